"""Pins of the oracle's noiseless state-vector simulation (Sec. 2.2) to textbook
identities and closed forms, so that a wrong matrix entry, qubit order or index
loop fails here and not only in a comparison with the CUDA path."""
import cmath
import math

import numpy as np
import pytest

from tqs_inputs import (Circuit, ghz, qft_on_basis, inverse_qft_on_fourier_state, qaoa_maxcut, qpe,
                        random_layers, random_regular_graph)

I2 = np.eye(2)


def M(orc, name, th=0.0, mat=None):
    return orc.core.gate_matrix(name, th, mat)


def test_pauli_and_clifford_identities(orc):
    X, Y, Z, H = (M(orc, g) for g in "xyzh")
    S, Sd, T, Td = M(orc, "s"), M(orc, "sdg"), M(orc, "t"), M(orc, "tdg")
    assert np.allclose(X @ X, I2) and np.allclose(Y @ Y, I2) and np.allclose(Z @ Z, I2)
    assert np.allclose(X @ Y, 1j * Z)          # XY = iZ
    assert np.allclose(H @ X @ H, Z) and np.allclose(H @ Z @ H, X)
    assert np.allclose(H @ H, I2)
    assert np.allclose(S @ S, Z) and np.allclose(T @ T, S)
    assert np.allclose(S @ Sd, I2) and np.allclose(T @ Td, I2)
    assert np.allclose(S @ X @ Sd, Y)          # S X S^dag = Y


@pytest.mark.parametrize("th", [0.0, 0.3, 1.0, math.pi, 4.5])
def test_rotation_identities(orc, th):
    X, Y, Z, H, S, Sd = (M(orc, g) for g in ("x", "y", "z", "h", "s", "sdg"))
    RX, RY, RZ, P = M(orc, "rx", th), M(orc, "ry", th), M(orc, "rz", th), M(orc, "p", th)
    c, s = math.cos(th / 2), math.sin(th / 2)
    # R_P(t) = cos(t/2) I - i sin(t/2) P
    assert np.allclose(RX, c * I2 - 1j * s * X)
    assert np.allclose(RY, c * I2 - 1j * s * Y)
    assert np.allclose(RZ, c * I2 - 1j * s * Z)
    assert np.allclose(H @ RZ @ H, RX)
    assert np.allclose(S @ RX @ Sd, RY)
    assert np.allclose(P, cmath.exp(1j * th / 2) * RZ)   # P = e^{i t/2} RZ
    for U in (RX, RY, RZ, P):
        assert np.allclose(U.conj().T @ U, I2)


def basis(n, x):
    v = np.zeros(1 << n, dtype=complex)
    v[x] = 1.0
    return v


def test_cx_truth_table_control_is_q0(orc):
    # X on qubit 0 then CX(0 -> 1): |01> (index 1) -> |11> (index 3)
    c = Circuit(2).add("x", 0).add("cx", 0, 1)
    assert np.allclose(orc.core.ideal_state(c), basis(2, 3))
    # control 0 unset: target untouched
    c = Circuit(2).add("x", 1).add("cx", 0, 1)
    assert np.allclose(orc.core.ideal_state(c), basis(2, 2))
    # on non-adjacent qubits of a wider register
    c = Circuit(4).add("x", 3).add("cx", 3, 1)
    assert np.allclose(orc.core.ideal_state(c), basis(4, 0b1010))


def test_swap_cz_cp_definitions(orc):
    c = Circuit(3).add("x", 0).add("swap", 0, 2)
    assert np.allclose(orc.core.ideal_state(c), basis(3, 4))
    c = Circuit(2).add("x", 0).add("x", 1).add("cz", 0, 1)
    assert np.allclose(orc.core.ideal_state(c), -basis(2, 3))
    c = Circuit(2).add("x", 0).add("x", 1).add("cp", 1, 0, 0.7)
    assert np.allclose(orc.core.ideal_state(c), cmath.exp(0.7j) * basis(2, 3))
    c = Circuit(2).add("x", 0).add("cp", 0, 1, 0.7)   # only one bit set: no phase
    assert np.allclose(orc.core.ideal_state(c), basis(2, 1))
    assert np.allclose(M(orc, "cp", math.pi), M(orc, "cz"))


def test_u1_u2_match_named_gates(orc):
    h = M(orc, "h")
    a = orc.core.ideal_state(Circuit(3).add("h", 1).add("cx", 1, 2))
    b = orc.core.ideal_state(Circuit(3).add("u1", 1, -1, 0.0, h).add("u2", 1, 2, 0.0, M(orc, "cx")))
    assert np.allclose(a, b)


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_ghz(orc, n):
    psi = orc.core.ideal_state(ghz(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    if n == 1:
        want[:] = 1 / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-14)


@pytest.mark.parametrize("n,x", [(1, 1), (3, 5), (6, 0), (6, 37), (10, 123), (12, 4095)])
def test_qft_closed_form(orc, n, x):
    psi = orc.core.ideal_state(qft_on_basis(n, x))
    y = np.arange(1 << n)
    want = np.exp(2j * np.pi * x * y / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(psi - want)) < 1e-12


@pytest.mark.parametrize("n,b", [(4, 9), (8, 170), (11, 1234)])
def test_inverse_qft_on_fourier_state_returns_basis(orc, n, b):
    psi = orc.core.ideal_state(inverse_qft_on_fourier_state(n, b))
    assert abs(abs(psi[b]) - 1.0) < 1e-12
    assert np.sum(np.abs(psi) ** 2) - abs(psi[b]) ** 2 < 1e-20 + 1e-12


@pytest.mark.parametrize("m,phi", [(4, 0.3), (6, 1.0 / 3.0), (8, 0.3), (5, 5.0 / 32.0)])
def test_qpe_textbook_distribution(orc, m, phi):
    """Phase estimation with m counting qubits: the target stays in |1> and the
    counting register reads y with probability
    |2^-m sum_k exp(2 pi i k (phi - y/2^m))|^2 = sin^2(pi 2^m d) / (2^2m sin^2(pi d)),
    d = phi - y/2^m (exactly 1 at y = phi 2^m when that is an integer)."""
    M_ = 1 << m
    psi = orc.core.ideal_state(qpe(m, phi))
    p = np.abs(psi) ** 2
    assert p[:M_].sum() < 1e-24 + 1e-14  # target qubit m is 1 throughout
    d = phi - np.arange(M_) / M_
    s = np.sin(np.pi * d)
    want = np.where(np.abs(s) < 1e-12, 1.0, np.sin(np.pi * M_ * d) ** 2 / np.where(np.abs(s) < 1e-12, 1.0, M_ * M_ * s * s))
    assert np.max(np.abs(p[M_:] - want)) < 1e-12


@pytest.mark.parametrize("n,d,gseed", [(10, 3, 5), (8, 3, 11), (9, 4, 2)])
def test_qaoa_p1_maxcut_closed_form(orc, n, d, gseed):
    """One QAOA layer for MaxCut: the expected cut has the closed form of Wang,
    Hadfield, Jiang and Rieffel (Phys. Rev. A 97, 022304, 2018) for any graph,
    per edge uv with D_u = deg(u) - 1, D_v = deg(v) - 1 and t_uv triangles on uv:
    1/2 + sin(4b) sin(g) (cos^D_u g + cos^D_v g) / 4
        - sin^2(2b) cos^(D_u + D_v - 2 t_uv) g (1 - cos^t_uv 2g) / 4.
    It pins the oracle's H, CX, RZ and RX and the generator's decomposition."""
    E = random_regular_graph(n, d, gseed)
    nb = {v: set() for v in range(n)}
    for u, v in E:
        nb[u].add(v)
        nb[v].add(u)
    x = np.arange(1 << n)
    cut = np.zeros(1 << n)
    for u, v in E:
        cut += ((x >> u) & 1) != ((x >> v) & 1)
    for g, b in [(0.3, 0.2), (1.1, 0.7), (2.5, 1.3), (0.7, -0.4)]:
        want = 0.0
        for u, v in E:
            du, dv, t = len(nb[u]) - 1, len(nb[v]) - 1, len(nb[u] & nb[v])
            want += (0.5 + 0.25 * math.sin(4 * b) * math.sin(g) * (math.cos(g) ** du + math.cos(g) ** dv)
                     - 0.25 * math.sin(2 * b) ** 2 * math.cos(g) ** (du + dv - 2 * t) * (1 - math.cos(2 * g) ** t))
        p = np.abs(orc.core.ideal_state(qaoa_maxcut(n, E, g, b))) ** 2
        assert abs(float(p @ cut) - want) < 1e-11, (g, b)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_norm_preserved_random_circuit(orc, seed):
    c = random_layers(11, 12, seed)
    psi = orc.core.ideal_state(c)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13


def test_apply_matches_full_matrix_product(orc):
    """The oracle's in-place index loops agree with the product of embedded full
    matrices (the density module's independent element-wise embedding)."""
    c = random_layers(5, 3, 77)
    c.add("cx", 4, 0).add("swap", 1, 3).add("cp", 2, 4, 0.9).add("h", 2)
    psi = np.zeros(32, dtype=complex)
    psi[0] = 1
    for name, q0, q1, th, mat in c.gates:
        u = orc.core.gate_matrix(name, th, mat)
        qs = (q0,) if u.shape[0] == 2 else (q0, q1)
        psi = orc.density.embed(u, qs, 5) @ psi
    assert np.max(np.abs(orc.core.ideal_state(c) - psi)) < 1e-13
