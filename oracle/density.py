"""Exact density-matrix simulation of the noisy circuit for small n (Sec. 2.3.1).

TEST INFRASTRUCTURE ONLY.  O(4^n) memory; meant for n <= 6.

Each gate U acts as rho <- U rho U^dagger; the depolarizing site after it is the
channel rho <- (1-p) rho + p/3 sum_{P in X,Y,Z} P rho P (one qubit) or
(1-p) rho + p/15 sum_{(a,b) != (I,I)} (P_a x P_b) rho (P_a x P_b) (two qubits,
a on q0, b on q1); the damping channels, when given, act as rho <- sum_i K_i rho
K_i^dagger (Sec. 4.3); measurement with readout error gives
P(y) = sum_x rho_xx prod_q (pm if x_q != y_q else 1 - pm).
The embedding of a local operator into the full space is written directly from
its definition (matrix element between full basis states), independent of the C
oracle's index loops.
"""
from __future__ import annotations

import numpy as np

from . import core

_PAULI = [
    np.eye(2, dtype=complex),
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]


def embed(u: np.ndarray, qubits, n: int) -> np.ndarray:
    """Full 2^n x 2^n matrix of the local operator u on `qubits` (local index
    k = sum_j bit(q_j) 2^j): <r|U|c> = u[k(r), k(c)] if r and c agree on every
    other qubit, else 0."""
    idx = np.arange(1 << n)
    k = np.zeros(1 << n, dtype=np.int64)
    other = idx.copy()
    for j, q in enumerate(qubits):
        k += ((idx >> q) & 1) << j
        other &= ~(1 << q)
    same = other[:, None] == other[None, :]
    return np.where(same, u[k[:, None], k[None, :]], 0.0)


def _depolarize(rho, qubits, p, n):
    if p == 0.0:
        return rho
    if len(qubits) == 1:
        acc = np.zeros_like(rho)
        for a in (1, 2, 3):
            P = embed(_PAULI[a], qubits, n)
            acc += P @ rho @ P.conj().T
        return (1.0 - p) * rho + (p / 3.0) * acc
    acc = np.zeros_like(rho)
    for t in range(1, 16):
        a, b = t >> 2, t & 3
        P = embed(np.kron(_PAULI[b], _PAULI[a]), qubits, n)  # local index bit0 = q0 (a)
        acc += P @ rho @ P.conj().T
    return (1.0 - p) * rho + (p / 15.0) * acc


def damping_kraus(r: float, amplitude: bool):
    """Kraus operators of amplitude damping (K0 = diag(1, sqrt(1-r)), K1 = sqrt(r) |0><1|)
    or phase damping (K0 = diag(1, sqrt(1-r)), K1 = sqrt(r) |1><1|), Nielsen & Chuang 8.3.5-8.3.6."""
    k0 = np.array([[1.0, 0.0], [0.0, np.sqrt(1.0 - r)]], dtype=complex)
    k1 = np.zeros((2, 2), dtype=complex)
    if amplitude:
        k1[0, 1] = np.sqrt(r)
    else:
        k1[1, 1] = np.sqrt(r)
    return k0, k1


def _channel(rho, q, kraus_ops, n):
    acc = np.zeros_like(rho)
    for k in kraus_ops:
        K = embed(k, (q,), n)
        acc += K @ rho @ K.conj().T
    return acc


def _damp(rho, qubits, kraus, n):
    """The non-unitary channels after a gate (as the trajectory oracle orders them):
    for each qubit of the gate, thermal relaxation's damping and dephasing, then
    amplitude damping, then phase damping; kraus = [AD gamma, PD lambda, TR pair
    after a one-qubit gate, TR pair after a two-qubit gate]."""
    if kraus is None:
        return rho
    two = len(qubits) == 2
    rates = [(kraus[4 if two else 2], True), (kraus[5 if two else 3], False), (kraus[0], True), (kraus[1], False)]
    for q in qubits:
        for r, amp in rates:
            if r > 0.0:
                rho = _channel(rho, q, damping_kraus(r, amp), n)
    return rho


def final_density(circuit, p1: float, p2: float, kraus=None) -> np.ndarray:
    n = circuit.n
    rho = np.zeros((1 << n, 1 << n), dtype=complex)
    rho[0, 0] = 1.0
    for name, q0, q1, th, mat in circuit.gates:
        u = core.gate_matrix(name, th, mat)
        qs = (q0,) if u.shape[0] == 2 else (q0, q1)
        U = embed(u, qs, n)
        rho = U @ rho @ U.conj().T
        rho = _depolarize(rho, qs, p1 if len(qs) == 1 else p2, n)
        rho = _damp(rho, qs, kraus, n)
    return rho


def outcome_distribution(circuit, p1: float, p2: float, pm: float, kraus=None) -> np.ndarray:
    """P(y) of the measured bitstring including readout error."""
    n = circuit.n
    diag = np.real(np.diag(final_density(circuit, p1, p2, kraus)))
    x = np.arange(1 << n)
    out = np.zeros(1 << n)
    for y in range(1 << n):
        d = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            d += ((x >> q) & 1) != ((y >> q) & 1)
        out[y] = np.sum(diag * (pm ** d) * ((1.0 - pm) ** (n - d)))
    return out
