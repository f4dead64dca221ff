"""Host side of the specialised pass kernels (no device): the generator turns
every pass program into statements that NVRTC compiles for sm_103a, one
statement per dense gate in the pass's program order, and the entry points
refuse what they do not cover."""
import re

import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

P = (1e-3, 1e-2, 2e-2)
DENSE1 = {"h", "x", "y", "rx", "ry", "u1"}
DENSE2 = {"cx", "u2"}


def _mixed(n, seed):
    c = random_layers(n, 3, seed)
    rng = np.random.default_rng(seed)
    u = np.linalg.qr(rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))[0]
    v = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))[0]
    c.add("swap", 0, n - 1).add("cx", n - 2, 1).add("u2", 2, n - 1, 0.0, u).add("u1", n // 2, -1, 0.0, v)
    for g in ("h", "x", "y", "z", "s", "sdg", "t", "tdg"):
        c.add(g, int(rng.integers(n)))
    c.add("p", 1, -1, 0.3).add("cp", n - 1, 0, 1.1).add("cz", 1, n - 2).add("rx", n - 1, -1, 0.7)
    c.add("ry", 0, -1, 2.2).add("rz", n - 2, -1, 0.4)
    return c


def _nvrtc_or_skip(c, nz, shots, o):
    try:
        return tqs.tqs_debug_spec_check(c, nz, shots, o)
    except capi.TqsError as e:
        if e.status == capi.TQS_EUNSUPPORTED:
            pytest.skip(str(e))
        raise


@pytest.mark.parametrize("name,circ_fn,shots,kw", [
    ("qft20", lambda: qft(20), 32000, {}),
    ("mixed13_t8", lambda: _mixed(13, 5), 64, {"tile_qubits": 8}),
    ("mixed13_t12", lambda: _mixed(13, 5), 64, {"tile_qubits": 12}),
    ("rc12_t10", lambda: random_layers(12, 6, 2), 512, {"tile_qubits": 10}),
])
def test_every_specialised_kernel_compiles(name, circ_fn, shots, kw):
    circ = circ_fn()
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    o = tqs.options(prec="fp32", **kw)
    nk, nbytes = _nvrtc_or_skip(c, nz, shots, o)
    _, _, tiles = tqs.tqs_debug_plan_order(c, nz, shots, o, len(circ.gates))
    assert nk == len(tiles) + 2  # a store kernel per pass, and the last pass's two measuring modes
    assert nbytes > 0


def test_damping_channel_programs_compile():
    circ = random_layers(8, 2, 77)
    circ.add("cx", 0, 7).add("h", 3)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model_ex(*P, ad_gamma=0.01, pd_lambda=0.01, t1=50e-6, t2=70e-6, time_1q=0.5e-6,
                                time_2q=2e-6)
    nk, _ = _nvrtc_or_skip(c, nz, 100, tqs.options(prec="fp32", tile_qubits=8))
    assert nk == len(circ.gates) + 1 + 2  # one gate per pass, a closing pass, two measuring modes


def test_one_statement_per_dense_gate_in_program_order():
    """Pin of the generator against the planner's own record of the plan: each
    pass's source holds one dense1 / dense1_real / dense2 call per dense gate of
    that pass, in the order the plan applies them, on the gate's tile position."""
    circ = _mixed(13, 5)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    o = tqs.options(prec="fp32", tile_qubits=8)
    order, pass_of, tiles = tqs.tqs_debug_plan_order(c, nz, 64, o, len(circ.gates))
    for p in range(len(tiles)):
        src = tqs.tqs_debug_spec_source(c, nz, 64, o, p, 0)
        calls = re.findall(r"\b(dense1_real|dense1|dense2)\(", src)
        kinds = [circ.gates[g][0] for g, q in zip(order, pass_of) if q == p]
        want = ["dense2" if k in DENSE2 else "dense1" for k in kinds if k in DENSE1 | DENSE2]
        got = ["dense1" if k == "dense1_real" else k for k in calls]
        assert got == want, (p, got, want)
        # the pass's tile width is a compile-time constant of its kernel
        tile = [b for b in range(circ.n) if (int(tiles[p]) >> b) & 1]
        assert src.count("flush();") >= len(want)
        assert "kT = " + str(len(tile)) + "u" in src


def test_leaf_of_the_qft20_tree_is_straight_line():
    """The benchmark's leaf pass: six Hadamards (real matrices), five diagonal
    runs whose phases all sit on thread bits and the run of the final lazy
    swaps (noise sites only), nothing interpreted."""
    circ = qft(20)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    o = tqs.options(prec="fp32")
    _, _, tiles = tqs.tqs_debug_plan_order(c, nz, 32000, o, len(circ.gates))
    src = tqs.tqs_debug_spec_source(c, nz, 32000, o, len(tiles) - 1, 1)
    assert src.count("dense1_real(") == 6 and "dense2(" not in src
    assert src.count("// diagonal run") == 6
    assert "acc.E[" not in src and "acc.Gs[" not in src
    assert "chunk_begin" not in src and "pbuf" not in src


def test_refusals():
    circ = qft(8)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_debug_spec_check(c, nz, 64, tqs.options(prec="fp64"))
    assert e.value.status == capi.TQS_EINVAL
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_debug_spec_source(c, nz, 64, tqs.options(prec="fp32"), 999, 0)
    assert e.value.status == capi.TQS_EINVAL
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_debug_spec_source(c, nz, 64, tqs.options(prec="fp32"), 0, 3)
    assert e.value.status == capi.TQS_EINVAL


def test_test_plans_reach_every_record_form():
    """The plans the GPU parity tests run with specialised kernels produce every
    form the generator writes: real and complex one-qubit matrices, 4x4
    matrices, base, slot and pair phase terms, the per-gate fallback of runs,
    damping records."""
    def all_sources(circ, nz, shots, o):
        _, _, tiles = tqs.tqs_debug_plan_order(tqs.circuit(circ), nz, shots, o, len(circ.gates))
        return "".join(tqs.tqs_debug_spec_source(tqs.circuit(circ), nz, shots, o, p, 0) for p in range(len(tiles)))

    from test_gpu_parity import mixed_circuit

    nz = tqs.tqs_noise_model(0.15, 0.3, 0.0)
    src = ""
    for tile in (8, 10, 12):
        circ = mixed_circuit(13, 5)
        o = tqs.options(prec="fp32", tile_qubits=tile, arity=[4, 2, 2, 2],
                        split=[0, 20, 61, 100, len(circ.gates)])
        src += all_sources(circ, nz, 32, o)
    for form in ("dense1_real(", "dense1(", "dense2(", "acc.base += add", "acc.E[", "acc.Gs[", "acc_alpha(",
                 "acc_gamma(", "apply_noise("):
        assert form in src, form
    circ = random_layers(10, 4, 77)
    circ.add("h", 0).add("cx", 0, 9).add("cp", 3, 5, 0.4).add("swap", 2, 7).add("x", 4)
    G = len(circ.gates)
    nzk = tqs.tqs_noise_model_ex(*P, ad_gamma=0.01, pd_lambda=0.01, t1=50e-6, t2=70e-6, time_1q=0.5e-6,
                                 time_2q=2e-6)
    o = tqs.options(prec="fp32", tile_qubits=8, arity=[40, 3, 5], split=[0, G // 3, 2 * G // 3, G])
    assert "km[0].x" in all_sources(circ, nzk, 600, o)


def test_matrix_literals_are_the_gates_fp32_matrices(orc):
    """The generator's hexadecimal literals are exact: each one-qubit dense gate's
    statement holds the FP32 rounding of that gate's matrix (the oracle's FP64
    matrix, rounded), real ones as dense1_real with the four real parts."""
    circ = _mixed(13, 5)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    o = tqs.options(prec="fp32", tile_qubits=8)
    order, pass_of, tiles = tqs.tqs_debug_plan_order(c, nz, 64, o, len(circ.gates))
    lit = r"(-?0x[0-9a-f.]+p[-+]\d+)f"
    checked = 0
    for p in range(len(tiles)):
        src = tqs.tqs_debug_spec_source(c, nz, 64, o, p, 0)
        calls = re.findall(r"\b(dense1_real|dense1)\(\d+u, \d+u, (.*?)\);\n", src)
        gates = [circ.gates[g] for g, q in zip(order, pass_of) if q == p and circ.gates[g][0] in DENSE1]
        assert len(calls) == len(gates), p
        for (kind, args), (name, q0, q1, th, mat) in zip(calls, gates):
            vals = [float.fromhex(x) for x in re.findall(lit, args)]
            u = orc.core.gate_matrix(name, th, mat).astype(np.complex64).ravel()
            if kind == "dense1_real":
                assert np.all(u.imag == 0) and vals == [float(x) for x in u.real], (name, vals)
            else:
                want = [float(x) for z in u for x in (z.real, z.imag)]
                assert vals == want, (name, vals, want)
            checked += 1
    assert checked >= 10


def test_qft20_leaf_phase_entries_are_the_controlled_phases():
    """Each diagonal run of the benchmark's leaf pass, as generated, adds for a
    thread exactly the controlled phases of its CP gates: one entry per gate,
    mask = the two qubits' bits (no swaps precede them in this pass, so physical
    = logical), phase = theta / 2 pi in units of 2^-32 turns (to one unit of
    rounding)."""
    circ = qft(20)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    o = tqs.options(prec="fp32")
    order, pass_of, tiles = tqs.tqs_debug_plan_order(c, nz, 32000, o, len(circ.gates))
    last = len(tiles) - 1
    src = tqs.tqs_debug_spec_source(c, nz, 32000, o, last, 1)
    gates = [circ.gates[g] for g, q in zip(order, pass_of) if q == last]
    runs, cur = [], None
    for name, q0, q1, th, _ in gates:
        if name == "h":
            if cur is not None:
                runs.append(cur)
            cur = []
        elif name == "cp":
            cur.append((q0, q1, th))
    if cur:
        runs.append(cur)
    blocks = src.split("// diagonal run")[1:]
    for run, block in zip(runs, blocks):
        fast = block.split("} else {")[0]
        got = sorted((int(m, 16), int(ph, 16)) for m, _, ph in
                     re.findall(r"if \(\(xt & (0x[0-9a-f]+)u\) == (0x[0-9a-f]+)u\) add \+= (0x[0-9a-f]+)u;", fast))
        want = sorted(((1 << a) | (1 << b), round(th / (2 * np.pi) * 2 ** 32) % 2 ** 32) for a, b, th in run)
        assert [m for m, _ in got] == [m for m, _ in want]
        assert all(abs(x - y) <= 1 for (_, x), (_, y) in zip(got, want)), (got, want)
    assert len(runs) == 5
