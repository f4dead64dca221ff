"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: noise assignments and FP64 counts bit-exact for the same seed; node
amplitudes within 1e-12 (FP64) and 2e-5 (FP32) of the oracle; FP32 histograms
differ only where a sample lies within rounding of an outcome boundary."""
import math

import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from tqs_inputs import Circuit, ghz, inverse_qft_on_fourier_state, qft, random_layers

pytestmark = pytest.mark.gpu

P1, P2, PM = 1e-3, 1e-2, 2e-2
TWO = ("cx", "cz", "cp", "swap", "u2")


def run(circ, shots, seed, p=(P1, P2, PM), **opt):
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model(*p)
    return tqs.tqs_simulate(c, nz, shots, seed, tqs.options(**opt), n=circ.n)


def partition(circ, shots, p=(P1, P2, PM), **opt):
    return tqs.tqs_partition(tqs.circuit(circ), tqs.tqs_noise_model(*p), shots, tqs.options(**opt))


def mixed_circuit(n, seed):
    """Random layers plus every gate kind, swaps in the middle and at the end."""
    c = random_layers(n, 4, seed)
    rng = np.random.default_rng(seed)
    u = np.linalg.qr(rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))[0]
    v = np.linalg.qr(rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2)))[0]
    c.add("swap", 0, n - 1).add("cx", n - 2, 1).add("u2", 2, n - 1, 0.0, u).add("u1", n // 2, -1, 0.0, v)
    for g in ("h", "x", "y", "z", "s", "sdg", "t", "tdg"):
        c.add(g, int(rng.integers(n)))
    c.add("p", 1, -1, 0.3).add("cp", n - 1, 0, 1.1).add("cz", 1, n - 2).add("swap", 1, n - 3)
    c.add("rx", n - 1, -1, 0.7).add("ry", 0, -1, 2.2).add("rz", n - 2, -1, 0.4)
    c.gates.extend(random_layers(n, 2, seed + 1).gates)
    c.add("swap", 2, n - 2)
    return c


def test_config1_qft10_baseline_fp64_bit_exact(orc):
    circ = qft(10)
    counts, F, rep = run(circ, 1000, 0, mode="baseline", prec="fp64")
    want = orc.core.run_baseline(circ, P1, P2, PM, 1000, 0)
    assert counts.sum() == 1000
    assert np.array_equal(counts, want)
    assert math.isnan(F)  # QFT|0> has a uniform ideal distribution


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noise_assignment_bit_exact(orc, prec):
    circ = mixed_circuit(9, 3)
    p = (0.2, 0.35, 0.0)
    arity, split = partition(circ, 400, p, part="ucp", k=3)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*p)
    o = tqs.options(part="ucp", k=3, prec=prec)
    for level, node in [(0, 0), (0, 3), (1, 13), (2, 50), (3, 399)]:
        sites = split[level + 1] - split[level]
        got = tqs.tqs_debug_node_noise(c, nz, 400, 77, o, level, node, sites)
        want = orc.core.node_noise(circ, p[0], p[1], 77, split, level, node)
        assert np.array_equal(got.astype(np.int64), want.astype(np.int64)), (level, node)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("tile", [6, 8, 12])
def test_node_amplitudes(orc, prec, tol, tile):
    """Multi-tile (n=13 with 6/8-qubit tiles), multi-pass, every gate kind, lazy
    swaps and a high noise rate so that X/Y/Z frames are exercised."""
    circ = mixed_circuit(13, 5)
    p = (0.15, 0.3, 0.0)
    shots = 32
    arity, split = [4, 2, 2, 2], [0, 20, 61, 100, len(circ.gates)]
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*p)
    o = tqs.options(arity=arity, split=split, prec=prec, tile_qubits=tile)
    for level, node in [(0, 1), (1, 6), (2, 9), (3, 31)]:
        got = tqs.tqs_debug_node_state(c, nz, shots, 11, o, level, node, circ.n)
        want = orc.core.node_state(circ, p[0], p[1], 11, arity, split, level, node)
        err = np.max(np.abs(got - want))
        assert err < tol, (level, node, err)


@pytest.mark.parametrize("circ_fn,tile", [(lambda: qft(12), 7), (lambda: random_layers(11, 9, 4), 6),
                                          (lambda: mixed_circuit(10, 8), 12), (lambda: ghz(12), 5 + 1),
                                          (lambda: qft(14), 10), (lambda: mixed_circuit(12, 6), 11)])
def test_tree_counts_fp64_bit_exact(orc, circ_fn, tile):
    circ = circ_fn()
    shots, seed = 3000, 4
    arity, split = partition(circ, shots)
    counts, F, rep = run(circ, shots, seed, prec="fp64", tile_qubits=tile)
    want = orc.core.run_tree(circ, P1, P2, PM, shots, seed, arity, split)
    assert counts.sum() == shots
    assert np.array_equal(counts, want)
    assert rep["arity"] == arity and rep["split"] == split


@pytest.mark.parametrize("arity,split_fn", [
    ([7, 3, 5], lambda G: [0, 10, 10, G]),          # empty middle level, 105 leaves for 100 shots
    ([100, 1, 1], lambda G: [0, 5, 30, G]),         # degenerate tree
    ([1, 1, 100], lambda G: [0, 12, 40, G]),        # the (1, N) tree of Sec. 3.6
    ([2, 3, 4, 5], lambda G: [0, 1, 2, 3, G]),
])
def test_explicit_trees_fp64_bit_exact(orc, arity, split_fn):
    circ = mixed_circuit(8, 2)
    split = split_fn(len(circ.gates))
    shots = 100
    p = (0.05, 0.1, 0.05)
    counts, _, rep = run(circ, shots, 9, p, prec="fp64", arity=arity, split=split)
    want = orc.core.run_tree(circ, p[0], p[1], p[2], shots, 9, arity, split)
    assert np.array_equal(counts, want)


@pytest.mark.parametrize("idx", range(6))
def test_speed_accuracy_study_trees_fp64_bit_exact(orc, idx):
    """The six tree structures of the speed-against-accuracy study (Sec. 5.6:
    DCP, XCP (20,10,5), UCP (10,10,10), (5,10,20), (2,2,250) and (250,1,1)) on
    its phase-estimation workload: FP64 counts bit-exact for two seeds, so the
    study's fidelities are the oracle's."""
    from paper_2203_13892_gb300 import sweep

    circ = sweep.workload()
    label, arity, split, shots = sweep.structures(circ)[idx]
    for seed in (0, 7):
        counts, F, rep = run(circ, shots, seed, prec="fp64", arity=arity, split=split)
        want = orc.core.run_tree(circ, P1, P2, PM, shots, seed, arity, split)
        assert rep["arity"] == arity and int(counts.sum()) == shots
        assert np.array_equal(counts, want), (label, seed)


def test_degenerate_tree_equals_baseline_on_gpu():
    circ = random_layers(10, 6, 1)
    G = len(circ.gates)
    a, _, _ = run(circ, 500, 3, mode="baseline", prec="fp64")
    b, _, _ = run(circ, 500, 3, prec="fp64", arity=[500, 1, 1], split=[0, 7, 33, G])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("circ", [Circuit(1).add("h", 0), Circuit(3), Circuit(2).add("swap", 0, 1),
                                  Circuit(1).add("x", 0).add("rz", 0, -1, 0.2)])
@pytest.mark.parametrize("shots", [1, 37])
def test_edge_cases_fp64(orc, circ, shots):
    for mode in ("baseline", "tree"):
        counts, _, _ = run(circ, shots, 5, (0.3, 0.3, 0.1), mode=mode, prec="fp64")
        arity, split = partition(circ, shots, (0.3, 0.3, 0.1), mode=mode)
        want = orc.core.run_tree(circ, 0.3, 0.3, 0.1, shots, 5, arity, split)
        assert np.array_equal(counts, want)


def test_fp32_histogram_close_to_oracle(orc):
    circ = qft(11)
    shots = 4000
    arity, split = partition(circ, shots)
    counts, _, _ = run(circ, shots, 6, prec="fp32", tile_qubits=8)
    want = orc.core.run_tree(circ, P1, P2, PM, shots, 6, arity, split)
    assert counts.sum() == shots
    # identical noise; FP32 amplitudes only move samples that fall within ~1e-6 of a boundary
    assert np.abs(counts.astype(np.int64) - want.astype(np.int64)).sum() <= 8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fidelity_matches_oracle(orc, prec):
    circ = inverse_qft_on_fourier_state(9, 300)
    shots = 2000
    arity, split = partition(circ, shots)
    counts, F, rep = run(circ, shots, 1, prec=prec)
    ideal = np.abs(orc.core.ideal_state(circ)) ** 2
    want = orc.fidelity.normalized_fidelity(ideal, counts / shots)
    assert abs(F - want) < 1e-9
    assert 0.0 < F < 1.0
    orc_counts = orc.core.run_tree(circ, P1, P2, PM, shots, 1, arity, split)
    Fo = orc.fidelity.normalized_fidelity(ideal, orc_counts / shots)
    assert abs(F - Fo) < (1e-9 if prec == "fp64" else 0.01)


def test_plan_execute_device_counts(orc):
    torch = pytest.importorskip("torch")
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    plan = tqs.tqs_plan_create(c, nz, 1000, tqs.options(mode="baseline", prec="fp64"))
    d = torch.zeros(1 << 10, dtype=torch.int64, device="cuda")
    rep = tqs.tqs_plan_execute(plan, 0, d.data_ptr(), report=True)
    want = orc.core.run_baseline(circ, P1, P2, PM, 1000, 0)
    assert np.array_equal(d.cpu().numpy().astype(np.uint64), want)
    assert rep["kernel_ms"] > 0 and rep["kernel_launches"] >= 3
    # a second execution with the same seed reproduces the histogram
    tqs.tqs_plan_execute(plan, 0, d.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().astype(np.uint64), want)
