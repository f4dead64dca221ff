"""Batched execution replayed from one CUDA graph (uneven circuits) and the
autotuner: the histograms must equal the single-simulation path bit for bit in
FP64, replays with new seeds must not need a new capture, and a tuned plan must
reproduce the untuned counts."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import batch_circuits_spec, qft, random_layers

pytestmark = pytest.mark.gpu

P = (2e-3, 1.5e-2, 2e-2)


def uneven_circuits():
    return [random_layers(6, 5, 1), qft(9), random_layers(13, 7, 2), qft(4), random_layers(11, 3, 3),
            random_layers(14, 4, 4)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_single_simulations(orc, prec):
    circs = uneven_circuits()
    shots = [300, 1000, 700, 64, 512, 400]
    handles = [tqs.circuit(c) for c in circs]
    noises = [tqs.tqs_noise_model(*P) for _ in circs]
    o = tqs.options(prec=prec)
    b = tqs.tqs_batch_create(handles, noises, shots, o)
    assert tqs.tqs_batch_size(b) == len(circs)
    for seeds in ([1, 2, 3, 4, 5, 6], [70, 60, 50, 40, 30, 20]):
        rep = tqs.tqs_batch_execute(b, seeds, report=True)
        assert rep["shots_done"] == sum(shots) and rep["kernel_ms"] > 0
        for i, c in enumerate(circs):
            got = tqs.tqs_batch_counts(b, i, c.n)
            want, _, _ = tqs.tqs_simulate(handles[i], noises[i], shots[i], seeds[i],
                                          tqs.options(prec=prec, flags=capi.TQS_FLAG_NO_FIDELITY), n=c.n)
            assert np.array_equal(got, want), (i, seeds[i])
            if prec == "fp64" and c.n <= 9:
                arity, split = tqs.tqs_partition(handles[i], noises[i], shots[i], o)
                oracle = orc.core.run_tree(c, *P, shots[i], seeds[i], arity, split)
                assert np.array_equal(got, oracle)


def test_batch_device_counts_pointer():
    torch = pytest.importorskip("torch")
    circs = uneven_circuits()[:3]
    b = tqs.tqs_batch_create([tqs.circuit(c) for c in circs], [tqs.tqs_noise_model(*P)] * 3, [100, 200, 300])
    tqs.tqs_batch_execute(b, [5, 6, 7])
    for i, c in enumerate(circs):
        ptr = tqs.tqs_batch_device_counts(b, i)
        assert ptr != 0
        host = tqs.tqs_batch_counts(b, i, c.n)
        assert int(host.sum()) == [100, 200, 300][i]


def test_batch_spec_circuits_small_subset():
    """The uneven-batch generator's circuits (n 12..22) run in one graph; their
    counts sum to the shots."""
    spec = [s for s in batch_circuits_spec() if s[0] <= 14][:6]
    circs = [random_layers(n, L, seed) for n, L, seed in spec]
    b = tqs.tqs_batch_create([tqs.circuit(c) for c in circs], [tqs.tqs_noise_model(*P)] * len(circs),
                             [2048] * len(circs))
    tqs.tqs_batch_execute(b, list(range(len(circs))))
    for i, c in enumerate(circs):
        assert int(tqs.tqs_batch_counts(b, i, c.n).sum()) == 2048


def test_autotune_reproduces_untuned_counts():
    c = random_layers(14, 10, 9)
    h, nz = tqs.circuit(c), tqs.tqs_noise_model(*P)
    base, _, _ = tqs.tqs_simulate(h, nz, 2000, 3, tqs.options(prec="fp64", flags=capi.TQS_FLAG_NO_FIDELITY), n=c.n)
    tuned, _, rep = tqs.tqs_simulate(h, nz, 2000, 3, tqs.options(prec="fp64", flags=capi.TQS_FLAG_NO_FIDELITY
                                                                  | capi.TQS_FLAG_AUTOTUNE), n=c.n)
    assert np.array_equal(base, tuned)


def test_config3_batch64_error_per_circuit(orc):
    """The uneven 64-circuit batch (12-22 qubits, 20-60 layers, 2,048 shots each,
    FP32, one graph), error per circuit (first 16 circuits):
      * one leaf state, FP32 against FP64 with the same noise: relative L2 error
        within the FP32 rounding bound 2u per gate (u = 2^-24); for the circuits
        of <= 14 qubits also the FP32 amplitudes against the FP64 oracle;
      * the histogram against the FP64 path with the same seed.  Identical noise,
        so a sample can only move to a neighbouring outcome where FP32 rounding
        shifts a cumulative-probability boundary; with 2^22 outcomes that happens
        to a few per cent of the samples, so the check is on 256 coarse bins (the
        top 8 outcome bits), which such a shift almost never crosses."""
    spec = batch_circuits_spec()
    circs = [random_layers(n, L, seed) for n, L, seed in spec]
    noise = (1e-3, 1e-2, 2e-2)
    b = tqs.tqs_batch_create([tqs.circuit(c) for c in circs], [tqs.tqs_noise_model(*noise)] * 64, [2048] * 64,
                             tqs.options(prec="fp32"))
    seeds = list(range(500, 564))
    tv, tv_coarse, rel, amp = [], [], [], []
    tqs.tqs_batch_execute(b, seeds)
    for i, c in enumerate(circs[:16]):
        h, nz = tqs.circuit(c), tqs.tqs_noise_model(*noise)
        got = tqs.tqs_batch_counts(b, i, c.n).astype(np.int64)
        assert int(got.sum()) == 2048
        want, _, _ = tqs.tqs_simulate(h, nz, 2048, seeds[i], tqs.options(prec="fp64", flags=capi.TQS_FLAG_NO_FIDELITY),
                                      n=c.n)
        want = want.astype(np.int64)
        tv.append(0.5 * np.abs(got - want).sum() / 2048)
        sh = max(c.n - 8, 0)
        cg = np.bincount(np.arange(1 << c.n) >> sh, weights=got)
        cw = np.bincount(np.arange(1 << c.n) >> sh, weights=want)
        tv_coarse.append(0.5 * np.abs(cg - cw).sum() / 2048)
        arity, split = tqs.tqs_partition(h, nz, 2048, tqs.options())
        L = len(arity)
        p32 = tqs.tqs_debug_node_state(h, nz, 2048, seeds[i], tqs.options(prec="fp32"), L - 1, 2047, c.n)
        p64 = tqs.tqs_debug_node_state(h, nz, 2048, seeds[i], tqs.options(prec="fp64"), L - 1, 2047, c.n)
        r = float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))
        rel.append(r)
        assert r <= 2 * 2.0 ** -24 * len(c.gates), (i, r)
        if c.n <= 14:
            ref = orc.core.node_state(c, noise[0], noise[1], seeds[i], arity, split, L - 1, 2047)
            amp.append(float(np.max(np.abs(p32 - ref))))
    for i in range(16, 64):
        assert int(tqs.tqs_batch_counts(b, i, circs[i].n).sum()) == 2048
    print("config3 qubits:", [c.n for c in circs[:16]])
    print("config3 leaf-state relative L2 error FP32 vs FP64:", [f"{x:.2e}" for x in rel])
    print("config3 histogram TV vs FP64 (outcomes / 256 coarse bins):",
          [f"{x:.4f}/{y:.4f}" for x, y in zip(tv, tv_coarse)])
    print("config3 max |amp - oracle| (n <= 14):", amp)
    assert max(tv_coarse) <= 4 / 2048, tv_coarse
    assert amp and max(amp) < 2e-5, amp
