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
