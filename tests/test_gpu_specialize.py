"""Pass kernels specialised per pass program (TQS_FLAG_SPECIALIZE) against the
FP64 oracle and against the generic FP32 kernel that interprets the same
records.  The specialised kernels run the same arithmetic as the generic FP32
path, so they meet its bars: node amplitudes within 2e-5 of the oracle, sampled
leaves of the 20-qubit QFT workload present in the histogram (or a neighbour,
where FP32 rounding moves a cumulative-probability boundary), and histograms
equal to the generic kernel's up to such moves.  The circuits cover every
record kind: dense one- and two-qubit gates (real and complex matrices),
diagonal runs with thread, slot and pair terms, the per-gate fallback of runs
that hold a Pauli (heavy noise), lazy swaps and the damping channels' records."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

from test_gpu_parity import mixed_circuit

pytestmark = pytest.mark.gpu

SPEC = capi.TQS_FLAG_SPECIALIZE
P1, P2, PM = 1e-3, 1e-2, 2e-2


@pytest.mark.parametrize("tile", [8, 10, 12])
def test_node_amplitudes_specialized(orc, tile):
    circ = mixed_circuit(13, 5)
    p = (0.15, 0.3, 0.0)
    shots = 32
    arity, split = [4, 2, 2, 2], [0, 20, 61, 100, len(circ.gates)]
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*p)
    o = tqs.options(arity=arity, split=split, prec="fp32", tile_qubits=tile, flags=SPEC)
    for level, node in [(0, 1), (1, 6), (2, 9), (3, 31)]:
        got = tqs.tqs_debug_node_state(c, nz, shots, 11, o, level, node, circ.n)
        want = orc.core.node_state(circ, p[0], p[1], 11, arity, split, level, node)
        err = np.max(np.abs(got - want))
        assert err < 2e-5, (tile, level, node, err)


def test_damping_channels_specialized(orc):
    ch = dict(ad_gamma=0.01, pd_lambda=0.01, t1=50e-6, t2=70e-6, time_1q=0.5e-6, time_2q=2e-6)
    circ = random_layers(10, 4, 77)
    circ.add("h", 0).add("cx", 0, 9).add("cp", 3, 5, 0.4).add("swap", 2, 7).add("x", 4)
    G = len(circ.gates)
    arity, split = [40, 3, 5], [0, G // 3, 2 * G // 3, G]
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model_ex(P1, P2, PM, **ch)
    kr = orc.core.kraus_params(ad=ch["ad_gamma"], pd=ch["pd_lambda"], t1=ch["t1"], t2=ch["t2"],
                               time_1q=ch["time_1q"], time_2q=ch["time_2q"])
    o = tqs.options(prec="fp32", arity=arity, split=split, tile_qubits=8, flags=SPEC)
    for level, node in [(0, 7), (1, 100), (2, 599)]:
        got = tqs.tqs_debug_node_state(c, nz, 600, 11, o, level, node, circ.n)
        want = orc.core.node_state(circ, P1, P2, 11, arity, split, level, node, kraus=kr)
        assert np.max(np.abs(got - want)) < 2e-5, (level, node)


@pytest.mark.parametrize("circ_fn", [lambda: qft(14), lambda: random_layers(14, 12, 3), lambda: mixed_circuit(12, 6)])
def test_histogram_matches_generic_fp32(circ_fn):
    circ = circ_fn()
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    shots = 4096
    a, Fa, ra = tqs.tqs_simulate(c, nz, shots, 9, tqs.options(prec="fp32", flags=SPEC), n=circ.n)
    b, Fb, rb = tqs.tqs_simulate(c, nz, shots, 9, tqs.options(prec="fp32"), n=circ.n)
    assert int(a.sum()) == shots and ra["arity"] == rb["arity"]
    moved = int(np.abs(a.astype(np.int64) - b.astype(np.int64)).sum())
    print(f"{circ.n} qubits: {moved} samples differ between specialised and generic kernels")
    assert moved <= shots // 100
    # (NaN both times when the ideal distribution is uniform, as for the QFT of |0...0>)
    assert (np.isnan(Fa) and np.isnan(Fb)) or abs(Fa - Fb) < 0.02


def test_fp64_plans_ignore_the_flag(orc):
    circ = mixed_circuit(10, 8)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    a, _, _ = tqs.tqs_simulate(c, nz, 2000, 4, tqs.options(prec="fp64", flags=SPEC), n=circ.n)
    arity, split = tqs.tqs_partition(c, nz, 2000, tqs.options())
    want = orc.core.run_tree(circ, P1, P2, PM, 2000, 4, arity, split)
    assert np.array_equal(a, want)


def test_static_entry_refuses_specialisation():
    torch = pytest.importorskip("torch")
    circ = qft(8)
    d = torch.zeros(1 << circ.n, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_simulate_static(tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM), 64, 1,
                                tqs.options(prec="fp32", flags=SPEC), d.data_ptr())
    assert e.value.status == capi.TQS_EUNSUPPORTED


N, SHOTS = 20, 32000
LEAVES = [0, 1, 63, 64, 12345, 20000, 31936, 31999]


def _device_histogram(c, nz, seed, flags):
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    o = tqs.options(prec="fp32", stream=stream.cuda_stream, flags=flags)
    plan = tqs.tqs_plan_create(c, nz, SHOTS, o)
    d = torch.zeros(1 << N, dtype=torch.int64, device="cuda")
    rep = tqs.tqs_plan_execute(plan, seed, d.data_ptr(), report=True)
    stream.synchronize()
    plan.close()
    return d.cpu().numpy().astype(np.uint64), rep


def test_metric_workload_specialized(orc):
    """The benchmark's workload (20-qubit QFT, 32,000 shots, DCP tree) through the
    device-resident entry point with specialised kernels: oracle leaves present,
    and the histogram equal to the generic kernel's up to boundary moves."""
    from concurrent.futures import ThreadPoolExecutor

    circ = qft(N)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    arity, split = tqs.tqs_partition(c, nz, SHOTS, tqs.options())
    with ThreadPoolExecutor(max_workers=len(LEAVES)) as ex:
        ys = list(ex.map(lambda m: orc.core.leaf_outcome(circ, P1, P2, PM, 5, arity, split, m), LEAVES))
    spec, rep = _device_histogram(c, nz, 5, SPEC)
    assert rep["arity"] == arity and int(spec.sum()) == SHOTS
    for m, y in zip(LEAVES, ys):
        assert spec[max(y - 1, 0):min(y + 2, 1 << N)].sum() > 0, (m, y)
    assert sum(int(spec[y] > 0) for y in ys) >= len(LEAVES) - 1
    gen, _ = _device_histogram(c, nz, 5, 0)
    moved = int(np.abs(spec.astype(np.int64) - gen.astype(np.int64)).sum())
    print(f"QFT-20: {moved} of {SHOTS} samples differ between specialised and generic kernels")
    assert moved <= SHOTS // 100
    # a node state deep in the tree, element by element
    o = tqs.options(prec="fp32", flags=SPEC)
    L = len(arity)
    got = tqs.tqs_debug_node_state(c, nz, SHOTS, 5, o, L - 1, 31999, N)
    want = orc.core.node_state(circ, P1, P2, 5, arity, split, L - 1, 31999)
    assert np.max(np.abs(got - want)) < 2e-5


def test_batch_graph_with_specialised_kernels():
    """A batch of uneven circuits captured in one CUDA graph with the specialised
    kernels (driver-API launches inside the capture) gives the histograms of the
    single simulations with the same kernels, replay after replay."""
    circs = [random_layers(6, 5, 1), qft(9), random_layers(13, 7, 2), qft(4)]
    shots = [300, 1000, 700, 64]
    handles = [tqs.circuit(c) for c in circs]
    noises = [tqs.tqs_noise_model(P1, P2, PM) for _ in circs]
    b = tqs.tqs_batch_create(handles, noises, shots, tqs.options(prec="fp32", flags=SPEC))
    for seeds in ([1, 2, 3, 4], [40, 30, 20, 10]):
        tqs.tqs_batch_execute(b, seeds)
        for i, c in enumerate(circs):
            got = tqs.tqs_batch_counts(b, i, c.n)
            want, _, _ = tqs.tqs_simulate(handles[i], noises[i], shots[i], seeds[i],
                                          tqs.options(prec="fp32", flags=SPEC | capi.TQS_FLAG_NO_FIDELITY), n=c.n)
            assert np.array_equal(got, want), (i, seeds[i])


def test_index_checks_in_specialised_kernels():
    """TQS_FLAG_DEBUG_BOUNDS reaches the specialised kernels (their prologue is the
    generic one): valid input changes nothing, an understated output pool is caught
    before any access (TQS_EBOUNDS), and the next call is correct."""
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    base = capi.TQS_FLAG_NO_FIDELITY | SPEC
    o = dict(prec="fp32", batch=4)
    want, _, _ = tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=base, **o), n=circ.n)
    checked, _, _ = tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=base | capi.TQS_FLAG_DEBUG_BOUNDS, **o),
                                     n=circ.n)
    assert np.array_equal(checked, want)
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=base | capi.TQS_FLAG_DEBUG_BOUNDS |
                                                     capi.TQS_FLAG_FAULT_BOUNDS, **o), n=circ.n)
    assert e.value.status == capi.TQS_EBOUNDS
    again, _, _ = tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=base, **o), n=circ.n)
    assert np.array_equal(again, want)
