"""The allocation-free entry point tqs_simulate_static, called through the C ABI.

Some callers cannot allocate device memory (a pool allocator owns the device,
a latency-critical loop must not synchronise on cudaMalloc, a plugin host
forbids it).  tqs_simulate_static serves them from a static scratch array inside
the library; here it must reproduce the histograms of the regular entry points
on two calls in a row (the array keeps the previous call's contents)."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

pytestmark = pytest.mark.gpu


def _device_counts(torch, n, fill):
    d = torch.empty(1 << n, dtype=torch.int64, device="cuda")
    d.fill_(fill)  # stale contents must not leak into the result
    return d


def test_static_matches_simulate_fp64_baseline_twice():
    torch = pytest.importorskip("torch")
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    o = tqs.options(mode="baseline", prec="fp64")
    want, _, _ = tqs.tqs_simulate(c, nz, 1000, 0, o, n=circ.n)
    for call in range(2):
        d = _device_counts(torch, circ.n, 7 + call)
        tqs.tqs_simulate_static(c, nz, 1000, 0, o, d.data_ptr())
        got = d.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, want), call


def test_static_matches_plan_execute_fp32_tree_twice():
    torch = pytest.importorskip("torch")
    circ = random_layers(12, 8, 5)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-2, 3e-2, 2e-2)
    o = tqs.options(prec="fp32")
    plan = tqs.tqs_plan_create(c, nz, 3000, o)
    ref = torch.zeros(1 << circ.n, dtype=torch.int64, device="cuda")
    tqs.tqs_plan_execute(plan, 11, ref.data_ptr())
    torch.cuda.synchronize()
    want = ref.cpu().numpy()
    for call in range(2):
        d = _device_counts(torch, circ.n, -1)
        tqs.tqs_simulate_static(c, nz, 3000, 11, o, d.data_ptr())
        assert np.array_equal(d.cpu().numpy(), want), call
        assert int(d.sum().item()) == 3000


def test_static_rejects_requests_beyond_the_array():
    torch = pytest.importorskip("torch")
    circ = qft(22)  # one FP32 state is 32 MiB: no room for one node per level
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    d = torch.zeros(1 << circ.n, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_simulate_static(c, nz, 100, 0, tqs.options(), d.data_ptr())
    assert e.value.status == capi.TQS_EINVAL
    assert "static scratch" in str(e.value)


def test_static_uses_the_whole_array_for_states():
    """QFT-20 in FP32 with three stored levels needs 24 MiB of states plus small
    tables: it fits the 32 MiB array only because this path reserves no internal
    histogram (8 MiB at 20 qubits) and no fidelity scratch."""
    torch = pytest.importorskip("torch")
    circ = qft(20)
    G = len(circ.gates)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    o = tqs.options(prec="fp32", arity=[4, 2, 2, 2], split=[0, 55, 110, 165, G])
    plan = tqs.tqs_plan_create(c, nz, 32, o)
    ref = torch.zeros(1 << circ.n, dtype=torch.int64, device="cuda")
    tqs.tqs_plan_execute(plan, 3, ref.data_ptr())
    torch.cuda.synchronize()
    for call in range(2):
        d = _device_counts(torch, circ.n, 5)
        tqs.tqs_simulate_static(c, nz, 32, 3, o, d.data_ptr())
        assert np.array_equal(d.cpu().numpy(), ref.cpu().numpy()), call


def test_static_refuses_the_learned_partitioner():
    """The learned partitioner's network runs through allocating kernels, so the
    allocation-free entry point refuses it before any device work."""
    torch = pytest.importorskip("torch")
    circ = qft(8)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    d = torch.zeros(1 << circ.n, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_simulate_static(c, nz, 100, 0, tqs.options(part="learned"), d.data_ptr())
    assert e.value.status == capi.TQS_EUNSUPPORTED
