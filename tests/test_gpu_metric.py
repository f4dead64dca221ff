"""Parity at the size of the throughput workload, in the launch configuration
the benchmark times: the 20-qubit QFT (220 gates: 20 H, 190 CP, 10 SWAP) from
|0...0>, 32,000 shots, depolarizing p1 = 1e-3 / p2 = 1e-2 and readout pm = 2e-2,
DCP tree, run through the device-resident entry point (tqs_plan_create /
tqs_plan_execute) with a caller-owned workspace and stream.

The oracle cannot run all 32,000 shots in test time, so it checks outputs it
can compute one by one, plus properties that hold at any size:
  * sampled leaves: the oracle follows one leaf's chain of nodes (gates, noise
    draws, measurement and readout draws) to its outcome, and that outcome must
    be in the device histogram.  In FP64 every sampled outcome must be present;
    a wrong outcome would land on one of the ~31k occupied bins of 2^20 with
    probability ~3 %, so eight leaves leave a false pass at ~1e-12.  In FP32 a
    sample may move to the neighbouring outcome when rounding shifts a
    cumulative-probability boundary past it (the inverse-CDF rule of Sec. 2.4
    reads outcomes in ascending order), so the outcome or a neighbour must be
    present;
  * launch independence: the histogram does not depend on how many tree nodes
    share one launch (the library's choice, 256 here, against 64 and a ragged
    97);
  * sampled node states within 2e-5 of the FP64 oracle (FP32) and their noise
    assignments bit-exact."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from tqs_inputs import qft

pytestmark = pytest.mark.gpu

N, SHOTS = 20, 32000
P1, P2, PM = 1e-3, 1e-2, 2e-2
LEAVES = [0, 1, 63, 64, 12345, 20000, 31936, 31999]


@pytest.fixture(scope="module")
def workload():
    circ = qft(N)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(P1, P2, PM)
    arity, split = tqs.tqs_partition(c, nz, SHOTS, tqs.options())
    return circ, c, nz, arity, split


@pytest.fixture(scope="module")
def oracle_outcomes(orc, workload):
    """Outcomes of the sampled leaves by the oracle (one chain each, in threads:
    the oracle's C calls release the interpreter lock)."""
    circ, _, _, arity, split = workload
    with ThreadPoolExecutor(max_workers=len(LEAVES)) as ex:
        ys = list(ex.map(lambda m: orc.core.leaf_outcome(circ, P1, P2, PM, 5, arity, split, m), LEAVES))
    return dict(zip(LEAVES, ys))


def device_histogram(c, nz, seed, prec, batch):
    """One execution as the benchmark runs it: plan sized by the library, the
    workspace and the histogram in device memory owned by the caller."""
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    o = tqs.options(prec=prec, stream=stream.cuda_stream, batch=batch)
    probe = tqs.tqs_plan_create(c, nz, SHOTS, o)
    nbytes = tqs.tqs_plan_workspace_bytes(probe)
    probe.close()
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    o.workspace, o.workspace_bytes = ws.data_ptr(), nbytes
    plan = tqs.tqs_plan_create(c, nz, SHOTS, o)
    d = torch.zeros(1 << N, dtype=torch.int64, device="cuda")
    rep = tqs.tqs_plan_execute(plan, seed, d.data_ptr(), report=True)
    stream.synchronize()
    plan.close()
    return d.cpu().numpy().astype(np.uint64), rep


def test_metric_fp64_sampled_leaves_exact(workload, oracle_outcomes):
    circ, c, nz, arity, split = workload
    counts, rep = device_histogram(c, nz, 5, "fp64", 0)
    assert rep["arity"] == arity and int(counts.sum()) == SHOTS
    missing = {m: y for m, y in oracle_outcomes.items() if counts[y] == 0}
    assert not missing, f"oracle outcomes absent from the FP64 histogram: {missing}"


def test_metric_fp32_sampled_leaves_and_launch_independence(workload, oracle_outcomes):
    circ, c, nz, arity, split = workload
    counts, rep = device_histogram(c, nz, 5, "fp32", 0)
    assert rep["arity"] == arity and int(counts.sum()) == SHOTS
    for m, y in oracle_outcomes.items():
        near = counts[max(y - 1, 0):min(y + 2, 1 << N)]
        assert near.sum() > 0, (m, y)
    exact = sum(int(counts[y] > 0) for y in oracle_outcomes.values())
    assert exact >= len(LEAVES) - 1, exact
    for batch in (64, 97):
        other, rep_b = device_histogram(c, nz, 5, "fp32", batch)
        assert rep_b["arity"] == arity
        assert np.array_equal(other, counts), batch


def test_metric_fp32_node_states_and_noise(orc, workload):
    circ, c, nz, arity, split = workload
    o = tqs.options(prec="fp32")
    L = len(arity)
    for level, node in [(L - 1, 31999), (L // 2, 3999)]:
        got = tqs.tqs_debug_node_state(c, nz, SHOTS, 5, o, level, node, N)
        want = orc.core.node_state(circ, P1, P2, 5, arity, split, level, node)
        assert np.max(np.abs(got - want)) < 2e-5, (level, node)
        sites = split[level + 1] - split[level]
        nzg = tqs.tqs_debug_node_noise(c, nz, SHOTS, 5, o, level, node, sites)
        assert np.array_equal(nzg.astype(np.int64), orc.core.node_noise(circ, P1, P2, 5, split, level, node))
