"""The state pool in mapped host memory (TQS_FLAG_HOST_POOL, and the automatic
move of the upper levels there when one node per level does not fit in the
device budget): the pass kernels read parents from and write children to host
memory in place, so the histograms must be identical to those of the
device-resident pool, and FP64 counts identical to the oracle's."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

pytestmark = pytest.mark.gpu

P = (1e-3, 1e-2, 2e-2)


def _counts(c, nz, shots, seed, n, **opt):
    torch = pytest.importorskip("torch")
    plan = tqs.tqs_plan_create(c, nz, shots, tqs.options(**opt))
    d = torch.zeros(1 << n, dtype=torch.int64, device="cuda")
    tqs.tqs_plan_execute(plan, seed, d.data_ptr())
    torch.cuda.synchronize()
    host = tqs.tqs_plan_host_pool_bytes(plan)
    ws = tqs.tqs_plan_workspace_bytes(plan)
    plan.close()
    return d.cpu().numpy().astype(np.uint64), host, ws


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_pool_flag_matches_device_pool(orc, prec):
    circ = qft(12)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    want, host0, _ = _counts(c, nz, 2000, 4, circ.n, prec=prec)
    got, host1, _ = _counts(c, nz, 2000, 4, circ.n, prec=prec, flags=capi.TQS_FLAG_HOST_POOL)
    assert host0 == 0 and host1 > 0
    assert np.array_equal(got, want)
    if prec == "fp64":
        arity, split = tqs.tqs_partition(c, nz, 2000, tqs.options())
        assert np.array_equal(got, orc.core.run_tree(circ, *P, 2000, 4, arity, split))


def test_small_device_budget_moves_upper_levels_to_host():
    circ = random_layers(16, 12, 3)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    shots = 1024
    want, _, ws1 = _counts(c, nz, shots, 9, circ.n, prec="fp32", batch=1)
    state = 8 << circ.n
    # a cap two states short of one node per level on the device
    got, host, ws = _counts(c, nz, shots, 9, circ.n, prec="fp32", batch=1, workspace_bytes=ws1 - 2 * state)
    assert host >= 2 * state and ws <= ws1 - 2 * state
    assert np.array_equal(got, want)


def test_host_pool_debug_state_matches(orc):
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    arity, split = tqs.tqs_partition(c, nz, 500, tqs.options())
    o = tqs.options(prec="fp64", flags=capi.TQS_FLAG_HOST_POOL)
    level = len(arity) // 2
    got = tqs.tqs_debug_node_state(c, nz, 500, 2, o, level, 7, circ.n)
    want = orc.core.node_state(circ, *P[:2], 2, arity, split, level, 7)
    assert np.max(np.abs(got - want)) < 1e-12
