"""Damping channels on the GPU (Sec. 4.3: thermal relaxation, amplitude damping,
phase damping as quantum trajectories) against the oracle: FP64 histograms bit
for bit in baseline and tree mode on a 10-qubit circuit with all three
channels, FP32 node states within 2e-5, and the choices keyed by node so that a
node's subtree shares them."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qpe, random_layers

pytestmark = pytest.mark.gpu

P1, P2, PM = 1e-3, 1e-2, 2e-2
CH = dict(ad_gamma=0.01, pd_lambda=0.01, t1=50e-6, t2=70e-6, time_1q=0.5e-6, time_2q=2e-6)


def _noise():
    return tqs.tqs_noise_model_ex(P1, P2, PM, **CH)


def _kr(orc):
    return orc.core.kraus_params(ad=CH["ad_gamma"], pd=CH["pd_lambda"], t1=CH["t1"], t2=CH["t2"],
                                 time_1q=CH["time_1q"], time_2q=CH["time_2q"])


def _circuit():
    c = random_layers(10, 4, 77)
    c.add("h", 0).add("cx", 0, 9).add("cp", 3, 5, 0.4).add("swap", 2, 7).add("x", 4)
    return c


def test_kraus_baseline_fp64_counts_bit_exact(orc):
    circ = _circuit()
    c, nz = tqs.circuit(circ), _noise()
    got, _, rep = tqs.tqs_simulate(c, nz, 600, 3, tqs.options(mode="baseline", prec="fp64",
                                                               flags=capi.TQS_FLAG_NO_FIDELITY), n=circ.n)
    want = orc.core.run_baseline(circ, P1, P2, PM, 600, 3, kraus=_kr(orc))
    assert rep["passes"][0] == len(circ.gates) + 1  # every gate ends a pass
    assert np.array_equal(got, want)


def test_kraus_tree_fp64_counts_bit_exact(orc):
    circ = _circuit()
    G = len(circ.gates)
    arity, split = [40, 3, 5], [0, G // 3, 2 * G // 3, G]
    c, nz = tqs.circuit(circ), _noise()
    got, _, _ = tqs.tqs_simulate(c, nz, 600, 11, tqs.options(prec="fp64", arity=arity, split=split,
                                                              flags=capi.TQS_FLAG_NO_FIDELITY), n=circ.n)
    want = orc.core.run_tree(circ, P1, P2, PM, 600, 11, arity, split, kraus=_kr(orc))
    assert np.array_equal(got, want)


def test_kraus_dcp_tree_fp64_bit_exact_on_phase_estimation(orc):
    """The circuit family of the paper's noise-model study (phase estimation),
    partitioned by DCP with the damping rates in its error estimate."""
    circ = qpe(8, 0.3)
    c, nz = tqs.circuit(circ), _noise()
    arity, split = tqs.tqs_partition(c, nz, 1000, tqs.options())
    assert len(arity) > 1
    got, _, _ = tqs.tqs_simulate(c, nz, 1000, 5, tqs.options(prec="fp64", flags=capi.TQS_FLAG_NO_FIDELITY),
                                 n=circ.n)
    want = orc.core.run_tree(circ, P1, P2, PM, 1000, 5, arity, split, kraus=_kr(orc))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_kraus_node_states(orc, prec, tol):
    circ = _circuit()
    G = len(circ.gates)
    arity, split = [40, 3, 5], [0, G // 3, 2 * G // 3, G]
    c, nz = tqs.circuit(circ), _noise()
    o = tqs.options(prec=prec, arity=arity, split=split, tile_qubits=8)
    for level, node in [(0, 7), (1, 100), (2, 599)]:
        got = tqs.tqs_debug_node_state(c, nz, 600, 11, o, level, node, circ.n)
        want = orc.core.node_state(circ, P1, P2, 11, arity, split, level, node, kraus=_kr(orc))
        assert np.max(np.abs(got - want)) < tol, (level, node)


def test_kraus_fp32_histogram_close_to_fp64():
    circ = _circuit()
    c, nz = tqs.circuit(circ), _noise()
    a, _, _ = tqs.tqs_simulate(c, nz, 4000, 2, tqs.options(prec="fp32", flags=capi.TQS_FLAG_NO_FIDELITY), n=circ.n)
    b, _, _ = tqs.tqs_simulate(c, nz, 4000, 2, tqs.options(prec="fp64", flags=capi.TQS_FLAG_NO_FIDELITY), n=circ.n)
    assert int(a.sum()) == 4000
    assert np.abs(a.astype(np.int64) - b.astype(np.int64)).sum() <= 8
