"""Failure detection without a GPU fault.

A fused tensor-core block waits for its products on an mbarrier with an
iteration cap.  TQS_FLAG_FAULT_TIMEOUT makes the fused blocks issue no MMA and no
commit and wait with a short cap, so the wait gives up with nothing in flight:
the call must return TQS_ETIMEOUT and the next ordinary call in the same process
must give the same histogram as before.  TQS_FLAG_DEBUG_BOUNDS makes every
state-pass CTA check its indices before touching memory; TQS_FLAG_FAULT_BOUNDS
understates the output pool by one slot on the host, so the kernels' own check
must catch the last node of a full launch (no access is made out of range)."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

pytestmark = pytest.mark.gpu


def _fused_setup():
    circ = random_layers(14, 6, 21)
    arity, split = [8, 2, 2], [0, 30, 70, len(circ.gates)]
    return circ, tqs.circuit(circ), tqs.tqs_noise_model(0.0, 0.0, 0.0), arity, split


def test_fused_wait_timeout_returns_etimeout_and_library_recovers():
    circ, c, nz, arity, split = _fused_setup()
    base = capi.TQS_FLAG_NO_FIDELITY | capi.TQS_FLAG_FUSE

    def run(extra=0):
        return tqs.tqs_simulate(c, nz, 32, 7, tqs.options(arity=arity, split=split, prec="fp32", tile_qubits=12,
                                                          flags=base | extra), n=circ.n)

    want, _, rep = run()
    assert sum(rep["fused_blocks"]) > 0  # the fused path is what the fault exercises
    with pytest.raises(capi.TqsError) as e:
        run(capi.TQS_FLAG_FAULT_TIMEOUT)
    assert e.value.status == capi.TQS_ETIMEOUT
    got, _, _ = run()
    assert np.array_equal(got, want)
    got2, _, _ = run()
    assert np.array_equal(got2, want)


def test_debug_bounds_on_valid_input_changes_nothing():
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    for prec in ("fp64", "fp32"):
        a, _, _ = tqs.tqs_simulate(c, nz, 1000, 3, tqs.options(prec=prec, flags=capi.TQS_FLAG_NO_FIDELITY), n=circ.n)
        b, _, _ = tqs.tqs_simulate(c, nz, 1000, 3, tqs.options(prec=prec, flags=capi.TQS_FLAG_NO_FIDELITY |
                                                               capi.TQS_FLAG_DEBUG_BOUNDS), n=circ.n)
        assert np.array_equal(a, b), prec


def test_debug_bounds_catches_an_understated_pool_and_library_recovers():
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    flags = capi.TQS_FLAG_NO_FIDELITY | capi.TQS_FLAG_DEBUG_BOUNDS
    o = dict(prec="fp64", batch=4)
    want, _, _ = tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=flags, **o), n=circ.n)
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=flags | capi.TQS_FLAG_FAULT_BOUNDS, **o), n=circ.n)
    assert e.value.status == capi.TQS_EBOUNDS
    assert "output slot 3" in str(e.value)
    got, _, _ = tqs.tqs_simulate(c, nz, 256, 5, tqs.options(flags=flags, **o), n=circ.n)
    assert np.array_equal(got, want)
