"""Fused k-qubit gates on the tensor cores (TQS_FLAG_FUSE; FP32 states, 3xTF32
products on tcgen05 with FP32 accumulation in tensor memory): node amplitudes within 2e-5
of the FP64 oracle, both when the fused blocks run on the tensor cores (no noise
inside them) and when a noise site inside a block sends it down the per-gate path."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import random_layers

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile", [12, 11])
@pytest.mark.parametrize("p", [(0.0, 0.0), (0.02, 0.05)])
def test_fused_blocks_match_oracle(orc, tile, p):
    circ = random_layers(14, 6, 21)
    arity, split = [8, 2, 2], [0, 30, 70, len(circ.gates)]
    shots = 32
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(p[0], p[1], 0.0)
    o = tqs.options(arity=arity, split=split, prec="fp32", tile_qubits=tile, flags=capi.TQS_FLAG_FUSE)
    for level, node in [(0, 0), (0, 5), (1, 9), (2, 31)]:
        got = tqs.tqs_debug_node_state(c, nz, shots, 7, o, level, node, circ.n)
        want = orc.core.node_state(circ, p[0], p[1], 7, arity, split, level, node)
        err = np.max(np.abs(got - want))
        assert err < 2e-5, (level, node, err)
    _, _, rep = tqs.tqs_simulate(c, nz, shots, 7, tqs.options(arity=arity, split=split, prec="fp32",
                                                            tile_qubits=tile,
                                                            flags=capi.TQS_FLAG_NO_FIDELITY | capi.TQS_FLAG_FUSE),
                                 n=circ.n)
    assert sum(rep["fused_blocks"]) > 0  # the tensor-core blocks really ran


def test_fusion_only_when_asked_and_only_for_fp32():
    circ = random_layers(12, 6, 21)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 0.0)
    for prec, flags in (("fp64", capi.TQS_FLAG_FUSE), ("fp32", 0)):
        _, _, rep = tqs.tqs_simulate(c, nz, 64, 1, tqs.options(prec=prec, flags=capi.TQS_FLAG_NO_FIDELITY | flags),
                                     n=circ.n)
        assert sum(rep["fused_blocks"]) == 0


def test_autotune_with_fusion_candidates_gives_valid_counts():
    circ = random_layers(14, 8, 77)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    a, _, _ = tqs.tqs_simulate(c, nz, 4000, 4, tqs.options(prec="fp32", flags=capi.TQS_FLAG_AUTOTUNE), n=circ.n)
    b, _, _ = tqs.tqs_simulate(c, nz, 4000, 4, tqs.options(prec="fp64"), n=circ.n)
    assert int(a.sum()) == 4000
    assert np.abs(a.astype(np.int64) - b.astype(np.int64)).sum() <= 8


def test_fused_counts_close_to_fp64():
    circ = random_layers(13, 10, 5)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    a, _, ra = tqs.tqs_simulate(c, nz, 4000, 2, tqs.options(prec="fp32", tile_qubits=12, flags=capi.TQS_FLAG_FUSE),
                                n=circ.n)
    assert sum(ra["fused_blocks"]) > 0
    b, _, _ = tqs.tqs_simulate(c, nz, 4000, 2, tqs.options(prec="fp64"), n=circ.n)
    assert int(a.sum()) == 4000
    assert np.abs(a.astype(np.int64) - b.astype(np.int64)).sum() <= 8
