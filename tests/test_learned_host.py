"""Host-only parts of the learned partitioner, on CPU: the feature vector, the
mask of candidate trees DCP allows, and the candidate trees themselves.  Every
allowed candidate keeps DCP's sample-size guarantee (a first-level arity A_0 at
least DCP's, no more levels than DCP) and is a valid tree for the shot count
(product of arities >= shots, cuts non-decreasing from 0 to the gate count)."""
import math

import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import qft, random_layers

P = (1e-3, 1e-2, 2e-2)
CASES = [(lambda: random_layers(14, 20, 3), 8192), (lambda: random_layers(20, 40, 11), 8192),
         (lambda: qft(16), 8192), (lambda: random_layers(12, 60, 5), 2048)]


@pytest.mark.parametrize("make,shots", CASES)
def test_features_and_allowed_candidates_respect_dcp(make, shots):
    circ = make()
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    feat, allowed = tqs.tqs_learned_features(c, nz, shots)
    assert feat.shape == (capi.TQS_LEARNED_FEATURES,) and np.all(np.isfinite(feat))
    assert set(np.unique(allowed)) <= {0, 1} and allowed.sum() >= 1
    dcp_arity, dcp_split = tqs.tqs_partition(c, nz, shots, tqs.options())
    G = len(circ.gates)
    for cls in np.nonzero(allowed)[0]:
        arity, split = tqs.tqs_learned_candidate(c, nz, shots, None, int(cls))
        assert arity[0] >= dcp_arity[0] and len(arity) <= len(dcp_arity), (cls, arity, dcp_arity)
        assert math.prod(arity) >= shots
        assert split[0] == 0 and split[-1] == G and all(a <= b for a, b in zip(split, split[1:]))
        assert len(split) == len(arity) + 1


def test_features_are_deterministic_and_shot_dependent():
    circ = random_layers(16, 30, 7)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    f1, a1 = tqs.tqs_learned_features(c, nz, 8192)
    f2, a2 = tqs.tqs_learned_features(c, nz, 8192)
    assert np.array_equal(f1, f2) and np.array_equal(a1, a2)
    f3, _ = tqs.tqs_learned_features(c, nz, 1024)
    assert not np.array_equal(f1, f3)


def test_learned_partition_without_model_is_unsupported():
    circ = random_layers(12, 10, 1)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    tqs.tqs_learned_set_model(None)
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_partition(c, nz, 4096, tqs.options(part="learned"))
    assert e.value.status == capi.TQS_EUNSUPPORTED


def test_invalid_candidate_class_is_rejected():
    circ = random_layers(12, 10, 1)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(*P)
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_learned_candidate(c, nz, 4096, None, capi.TQS_LEARNED_CLASSES)
    assert e.value.status == capi.TQS_EINVAL
