"""The learned partitioner's GPU kernels against the FP64 oracle network, its
training, and its use inside the partition step with DCP as fallback and arbiter."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from oracle import mlp
from tqs_inputs import qft, random_layers

pytestmark = pytest.mark.gpu


def test_param_count_matches_oracle():
    assert tqs.tqs_learned_param_count() == mlp.param_count()


@pytest.mark.parametrize("rows", [1, 37, 256])
def test_loss_and_gradient_match_oracle(rows):
    rng = np.random.default_rng(rows)
    w = mlp.he_init(rows).astype(np.float32)
    w[-mlp.C:] = rng.normal(size=mlp.C) * 0.1
    X = rng.normal(size=(rows, mlp.F)).astype(np.float32)
    y = rng.integers(0, mlp.C, size=rows).astype(np.int32)
    loss, g = tqs.tqs_learned_loss_grad(w, X, y)
    L, G = mlp.loss_grad(w.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    rel = np.linalg.norm(g - G) / np.linalg.norm(G)
    assert rel <= 1e-4, rel


def test_forward_matches_oracle():
    rng = np.random.default_rng(3)
    w = mlp.he_init(9).astype(np.float32)
    X = rng.normal(size=(50, mlp.F)).astype(np.float32)
    got = tqs.tqs_learned_predict(w, X)
    _, _, Z = mlp.forward(w.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(got - Z)) <= 1e-4 * max(1.0, np.max(np.abs(Z)))


def test_training_fits_separable_labels():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(2048, mlp.F)).astype(np.float32)
    P = rng.normal(size=(mlp.F, mlp.C))
    y = np.argmax(X @ P, axis=1).astype(np.int32)
    w, loss = tqs.tqs_learned_train(X, y, epochs=40, batch=128, lr=3e-3, seed=1)
    L0 = mlp.loss(mlp.he_init(0), X, y)
    assert loss < 0.5 * L0
    acc = np.mean(np.argmax(tqs.tqs_learned_predict(w, X), axis=1) == y)
    assert acc > 0.8, acc
    # the trained weights give the oracle the same loss
    assert abs(mlp.loss(w.astype(np.float64), X, y) - loss) < 1e-3


def test_learned_partition_uses_model_and_respects_dcp():
    circ = random_layers(14, 20, 3)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    shots = 8192
    with pytest.raises(capi.TqsError) as e:
        tqs.tqs_partition(c, nz, shots, tqs.options(part="learned"))
    assert e.value.status == capi.TQS_EUNSUPPORTED
    feat, allowed = tqs.tqs_learned_features(c, nz, shots)
    dcp_arity, _ = tqs.tqs_partition(c, nz, shots, tqs.options())
    assert allowed.sum() >= 1
    # a model that prefers class `pick` (bias only) must produce exactly that candidate
    pick = int(np.nonzero(allowed)[0][-1])
    w = np.zeros(tqs.tqs_learned_param_count(), dtype=np.float32)
    w[-mlp.C + pick] = 5.0
    tqs.tqs_learned_set_model(w)
    try:
        arity, split = tqs.tqs_partition(c, nz, shots, tqs.options(part="learned"))
        assert (arity, split) == tuple(tqs.tqs_learned_candidate(c, nz, shots, None, pick))
        assert arity[0] >= dcp_arity[0] and len(arity) <= len(dcp_arity)
        # a model preferring a class DCP forbids falls back to the best allowed one
        bad = [k for k in range(mlp.C) if not allowed[k]]
        if bad:
            w2 = np.zeros_like(w)
            w2[-mlp.C + bad[0]] = 9.0
            tqs.tqs_learned_set_model(w2)
            a2, _ = tqs.tqs_partition(c, nz, shots, tqs.options(part="learned"))
            assert a2[0] >= dcp_arity[0]
        counts, _, _ = tqs.tqs_simulate(c, nz, shots, 5, tqs.options(part="learned"), n=circ.n)
        assert int(counts.sum()) == shots
    finally:
        tqs.tqs_learned_set_model(None)
