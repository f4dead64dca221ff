"""Pins of the oracle's partitioners (Sec. 3.2, 3.6) against values printed in the
paper, and of the fidelity metric (Sec. 4.1) against closed forms."""
import json
import math
import os
import random

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def qpe9_like_rates():
    """Stand-in for QPE_9 (120 gates, circuit not available): a uniform per-gate
    error of 0.65% puts the first-third error rate at about 0.23."""
    return [0.0065] * 120


def qft14_like_rates():
    """Stand-in for the basis-decomposed QFT_14 (472 gates, about 40% CX): Sycamore
    rates (0.1% / 1.5%) with two two-qubit gates in every five."""
    g = GOLD["sycamore_rates"]
    return [g["p2"] if i % 5 in (1, 3) else g["p1"] for i in range(472)]


def test_dcp_reproduces_qpe9_tree(orc):
    g = GOLD["qpe9_dcp"]
    arity, split, info = orc.partition.dcp(qpe9_like_rates(), g["shots"])
    assert arity == g["arity"]
    assert split == [0, 40, 80, 120]
    assert 125 < info["a0_min"] <= 250


def test_dcp_reproduces_qft14_tree_and_speedup(orc):
    g = GOLD["qft14_dcp"]
    arity, split, info = orc.partition.dcp(qft14_like_rates(), g["shots"])
    assert len(arity) == g["subcircuits"]
    assert arity[0] == g["a0"] and all(a == 2 for a in arity[1:])
    sp = orc.partition.theoretical_speedup(arity, g["shots"])
    assert round(sp, 2) == g["theoretical_speedup"]
    assert sp > g["measured_speedup_cpu"]


def test_ucp_and_xcp_examples(orc):
    u = GOLD["ucp_example"]
    arity, split = orc.partition.ucp(u["shots"], u["levels"], 30)
    assert arity == u["arity"]
    assert orc.partition.level_sizes(arity) == u["instances"]
    x = GOLD["xcp_example"]
    assert orc.partition.xcp(x["shots"], x["levels"], 30)[0] == x["arity"]


@pytest.mark.parametrize("k,N", [(2, 1000), (3, 32000), (7, 8192)])
def test_max_speedup_formula_is_the_one_n_tree(orc, k, N):
    """Sec. 3.6: kN/((k-1)+N) is the speedup of the tree (1,...,1,N) with k equal subcircuits."""
    arity = [1] * (k - 1) + [N]
    assert math.isclose(orc.partition.theoretical_speedup(arity, N),
                        orc.partition.max_speedup_formula(k, N), rel_tol=1e-15)
    assert math.isclose(orc.partition.max_speedup_formula(2, N), 2 * N / (N + 1))


def test_dcp_invariants_random(orc):
    rnd = random.Random(0)
    for _ in range(300):
        G = rnd.randint(0, 600)
        N = rnd.randint(1, 100000)
        p1, p2 = rnd.choice([1e-4, 1e-3, 5e-3]), rnd.choice([1e-3, 1e-2, 3e-2])
        rates = [p2 if rnd.random() < 0.5 else p1 for _ in range(G)]
        c = rnd.choice([1, 5, 10, 30])
        arity, split, info = orc.partition.dcp(rates, N, copy_gates=c)
        assert int(np.prod(arity)) >= N
        assert split[0] == 0 and split[-1] == G and len(split) == len(arity) + 1
        assert all(b >= a for a, b in zip(split, split[1:]))
        if len(arity) > 1:
            assert all(a == arity[1] for a in arity[1:]) and arity[1] >= 2
            assert len(arity) <= max(1, G // c)
            # removing one from A_0 would drop below N leaves
            assert (arity[0] - 1) * int(np.prod(arity[1:])) < N


def test_fidelity_closed_forms(orc):
    F = orc.fidelity
    p = np.array([0.5, 0.3, 0.2, 0.0])
    u = np.full(4, 0.25)
    assert math.isclose(F.normalized_fidelity(p, p), 1.0, rel_tol=1e-14)
    assert abs(F.normalized_fidelity(p, u)) < 1e-14
    for q in (0.0, 0.3, 0.9):
        # P = delta_0, Q = (q, 1-q): F_s = q, F_s(P,U) = 1/2, so F = 2q - 1
        assert math.isclose(F.normalized_fidelity([1.0, 0.0], [q, 1 - q]), 2 * q - 1, abs_tol=1e-14)
    assert math.isnan(F.normalized_fidelity(u, p))
    assert math.isclose(F.state_fidelity([0.5, 0.5], [1.0, 0.0]), 0.5)
