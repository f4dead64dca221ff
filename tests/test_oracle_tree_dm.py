"""Pins of the oracle's tree Monte-Carlo (Sec. 3.1) and of its density-matrix
reference (Sec. 2.3.1): invariants of the tree, closed forms of the density
matrix, and Hoeffding-bounded agreement of both Monte-Carlo modes with it."""
import json
import math
import os

import numpy as np
import pytest

from tqs_inputs import Circuit, ghz, random_layers, qft

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _hoeffding(n_bins, samples, delta=1e-6):
    return math.sqrt(math.log(2 * n_bins / delta) / (2 * samples))


def small_noisy_circuit(n=4, seed=3):
    c = random_layers(n, 3, seed)
    c.add("cx", 0, n - 1).add("h", 1).add("cp", 1, 2, 0.7).add("swap", 0, 2).add("y", n - 1)
    return c


def test_paper_node_counts(orc):
    for key in ("baseline_tree_nodes", "dcp_tree_nodes"):
        g = GOLD[key]
        assert orc.partition.tree_node_count(g["arity"]) == g["nodes"]
        assert orc.partition.level_sizes(g["arity"])[-1] == g["outcomes"]


def test_density_matrix_pins(orc):
    c = small_noisy_circuit()
    rho0 = orc.density.final_density(c, 0.0, 0.0)
    psi = orc.core.ideal_state(c)
    assert np.allclose(np.real(np.diag(rho0)), np.abs(psi) ** 2, atol=1e-13)
    rho = orc.density.final_density(c, 0.05, 0.1)
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.allclose(rho, rho.conj().T, atol=1e-13)
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12
    # closed forms of the channels
    one = orc.density.outcome_distribution(Circuit(1).add("rz", 0, -1, 0.0), 0.3, 0.0, 0.0)
    assert abs(one[1] - 0.2) < 1e-14
    two = orc.density.outcome_distribution(Circuit(2).add("cz", 0, 1), 0.0, 0.45, 0.0)
    assert np.allclose(two, [1 - 0.45 + 0.09, 0.12, 0.12, 0.12], atol=1e-14)
    unif = ghz(3)
    for q in range(3):
        unif.add("rz", q, -1, 0.0)
    assert np.allclose(orc.density.outcome_distribution(unif, 0.75, 0.02, 0.0), 1 / 8, atol=1e-13)
    ro = orc.density.outcome_distribution(Circuit(2).add("x", 0), 0.0, 0.0, 0.1)
    assert np.allclose(ro, [0.09, 0.81, 0.01, 0.09], atol=1e-14)


@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (5, 3)])
def test_baseline_mc_matches_density_matrix(orc, n, seed):
    c = small_noisy_circuit(n, seed)
    p1, p2, pm, N = 0.04, 0.12, 0.03, 20000
    want = orc.density.outcome_distribution(c, p1, p2, pm)
    got = orc.core.run_baseline(c, p1, p2, pm, N, seed=seed) / N
    assert np.max(np.abs(got - want)) < _hoeffding(1 << n, N)


@pytest.mark.parametrize("arity", [[2500, 2, 2], [625, 4, 2, 2]])
def test_tree_mc_matches_density_matrix(orc, arity):
    """The A_0 top-level subtrees are i.i.d. and each leaf is marginally one
    baseline shot, so the leaf frequencies concentrate around the exact
    distribution with A_0 independent samples (Hoeffding on A_0)."""
    n = 4
    c = small_noisy_circuit(n, 9)
    p1, p2, pm = 0.04, 0.12, 0.03
    N = int(np.prod(arity))
    split = orc.partition.equal_splits(len(c.gates), len(arity))
    want = orc.density.outcome_distribution(c, p1, p2, pm)
    got = orc.core.run_tree(c, p1, p2, pm, N, 21, arity, split) / N
    assert np.max(np.abs(got - want)) < _hoeffding(1 << n, arity[0])


def test_degenerate_tree_equals_baseline_bitwise(orc):
    """Tree (N,1,...,1) reuses nothing: node id m at every level is shot m, so the
    counts equal the baseline's bit for bit."""
    c = random_layers(7, 5, 4)
    N = 700
    base = orc.core.run_baseline(c, 0.01, 0.05, 0.02, N, seed=5)
    G = len(c.gates)
    tree = orc.core.run_tree(c, 0.01, 0.05, 0.02, N, 5, [N, 1, 1, 1], [0, 3, 17, 40, G])
    assert np.array_equal(base, tree)


def test_zero_noise_leaves_equal_ideal(orc):
    c = qft(6)
    ideal = orc.core.ideal_state(c)
    arity, split = [4, 3, 2], [0, 5, 12, len(c.gates)]
    for m in (0, 7, 23):
        st = orc.core.node_state(c, 0.0, 0.0, 3, arity, split, 2, m)
        assert np.max(np.abs(st - ideal)) < 1e-13


def test_tree_reuse_equals_per_leaf_chains(orc):
    """The reusing recursion and an independent recomputation of every leaf along
    its ancestor chain give the same histogram (reuse is exact)."""
    c = small_noisy_circuit(5, 8)
    arity, split = [3, 4, 2], orc.partition.equal_splits(len(c.gates), 3)
    N = 21  # < 24 leaves: the trailing leaves are skipped
    p1, p2, pm = 0.05, 0.2, 0.05
    counts = orc.core.run_tree(c, p1, p2, pm, N, 17, arity, split)
    chain = np.zeros_like(counts)
    for leaf in range(N):
        chain[orc.core.leaf_outcome(c, p1, p2, pm, 17, arity, split, leaf)] += 1
    assert np.array_equal(counts, chain)
    assert counts.sum() == N


def test_thread_count_does_not_change_counts(orc):
    c = random_layers(8, 4, 6)
    arity, split = [50, 2, 2], orc.partition.equal_splits(len(c.gates), 3)
    a = orc.core.run_tree(c, 0.01, 0.05, 0.02, 200, 9, arity, split, threads=1)
    b = orc.core.run_tree(c, 0.01, 0.05, 0.02, 200, 9, arity, split, threads=4)
    assert np.array_equal(a, b)


def test_node_noise_matches_draws(orc):
    c = random_layers(5, 4, 2)
    split = [0, 10, len(c.gates)]
    nz = orc.core.node_noise(c, 0.3, 0.6, 8, split, 1, 5)
    for g in range(10, len(c.gates)):
        two = c.gates[g][0] in ("cz", "cx", "cp", "swap", "u2")
        want = orc.core.noise_draw(8, 5, g, 0.6 if two else 0.3, 15 if two else 3)
        assert nz[g - 10] == want
