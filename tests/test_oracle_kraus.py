"""Pins of the oracle's non-unitary channels (Sec. 4.3: thermal relaxation,
amplitude damping and phase damping as Kraus operators, run by quantum
trajectories): closed forms of the channels in the density-matrix oracle,
the thermal-relaxation decay times, frequencies of the trajectory choices, and
Hoeffding-bounded agreement of the trajectory histograms (baseline and tree
mode) with the density matrix."""
import math

import numpy as np
import pytest

from tqs_inputs import Circuit, random_layers


def _hoeffding(n_bins, samples, delta=1e-6):
    return math.sqrt(math.log(2 * n_bins / delta) / (2 * samples))


def _idle(c, q, k):
    for _ in range(k):
        c.add("rz", q, -1, 0.0)  # an identity gate: only its noise sites act
    return c


def test_amplitude_damping_population_decay(orc):
    """|1> under k+1 amplitude-damping sites keeps P(1) = (1-gamma)^(k+1)."""
    g = 0.07
    for k in (0, 3, 9):
        c = _idle(Circuit(1).add("x", 0), 0, k)
        p = orc.density.outcome_distribution(c, 0.0, 0.0, 0.0, orc.core.kraus_params(ad=g))
        assert abs(p[1] - (1 - g) ** (k + 1)) < 1e-13, k


def test_phase_damping_coherence_decay(orc):
    """H, m idle gates, H: the coherence between the two H gates decays by
    sqrt(1-lambda) per site (the first H's site and the m idle ones), so
    P(0) = (1 + (1-lambda)^((m+1)/2)) / 2; populations never change."""
    lam = 0.11
    for m in (0, 2, 5):
        c = _idle(Circuit(1).add("h", 0), 0, m).add("h", 0)
        p = orc.density.outcome_distribution(c, 0.0, 0.0, 0.0, orc.core.kraus_params(pd=lam))
        assert abs(p[0] - 0.5 * (1 + (1 - lam) ** ((m + 1) / 2))) < 1e-13, m
    c = _idle(Circuit(1).add("h", 0), 0, 4)
    p = orc.density.outcome_distribution(c, 0.0, 0.0, 0.0, orc.core.kraus_params(pd=lam))
    assert np.allclose(p, 0.5, atol=1e-14)


def test_thermal_relaxation_times(orc):
    """Thermal relaxation over gates of duration t: the excited population decays
    as exp(-t/T1) per gate and the coherence as exp(-t/T2), both read off the
    density matrix built from the Kraus operators."""
    t1, t2, t = 50e-6, 70e-6, 2e-6
    kr = orc.core.kraus_params(t1=t1, t2=t2, time_1q=t, time_2q=3 * t)
    for k in (1, 4):
        c = _idle(Circuit(1).add("x", 0), 0, k - 1)
        rho = orc.density.final_density(c, 0.0, 0.0, kr)
        assert abs(rho[1, 1].real - math.exp(-k * t / t1)) < 1e-12
        c = _idle(Circuit(1).add("h", 0), 0, k - 1)
        rho = orc.density.final_density(c, 0.0, 0.0, kr)
        assert abs(abs(rho[0, 1]) - 0.5 * math.exp(-k * t / t2)) < 1e-12
    # a two-qubit gate relaxes both qubits over the longer duration
    c = Circuit(2).add("x", 0).add("x", 1).add("cz", 0, 1)
    rho = orc.density.final_density(c, 0.0, 0.0, kr)
    assert abs(rho[3, 3].real - math.exp(-(t + 3 * t) / t1) ** 2) < 1e-12
    # T2 = 2 T1 is pure damping; T2 > 2 T1 is unphysical
    g, l = orc.core.thermal_params(t1, 2 * t1, t)
    assert abs(g - (1 - math.exp(-t / t1))) < 1e-15 and l == 0.0
    with pytest.raises(ValueError):
        orc.core.thermal_params(t1, 2.5 * t1, t)


def test_zero_rates_change_nothing(orc):
    c = random_layers(5, 4, 8)
    a = orc.core.run_baseline(c, 1e-2, 3e-2, 1e-2, 2000, 4)
    b = orc.core.run_baseline(c, 1e-2, 3e-2, 1e-2, 2000, 4, kraus=np.zeros(6))
    assert np.array_equal(a, b)


def test_damping_jump_frequency(orc):
    """One amplitude-damping site on |1>: a fraction gamma of the trajectories
    decays to |0> (binomial, 6 sigma)."""
    g, N = 0.3, 20000
    c = Circuit(1).add("x", 0)
    counts = orc.core.run_baseline(c, 0.0, 0.0, 0.0, N, 9, kraus=orc.core.kraus_params(ad=g))
    assert abs(counts[0] / N - g) < 6 * math.sqrt(g * (1 - g) / N)


def _kraus_circuit(n, seed):
    c = random_layers(n, 3, seed)
    c.add("cx", 0, n - 1).add("h", 1).add("cp", 1, 2, 0.7).add("x", n - 1).add("h", 0)
    return c


@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (5, 3)])
def test_trajectories_match_density_matrix(orc, n, seed):
    """Every channel at once (depolarizing, thermal relaxation, amplitude and
    phase damping, readout): the baseline trajectory histogram and a tree-mode
    histogram are within the Hoeffding bound of the exact distribution (for the
    tree, on its A_0 independent top-level subtrees)."""
    c = _kraus_circuit(n, seed)
    kr = orc.core.kraus_params(ad=0.05, pd=0.08, t1=40e-6, t2=50e-6, time_1q=1e-6, time_2q=4e-6)
    p1, p2, pm = 0.02, 0.05, 0.02
    want = orc.density.outcome_distribution(c, p1, p2, pm, kr)
    assert abs(want.sum() - 1) < 1e-12
    N = 20000
    got = orc.core.run_baseline(c, p1, p2, pm, N, seed, kraus=kr) / N
    assert np.max(np.abs(got - want)) < _hoeffding(1 << n, N)
    G = len(c.gates)
    arity, split = [2000, 2, 5], [0, G // 3, 2 * G // 3, G]
    got_t = orc.core.run_tree(c, p1, p2, pm, N, seed, arity, split, kraus=kr) / N
    assert np.max(np.abs(got_t - want)) < _hoeffding(1 << n, arity[0])
