"""Tree arithmetic and circuit partitioners, written step by step from Sec. 3.1-3.2 and 3.6.

TEST INFRASTRUCTURE ONLY.

Readings taken where the paper is silent or inconsistent (each is pinned by a
printed value in the tests):
  * Eq. (circuit-instances) is read as M_i = prod_{j<=i} A_j instances of
    subcircuit i: this is what reproduces the printed node counts 193 for the
    baseline tree (64,1,1) and 113 for (16,2,2) (Sec. 3, Fig. 5 and Fig. 6).
  * z = 1.96, eps = 0.05 (the paper gives neither); they reproduce (250,2,2)
    for QPE_9 at 1000 shots (Sec. 5.6) and A_0 = 500 with seven subcircuits
    for QFT_14 at 32,000 shots (Sec. 5.1).
  * the top-up of the uniform arities until the leaves reach the requested
    shot count (Sec. 3.2.4 adds shots one at a time from the first subcircuit
    on) is read as A_0 = ceil(N / A_r^k).
  * all k+1 subcircuits get an equal share of the gates (this matches the
    printed 3.53x theoretical speedup of QFT_14, Sec. 5.1).
  * the copy-cost limit bounds the subcircuit count: every subcircuit needs at
    least c gates, so at most floor(G / c) subcircuits (Sec. 3.6).
  * the iteration over k never raises k (it starts from the copy limit and
    stops at the first fixed point), so it always terminates.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def level_sizes(arity: Sequence[int]) -> List[int]:
    """M_i = prod_{j<=i} A_j for every level i."""
    out, m = [], 1
    for a in arity:
        m *= int(a)
        out.append(m)
    return out


def active_nodes(arity: Sequence[int], shots: int) -> List[int]:
    """Nodes simulated per level when only leaves m < shots are kept:
    ceil(shots / prod_{j>i} A_j)."""
    out = []
    for i in range(len(arity)):
        below = 1
        for a in arity[i + 1:]:
            below *= int(a)
        out.append(-(-int(shots) // below))
    return out


def tree_node_count(arity: Sequence[int]) -> int:
    """Nodes of the full simulation tree including the initial-state root."""
    return 1 + sum(level_sizes(arity))


def theoretical_speedup(arity: Sequence[int], shots: int) -> float:
    """Subcircuit executions of the baseline over those of the tree, for
    equal-length subcircuits: L * N / sum_i (active nodes of level i)."""
    L = len(arity)
    return L * shots / float(sum(active_nodes(arity, shots)))


def max_speedup_formula(k: int, shots: int) -> float:
    """Sec. 3.6: the speedup bound with k equal subcircuits, kN / ((k-1) + N)."""
    return k * shots / float((k - 1) + shots)


def equal_splits(G: int, L: int) -> List[int]:
    """Gate boundaries of L subcircuits of equal length: g_i = floor(i G / L)."""
    return [(i * G) // L for i in range(L + 1)]


def first_subcircuit_error(rates: Sequence[float], length: int) -> float:
    """Eq. (error_rate): 1 - prod_i (1 - e_i) over the first subcircuit."""
    prod = 1.0
    for e in rates[:length]:
        prod *= (1.0 - e)
    return 1.0 - prod


def min_first_arity(p_hat: float, shots: int, z: float, eps: float) -> int:
    """Eq. (sample_size_formula): the smallest integer A_0 with
    A_0 >= n0 / (1 + n0 / N), n0 = z^2 p(1-p) / eps^2 (at least 1)."""
    n0 = z * z * p_hat * (1.0 - p_hat) / (eps * eps)
    return max(1, math.ceil(n0 / (1.0 + n0 / shots)))


def _largest_base(k: int, a0: int, shots: int) -> int:
    """floor((N / a0)^(1/k)) computed exactly: the largest a with a^k * a0 <= N."""
    a = 1
    while (a + 1) ** k * a0 <= shots:
        a += 1
    return a


def dcp(rates: Sequence[float], shots: int, z: float = 1.96, eps: float = 0.05,
        copy_gates: int = 10) -> Tuple[List[int], List[int], dict]:
    """Dynamic Circuit Partition (Sec. 3.2).

    rates      -- per-gate error rate e_i (p1 for one-qubit, p2 for two-qubit gates)
    shots      -- N, the number of outcomes wanted
    copy_gates -- c, the state-copy cost in gates = the minimum subcircuit length
    Returns (arity, split, info)."""
    G = len(rates)
    N = int(shots)
    cap = max(0, G // max(1, int(copy_gates)) - 1)
    K = cap
    while True:
        first = -(-G // (K + 1)) if G else 0
        p_hat = first_subcircuit_error(rates, first)
        a0min = min_first_arity(p_hat, N, z, eps)
        k_shots = 0
        while (2 ** (k_shots + 1)) * a0min <= N:
            k_shots += 1
        K_next = min(k_shots, cap, K)
        if K_next == K:
            break
        K = K_next
    k = K
    info = {"p_hat": p_hat, "a0_min": a0min, "copy_limit": cap}
    if k == 0:
        return [N], [0, G], info
    a_r = _largest_base(k, a0min, N)
    a0 = -(-N // (a_r ** k))
    return [a0] + [a_r] * k, equal_splits(G, k + 1), info


def ucp(shots: int, levels: int, G: int) -> Tuple[List[int], List[int]]:
    """Uniform Circuit Partition: `levels` equal subcircuits, all arities equal to
    the smallest a with a^levels >= N (Sec. 3.2.1: (10,10,10) for 1000 shots)."""
    a = 1
    while a ** levels < shots:
        a += 1
    return [a] * levels, equal_splits(G, levels)


def xcp(shots: int, levels: int, G: int, ratio: int = 2) -> Tuple[List[int], List[int]]:
    """Exponential Circuit Partition: A_i = a * ratio^(levels-1-i) with the smallest
    integer a whose product reaches N ((20,10,5) for 1000 shots, Sec. 5.6)."""
    a = 1
    while True:
        ar = [a * ratio ** (levels - 1 - i) for i in range(levels)]
        prod = 1
        for x in ar:
            prod *= x
        if prod >= shots:
            return ar, equal_splits(G, levels)
        a += 1


def gate_rates(circuit, p1: float, p2: float, kraus=None) -> List[float]:
    """Per-gate error rate e_i for DCP: the depolarizing probability and, with
    damping channels (the oracle's channel array, core.kraus_params), the
    probability that any of them jumps, bounded by its rate on each of the
    gate's qubits."""
    two = {"cx", "cz", "cp", "swap", "u2"}
    out = []
    for g in circuit.gates:
        t = g[0] in two
        keep = 1.0 - (p2 if t else p1)
        if kraus is not None:
            rates = [kraus[4] if t else kraus[2], kraus[5] if t else kraus[3], kraus[0], kraus[1]]
            for _ in range(2 if t else 1):
                for r in rates:
                    keep *= 1.0 - r
        out.append(1.0 - keep)
    return out
