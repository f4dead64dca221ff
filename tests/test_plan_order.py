"""Host-side checks of the pass planner (no GPU): the order in which a plan
applies the gates (tqs_debug_plan_order) is a permutation of the circuit that
keeps every pair of gates sharing a qubit (with its noise site) in circuit order,
each pass's dense gates act inside its tile, and list scheduling never needs more
passes than cutting the circuit greedily in gate order."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from tqs_inputs import Circuit, ghz, qft, random_layers

TWO = ("cx", "cz", "cp", "swap", "u2")
DIAG = ("z", "s", "sdg", "t", "tdg", "rz", "p", "cz", "cp")


def physical(circ):
    """Per gate: (physical qubit mask of the gate and its noise site, dense qubit
    mask), with SWAPs as a relabelling applied before the SWAP's own noise site."""
    perm = list(range(circ.n))
    out = []
    for name, q0, q1, _, _ in circ.gates:
        if name == "swap":
            perm[q0], perm[q1] = perm[q1], perm[q0]
            out.append(((1 << perm[q0]) | (1 << perm[q1]), 0))
            continue
        m = (1 << perm[q0]) | ((1 << perm[q1]) if name in TWO else 0)
        dense = 0 if name in DIAG else m
        out.append((m, dense))
    return out


def greedy_pass_count(circ, split, t):
    """Passes when each level is cut in gate order at the first dense gate whose
    qubits no longer fit the tile (with the 4 lowest qubits held for coalescing)."""
    phys = physical(circ)
    low = (1 << min(circ.n, 4)) - 1
    cap = min(circ.n, t)
    total = 0
    for lv in range(len(split) - 1):
        g, g1 = split[lv], split[lv + 1]
        passes = 0
        while True:
            need = 0
            while g < g1 and bin(need | phys[g][1] | low).count("1") <= cap:
                need |= phys[g][1]
                g += 1
            passes += 1
            if g >= g1:
                break
        total += passes
    return total


def mixed(n, seed):
    c = random_layers(n, 3, seed)
    rng = np.random.default_rng(seed)
    c.add("swap", 0, n - 1).add("cx", n - 2, 1).add("h", 2).add("swap", 1, n - 3).add("cp", n - 1, 0, 0.4)
    c.gates.extend(random_layers(n, 2, seed + 1).gates)
    for _ in range(10):
        a, b = rng.choice(n, 2, replace=False)
        c.add("cx", int(a), int(b)).add("rx", int(a), -1, 0.3).add("cz", int(b), int(a))
    return c


CASES = [(lambda: qft(14), 8), (lambda: qft(20), 12), (lambda: random_layers(16, 12, 3), 12),
         (lambda: random_layers(13, 20, 5), 6), (lambda: mixed(12, 7), 9), (lambda: ghz(10), 6),
         (lambda: mixed(18, 2), 11)]


@pytest.mark.parametrize("make,t", CASES)
def test_plan_order_keeps_qubit_order_and_tiles(make, t):
    circ = make()
    G = len(circ.gates)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    o = tqs.options(tile_qubits=t)
    arity, split = tqs.tqs_partition(c, nz, 4096, o)
    order, pass_of, tiles = tqs.tqs_debug_plan_order(c, nz, 4096, o, G)
    assert sorted(order.tolist()) == list(range(G))
    pos = np.empty(G, dtype=np.int64)
    pos[order] = np.arange(G)
    phys = physical(circ)
    # levels stay in place: every gate of level i comes before every gate of level i+1
    for lv in range(len(split) - 1):
        assert sorted(order[split[lv]:split[lv + 1]].tolist()) == list(range(split[lv], split[lv + 1]))
    # gates sharing a physical qubit keep circuit order
    for a in range(G):
        for b in range(a + 1, min(G, a + 400)):
            if phys[a][0] & phys[b][0]:
                assert pos[a] < pos[b], (a, b)
    # dense gates act inside the tile of the pass that applies them; tiles have t qubits
    for i, g in enumerate(order):
        tile = int(tiles[pass_of[i]])
        assert phys[g][1] & ~tile == 0
        assert bin(tile).count("1") == min(circ.n, t)
    # passes are contiguous runs of the order and never more than a greedy cut
    assert np.all(np.diff(pass_of.astype(np.int64)) >= 0)
    assert len(tiles) <= greedy_pass_count(circ, split, t)


def test_list_scheduling_saves_passes_on_layered_circuits():
    circ = random_layers(16, 40, 16040)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    o = tqs.options(tile_qubits=12)
    arity, split = tqs.tqs_partition(c, nz, 8192, o)
    _, _, tiles = tqs.tqs_debug_plan_order(c, nz, 8192, o, len(circ.gates))
    greedy = greedy_pass_count(circ, split, 12)
    assert len(tiles) * 2 <= greedy, (len(tiles), greedy)


def test_diagonal_gates_sink_to_the_dense_gate_that_needs_them():
    """QFT: before each H only the controlled phases touching its qubit remain."""
    circ = qft(10)
    c, nz = tqs.circuit(circ), tqs.tqs_noise_model(0.0, 0.0, 0.0)
    o = tqs.options(arity=[1], split=[0, len(circ.gates)], tile_qubits=10)
    order, _, _ = tqs.tqs_debug_plan_order(c, nz, 1, o, len(circ.gates))
    names = [circ.gates[g][0] for g in order]
    qs = [(circ.gates[g][1], circ.gates[g][2]) for g in order]
    for i, nm in enumerate(names):
        if nm == "h" and i > 0 and names[i - 1] == "cp":
            assert circ.gates[order[i]][1] in qs[i - 1]  # the phase just before touches this H's qubit
