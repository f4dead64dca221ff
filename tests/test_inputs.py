"""Shape of the synthetic workloads: gate counts of the QFT and random-layer
circuits and the determinism of the seeded generators."""
import os

from tqs_inputs import (batch_circuits_spec, qft, random_layers, read_text, write_text,
                        inverse_qft_on_fourier_state, qaoa_maxcut, qpe, random_regular_graph, splitmix64)


def test_qft_gate_counts():
    for n in (10, 16, 20, 26):
        c = qft(n)
        n1, n2 = c.counts()
        assert n1 == n and n2 == n * (n - 1) // 2 + n // 2
    assert len(qft(20)) == 220


def test_qpe_gate_counts():
    for m in (4, 8):
        c = qpe(m, 0.3)
        assert c.n == m + 1
        # X, m H, m controlled powers, m(m-1)/2 CP + m H (inverse QFT), m/2 SWAP
        assert len(c) == 1 + 3 * m + m * (m - 1) // 2 + m // 2
    assert len(qpe(8, 0.3)) == 57


def test_random_regular_graph_and_qaoa_counts():
    for n, d, seed in [(16, 3, 7), (10, 3, 5), (9, 4, 2)]:
        E = random_regular_graph(n, d, seed)
        assert E == random_regular_graph(n, d, seed)
        assert len(E) == n * d // 2 and len(set(E)) == len(E)
        assert all(0 <= u < v < n for u, v in E)
        deg = [0] * n
        for u, v in E:
            deg[u] += 1
            deg[v] += 1
        assert deg == [d] * n
    E = random_regular_graph(16, 3, 7)
    c = qaoa_maxcut(16, E, 0.4, 0.3)
    assert len(c) == 16 + 3 * len(E) + 16 and c.counts() == (16 + len(E) + 16, 2 * len(E))


def test_random_layer_counts_and_determinism():
    c = random_layers(16, 40, 16040)
    assert c.counts() == (640, 320)
    assert random_layers(16, 40, 16040).gates == c.gates
    assert random_layers(16, 40, 16041).gates != c.gates
    assert random_layers(26, 30, 26030).counts() == (780, 390)
    odd = random_layers(5, 2, 1)
    assert odd.counts() == (10, 4)
    for name, q0, q1, th, _ in c.gates:
        if name == "cz":
            assert q0 != q1
        else:
            assert name in ("rx", "ry", "rz") and 0.0 <= th < 6.2832


def test_batch_spec_ranges():
    spec = batch_circuits_spec()
    assert len(spec) == 64
    assert all(12 <= n <= 22 and 20 <= L <= 60 for n, L, _ in spec)
    assert spec == batch_circuits_spec()
    assert len({(n, L) for n, L, _ in spec}) > 30


def test_inverse_qft_counts():
    n1, n2 = inverse_qft_on_fourier_state(20, 5).counts()
    assert n1 == 60 and n2 == 200  # 20 H + 20 P (prep), 20 H; 190 CP + 10 SWAP


def test_text_round_trip(tmp_path):
    c = random_layers(6, 3, 9)
    c.add("u1", 2, -1, 0.0, [[0, 1], [1, 0]])
    p = os.path.join(tmp_path, "c.txt")
    write_text(c, p)
    d = read_text(p)
    assert d.n == c.n and len(d.gates) == len(c.gates)
    for a, b in zip(c.gates[:-1], d.gates[:-1]):
        assert a[:4] == b[:4]


def test_splitmix_below_range():
    r = splitmix64(3)
    vals = [r.below(7) for _ in range(5000)]
    assert min(vals) == 0 and max(vals) == 6
