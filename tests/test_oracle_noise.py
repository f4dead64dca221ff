"""Pins of the oracle's random draws and noise channels.

The Philox stream is pinned word for word against an independent
implementation, PyTorch's ATen Philox4x32-10 engine (compiled here from its
header by `philox_ref_aten.cpp`), and statistically (uniformity, avalanche,
independence of the counter domains).  The channels are pinned by closed forms
of the depolarizing and readout channels (Sec. 4.3) on states where the outcome
distribution is known exactly."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import stats

from tqs_inputs import Circuit, ghz


def _words(orc, count, seed=12345, domain=7):
    out = np.zeros((count, 4), dtype=np.uint64)
    for i in range(count):
        out[i] = orc.core.philox([i & 0xFFFFFFFF, i >> 32, 3, domain], [seed & 0xFFFFFFFF, seed >> 32])
    return out


def _aten_philox(tmp_path, rows):
    """Philox4x32-10 outputs of PyTorch's ATen engine for rows of (c0..c3, k0, k1)."""
    import torch.utils.cpp_extension as ext

    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is needed to compile the ATen Philox reference")
    exe = str(tmp_path / "philox_ref_aten")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "philox_ref_aten.cpp")
    inc = []
    for d in ext.include_paths():
        inc += ["-I", d]
    subprocess.run([gxx, "-std=c++17", "-O1", *inc, src, "-o", exe], check=True, capture_output=True)
    text = "\n".join(" ".join(str(int(x)) for x in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    return np.array(out, dtype=np.uint64).reshape(-1, 4)


def test_philox_matches_aten_engine(orc, tmp_path):
    """Every output word of the oracle's Philox4x32-10 equals that of PyTorch's
    ATen engine, an implementation written independently of this one, on
    12,000 (counter, key) pairs: the all-zero and all-ones inputs, single set
    bits in every counter and key word, counter words next to their carry
    boundaries, the counter layouts of the noise, measurement and readout
    draws, and uniformly random inputs."""
    M = 0xFFFFFFFF
    rows = [[0] * 6, [M] * 6, [0, 0, 0, 0, M, M], [M, M, M, M, 0, 0]]
    for w in range(6):
        for b in range(32):
            r = [0] * 6
            r[w] = 1 << b
            rows.append(r)
            r2 = [M] * 6
            r2[w] ^= 1 << b
            rows.append(r2)
    for v in (M - 1, M, 0x7FFFFFFF, 0x80000000):
        rows.append([v, v, v, v, 7, 9])
    rng = np.random.default_rng(2203)
    for dom in (1, 2, 3):  # (node_lo, node_hi, site, domain) with 64-bit seeds
        for _ in range(500):
            node = int(rng.integers(0, 2**40))
            seed = int(rng.integers(0, 2**63))
            rows.append([node & M, node >> 32, int(rng.integers(0, 1200)), dom, seed & M, seed >> 32])
    while len(rows) < 12000:
        rows.append([int(x) for x in rng.integers(0, 2**32, 6, dtype=np.uint64)])
    want = _aten_philox(tmp_path, rows)
    got = np.array([orc.core.philox(r[:4], r[4:]) for r in rows], dtype=np.uint64)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, ("first mismatch", rows[bad[0]], got[bad[0]], want[bad[0]])


def test_philox_uniform_bytes(orc):
    w = _words(orc, 40000)
    for col in range(4):
        for shift in (0, 24):
            b = ((w[:, col] >> np.uint64(shift)) & np.uint64(0xFF)).astype(np.int64)
            chi2, p = stats.chisquare(np.bincount(b, minlength=256))
            assert p > 1e-6, (col, shift, p)


def test_philox_avalanche(orc):
    """Flipping any single input bit (128 counter + 64 key bits) flips about
    half of the 128 output bits; too few rounds or a broken S-box fails this."""
    rng = np.random.default_rng(5)
    trials = 60
    for pos in range(192):
        flips = []
        for _ in range(trials):
            ctr = [int(x) for x in rng.integers(0, 2**32, 4)]
            key = [int(x) for x in rng.integers(0, 2**32, 2)]
            a = orc.core.philox(ctr, key)
            c2, k2 = list(ctr), list(key)
            if pos < 128:
                c2[pos // 32] ^= 1 << (pos % 32)
            else:
                k2[(pos - 128) // 32] ^= 1 << (pos % 32)
            b = orc.core.philox(c2, k2)
            flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
        m = np.mean(flips)
        # mean of `trials` Binomial(128, 1/2): sd 5.66/sqrt(trials) ~ 0.73
        assert abs(m - 64.0) < 6.0, (pos, m)


def test_philox_domains_and_seeds_differ(orc):
    a = orc.core.philox([1, 0, 5, 1], [0, 0])
    b = orc.core.philox([1, 0, 5, 2], [0, 0])
    c = orc.core.philox([1, 0, 5, 1], [1, 0])
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("p,npaulis", [(0.01, 15), (0.2, 3)])
def test_error_frequency_binomial(orc, p, npaulis):
    n = 60000
    hits = sum(1 for s in range(n) if orc.core.noise_draw(3, s // 50, s % 50, p, npaulis))
    sd = math.sqrt(n * p * (1 - p))
    assert abs(hits - n * p) < 5 * sd


def test_error_extremes(orc):
    assert all(orc.core.noise_draw(1, m, 7, 0.0, 3) == 0 for m in range(2000))
    assert all(orc.core.noise_draw(1, m, 7, 1.0, 3) != 0 for m in range(2000))


@pytest.mark.parametrize("npaulis", [3, 15])
def test_pauli_index_uniform(orc, npaulis):
    vals = [orc.core.noise_draw(9, m, 2, 1.0, npaulis) for m in range(30000)]
    assert min(vals) == 1 and max(vals) == npaulis
    chi2, pv = stats.chisquare(np.bincount(vals, minlength=npaulis + 1)[1:])
    assert pv > 1e-6


def test_measure_u_uniform(orc):
    u = np.array([orc.core.measure_u(4, m) for m in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-6


def test_readout_mask_frequency(orc):
    n, pm, trials = 12, 0.02, 5000
    ones = sum(bin(orc.core.readout_mask(2, m, n, pm)).count("1") for m in range(trials))
    tot = n * trials
    assert abs(ones - tot * pm) < 5 * math.sqrt(tot * pm * (1 - pm))


def _hoeffding(n_bins, shots, delta=1e-6):
    return math.sqrt(math.log(2 * n_bins / delta) / (2 * shots))


def test_one_qubit_depolarizing_closed_form(orc):
    """|0> then an identity gate then the 1q channel: P(1) = 2p/3 (X and Y flip)."""
    p, N = 0.3, 20000
    c = Circuit(1).add("rz", 0, -1, 0.0)
    cnt = orc.core.run_baseline(c, p, 0.0, 0.0, N, seed=11)
    assert abs(cnt[1] / N - 2 * p / 3) < _hoeffding(2, N)


def test_two_qubit_depolarizing_closed_form(orc):
    """|00>, CZ (identity on |00>), 2q channel: of the 15 Paulis, 4 flip only q0,
    4 only q1, 4 both, 3 neither."""
    p, N = 0.45, 30000
    c = Circuit(2).add("cz", 0, 1)
    cnt = orc.core.run_baseline(c, 0.0, p, 0.0, N, seed=12) / N
    want = np.array([1 - p + 3 * p / 15, 4 * p / 15, 4 * p / 15, 4 * p / 15])
    assert np.max(np.abs(cnt - want)) < _hoeffding(4, N)


def test_readout_only_closed_form(orc):
    n, x, pm, N = 4, 0b1011, 0.1, 30000
    c = Circuit(n)
    for q in range(n):
        if (x >> q) & 1:
            c.add("x", q)
    cnt = orc.core.run_baseline(c, 0.0, 0.0, pm, N, seed=13) / N
    y = np.arange(1 << n)
    d = np.array([bin(int(v) ^ x).count("1") for v in y])
    want = pm ** d * (1 - pm) ** (n - d)
    assert np.max(np.abs(cnt - want)) < _hoeffding(1 << n, N)


def test_complete_depolarizer_gives_uniform(orc):
    """p1 = 3/4 is the completely depolarizing one-qubit channel; after a final
    identity gate on every qubit the output is exactly uniform."""
    n, N = 4, 40000
    c = ghz(n)
    for q in range(n):
        c.add("rz", q, -1, 0.0)
    cnt = orc.core.run_baseline(c, 0.75, 0.05, 0.0, N, seed=14) / N
    assert np.max(np.abs(cnt - 1.0 / (1 << n))) < _hoeffding(1 << n, N)


def test_zero_noise_deterministic_and_ghz(orc):
    c = Circuit(5).add("x", 1).add("x", 4)
    cnt = orc.core.run_baseline(c, 0.0, 0.0, 0.0, 500, seed=1)
    assert cnt[0b10010] == 500
    N = 4000
    cnt = orc.core.run_baseline(ghz(6), 0.0, 0.0, 0.0, N, seed=2)
    assert cnt[0] + cnt[63] == N
    assert abs(cnt[0] - N / 2) < 5 * math.sqrt(N / 4)
