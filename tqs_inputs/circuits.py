"""Circuit generators for the synthetic workloads (QFT, random layers, GHZ, QPE, QAOA).

The paper's 48 benchmark circuits are not available; these generators stand in
for the *shape* of its QFT and random-circuit (QV/QSC-like) classes
(Sec. 4.2, Table 2).  Everything here is deterministic in its arguments.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

Gate = Tuple[str, int, int, float, Optional[np.ndarray]]

ONE_QUBIT = ("h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "p", "u1")
TWO_QUBIT = ("cx", "cz", "cp", "swap", "u2")
_MASK64 = (1 << 64) - 1


@dataclass
class Circuit:
    n: int
    gates: List[Gate] = field(default_factory=list)
    name: str = ""

    def add(self, name: str, q0: int, q1: int = -1, theta: float = 0.0, mat=None) -> "Circuit":
        self.gates.append((name, int(q0), int(q1), float(theta), mat))
        return self

    def counts(self) -> Tuple[int, int]:
        """(#one-qubit gates, #two-qubit gates)."""
        n1 = sum(1 for g in self.gates if g[0] in ONE_QUBIT)
        return n1, len(self.gates) - n1

    def __len__(self) -> int:
        return len(self.gates)


class splitmix64:
    """SplitMix64 (Steele, Lea, Flood 2014): a 64-bit counter with a finaliser."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def below(self, k: int) -> int:
        """Uniform integer in [0, k) from the top 32 bits (multiply-shift)."""
        return ((self.next() >> 32) * k) >> 32

    def unit(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


def _qft_body(c: Circuit, n: int) -> None:
    # Textbook QFT in little-endian order: the most significant qubit first,
    # controlled phases pi/2^(j-k) from every lower qubit, then the bit reversal.
    for j in range(n - 1, -1, -1):
        c.add("h", j)
        for k in range(j - 1, -1, -1):
            c.add("cp", k, j, math.pi / (1 << (j - k)))
    for q in range(n // 2):
        c.add("swap", q, n - 1 - q)


def qft(n: int) -> Circuit:
    """n-qubit QFT on |0...0>: n H + n(n-1)/2 CP + floor(n/2) SWAP gates."""
    c = Circuit(n, name=f"qft{n}")
    _qft_body(c, n)
    return c


def qft_on_basis(n: int, x: int) -> Circuit:
    """X gates preparing |x>, then the QFT (output amplitudes 2^-n/2 e^{2 pi i x y / 2^n})."""
    c = Circuit(n, name=f"qft{n}_on_{x}")
    for q in range(n):
        if (x >> q) & 1:
            c.add("x", q)
    _qft_body(c, n)
    return c


def inverse_qft_on_fourier_state(n: int, b: int) -> Circuit:
    """Prepare QFT|b> qubit by qubit (H then a phase 2 pi b / 2^(n-q)), then run the
    inverse QFT; the ideal output is the basis state |b>, so the normalised
    fidelity is well defined (the plain QFT|0> output is uniform)."""
    c = Circuit(n, name=f"iqft{n}_fourier_{b}")
    for q in range(n):
        c.add("h", q)
        c.add("p", q, -1, 2.0 * math.pi * b / float(1 << (n - q)))
    for q in range(n // 2):
        c.add("swap", q, n - 1 - q)
    for j in range(n):
        for k in range(j):
            c.add("cp", k, j, -math.pi / (1 << (j - k)))
        c.add("h", j)
    return c


def qpe(m: int, phi: float) -> Circuit:
    """Textbook phase estimation with m counting qubits (0..m-1) and one target
    qubit m prepared in |1>, the eigenstate of the phase gate P(2 pi phi):
    X on the target, H on every counting qubit, a controlled P(2 pi phi)^(2^q)
    from counting qubit q (one CP of angle 2 pi phi 2^q), then the inverse QFT
    of the counting register (the same swaps and gate order as
    inverse_qft_on_fourier_state).  The counting register ends near
    |round(phi 2^m)>; for phi not a multiple of 2^-m its outcome distribution is
    a narrow peak of width ~1 around phi 2^m.  m = 8 gives a 9-qubit circuit of
    57 gates (8 + 1 one-qubit H/X, 8 CP for the controlled powers, 28 CP and 8 H
    for the inverse QFT, 4 SWAP)."""
    c = Circuit(m + 1, name=f"qpe{m + 1}")
    c.add("x", m)
    for q in range(m):
        c.add("h", q)
    for q in range(m):
        c.add("cp", q, m, math.remainder(2.0 * math.pi * phi * float(1 << q), 2.0 * math.pi))
    for q in range(m // 2):
        c.add("swap", q, m - 1 - q)
    for j in range(m):
        for k in range(j):
            c.add("cp", k, j, -math.pi / (1 << (j - k)))
        c.add("h", j)
    return c


def random_layers(n: int, layers: int, seed: int) -> Circuit:
    """Random layered circuit: per layer one rotation per qubit (axis uniform in
    {X,Y,Z}, angle uniform in [0, 2 pi)), then CZ on a uniformly random perfect
    matching (Fisher-Yates permutation paired consecutively; one qubit idles when
    n is odd).  Randomness: SplitMix64 seeded with ``seed``."""
    rng = splitmix64(seed)
    c = Circuit(n, name=f"rc{n}x{layers}_s{seed}")
    axes = ("rx", "ry", "rz")
    for _ in range(layers):
        for q in range(n):
            ax = axes[rng.below(3)]
            c.add(ax, q, -1, 2.0 * math.pi * rng.unit())
        perm = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.below(i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        for i in range(n // 2):
            c.add("cz", perm[2 * i], perm[2 * i + 1])
    return c


def random_regular_graph(n: int, d: int, seed: int) -> List[Tuple[int, int]]:
    """A random simple d-regular graph on n vertices (n*d even) by the pairing
    model: n*d half-edges are shuffled (Fisher-Yates, SplitMix64(seed)) and paired
    consecutively; a pairing with a loop or a repeated edge is drawn again.
    Edges as (u, v) with u < v, sorted."""
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    rng = splitmix64(seed)
    while True:
        stubs = [v for v in range(n) for _ in range(d)]
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            u, v = sorted((stubs[i], stubs[i + 1]))
            if u == v or (u, v) in edges:
                ok = False
                break
            edges.add((u, v))
        if ok:
            return sorted(edges)


def qaoa_maxcut(n: int, edges: List[Tuple[int, int]], gamma: float, beta: float) -> Circuit:
    """One QAOA layer for MaxCut (cost C = sum over edges of (1 - Z_u Z_v)/2):
    H on every qubit, then exp(-i gamma C) edge by edge as CX(u,v) RZ_v(-gamma)
    CX(u,v) (exp(+i gamma Z_u Z_v / 2), the global phase dropped), then the mixer
    exp(-i beta sum_q X_q) as RX(2 beta) on every qubit.  n + 3|E| + n gates."""
    c = Circuit(n, name=f"qaoa{n}_g{gamma:.4f}_b{beta:.4f}")
    for q in range(n):
        c.add("h", q)
    for u, v in edges:
        c.add("cx", u, v)
        c.add("rz", v, -1, -gamma)
        c.add("cx", u, v)
    for q in range(n):
        c.add("rx", q, -1, 2.0 * beta)
    return c


def ghz(n: int) -> Circuit:
    c = Circuit(n, name=f"ghz{n}")
    c.add("h", 0)
    for k in range(1, n):
        c.add("cx", 0, k)
    return c


def batch_circuits_spec(count: int = 64, base_seed: int = 1000) -> List[Tuple[int, int, int]]:
    """(n, layers, circuit_seed) for the uneven batch: circuit i draws
    n ~ U{12..22} and layers ~ U{20..60} from SplitMix64(base_seed + i) and uses
    circuit seed i for its gates."""
    out = []
    for i in range(count):
        r = splitmix64(base_seed + i)
        n = 12 + r.below(11)
        layers = 20 + r.below(41)
        out.append((n, layers, i))
    return out


def write_text(c: Circuit, path: str) -> None:
    """Plain text form: ``n <n>`` then one gate per line ``name q0 q1 theta [re im ...]``."""
    with open(path, "w") as f:
        f.write(f"n {c.n}\n")
        for name, q0, q1, th, mat in c.gates:
            extra = ""
            if mat is not None:
                m = np.asarray(mat, dtype=complex).ravel()
                extra = " " + " ".join(f"{float(v.real)!r} {float(v.imag)!r}" for v in m)
            f.write(f"{name} {q0} {q1} {th!r}{extra}\n")


def read_text(path: str) -> Circuit:
    with open(path) as f:
        head = f.readline().split()
        c = Circuit(int(head[1]))
        for line in f:
            p = line.split()
            if not p:
                continue
            mat = None
            if len(p) > 4:
                v = np.array([float(x) for x in p[4:]])
                z = v[0::2] + 1j * v[1::2]
                d = int(round(math.sqrt(len(z))))
                mat = z.reshape(d, d)
            c.add(p[0], int(p[1]), int(p[2]), float(p[3]), mat)
    return c
