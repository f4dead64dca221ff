"""State fidelity F_s and normalised fidelity F of output distributions (Sec. 4.1).

TEST INFRASTRUCTURE ONLY.

F_s(P, Q) = (sum_x sqrt(P(x) Q(x)))^2   (Eq. fidelity)
F(P, Q)   = (F_s(P, Q) - F_s(P, U)) / (1 - F_s(P, U)),  U uniform   (Eq. norm-fidelity)
When the ideal distribution P is itself uniform the normalised fidelity is 0/0;
it is returned as NaN.
"""
from __future__ import annotations

import math

import numpy as np


def state_fidelity(p, q) -> float:
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    s = 0.0
    for a, b in zip(p.tolist(), q.tolist()):
        s += math.sqrt(a * b)
    return s * s


def normalized_fidelity(p_ideal, q_out) -> float:
    p = np.asarray(p_ideal, dtype=np.float64)
    u = np.full(p.shape, 1.0 / p.size)
    fu = state_fidelity(p, u)
    den = 1.0 - fu
    if abs(den) < 1e-12:
        return float("nan")
    return (state_fidelity(p, q_out) - fu) / den


def counts_to_distribution(counts) -> np.ndarray:
    c = np.asarray(counts, dtype=np.float64)
    return c / c.sum()
