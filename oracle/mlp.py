"""FP64 reference of the learned partitioner's network (numpy).

TEST INFRASTRUCTURE ONLY.  F -> 128 -> 128 -> C with ReLU hidden layers and
mean softmax cross-entropy; parameters in one flat vector laid out W1[F][H],
b1[H], W2[H][H], b2[H], W3[H][C], b3[C] (W[i][o] maps input i to output o).
The analytic gradient is pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

F, H, C = 40, 128, 20


def shapes(f=F, h=H, c=C):
    return [(f, h), (h,), (h, h), (h,), (h, c), (c,)]


def param_count(f=F, h=H, c=C) -> int:
    return int(sum(np.prod(s) for s in shapes(f, h, c)))


def unpack(w, f=F, h=H, c=C):
    w = np.asarray(w, dtype=np.float64)
    out, off = [], 0
    for s in shapes(f, h, c):
        n = int(np.prod(s))
        out.append(w[off:off + n].reshape(s))
        off += n
    return out


def forward(w, X, f=F, h=H, c=C):
    W1, b1, W2, b2, W3, b3 = unpack(w, f, h, c)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return H1, H2, H2 @ W3 + b3


def loss(w, X, y, f=F, h=H, c=C) -> float:
    _, _, Z = forward(w, X, f, h, c)
    m = Z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(Z - m).sum(axis=1)) + m[:, 0]
    return float(np.mean(lse - Z[np.arange(len(y)), y]))


def loss_grad(w, X, y, f=F, h=H, c=C):
    """Mean cross-entropy and its gradient by the chain rule, layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(w, f, h, c)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y)
    B = X.shape[0]
    H1, H2, Z = forward(w, X, f, h, c)
    m = Z.max(axis=1, keepdims=True)
    E = np.exp(Z - m)
    P = E / E.sum(axis=1, keepdims=True)
    L = float(np.mean(np.log(E.sum(axis=1)) + m[:, 0] - Z[np.arange(B), y]))
    dZ = P.copy()
    dZ[np.arange(B), y] -= 1.0
    dZ /= B
    gW3 = H2.T @ dZ
    gb3 = dZ.sum(axis=0)
    dH2 = (dZ @ W3.T) * (H2 > 0)
    gW2 = H1.T @ dH2
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0)
    gW1 = X.T @ dH1
    gb1 = dH1.sum(axis=0)
    return L, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def he_init(seed: int, f=F, h=H, c=C) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(f, h, c):
        if len(s) == 2:
            parts.append(rng.normal(size=s).ravel() * np.sqrt(2.0 / s[0]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)
