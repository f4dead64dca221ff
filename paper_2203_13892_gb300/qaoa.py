"""Noisy QAOA cost landscape (Sec. 5.7): a grid search over the two angles of
one QAOA layer for MaxCut, every grid point a noisy simulation, run in tree
mode and in plain baseline mode, and the two landscapes compared.

The workload stands in for the paper's 16-qubit study (961 circuits, 0.1 %
depolarizing noise): a random 3-regular graph on 16 vertices (pairing model,
SplitMix64 seed 7; 24 edges), one layer H^16, exp(-i gamma C) as CX-RZ-CX per
edge and RX(2 beta) on every qubit (104 gates), on a 31 x 31 grid of
gamma in [0, pi] and beta in [0, pi/2], depolarizing p1 = p2 = 1e-3 after every
gate and no readout error, 2,048 shots per circuit.  Each row of the grid (31
circuits of one gamma) is one batch: its circuits are planned once, captured
into one CUDA graph and replayed once (tqs_batch_*); the device time of the
replays is what both modes are compared on.

The landscape value is the expected cut fraction <C>/|E| estimated from each
histogram.  Reported: device time of both modes, their ratio, the mean squared
difference between the two landscapes, and for scale the mean squared
difference that sampling alone gives two independent baseline estimates
(2 Var/shots, Var taken from each baseline histogram).

    python -m paper_2203_13892_gb300.qaoa [--grid 31] [--shots 2048] [--prec fp32] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import capi
from tqs_inputs import qaoa_maxcut, random_regular_graph

NOISE = (1e-3, 1e-3, 0.0)
N, DEG, GRAPH_SEED = 16, 3, 7


def graph():
    return random_regular_graph(N, DEG, GRAPH_SEED)


def angles(G):
    gammas = [math.pi * i / (G - 1) for i in range(G)]
    betas = [0.5 * math.pi * j / (G - 1) for j in range(G)]
    return gammas, betas


def cut_values(E, n=N):
    x = np.arange(1 << n, dtype=np.int64)
    cut = np.zeros(1 << n, dtype=np.float64)
    for u, v in E:
        cut += ((x >> u) & 1) != ((x >> v) & 1)
    return cut


def row_histograms(E, gamma, betas, shots, seeds, mode, prec):
    """Histograms of one grid row (one batch: one captured graph, replayed once)
    and the device time of that replay."""
    circs = [qaoa_maxcut(N, E, gamma, b) for b in betas]
    handles = [capi.circuit(c) for c in circs]
    noises = [capi.tqs_noise_model(*NOISE) for _ in circs]
    b = capi.tqs_batch_create(handles, noises, [shots] * len(circs), capi.options(mode=mode, prec=prec))
    rep = capi.tqs_batch_execute(b, seeds, report=True)
    hist = [capi.tqs_batch_counts(b, j, N) for j in range(len(circs))]
    b.close()
    return hist, rep["kernel_ms"], rep["kernel_launches"]


def landscape(mode, prec, G, shots, E, cut):
    gammas, betas = angles(G)
    L = np.zeros((G, G))
    var = np.zeros((G, G))
    ms = 0.0
    launches = 0
    for i, g in enumerate(gammas):
        seeds = [i * G + j for j in range(G)]
        hist, t, nl = row_histograms(E, g, betas, shots, seeds, mode, prec)
        ms += t
        launches += nl
        for j, h in enumerate(hist):
            p = h.astype(np.float64) / shots
            m = float(p @ cut) / len(E)
            L[i, j] = m
            var[i, j] = float(p @ (cut / len(E)) ** 2) - m * m
    return L, var, ms, launches


def run(G=31, shots=2048, prec="fp32"):
    E = graph()
    cut = cut_values(E)
    c0 = capi.circuit(qaoa_maxcut(N, E, 0.0, 0.0))
    tree, split = capi.tqs_partition(c0, capi.tqs_noise_model(*NOISE), shots, capi.options())
    Lt, _, ms_t, nl_t = landscape("tree", prec, G, shots, E, cut)
    Lb, var_b, ms_b, nl_b = landscape("baseline", prec, G, shots, E, cut)
    d = Lt - Lb
    return {
        "workload": f"QAOA p=1 MaxCut, random 3-regular graph on {N} vertices ({len(E)} edges), "
                    f"{G}x{G} grid, {shots} shots per circuit",
        "noise": {"p1": NOISE[0], "p2": NOISE[1], "pm": NOISE[2]}, "precision": prec,
        "circuits": G * G, "gates_per_circuit": 2 * N + 3 * len(E), "dcp_tree": tree, "dcp_split": split,
        "tree_ms": ms_t, "baseline_ms": ms_b, "tree_launches": nl_t, "baseline_launches": nl_b,
        "speedup": ms_b / ms_t,
        "mse_tree_vs_baseline": float(np.mean(d * d)), "max_abs_diff": float(np.max(np.abs(d))),
        "mse_two_independent_baselines": float(np.mean(2.0 * var_b / shots)),
        "landscape_tree": Lt.tolist(), "landscape_baseline": Lb.tolist(),
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=31)
    ap.add_argument("--shots", type=int, default=2048)
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = run(a.grid, a.shots, a.prec)
    print(json.dumps({k: v for k, v in res.items() if not k.startswith("landscape")}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
