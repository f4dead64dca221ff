"""Learned partitioner: simulator-generated training data, GPU training and
evaluation against DCP (argument marshalling around the C ABI).

Data: for each random layered circuit the simulator times every candidate tree
that DCP allows (tqs_learned_features' `allowed` mask) on a few whole level-0
subtrees, and the label is the fastest.  Training runs the library's own GPU
kernels (tqs_learned_train).  At run time TQS_PART_LEARNED consults the loaded
model and keeps DCP as the fallback and the arbiter.

    python -m paper_2203_13892_gb300.learned generate --count 5000 --out data.npz
    python -m paper_2203_13892_gb300.learned train --data data.npz --out model.npz
    python -m paper_2203_13892_gb300.learned evaluate --model model.npz --count 200
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import capi
from tqs_inputs import random_layers, splitmix64

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "learned_model.npz")
NOISE = (1e-3, 1e-2, 2e-2)


def training_circuit(i: int, base: int = 100000, n_range=(12, 22), layers=(20, 60)):
    r = splitmix64(base + i)
    n = n_range[0] + r.below(n_range[1] - n_range[0] + 1)
    L = layers[0] + r.below(layers[1] - layers[0] + 1)
    return random_layers(n, L, base + i)


_WS = {}


def _workspace(nbytes=4 << 30):
    """One device workspace (and histogram) reused by every trial run."""
    import torch

    if "ws" not in _WS:
        _WS["ws"] = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        _WS["counts"] = torch.zeros(1 << 24, dtype=torch.int64, device="cuda")
    return _WS["ws"], _WS["counts"]


def trial_leaves_for(n: int) -> int:
    """Leaves timed per candidate: about 2^26 amplitude-leaves of work at any n."""
    return int(min(4096, max(64, 1 << max(0, 26 - n))))


def time_tree(c, nz, shots, arity, split, prec="fp32", trial_leaves=4096, reps=1, warmup=0):
    """ms per leaf of `arity`/`split` measured on whole level-0 subtrees."""
    below = int(np.prod(arity[1:])) if len(arity) > 1 else 1
    roots = max(1, min(-(-shots // below), max(1, trial_leaves // below)))
    leaves = min(shots, roots * below)
    ws, d = _workspace()
    o = capi.options(arity=arity, split=split, prec=prec, flags=capi.TQS_FLAG_NO_FIDELITY,
                     workspace=ws.data_ptr(), workspace_bytes=ws.numel())
    plan = capi.tqs_plan_create(c, nz, leaves, o)
    best = float("inf")
    for r in range(warmup + reps):
        rep = capi.tqs_plan_execute(plan, r, d.data_ptr(), report=True)
        if r >= warmup:
            best = min(best, rep["kernel_ms"] / leaves)
    plan.close()
    return best


def label_circuit(circ, shots, prec="fp32"):
    c = capi.circuit(circ)
    nz = capi.tqs_noise_model(*NOISE)
    o = capi.options(prec=prec)
    feat, allowed = capi.tqs_learned_features(c, nz, shots, o)
    times = np.full(capi.TQS_LEARNED_CLASSES, np.inf)
    for cls in np.nonzero(allowed)[0]:
        arity, split = capi.tqs_learned_candidate(c, nz, shots, o, int(cls))
        times[cls] = time_tree(c, nz, shots, arity, split, prec, trial_leaves_for(circ.n))
    return feat, allowed, times


def generate(count, out, shots=8192, base=100000, n_range=(12, 22), layers=(20, 60), log_every=100):
    X = np.zeros((count, capi.TQS_LEARNED_FEATURES), dtype=np.float32)
    A = np.zeros((count, capi.TQS_LEARNED_CLASSES), dtype=np.uint8)
    T = np.zeros((count, capi.TQS_LEARNED_CLASSES), dtype=np.float32)
    t0 = time.time()
    for i in range(count):
        X[i], A[i], T[i] = label_circuit(training_circuit(i, base, n_range, layers), shots)
        if log_every and (i + 1) % log_every == 0:
            print(f"{i + 1}/{count} circuits labelled in {time.time() - t0:.0f} s", file=sys.stderr, flush=True)
    y = np.argmin(T, axis=1).astype(np.int32)
    np.savez_compressed(out, X=X, allowed=A, times=T, y=y, shots=shots, base=base)
    return X, A, T, y


def train(X, y, epochs=300, batch=256, lr=2e-3, seed=7):
    return capi.tqs_learned_train(X, y, epochs, batch, lr, seed)


def predict_classes(w, X, allowed):
    logits = capi.tqs_learned_predict(w, X)
    logits = np.where(allowed.astype(bool), logits, -np.inf)
    return np.argmax(logits, axis=1)


def load_model(path=MODEL_PATH):
    return np.load(path)["w"].astype(np.float32)


def evaluate(w, count=200, shots=8192, base=200000, n_range=(20, 24), layers=(20, 60), prec="fp32",
             full_runs=True):
    """Held-out comparison with DCP: shots/s of both trees and the normalised
    fidelity difference between their histograms (inverse-free random circuits
    have a non-uniform ideal distribution)."""
    capi.tqs_learned_set_model(w)
    rows = []
    for i in range(count):
        circ = training_circuit(i, base, n_range, layers)
        c = capi.circuit(circ)
        nz = capi.tqs_noise_model(*NOISE)
        res = {}
        for part in ("dcp", "learned"):
            o = capi.options(prec=prec, part=part)
            arity, split = capi.tqs_partition(c, nz, shots, o)
            if full_runs:
                counts, F, rep = capi.tqs_simulate(c, nz, shots, 11, o, n=circ.n)
                res[part] = {"tree": arity, "split": split, "shots_per_s": rep["shots_per_s"], "F": F}
            else:
                ms = time_tree(c, nz, shots, arity, split, prec, trial_leaves_for(circ.n), reps=2, warmup=1)
                res[part] = {"tree": arity, "split": split, "shots_per_s": 1e3 / ms}
        rows.append({"n": circ.n, "gates": len(circ.gates), **res})
    capi.tqs_learned_set_model(None)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("generate")
    g.add_argument("--count", type=int, default=5000)
    g.add_argument("--shots", type=int, default=8192)
    g.add_argument("--out", required=True)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", default=MODEL_PATH)
    t.add_argument("--epochs", type=int, default=300)
    e = sub.add_parser("evaluate")
    e.add_argument("--model", default=MODEL_PATH)
    e.add_argument("--count", type=int, default=200)
    e.add_argument("--shots", type=int, default=8192)
    e.add_argument("--out", default=None)
    e.add_argument("--trial", action="store_true", help="time trial subtrees instead of full runs")
    a = ap.parse_args(argv)
    if a.cmd == "generate":
        generate(a.count, a.out, a.shots)
    elif a.cmd == "train":
        d = np.load(a.data)
        w, loss = train(d["X"], d["y"], epochs=a.epochs)
        pred = predict_classes(w, d["X"], d["allowed"])
        acc = float(np.mean(pred == d["y"]))
        T = d["times"]
        regret = float(np.mean(T[np.arange(len(pred)), pred] / T[np.arange(len(pred)), d["y"]]))
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        np.savez_compressed(a.out, w=w, loss=loss, train_acc=acc, train_time_ratio=regret)
        print(json.dumps({"loss": loss, "train_acc": acc, "time_ratio_vs_best": regret}))
    else:
        rows = evaluate(load_model(a.model), a.count, a.shots, full_runs=not a.trial)
        ratio = [r["learned"]["shots_per_s"] / r["dcp"]["shots_per_s"] for r in rows]
        dF = [abs(r["learned"].get("F", np.nan) - r["dcp"].get("F", np.nan)) for r in rows]
        summary = {"circuits": len(rows), "speed_ratio_mean": float(np.mean(ratio)),
                   "speed_ratio_min": float(np.min(ratio)), "speed_ratio_max": float(np.max(ratio)),
                   "fid_diff_mean": float(np.nanmean(dF)) if rows and "F" in rows[0]["dcp"] else None,
                   "fid_diff_max": float(np.nanmax(dF)) if rows and "F" in rows[0]["dcp"] else None}
        print(json.dumps(summary))
        if a.out:
            with open(a.out, "w") as f:
                json.dump({"summary": summary, "rows": rows}, f)


if __name__ == "__main__":
    main()
