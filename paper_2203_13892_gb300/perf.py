"""Throughput of the library on the benchmark configurations other than the
headline one (which bench.py measures): one JSON line per configuration.

    python -m paper_2203_13892_gb300.perf [--config NAME ...] [--reps K]

  qft16 / rc16   16-qubit QFT and random 16x40 circuit, 8,192 shots, tree FP32
                 (DCP) with the specialised and with the generic pass kernels,
                 beside plain baseline mode in FP64 on the same GPU
  batch64        64 random circuits, 12-22 qubits, 20-60 layers, 2,048 shots
                 each, one captured CUDA graph replayed (FP32, DCP trees),
                 optionally autotuned (--autotune)
  qft26 / rc26   26-qubit QFT (32,768 shots) and random 26x30 circuit (2,048
                 shots: its ~30 passes per level make 32,768 shots a minutes-long
                 run), 512 MiB FP32 states, tree FP32 (DCP), specialised and
                 generic pass kernels
  qft20_host     the 20-qubit QFT, 32,000 shots, tree FP32, with the state pool
                 in device memory and in mapped host memory (not in the default
                 list)
  batch64_serial the batch64 circuits as 64 plans run back to back on one stream
  rc16_fused / rc20_fused
                 random 16x40 / 20x40 circuits, 8,192 shots, tree FP32 with and
                 without the fused tensor-core blocks

Device time comes from the library's CUDA events (report.kernel_ms); noise
p1 = 1e-3, p2 = 1e-2, pm = 2e-2 throughout.  Inputs are synthetic circuits of
the shapes above (tqs_inputs)."""
from __future__ import annotations

import argparse
import json
import time


from . import capi
from tqs_inputs import batch_circuits_spec, qft, random_layers

NOISE = (1e-3, 1e-2, 2e-2)


def _device_counts(n):
    import torch

    return torch.zeros(1 << n, dtype=torch.int64, device="cuda")


SPEC_AND_GENERIC = (("tree", "fp32", True), ("tree", "fp32", False), ("baseline", "fp64", False))


def single(name, circ, shots, reps, modes=SPEC_AND_GENERIC):
    """Each mode is (tree or baseline, precision, specialised pass kernels)."""
    c, nz = capi.circuit(circ), capi.tqs_noise_model(*NOISE)
    d = _device_counts(circ.n)
    out = {"config": name, "n": circ.n, "gates": len(circ.gates), "shots": shots}
    for mode, prec, spec in modes:
        sh = shots if mode == "tree" else max(64, shots // 16)
        flags = capi.TQS_FLAG_PROFILE | (capi.TQS_FLAG_SPECIALIZE if spec else 0)
        t0 = time.perf_counter()
        plan = capi.tqs_plan_create(c, nz, sh, capi.options(mode=mode, prec=prec, flags=flags))
        create_s = time.perf_counter() - t0
        capi.tqs_plan_execute(plan, 0, d.data_ptr())
        ms = []
        for r in range(reps):
            rep = capi.tqs_plan_execute(plan, 1 + r, d.data_ptr(), report=True)
            ms.append(rep["kernel_ms"])
        plan.close()
        best = min(ms)
        out[f"{mode}_{prec}" + ("_spec" if spec else "")] = {
            "shots": sh, "ms": best, "shots_per_s": sh / (best * 1e-3), "tree": rep["arity"],
            "plan_create_s": round(create_s, 2),
            "passes": rep["passes"], "theo_speedup": rep["theo_speedup"],
            "classes_ms": {k: v["ms"] for k, v in rep["prof"].items() if v["launches"]},
            "classes_alg_GBps": {k: v["bytes"] / (v["ms"] * 1e-3) / 1e9 for k, v in rep["prof"].items()
                                 if v["launches"] and v["ms"] > 0},
        }
    if "tree_fp32" in out and "baseline_fp64" in out:
        out["tree_fp32_over_baseline_fp64"] = out["tree_fp32"]["shots_per_s"] / out["baseline_fp64"]["shots_per_s"]
    if "tree_fp32_spec" in out and "baseline_fp64" in out:
        out["tree_fp32_spec_over_baseline_fp64"] = (out["tree_fp32_spec"]["shots_per_s"] /
                                                    out["baseline_fp64"]["shots_per_s"])
    return out


def batch64(reps, autotune):
    spec = batch_circuits_spec()
    circs = [random_layers(n, L, seed) for n, L, seed in spec]
    handles = [capi.circuit(c) for c in circs]
    noises = [capi.tqs_noise_model(*NOISE) for _ in circs]
    shots = [2048] * len(circs)
    flags = capi.TQS_FLAG_AUTOTUNE if autotune else 0
    t0 = time.perf_counter()
    b = capi.tqs_batch_create(handles, noises, shots, capi.options(prec="fp32", flags=flags))
    create_s = time.perf_counter() - t0
    capi.tqs_batch_execute(b, list(range(len(circs))))
    ms = []
    for r in range(reps):
        rep = capi.tqs_batch_execute(b, [1000 * (r + 1) + i for i in range(len(circs))], report=True)
        ms.append(rep["kernel_ms"])
    best = min(ms)
    total = sum(shots)
    return {"config": "batch64" + ("_autotune" if autotune else ""), "circuits": len(circs),
            "qubits": [c.n for c in circs], "shots_each": 2048, "ms": best,
            "shots_per_s": total / (best * 1e-3), "graph_replay": True, "create_s": create_s}


def batch64_serial(reps):
    """The batch64 circuits as 64 separate plans executed back to back on one
    stream (no graph): the comparison for the graph-branch batch."""
    import torch

    spec = batch_circuits_spec()
    circs = [random_layers(n, L, seed) for n, L, seed in spec]
    noises = [capi.tqs_noise_model(*NOISE) for _ in circs]
    stream = torch.cuda.Stream()
    plans, counts = [], []
    for c, nz in zip(circs, noises):
        o = capi.options(prec="fp32", stream=stream.cuda_stream, workspace_bytes=2 << 30)
        plans.append(capi.tqs_plan_create(capi.circuit(c), nz, 2048, o))
        counts.append(torch.zeros(1 << c.n, dtype=torch.int64, device="cuda"))
    def run(seed0):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            for i, (p, d) in enumerate(zip(plans, counts)):
                capi.tqs_plan_execute(p, seed0 + i, d.data_ptr())
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b)
    run(0)
    best = min(run(1000 * (r + 1)) for r in range(reps))
    for p in plans:
        p.close()
    return {"config": "batch64_serial", "circuits": len(circs), "shots_each": 2048, "ms": best,
            "shots_per_s": 2048 * len(circs) / (best * 1e-3), "graph_replay": False}


def fused(name, circ, shots, reps):
    """Tree FP32 with and without the fused tensor-core blocks (TQS_FLAG_FUSE)."""
    c, nz = capi.circuit(circ), capi.tqs_noise_model(*NOISE)
    d = _device_counts(circ.n)
    out = {"config": name, "n": circ.n, "gates": len(circ.gates), "shots": shots}
    for label, flags in (("per_gate", 0), ("fused", capi.TQS_FLAG_FUSE)):
        plan = capi.tqs_plan_create(c, nz, shots, capi.options(prec="fp32", flags=flags | capi.TQS_FLAG_PROFILE))
        capi.tqs_plan_execute(plan, 0, d.data_ptr())
        reps_ = [capi.tqs_plan_execute(plan, 1 + r, d.data_ptr(), report=True) for r in range(reps)]
        best = min(r["kernel_ms"] for r in reps_)
        out[label] = {"ms": best, "shots_per_s": shots / (best * 1e-3), "fused_blocks": reps_[-1]["fused_blocks"],
                      "passes": reps_[-1]["passes"]}
        plan.close()
    out["fused_over_per_gate"] = out["fused"]["shots_per_s"] / out["per_gate"]["shots_per_s"]
    return out


def host_pool(name, circ, shots, reps):
    """Tree FP32 with the state pool in device memory and in mapped host memory
    (TQS_FLAG_HOST_POOL: the pass kernels read parents from and write children
    to host memory in place)."""
    c, nz = capi.circuit(circ), capi.tqs_noise_model(*NOISE)
    d = _device_counts(circ.n)
    out = {"config": name, "n": circ.n, "gates": len(circ.gates), "shots": shots}
    for label, flags in (("device_pool", 0), ("host_pool", capi.TQS_FLAG_HOST_POOL)):
        t0 = time.perf_counter()
        plan = capi.tqs_plan_create(c, nz, shots, capi.options(prec="fp32", flags=flags))
        create_s = time.perf_counter() - t0
        capi.tqs_plan_execute(plan, 0, d.data_ptr())
        ms = [capi.tqs_plan_execute(plan, 1 + r, d.data_ptr(), report=True)["kernel_ms"] for r in range(reps)]
        out[label] = {"ms": min(ms), "shots_per_s": shots / (min(ms) * 1e-3), "create_s": create_s,
                      "host_pool_bytes": capi.tqs_plan_host_pool_bytes(plan),
                      "workspace_bytes": capi.tqs_plan_workspace_bytes(plan)}
        plan.close()
    out["host_over_device"] = out["host_pool"]["shots_per_s"] / out["device_pool"]["shots_per_s"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", nargs="*", default=["qft16", "rc16", "batch64", "qft26", "rc26"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--autotune", action="store_true", help="batch64: tune every circuit first (slow)")
    a = ap.parse_args(argv)
    for name in a.config:
        if name == "qft16":
            r = single(name, qft(16), 8192, a.reps)
        elif name == "rc16":
            r = single(name, random_layers(16, 40, 16040), 8192, a.reps)
        elif name == "qft26":
            r = single(name, qft(26), 32768, 1, modes=(("tree", "fp32", True), ("tree", "fp32", False)))
        elif name == "rc26":
            r = single(name, random_layers(26, 30, 26030), 2048, 1, modes=(("tree", "fp32", True), ("tree", "fp32", False)))
        elif name == "qft20_host":
            r = host_pool(name, qft(20), 32000, a.reps)
        elif name == "batch64":
            r = batch64(a.reps, a.autotune)
        elif name == "batch64_serial":
            r = batch64_serial(a.reps)
        elif name == "rc16_fused":
            r = fused(name, random_layers(16, 40, 16040), 8192, a.reps)
        elif name == "rc20_fused":
            r = fused(name, random_layers(20, 40, 20040), 8192, a.reps)
        else:
            raise SystemExit(f"unknown config {name}")
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
