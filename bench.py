#!/usr/bin/env python3
"""Benchmark: noisy shots/sec of the 20-qubit QFT in tree mode (FP32 state
vectors, dynamic circuit partition) on one GB300, against the HBM roofline.

A step is one full noisy simulation of the workload: 32,000 shots of the
220-gate QFT-20 (20 H, 190 CP, 10 SWAP) from |0...0> with depolarizing noise
p1 = 1e-3 after one-qubit gates, p2 = 1e-2 after two-qubit gates and readout
flips pm = 2e-2 (the paper's 32,000-shot count, Sec. 4.3), planned by DCP
(Sec. 3.2) and run through the library's device-resident entry point.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent 32,000-shot problem
with a rank-specific seed (weak scaling, no data-path collective); `value` is
the shots of all ranks divided by the slowest rank's time.

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores: each step is a bounded sample of the same tree (whole level-0 subtrees,
one per core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "noisy shots/sec at 20q QFT (tree FP32 vs plain FP64), % of HBM roofline"
UNIT = "shots/s"
N_QUBITS, SHOTS = 20, 32000
P1, P2, PM = 1e-3, 1e-2, 2e-2
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def workload_config(tree=None, split=None, extra=None, shots=SHOTS):
    cfg = {
        "workload": f"qft20_noisy_tree_fp32_dcp_{shots}shots",
        "n_qubits": N_QUBITS, "gates": 220, "shots_per_step": shots,
        "noise": {"p1": P1, "p2": P2, "pm": PM, "channel": "depolarizing+readout"},
        "mode": "tree", "precision": "fp32", "partitioner": "dcp",
        "input": "|0...0>", "l2": "512 MiB buffer written between timed steps",
    }
    if tree is not None:
        cfg["tree"] = tree
        cfg["split"] = split
    if extra:
        cfg.update(extra)
    return cfg


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(kernels="generic"):
    """Hash of the files the pass kernel is compiled and launched from: its six
    instantiation units, the headers of csrc they include, and kernels.cu (which
    sets its grid and shared memory); for the specialised kernels also the
    generator that writes their statements (specialize.cpp and its header).
    Host-only sources (the NVRTC / driver runtime among them) do not enter."""
    d = os.path.join(ROOT, "paper_2203_13892_gb300", "csrc")
    names = sorted(f for f in os.listdir(d) if f.startswith("pass_") and f.endswith(".cu"))
    names += ["pass_kernel.cuh", "pass_kernel.h", "device_common.cuh", "internal.h", "kernels.cu"]
    if kernels == "specialized":
        names += ["specialize.cpp", "specialize.h"]
    h = hashlib.sha256()
    for f in names:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kind, alg_bytes_per_launch, kernels="generic"):
    """DRAM bytes per launch of kernel class `kind`, from the committed ncu
    capture of a small case of the same kernel: its DRAM bytes per CTA (one
    tile of one node) times the CTAs of a full launch, or None when the kernels
    changed since the counters were taken."""
    name = "traffic_qft20_tree_fp32" + ("_specialized" if kernels == "specialized" else "") + ".json"
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash(kernels):
        return None
    ent = d.get("kernels", {}).get(kind)
    if not ent:
        return None
    ctas = alg_bytes_per_launch / ent["alg_bytes_per_cta"]
    return ent["dram_bytes_per_cta"] * ctas


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        top = max(sm)
        loaded = [x for x in sm if x >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        return dist, world, rank, local
    return None, 1, 0, local


def max_over_ranks(dist, value):
    if dist is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value):
    if dist is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(arity, split, subtrees, threads, seed=0):
    """Run the FP64 oracle on the first `subtrees` level-0 subtrees of the tree."""
    import oracle
    from tqs_inputs import qft

    below = 1
    for a in arity[1:]:
        below *= a
    leaves = subtrees * below
    t0 = time.perf_counter()
    counts = oracle.core.run_tree(qft(N_QUBITS), P1, P2, PM, leaves, seed, arity, split, threads=threads)
    dt = time.perf_counter() - t0
    assert int(counts.sum()) == leaves
    return leaves, dt


def oracle_dcp_tree(shots=SHOTS):
    """DCP tree of the workload from the oracle's own partitioner (Sec. 3.2), so
    the reference arm loads nothing of the CUDA library."""
    import oracle.partition as part
    from tqs_inputs import qft

    arity, split, _ = part.dcp(part.gate_rates(qft(N_QUBITS), P1, P2), shots)
    return arity, split


def run_reference(args, dist, world, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    arity, split = oracle_dcp_tree(args.shots)
    subtrees = max(1, cores)
    steps = []
    for i in range(args.warmup + args.steps):
        leaves, dt = oracle_sample(arity, split, subtrees, cores, seed=i)
        if i >= args.warmup:
            steps.append((leaves, dt))
    shots = sum(s for s, _ in steps)
    secs = sum(t for _, t in steps)
    value = shots / secs
    sample = (f"{subtrees} whole level-0 subtrees ({steps[0][0]} leaves) of the DCP tree {arity} per step, "
              f"FP64 oracle, {cores} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(arity, split, {"l2": "host run"}, args.shots),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--baseline-shots", type=int, default=2000,
                    help="shots of the FP64 baseline-mode comparison run")
    ap.add_argument("--baseline-reps", type=int, default=6,
                    help="runs of the FP64 baseline-mode comparison (the first is not timed)")
    ap.add_argument("--shots", type=int, default=SHOTS,
                    help="shots per step (smaller values make the small case of a profiler capture)")
    ap.add_argument("--batch", type=int, default=0,
                    help="tree nodes per launch (0: the library's choice)")
    ap.add_argument("--kernels", default="specialized", choices=["specialized", "generic"],
                    help="FP32 tree pass kernels: compiled per pass program at plan time (TQS_FLAG_SPECIALIZE), "
                         "or the generic kernel that interprets the pass programs")
    ap.add_argument("--arity", default="",
                    help="comma-separated tree arities overriding DCP (with --shots below the workload's, the "
                         "small case of a profiler capture runs the workload's own tree); split: equal gate counts")
    args = ap.parse_args()
    dist, world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, dist, world, rank)
        if dist is not None:
            dist.barrier()
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import numpy as np
    import torch

    import paper_2203_13892_gb300 as tqs
    from paper_2203_13892_gb300 import capi
    from tqs_inputs import qft

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    circ = qft(N_QUBITS)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model(P1, P2, PM)
    seed0 = args.seed + 1000003 * rank

    SH = args.shots

    tree_kw = {}
    if args.arity:
        ar = [int(x) for x in args.arity.split(",")]
        G = len(circ.gates)
        tree_kw = {"arity": ar, "split": [G * i // len(ar) for i in range(len(ar) + 1)]}

    def make_plan(shots, **kw):
        if kw.get("mode") != "baseline":
            kw = {**tree_kw, **kw}
        o = tqs.options(stream=stream.cuda_stream, batch=args.batch, **kw)
        probe = tqs.tqs_plan_create(c, nz, shots, o)
        nbytes = tqs.tqs_plan_workspace_bytes(probe)
        probe.close()
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        o.workspace = ws.data_ptr()
        o.workspace_bytes = nbytes
        return tqs.tqs_plan_create(c, nz, shots, o), ws

    spec_flag = capi.TQS_FLAG_SPECIALIZE if args.kernels == "specialized" else 0
    t_plan = time.perf_counter()
    plan, ws = make_plan(SH, flags=capi.TQS_FLAG_PROFILE | spec_flag)
    plan_create_s = time.perf_counter() - t_plan  # includes compiling the specialised kernels (first use)
    d_counts = torch.zeros(1 << N_QUBITS, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            tqs.tqs_plan_execute(plan, seed0 + i, d_counts.data_ptr())
    stream.synchronize()

    # ---- timed region ------------------------------------------------
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms, reps = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            rep = tqs.tqs_plan_execute(plan, seed0 + args.warmup + k, d_counts.data_ptr(), report=True)
            ev[k][1].record(stream)
        reps.append(rep)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    for a, b in ev:
        step_ms.append(a.elapsed_time(b))
    assert int(d_counts.sum().item()) == SH
    total_ms = max_over_ranks(dist, sum(step_ms))
    total_shots = sum_over_ranks(dist, SH * args.steps)
    value = total_shots / (total_ms * 1e-3)

    # ---- dominant kernel and roofline --------------------------------
    kinds = {}
    for r in reps:
        for name, d in r["prof"].items():
            k = kinds.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
            k["launches"] += d["launches"]
            k["ms"] += d["ms"]
            k["bytes"] += d["bytes"]
    dom = max(kinds, key=lambda n: kinds[n]["ms"])
    D = kinds[dom]
    peak, peak_src = load_peaks()
    per_launch_bytes = D["bytes"] / max(D["launches"], 1)
    avg_s = D["ms"] * 1e-3 / max(D["launches"], 1)
    achieved = per_launch_bytes / avg_s / 1e9
    gpu_launches = sum(int(r["kernel_launches"]) for r in reps)
    alg_bytes_step = statistics.mean(r["alg_bytes"] for r in reps)
    rep0 = reps[-1]

    # ---- plain FP64 baseline mode on the same GPU (the metric's comparison) --
    # The same circuit, noise and shot statistics, every shot from |0...0> in
    # FP64: one tree level of all 220 gates, split into tile passes by the same
    # planner.  Timed over `baseline_reps` runs after one warm-up run.
    bshots = args.baseline_shots
    bplan, bws = make_plan(bshots, mode="baseline", prec="fp64")
    bcounts = torch.zeros(1 << N_QUBITS, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        tqs.tqs_plan_execute(bplan, 7, bcounts.data_ptr())
    stream.synchronize()
    base_ms, brep = [], None
    for r in range(args.baseline_reps):
        with torch.cuda.stream(stream):
            ba, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(1.0)
            ba.record(stream)
            rep_r = tqs.tqs_plan_execute(bplan, 8 + r, bcounts.data_ptr(), report=(r == 0))
            bb.record(stream)
        if r == 0:
            brep = rep_r
        stream.synchronize()
        base_ms.append(ba.elapsed_time(bb) if r else None)
    # the first repeat carries the report (which synchronises): time the others
    timed_b = [t for t in base_ms if t is not None] or [ba.elapsed_time(bb)]
    base_sps = bshots * len(timed_b) / (sum(timed_b) * 1e-3)
    del bplan, bws, bcounts
    state_b64 = (1 << N_QUBITS) * 16
    state_b32 = (1 << N_QUBITS) * 8
    # Bytes per shot as the method defines them (read the input state once,
    # write the output once per node instance) and as the planner's passes move
    # them (the executor's count: every pass reads and writes the state).
    nodes_tree = sum(rep0["node_instances"])
    tree_alg_shot = 2.0 * state_b32 * nodes_tree / SH
    tree_pass_shot = alg_bytes_step / SH
    base_alg_shot = 2.0 * state_b64
    base_pass_shot = brep["alg_bytes"] / bshots
    baseline = {
        "value": base_sps, "unit": UNIT, "shots": bshots, "repeats": len(timed_b), "mode": "baseline",
        "precision": "fp64", "ms_per_run": [round(t, 3) for t in timed_b],
        "passes_per_shot": int(sum(brep["passes"])),
        "method_bytes_per_shot": base_alg_shot, "pass_bytes_per_shot": base_pass_shot,
        "method_GBps": base_sps * base_alg_shot / 1e9, "pass_GBps": base_sps * base_pass_shot / 1e9,
    }
    baseline["frac_of_peak"] = baseline["pass_GBps"] / peak

    # ---- end to end through the public call with host buffers --------
    o = tqs.options(stream=stream.cuda_stream, batch=args.batch, flags=spec_flag)
    o.workspace = ws.data_ptr()
    o.workspace_bytes = ws.numel()
    del plan
    tqs.tqs_simulate(c, nz, SH, 99, o, n=N_QUBITS)  # warm
    torch.cuda.synchronize()
    e2e_s = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        counts, fid, _ = tqs.tqs_simulate(c, nz, SH, 100 + k, o, n=N_QUBITS)
        e2e_s.append(time.perf_counter() - t0)
        assert int(counts.sum()) == SH
    e2e_time = max_over_ranks(dist, sum(e2e_s))
    e2e_value = total_shots / e2e_time
    G = len(circ.gates)
    h2d = 16 * G + 4 * 32 * G + 4 * (len(rep0["passes"]) + sum(rep0["passes"])) + 32  # instrs, FP32 mats, pass table, perm
    h2d += 16 * G + 8 * 32 * G + 4 * 2 + 32  # the noiseless FP64 run behind the fidelity
    d2h = 8 * (1 << N_QUBITS) + 24

    # ---- CPU baseline: the oracle on the host cores ------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        leaves, dt = oracle_sample(rep0["arity"], rep0["split"], cores, cores)
        cpu = {"value": leaves / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cores} whole level-0 subtrees ({leaves} leaves) of the same DCP tree, FP64, "
                         f"{dt:.1f} s on {cores} OpenMP threads"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(rep0["arity"], rep0["split"],
                                  {"parallelism": f"independent problem per GPU x{world}",
                                   "passes_per_level": rep0["passes"], "plan_create_s": round(plan_create_s, 2),
                                   "pass_kernels": ("specialised per pass program (NVRTC, sm_103a), compiled at plan "
                                                    "creation, outside the timed region" if args.kernels == "specialized"
                                                    else "generic (interprets the pass programs)")}, SH),
        "roofline": {"bound": "hbm", "kernel": f"pass_kernel[{dom}]", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic(dom, per_launch_bytes, args.kernels),
                     "alg_bytes_per_launch": per_launch_bytes,
                     "avg_launch_ms": avg_s * 1e3, "launches": D["launches"]},
        "kernel_classes": {n: {"launches": d["launches"], "ms_per_step": d["ms"] / args.steps,
                               "GBps": (d["bytes"] / (d["ms"] * 1e-3) / 1e9) if d["ms"] > 0 else None}
                           for n, d in kinds.items()},
        "path_alg_GBps": alg_bytes_step / (statistics.mean(step_ms) * 1e-3) / 1e9,
        "baseline_fp64": baseline,
        "tree_fp32": {"passes_per_node": rep0["passes"], "node_instances": rep0["node_instances"],
                      "method_bytes_per_shot": tree_alg_shot, "pass_bytes_per_shot": tree_pass_shot,
                      "pass_GBps": value / world * tree_pass_shot / 1e9,
                      "frac_of_peak": value / world * tree_pass_shot / 1e9 / peak},
        "tree_fp32_over_baseline_fp64": value / world / base_sps,
        "theo_speedup_tree": rep0["theo_speedup"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
