"""Speed against accuracy for different tree structures (Sec. 5.6, Fig. 17).

The workload stands in for the paper's 9-qubit phase-estimation study: textbook
phase estimation with 8 counting qubits and phase 0.3 (not a multiple of 2^-8,
so the output is a narrow peak rather than one basis state; 57 gates with
native controlled-phase gates), 1,000 shots, depolarizing p1 = 1e-3 / p2 = 1e-2
and readout pm = 2e-2.  It runs as the plain baseline and as six trees with
equal-length subcircuits:

  DCP            the dynamic circuit partition's tree for this circuit
  XCP            (20, 10, 5)
  UCP            (10, 10, 10)
  manual         (5, 10, 20) and (2, 2, 250)
  extreme        (250, 1, 1), which yields only A_0 = 250 outcomes

For each structure and seeds 0..S-1 it reports the normalised fidelity F of the
histogram against the noiseless distribution (Sec. 4.1), the mean and largest
|F_tree - F_baseline| for the same seed (beside the same difference between
two baseline runs with different seeds, the spread of the estimate itself),
the theoretical speedup of the
1,000-shot task, levels * 1000 / sum_i M_i (Sec. 3.6), and the measured ratio of
device times.  The measured ratio is launch-bound at 9 qubits and says little;
the node counts are the meaningful cost.

    python -m paper_2203_13892_gb300.sweep [--seeds 10] [--prec fp64] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math

from . import capi
from tqs_inputs import qpe

NOISE = (1e-3, 1e-2, 2e-2)
SHOTS = 1000
MANUAL = (("XCP (20,10,5)", [20, 10, 5], 1000), ("UCP (10,10,10)", [10, 10, 10], 1000),
          ("manual (5,10,20)", [5, 10, 20], 1000), ("manual (2,2,250)", [2, 2, 250], 1000),
          ("extreme (250,1,1)", [250, 1, 1], 250))


def workload():
    return qpe(8, 0.3)


def structures(circ, shots=SHOTS):
    """(label, arity, split, shots) of the DCP tree and the five fixed trees; the
    fixed trees take the equal three-way split that UCP uses for k = 2."""
    c, nz = capi.circuit(circ), capi.tqs_noise_model(*NOISE)
    dcp = capi.tqs_partition(c, nz, shots, capi.options())
    _, split3 = capi.tqs_partition(c, nz, shots, capi.options(part="ucp", k=2))
    out = [("DCP", list(dcp[0]), list(dcp[1]), shots)]
    for label, arity, sh in MANUAL:
        out.append((label, list(arity), list(split3), sh))
    return out


def run(seeds=10, prec="fp64"):
    circ = workload()
    c, nz = capi.circuit(circ), capi.tqs_noise_model(*NOISE)
    base = []
    for s in range(seeds):
        _, F, rep = capi.tqs_simulate(c, nz, SHOTS, s, capi.options(mode="baseline", prec=prec), n=circ.n)
        base.append((F, rep["kernel_ms"]))
    rows = [{"structure": "baseline", "tree": [SHOTS], "shots": SHOTS, "theo_speedup": 1.0,
             "F_mean": sum(F for F, _ in base) / seeds, "ms_mean": sum(m for _, m in base) / seeds}]
    # the spread of the estimate itself: the baseline with seeds S..2S-1 against 0..S-1
    other = [capi.tqs_simulate(c, nz, SHOTS, seeds + s, capi.options(mode="baseline", prec=prec), n=circ.n)[1]
             for s in range(seeds)]
    dF = [abs(F - b[0]) for F, b in zip(other, base)]
    rows.append({"structure": "baseline, other seeds", "tree": [SHOTS], "shots": SHOTS, "theo_speedup": 1.0,
                 "F_mean": sum(other) / seeds, "dF_mean": sum(dF) / seeds, "dF_max": max(dF)})
    for label, arity, split, shots in structures(circ):
        Fs, ms, nodes = [], [], None
        for s in range(seeds):
            _, F, rep = capi.tqs_simulate(c, nz, shots, s, capi.options(arity=arity, split=split, prec=prec),
                                          n=circ.n)
            Fs.append(F)
            ms.append(rep["kernel_ms"])
            nodes = rep["node_instances"]
        dF = [abs(F - b[0]) for F, b in zip(Fs, base)]
        ms_mean = sum(ms) / seeds
        # both speedups are for the whole 1,000-shot task: the extreme tree
        # stands in for it with its 250 outcomes
        rows.append({"structure": label, "tree": arity, "split": split, "shots": shots,
                     "node_instances": nodes, "theo_speedup": len(arity) * SHOTS / sum(nodes),
                     "F_mean": sum(Fs) / seeds, "dF_mean": sum(dF) / seeds, "dF_max": max(dF),
                     "ms_mean": ms_mean, "measured_speedup": rows[0]["ms_mean"] / ms_mean})
    return {"circuit": f"qpe{circ.n} (8 counting qubits, phase 0.3, {len(circ.gates)} gates)",
            "noise": {"p1": NOISE[0], "p2": NOISE[1], "pm": NOISE[2]}, "precision": prec, "seeds": seeds,
            "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = run(a.seeds, a.prec)
    for r in res["rows"]:
        print(json.dumps({k: (round(v, 6) if isinstance(v, float) and math.isfinite(v) else v)
                          for k, v in r.items()}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
