"""Tree mode against plain baseline mode in normalised fidelity (Sec. 4.1, the
comparison of Sec. 5.4), computed with the FP64 oracle on the 16-qubit
configurations: 8,192 shots, p1 = 1e-3, p2 = 1e-2, pm = 2e-2, the DCP tree, seeds
0..S-1.  The GPU path's FP64 histograms are bit-exact with the oracle's wherever
the GPU tests compare them (QFT-16 and RC-16x40 at these sizes among them).

For each seed: F of the tree histogram and of the baseline histogram against the
noiseless distribution, their difference, and for scale the difference between
two baseline runs with different seeds (the spread of the estimate itself).  The
QFT of |0...0> has a uniform ideal distribution, for which F is undefined, so
the QFT case is the inverse QFT on a Fourier state (ideal output one basis state).

    python tests/oracle_fidelity_study.py [--circuit iqft16|rc16x40|iqft20] [--seeds 5] [--shots 8192]

iqft20 is the inverse QFT on a Fourier state of 20 qubits (260 gates), the
shape of the throughput workload with a defined fidelity; its baseline runs are
long on a CPU, so it is meant for a reduced shot count.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tqs_inputs import inverse_qft_on_fourier_state, random_layers  # noqa: E402

P1, P2, PM = 1e-3, 1e-2, 2e-2
SHOTS = 8192
TWO = ("cx", "cz", "cp", "swap", "u2")


def circuit(name):
    if name == "iqft16":
        return inverse_qft_on_fourier_state(16, 40503)
    if name == "rc16x40":
        return random_layers(16, 40, 16040)
    if name == "iqft20":
        return inverse_qft_on_fourier_state(20, 699051)
    raise SystemExit(f"unknown circuit {name}")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--circuit", default="iqft16", choices=["iqft16", "rc16x40", "iqft20"])
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--shots", type=int, default=SHOTS)
    a = ap.parse_args(argv)
    shots = a.shots
    oracle.core.build()
    circ = circuit(a.circuit)
    rates = [P2 if g[0] in TWO else P1 for g in circ.gates]
    arity, split = oracle.partition.dcp(rates, shots, copy_gates=10)[:2]
    ideal = np.abs(oracle.core.ideal_state(circ)) ** 2
    F = lambda counts: oracle.fidelity.normalized_fidelity(ideal, counts / shots)  # noqa: E731
    rows = []
    t0 = time.time()
    for s in range(a.seeds):
        ft = F(oracle.core.run_tree(circ, P1, P2, PM, shots, s, arity, split))
        fb = F(oracle.core.run_baseline(circ, P1, P2, PM, shots, s))
        fo = F(oracle.core.run_baseline(circ, P1, P2, PM, shots, 1000 + s))
        rows.append({"seed": s, "F_tree": ft, "F_baseline": fb, "F_baseline_other_seed": fo,
                     "dF_tree": abs(ft - fb), "dF_two_baselines": abs(fo - fb)})
        print(json.dumps(rows[-1]), flush=True)
    dft = [r["dF_tree"] for r in rows]
    dfb = [r["dF_two_baselines"] for r in rows]
    print(json.dumps({"circuit": a.circuit, "gates": len(circ.gates), "shots": shots, "tree": list(arity),
                      "seeds": a.seeds, "dF_tree_mean": float(np.mean(dft)), "dF_tree_max": float(np.max(dft)),
                      "dF_two_baselines_mean": float(np.mean(dfb)), "dF_two_baselines_max": float(np.max(dfb)),
                      "seconds": time.time() - t0}))


if __name__ == "__main__":
    main()
