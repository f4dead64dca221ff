"""Host-side checks of libtqs through its C ABI (no GPU needed): the library
loads and exports every function include/tqs.h declares, arguments are
validated, and the host partitioners agree with the oracle's and with the trees
printed in the paper."""
import json
import math
import os
import random
import re

import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import capi
from tqs_inputs import Circuit, qft, random_layers

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tqs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tqs_\w+)\s*\(", text)))


def test_exports_every_declared_symbol():
    lib = capi.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(capi.EXPORTS)
    assert tqs.tqs_abi_version() == 1


def _status(fn, *a):
    with pytest.raises(capi.TqsError) as e:
        fn(*a)
    return e.value.status


def test_argument_validation():
    assert _status(tqs.tqs_circuit_create, 3, [("h", 3, -1, 0.0, None)]) == capi.TQS_EINVAL
    assert _status(tqs.tqs_circuit_create, 3, [("cx", 1, 1, 0.0, None)]) == capi.TQS_EINVAL
    assert _status(tqs.tqs_circuit_create, 3, [("rx", 1, -1, float("nan"), None)]) == capi.TQS_EINVAL
    assert _status(tqs.tqs_circuit_create, 0, []) == capi.TQS_EINVAL
    assert _status(tqs.tqs_circuit_create, 31, []) == capi.TQS_EINVAL
    assert _status(tqs.tqs_noise_model, 0.1, 1.5, 0.0) == capi.TQS_EINVAL
    assert _status(tqs.tqs_noise_model, -0.1, 0.5, 0.0) == capi.TQS_EINVAL
    assert "probabilities" in tqs.tqs_last_error()
    c = tqs.circuit(qft(5))
    nz = tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    assert _status(tqs.tqs_partition, c, nz, 0, None) == capi.TQS_EINVAL
    assert _status(tqs.tqs_partition, c, nz, 100, tqs.options(part="learned")) == capi.TQS_EUNSUPPORTED
    bad = tqs.options(arity=[10, 10], split=[0, 3, 7])
    assert _status(tqs.tqs_partition, c, nz, 100, bad) == capi.TQS_EINVAL  # split must end at G=15
    small = tqs.options(arity=[5, 5], split=[0, 3, len(qft(5).gates)])
    assert _status(tqs.tqs_partition, c, nz, 100, small) == capi.TQS_EINVAL  # 25 < 100 leaves


def _rates(circ, p1, p2):
    return [p2 if g[0] in ("cx", "cz", "cp", "swap", "u2") else p1 for g in circ.gates]


def test_dcp_matches_oracle_on_random_workloads(orc):
    rnd = random.Random(1)
    for _ in range(120):
        n = rnd.randint(2, 12)
        circ = random_layers(n, rnd.randint(0, 30), rnd.randint(0, 10**6)) if rnd.random() < 0.6 else qft(n)
        p1, p2 = rnd.choice([1e-4, 1e-3, 4e-3]), rnd.choice([1e-3, 1e-2, 2e-2])
        shots = rnd.choice([1, 7, 100, 1000, 8192, 32000, 123457])
        cg = rnd.choice([1, 3, 10, 25])
        c = tqs.circuit(circ)
        nz = tqs.tqs_noise_model(p1, p2, 0.0)
        arity, split = tqs.tqs_partition(c, nz, shots, tqs.options(copy_gates=cg))
        oa, osplit, _ = orc.partition.dcp(_rates(circ, p1, p2), shots, copy_gates=cg)
        assert arity == oa and split == osplit, (n, len(circ), shots, cg)


def test_dcp_paper_trees():
    # QPE_9 stand-in: 120 gates with a uniform 0.65% error (first third ~ 0.23)
    g = GOLD["qpe9_dcp"]
    circ = Circuit(9)
    for i in range(120):
        circ.add("h", i % 9)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model(0.0065, 0.0065, 0.0)
    arity, split = tqs.tqs_partition(c, nz, g["shots"], tqs.options())
    assert arity == g["arity"] and split == [0, 40, 80, 120]
    # QFT_14 stand-in: 472 gates, two CX in every five, Sycamore rates
    q = GOLD["qft14_dcp"]
    circ = Circuit(14)
    for i in range(472):
        if i % 5 in (1, 3):
            circ.add("cx", i % 14, (i + 1) % 14)
        else:
            circ.add("h", i % 14)
    s = GOLD["sycamore_rates"]
    arity, split = tqs.tqs_partition(tqs.circuit(circ), tqs.tqs_noise_model(s["p1"], s["p2"], 0.0),
                                     q["shots"], tqs.options())
    assert len(arity) == q["subcircuits"] and arity[0] == q["a0"] and set(arity[1:]) == {2}


def test_ucp_xcp_explicit_baseline(orc):
    circ = qft(6)
    G = len(circ.gates)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model(1e-3, 1e-2, 0.0)
    u = GOLD["ucp_example"]
    assert tqs.tqs_partition(c, nz, u["shots"], tqs.options(part="ucp", k=2)) == \
        (u["arity"], orc.partition.equal_splits(G, 3))
    x = GOLD["xcp_example"]
    assert tqs.tqs_partition(c, nz, x["shots"], tqs.options(part="xcp", k=2))[0] == x["arity"]
    assert tqs.tqs_partition(c, nz, 777, tqs.options(mode="baseline")) == ([777], [0, G])
    ex = tqs.options(arity=[4, 3, 2], split=[0, 5, 5, G])
    assert tqs.tqs_partition(c, nz, 20, ex) == ([4, 3, 2], [0, 5, 5, G])


def test_noise_model_ex_validation():
    tqs.tqs_noise_model_ex(1e-3, 1e-2, 2e-2, 0.01, 0.01, 50e-6, 70e-6, 1e-6, 2e-6)
    bad = (dict(ad_gamma=1.5), dict(pd_lambda=-0.1), dict(t1=50e-6, t2=120e-6, time_1q=1e-6),
           dict(t1=50e-6, t2=0.0), dict(time_2q=-1.0))
    for kw in bad:
        with pytest.raises(capi.TqsError) as e:
            tqs.tqs_noise_model_ex(1e-3, 1e-2, 2e-2, **kw)
        assert e.value.status == capi.TQS_EINVAL, kw


def test_damping_plan_keeps_circuit_order_one_gate_per_pass():
    """With damping channels every gate's choice needs the state after it, so the
    plan keeps circuit order, one gate per tile pass, plus one closing pass per
    level that applies the last gate's choice."""
    circ = qft(6)
    G = len(circ.gates)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model_ex(1e-3, 1e-2, 2e-2, ad_gamma=0.01)
    o = tqs.options(arity=[8, 2, 4], split=[0, G // 3, 2 * G // 3, G])
    order, passes, tiles = tqs.tqs_debug_plan_order(c, nz, 64, o, G)
    assert list(order) == list(range(G))
    assert len(tiles) == G + 3
    plain = tqs.tqs_noise_model(1e-3, 1e-2, 2e-2)
    _, _, tiles_plain = tqs.tqs_debug_plan_order(c, plain, 64, o, G)
    assert len(tiles_plain) < G


def test_dcp_counts_damping_in_the_error_rate(orc):
    """DCP's first-subcircuit error estimate includes the damping rates; the
    library's tree equals the oracle partitioner's with the same rates."""
    circ = qft(12)
    kr = orc.core.kraus_params(ad=0.01, pd=0.01)
    arity, split, _ = orc.partition.dcp(orc.partition.gate_rates(circ, 1e-3, 1e-2, kr), 4000)
    c = tqs.circuit(circ)
    nz = tqs.tqs_noise_model_ex(1e-3, 1e-2, 2e-2, ad_gamma=0.01, pd_lambda=0.01)
    assert tqs.tqs_partition(c, nz, 4000, tqs.options()) == (arity, split)
    a_plain, _, _ = orc.partition.dcp(orc.partition.gate_rates(circ, 1e-3, 1e-2), 4000)
    assert arity[0] >= a_plain[0]
