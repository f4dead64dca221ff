"""ctypes wrapper of the FP64 C oracle (``tqs_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of bench.py).

``build()`` compiles the C file with gcc (OpenMP when available) into
``oracle/_build/liboracle.so``; it is the only native piece of the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tqs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

GATE_CODES = {
    "h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "sdg": 5, "t": 6, "tdg": 7,
    "rx": 8, "ry": 9, "rz": 10, "p": 11, "cx": 12, "cz": 13, "cp": 14, "swap": 15,
    "u1": 16, "u2": 17,
}
TWO_QUBIT = {"cx", "cz", "cp", "swap", "u2"}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            u32p = C.POINTER(C.c_uint32)
            ip, dp, u64p = C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_uint64)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_noise_draw.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_double, C.c_int]
            L.orc_noise_draw.restype = C.c_int
            L.orc_measure_u.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_measure_u.restype = C.c_double
            L.orc_readout_mask.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_double]
            L.orc_readout_mask.restype = C.c_uint64
            L.orc_gate_matrix.argtypes = [C.c_int, C.c_double, dp, dp]
            circ = [C.c_int, C.c_int, ip, ip, ip, dp, dp]
            L.orc_ideal_state.argtypes = circ + [dp]
            L.orc_ideal_state.restype = C.c_int
            L.orc_run_tree.argtypes = circ + [C.c_double] * 3 + [C.c_uint64, C.c_uint64, C.c_int, u64p, ip, C.c_int, u64p]
            L.orc_run_tree.restype = C.c_int
            L.orc_node_state.argtypes = circ + [C.c_double, C.c_double, C.c_uint64, C.c_int, u64p, ip, C.c_int, C.c_uint64, dp]
            L.orc_node_state.restype = C.c_int
            L.orc_leaf_outcome.argtypes = circ + [C.c_double] * 3 + [C.c_uint64, C.c_int, u64p, ip, C.c_uint64]
            L.orc_leaf_outcome.restype = C.c_int64
            L.orc_node_noise.argtypes = [C.c_int, ip, C.c_double, C.c_double, C.c_uint64, ip, C.c_int, C.c_uint64, ip]
            L.orc_max_threads.restype = C.c_int
            L.orc_run_tree_k.argtypes = circ + [C.c_double] * 3 + [dp, C.c_uint64, C.c_uint64, C.c_int, u64p, ip, C.c_int, u64p]
            L.orc_run_tree_k.restype = C.c_int
            L.orc_node_state_k.argtypes = circ + [C.c_double, C.c_double, dp, C.c_uint64, C.c_int, u64p, ip, C.c_int, C.c_uint64, dp]
            L.orc_node_state_k.restype = C.c_int
            L.orc_leaf_outcome_k.argtypes = circ + [C.c_double] * 3 + [dp, C.c_uint64, C.c_int, u64p, ip, C.c_uint64]
            L.orc_leaf_outcome_k.restype = C.c_int64
            L.orc_thermal_params.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
            L.orc_thermal_params.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Marshalled:
    """Gate list as the flat arrays the C oracle reads."""

    def __init__(self, circuit):
        G = len(circuit.gates)
        self.n = int(circuit.n)
        self.G = G
        self.kind = np.zeros(max(G, 1), dtype=np.int32)
        self.q0 = np.zeros(max(G, 1), dtype=np.int32)
        self.q1 = np.zeros(max(G, 1), dtype=np.int32)
        self.theta = np.zeros(max(G, 1), dtype=np.float64)
        self.mat = np.zeros((max(G, 1), 32), dtype=np.float64)
        for i, (name, a, b, th, m) in enumerate(circuit.gates):
            if not 0 <= a < self.n or (name in TWO_QUBIT and (not 0 <= b < self.n or a == b)):
                raise ValueError(f"gate {i} ({name} {a} {b}) is invalid on {self.n} qubits")
            self.kind[i] = GATE_CODES[name]
            self.q0[i] = a
            self.q1[i] = b if name in TWO_QUBIT else 0
            self.theta[i] = th
            if m is not None:
                z = np.asarray(m, dtype=complex).ravel()
                self.mat[i, 0:2 * len(z):2] = z.real
                self.mat[i, 1:2 * len(z):2] = z.imag

    def args(self):
        return [self.n, self.G, _ptr(self.kind, C.c_int), _ptr(self.q0, C.c_int), _ptr(self.q1, C.c_int),
                _ptr(self.theta, C.c_double), _ptr(self.mat, C.c_double)]


def _tree_arrays(arity: Sequence[int], split: Sequence[int]):
    a = np.ascontiguousarray(arity, dtype=np.uint64)
    s = np.ascontiguousarray(split, dtype=np.int32)
    assert len(s) == len(a) + 1
    return a, s


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def noise_draw(seed: int, node: int, site: int, p: float, npaulis: int) -> int:
    return lib().orc_noise_draw(seed, node, site, p, npaulis)


def measure_u(seed: int, leaf: int) -> float:
    return lib().orc_measure_u(seed, leaf)


def readout_mask(seed: int, leaf: int, n: int, pm: float) -> int:
    return int(lib().orc_readout_mask(seed, leaf, n, pm))


def gate_matrix(name: str, theta: float = 0.0, mat=None) -> np.ndarray:
    d = 4 if name in TWO_QUBIT else 2
    m = np.zeros(32, dtype=np.float64)
    if mat is not None:
        z = np.asarray(mat, dtype=complex).ravel()
        m[0:2 * len(z):2] = z.real
        m[1:2 * len(z):2] = z.imag
    out = np.zeros(32, dtype=np.float64)
    lib().orc_gate_matrix(GATE_CODES[name], theta, _ptr(m, C.c_double), _ptr(out, C.c_double))
    z = out[0:2 * d * d:2] + 1j * out[1:2 * d * d:2]
    return z.reshape(d, d)


def ideal_state(circuit) -> np.ndarray:
    m = _Marshalled(circuit)
    out = np.zeros(2 << m.n, dtype=np.float64)
    rc = lib().orc_ideal_state(*m.args(), _ptr(out, C.c_double))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out[0::2] + 1j * out[1::2]


def thermal_params(t1: float, t2: float, t: float):
    """(gamma, lambda) of the amplitude damping and phase damping that make up
    thermal relaxation over a gate of duration t (T2 <= 2 T1)."""
    g, l = C.c_double(), C.c_double()
    if lib().orc_thermal_params(t1, t2, t, C.byref(g), C.byref(l)) != 0:
        raise ValueError("thermal relaxation needs T1 > 0, 0 < T2 <= 2 T1 and t >= 0")
    return g.value, l.value


def kraus_params(ad: float = 0.0, pd: float = 0.0, t1: float = 0.0, t2: float = 0.0,
                 time_1q: float = 0.0, time_2q: float = 0.0) -> np.ndarray:
    """The oracle's channel array: [AD gamma, PD lambda, TR gamma/lambda after a
    one-qubit gate, TR gamma/lambda after a two-qubit gate] (zeros: no channel)."""
    kr = np.zeros(6)
    kr[0], kr[1] = ad, pd
    if t1 > 0.0:
        kr[2], kr[3] = thermal_params(t1, t2, time_1q)
        kr[4], kr[5] = thermal_params(t1, t2, time_2q)
    return kr


def _kr(kraus):
    if kraus is None:
        return None
    k = np.ascontiguousarray(kraus, dtype=np.float64)
    assert k.shape == (6,)
    return k


def run_tree(circuit, p1: float, p2: float, pm: float, shots: int, seed: int,
             arity: Sequence[int], split: Sequence[int], threads: int = 0, kraus=None) -> np.ndarray:
    """Histogram (uint64[2^n]) of the tree Monte-Carlo; ``arity=[N], split=[0, G]`` is the baseline.
    ``kraus``: the channel array of kraus_params (None: depolarizing and readout noise only)."""
    m = _Marshalled(circuit)
    a, s = _tree_arrays(arity, split)
    k = _kr(kraus)
    counts = np.zeros(1 << m.n, dtype=np.uint64)
    rc = lib().orc_run_tree_k(*m.args(), p1, p2, pm, None if k is None else _ptr(k, C.c_double), shots, seed,
                              len(a), _ptr(a, C.c_uint64), _ptr(s, C.c_int), threads, _ptr(counts, C.c_uint64))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return counts


def run_baseline(circuit, p1, p2, pm, shots, seed, threads: int = 0, kraus=None) -> np.ndarray:
    return run_tree(circuit, p1, p2, pm, shots, seed, [shots], [0, len(circuit.gates)], threads, kraus)


def node_state(circuit, p1, p2, seed, arity, split, level: int, node: int, kraus=None) -> np.ndarray:
    m = _Marshalled(circuit)
    a, s = _tree_arrays(arity, split)
    k = _kr(kraus)
    out = np.zeros(2 << m.n, dtype=np.float64)
    rc = lib().orc_node_state_k(*m.args(), p1, p2, None if k is None else _ptr(k, C.c_double), seed, len(a),
                                _ptr(a, C.c_uint64), _ptr(s, C.c_int), level, node, _ptr(out, C.c_double))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out[0::2] + 1j * out[1::2]


def leaf_outcome(circuit, p1, p2, pm, seed, arity, split, leaf: int, kraus=None) -> int:
    m = _Marshalled(circuit)
    a, s = _tree_arrays(arity, split)
    k = _kr(kraus)
    y = lib().orc_leaf_outcome_k(*m.args(), p1, p2, pm, None if k is None else _ptr(k, C.c_double), seed,
                                 len(a), _ptr(a, C.c_uint64), _ptr(s, C.c_int), leaf)
    if y < 0:
        raise MemoryError("oracle allocation failed")
    return int(y)


def node_noise(circuit, p1, p2, seed, split, level: int, node: int) -> np.ndarray:
    m = _Marshalled(circuit)
    s = np.ascontiguousarray(split, dtype=np.int32)
    cnt = int(s[level + 1] - s[level])
    out = np.zeros(max(cnt, 1), dtype=np.int32)
    lib().orc_node_noise(m.G, _ptr(m.kind, C.c_int), p1, p2, seed, _ptr(s, C.c_int), level, node,
                         _ptr(out, C.c_int))
    return out[:cnt]


def max_threads() -> int:
    return int(lib().orc_max_threads())
