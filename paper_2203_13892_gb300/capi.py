"""ctypes binding of libtqs (include/tqs.h): same names, argument marshalling only.

Every step of the simulation runs in the CUDA library; this module converts
Python values to the C structs and back.  Importing it loads ``_build/libtqs.so``
(building it with nvcc first if it is missing) and raises if that fails: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

TQS_OK, TQS_EINVAL, TQS_ENOMEM, TQS_ECUDA, TQS_ETIMEOUT, TQS_EUNSUPPORTED, TQS_EBOUNDS = range(7)
TQS_MODE_BASELINE, TQS_MODE_TREE = 0, 1
TQS_FP64, TQS_FP32 = 0, 1
TQS_PART_DCP, TQS_PART_UCP, TQS_PART_XCP, TQS_PART_EXPLICIT, TQS_PART_LEARNED = range(5)
TQS_FLAG_NO_FIDELITY = 0x1
TQS_FLAG_PROFILE = 0x2
TQS_FLAG_AUTOTUNE = 0x4
TQS_FLAG_FUSE = 0x8
TQS_FLAG_HOST_POOL = 0x10
TQS_FLAG_DEBUG_BOUNDS = 0x20
TQS_FLAG_FAULT_TIMEOUT = 0x40
TQS_FLAG_FAULT_BOUNDS = 0x80
TQS_FLAG_SPECIALIZE = 0x100
TQS_MAX_LEVELS = 17
TQS_PROF_KINDS = 4
PROF_NAMES = ("noise", "store", "sums", "sample")

GATE_KINDS = {
    "h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "sdg": 5, "t": 6, "tdg": 7,
    "rx": 8, "ry": 9, "rz": 10, "p": 11, "cx": 12, "cz": 13, "cp": 14, "swap": 15,
    "u1": 16, "u2": 17,
}
_TWO = {"cx", "cz", "cp", "swap", "u2"}


class TqsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tqs status {status}: {msg}")
        self.status = status


class tqs_gate(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("q0", C.c_uint32), ("q1", C.c_uint32),
                ("theta", C.c_double), ("mat", C.POINTER(C.c_double))]


class tqs_noise_params(C.Structure):
    _fields_ = [("p1", C.c_double), ("p2", C.c_double), ("pm", C.c_double), ("ad_gamma", C.c_double),
                ("pd_lambda", C.c_double), ("t1", C.c_double), ("t2", C.c_double), ("time_1q", C.c_double),
                ("time_2q", C.c_double)]


class tqs_options(C.Structure):
    _fields_ = [("mode", C.c_int), ("prec", C.c_int), ("part", C.c_int),
                ("z", C.c_double), ("eps", C.c_double), ("copy_gates", C.c_uint32),
                ("k", C.c_uint32), ("arity", C.POINTER(C.c_uint64)), ("split", C.POINTER(C.c_uint32)),
                ("tile_qubits", C.c_uint32), ("batch", C.c_uint32), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("stream", C.c_void_p), ("flags", C.c_uint32)]


class tqs_report(C.Structure):
    _fields_ = [("shots_done", C.c_uint64), ("levels", C.c_uint32),
                ("arity", C.c_uint64 * TQS_MAX_LEVELS), ("split", C.c_uint32 * (TQS_MAX_LEVELS + 1)),
                ("node_instances", C.c_uint64 * TQS_MAX_LEVELS), ("passes", C.c_uint32 * TQS_MAX_LEVELS),
                ("kernel_launches", C.c_uint64), ("kernel_ms", C.c_double), ("shots_per_s", C.c_double),
                ("alg_bytes", C.c_double), ("fid_norm", C.c_double), ("fid_s", C.c_double),
                ("theo_speedup", C.c_double), ("prof_launches", C.c_uint64 * TQS_PROF_KINDS),
                ("prof_ms", C.c_double * TQS_PROF_KINDS), ("prof_bytes", C.c_double * TQS_PROF_KINDS),
                ("fused_blocks", C.c_uint32 * TQS_MAX_LEVELS)]

    def as_dict(self) -> dict:
        L = self.levels
        return {
            "shots_done": self.shots_done, "levels": L,
            "arity": list(self.arity[:L]), "split": list(self.split[:L + 1]),
            "node_instances": list(self.node_instances[:L]), "passes": list(self.passes[:L]),
            "fused_blocks": list(self.fused_blocks[:L]),
            "kernel_launches": self.kernel_launches, "kernel_ms": self.kernel_ms,
            "shots_per_s": self.shots_per_s, "alg_bytes": self.alg_bytes,
            "fid_norm": self.fid_norm, "fid_s": self.fid_s, "theo_speedup": self.theo_speedup,
            "prof": {PROF_NAMES[k]: {"launches": self.prof_launches[k], "ms": self.prof_ms[k],
                                     "bytes": self.prof_bytes[k]} for k in range(TQS_PROF_KINDS)},
        }


_lock = threading.Lock()
_lib = None

# Exported symbols, by header declaration.
EXPORTS = (
    "tqs_circuit_create", "tqs_circuit_destroy", "tqs_noise_model", "tqs_noise_model_ex", "tqs_noise_destroy",
    "tqs_options_default", "tqs_partition", "tqs_simulate", "tqs_plan_create",
    "tqs_plan_execute", "tqs_plan_workspace_bytes", "tqs_plan_host_pool_bytes", "tqs_plan_destroy",
    "tqs_debug_node_state", "tqs_debug_node_noise", "tqs_debug_plan_order", "tqs_debug_spec_check",
    "tqs_debug_spec_source",
    "tqs_simulate_static",
    "tqs_last_error",
    "tqs_abi_version", "tqs_batch_create", "tqs_batch_execute", "tqs_batch_counts",
    "tqs_batch_device_counts", "tqs_batch_size", "tqs_batch_destroy", "tqs_learned_param_count",
    "tqs_learned_features", "tqs_learned_candidate", "tqs_learned_train", "tqs_learned_loss_grad",
    "tqs_learned_predict", "tqs_learned_set_model",
)
TQS_LEARNED_FEATURES = 40
TQS_LEARNED_CLASSES = 20
TQS_STATIC_SCRATCH_BYTES = 32 << 20


def lib():
    """The loaded libtqs (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                path = _build.build()
            L = C.CDLL(path)
            vp, u64p, u32p, dp = C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32), C.POINTER(C.c_double)
            st = C.c_int
            L.tqs_circuit_create.argtypes = [C.c_uint32, C.POINTER(tqs_gate), C.c_size_t, C.POINTER(vp)]
            L.tqs_circuit_create.restype = st
            L.tqs_circuit_destroy.argtypes = [vp]
            L.tqs_noise_model.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(vp)]
            L.tqs_noise_model.restype = st
            L.tqs_noise_model_ex.argtypes = [C.POINTER(tqs_noise_params), C.POINTER(vp)]
            L.tqs_noise_model_ex.restype = st
            L.tqs_noise_destroy.argtypes = [vp]
            L.tqs_options_default.argtypes = [C.POINTER(tqs_options)]
            L.tqs_partition.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), u32p, u64p, u32p]
            L.tqs_partition.restype = st
            L.tqs_simulate.argtypes = [vp, vp, C.c_uint64, C.c_uint64, C.POINTER(tqs_options), u64p, dp,
                                       C.POINTER(tqs_report)]
            L.tqs_simulate.restype = st
            L.tqs_plan_create.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), C.POINTER(vp)]
            L.tqs_plan_create.restype = st
            L.tqs_plan_execute.argtypes = [vp, C.c_uint64, vp, C.POINTER(tqs_report)]
            L.tqs_plan_execute.restype = st
            L.tqs_plan_workspace_bytes.argtypes = [vp]
            L.tqs_plan_workspace_bytes.restype = C.c_size_t
            L.tqs_plan_host_pool_bytes.argtypes = [vp]
            L.tqs_plan_host_pool_bytes.restype = C.c_size_t
            L.tqs_plan_destroy.argtypes = [vp]
            L.tqs_debug_node_state.argtypes = [vp, vp, C.c_uint64, C.c_uint64, C.POINTER(tqs_options),
                                               C.c_uint32, C.c_uint64, dp]
            L.tqs_debug_node_state.restype = st
            L.tqs_debug_node_noise.argtypes = [vp, vp, C.c_uint64, C.c_uint64, C.POINTER(tqs_options),
                                               C.c_uint32, C.c_uint64, C.POINTER(C.c_uint8)]
            L.tqs_debug_node_noise.restype = st
            u32p = C.POINTER(C.c_uint32)
            L.tqs_debug_plan_order.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), u32p, u32p, u32p, u32p]
            L.tqs_debug_plan_order.restype = st
            L.tqs_debug_spec_check.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), u32p,
                                               C.POINTER(C.c_uint64)]
            L.tqs_debug_spec_check.restype = st
            L.tqs_debug_spec_source.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), C.c_uint32, C.c_int,
                                                C.c_char_p, C.c_uint64, C.POINTER(C.c_uint64)]
            L.tqs_debug_spec_source.restype = st
            L.tqs_simulate_static.argtypes = [vp, vp, C.c_uint64, C.c_uint64, C.POINTER(tqs_options), vp]
            L.tqs_simulate_static.restype = st
            L.tqs_batch_create.argtypes = [C.c_size_t, C.POINTER(vp), C.POINTER(vp), u64p, C.POINTER(tqs_options),
                                           C.POINTER(vp)]
            L.tqs_batch_create.restype = st
            L.tqs_batch_execute.argtypes = [vp, u64p, C.POINTER(tqs_report)]
            L.tqs_batch_execute.restype = st
            L.tqs_batch_counts.argtypes = [vp, C.c_size_t, u64p]
            L.tqs_batch_counts.restype = st
            L.tqs_batch_device_counts.argtypes = [vp, C.c_size_t]
            L.tqs_batch_device_counts.restype = C.c_void_p
            L.tqs_batch_size.argtypes = [vp]
            L.tqs_batch_size.restype = C.c_size_t
            L.tqs_batch_destroy.argtypes = [vp]
            fp, i32p, u8p = C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
            L.tqs_learned_param_count.restype = C.c_size_t
            L.tqs_learned_features.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), fp, u8p]
            L.tqs_learned_features.restype = st
            L.tqs_learned_candidate.argtypes = [vp, vp, C.c_uint64, C.POINTER(tqs_options), C.c_uint32, u32p, u64p,
                                                u32p]
            L.tqs_learned_candidate.restype = st
            L.tqs_learned_train.argtypes = [fp, i32p, C.c_size_t, C.c_uint32, C.c_uint32, C.c_float, C.c_uint64, fp,
                                            fp, fp]
            L.tqs_learned_train.restype = st
            L.tqs_learned_loss_grad.argtypes = [fp, fp, i32p, C.c_size_t, fp, fp]
            L.tqs_learned_loss_grad.restype = st
            L.tqs_learned_predict.argtypes = [fp, fp, C.c_size_t, fp]
            L.tqs_learned_predict.restype = st
            L.tqs_learned_set_model.argtypes = [fp]
            L.tqs_learned_set_model.restype = st
            L.tqs_last_error.restype = C.c_char_p
            L.tqs_abi_version.restype = C.c_int
            _lib = L
    return _lib


def _check(status: int) -> None:
    if status != TQS_OK:
        raise TqsError(status, lib().tqs_last_error().decode())


def tqs_last_error() -> str:
    return lib().tqs_last_error().decode()


def tqs_abi_version() -> int:
    return int(lib().tqs_abi_version())


class Handle:
    """Owns a library handle and destroys it on close/garbage collection."""

    def __init__(self, ptr, destroy):
        self.ptr = ptr
        self._destroy = destroy

    def close(self):
        if self.ptr:
            self._destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tqs_circuit_create(n: int, gates) -> Handle:
    """gates: tqs_inputs-style tuples (name, q0, q1, theta, mat)."""
    G = len(gates)
    arr = (tqs_gate * max(G, 1))()
    keep = []
    for i, (name, q0, q1, th, mat) in enumerate(gates):
        arr[i].kind = GATE_KINDS[name]
        arr[i].q0 = int(q0)
        arr[i].q1 = int(q1) if name in _TWO else 0
        arr[i].theta = float(th)
        if mat is not None:
            z = np.asarray(mat, dtype=complex).ravel()
            buf = np.empty(2 * len(z), dtype=np.float64)
            buf[0::2], buf[1::2] = z.real, z.imag
            keep.append(buf)
            arr[i].mat = buf.ctypes.data_as(C.POINTER(C.c_double))
    out = C.c_void_p()
    _check(lib().tqs_circuit_create(int(n), arr, G, C.byref(out)))
    return Handle(out.value, lib().tqs_circuit_destroy)


def circuit(c) -> Handle:
    """tqs_circuit from a tqs_inputs.Circuit."""
    return tqs_circuit_create(c.n, c.gates)


def tqs_circuit_destroy(h: Handle) -> None:
    h.close()


def tqs_noise_model_ex(p1: float, p2: float, pm: float, ad_gamma: float = 0.0, pd_lambda: float = 0.0,
                       t1: float = 0.0, t2: float = 0.0, time_1q: float = 0.0, time_2q: float = 0.0) -> Handle:
    prm = tqs_noise_params(float(p1), float(p2), float(pm), float(ad_gamma), float(pd_lambda), float(t1),
                           float(t2), float(time_1q), float(time_2q))
    out = C.c_void_p()
    _check(lib().tqs_noise_model_ex(C.byref(prm), C.byref(out)))
    return Handle(out, lib().tqs_noise_destroy)


def tqs_noise_model(p1: float, p2: float, pm: float) -> Handle:
    out = C.c_void_p()
    _check(lib().tqs_noise_model(float(p1), float(p2), float(pm), C.byref(out)))
    return Handle(out.value, lib().tqs_noise_destroy)


def tqs_noise_destroy(h: Handle) -> None:
    h.close()


def tqs_options_default() -> tqs_options:
    o = tqs_options()
    lib().tqs_options_default(C.byref(o))
    return o


def options(mode: str = "tree", prec: str = "fp32", part: str = "dcp", arity: Optional[Sequence[int]] = None,
            split: Optional[Sequence[int]] = None, k: int = 0, **kw) -> tqs_options:
    """Build a tqs_options from keywords.  Arrays passed for an explicit tree are
    kept alive on the returned struct."""
    o = tqs_options_default()
    o.mode = {"baseline": TQS_MODE_BASELINE, "tree": TQS_MODE_TREE}[mode]
    o.prec = {"fp64": TQS_FP64, "fp32": TQS_FP32}[prec]
    o.part = {"dcp": TQS_PART_DCP, "ucp": TQS_PART_UCP, "xcp": TQS_PART_XCP,
              "explicit": TQS_PART_EXPLICIT, "learned": TQS_PART_LEARNED}[part]
    o.k = int(k)
    if arity is not None:
        a = np.ascontiguousarray(arity, dtype=np.uint64)
        s = np.ascontiguousarray(split, dtype=np.uint32)
        o._keep = (a, s)
        o.arity = a.ctypes.data_as(C.POINTER(C.c_uint64))
        o.split = s.ctypes.data_as(C.POINTER(C.c_uint32))
        o.k = len(a) - 1
        o.part = TQS_PART_EXPLICIT
    for key, v in kw.items():
        setattr(o, key, v)
    return o


def tqs_partition(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options] = None) -> Tuple[list, list]:
    L = C.c_uint32()
    a = (C.c_uint64 * TQS_MAX_LEVELS)()
    s = (C.c_uint32 * (TQS_MAX_LEVELS + 1))()
    _check(lib().tqs_partition(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None, C.byref(L), a, s))
    return list(a[:L.value]), list(s[:L.value + 1])


def tqs_simulate(c: Handle, nz: Handle, shots: int, seed: int, opts: Optional[tqs_options] = None,
                 n: Optional[int] = None):
    """Returns (counts uint64[2^n] on the host, normalised fidelity, report dict)."""
    if n is None:
        raise ValueError("n (qubit count) is required to size the histogram")
    counts = np.zeros(1 << n, dtype=np.uint64)
    fid = C.c_double()
    rep = tqs_report()
    _check(lib().tqs_simulate(c.ptr, nz.ptr, int(shots), int(seed), C.byref(opts) if opts else None,
                              counts.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(fid), C.byref(rep)))
    return counts, fid.value, rep.as_dict()


def tqs_plan_create(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options] = None) -> Handle:
    out = C.c_void_p()
    _check(lib().tqs_plan_create(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None, C.byref(out)))
    return Handle(out.value, lib().tqs_plan_destroy)


def tqs_plan_execute(plan: Handle, seed: int, d_counts: int, report: bool = False):
    rep = tqs_report() if report else None
    _check(lib().tqs_plan_execute(plan.ptr, int(seed), C.c_void_p(int(d_counts)),
                                  C.byref(rep) if rep is not None else None))
    return rep.as_dict() if rep is not None else None


def tqs_plan_workspace_bytes(plan: Handle) -> int:
    return int(lib().tqs_plan_workspace_bytes(plan.ptr))


def tqs_plan_host_pool_bytes(plan: Handle) -> int:
    return int(lib().tqs_plan_host_pool_bytes(plan.ptr))


def tqs_plan_destroy(plan: Handle) -> None:
    plan.close()


def tqs_debug_node_state(c: Handle, nz: Handle, shots: int, seed: int, opts: Optional[tqs_options],
                         level: int, node: int, n: int) -> np.ndarray:
    out = np.zeros(2 << n, dtype=np.float64)
    _check(lib().tqs_debug_node_state(c.ptr, nz.ptr, int(shots), int(seed), C.byref(opts) if opts else None,
                                      int(level), int(node), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out[0::2] + 1j * out[1::2]


def tqs_debug_node_noise(c: Handle, nz: Handle, shots: int, seed: int, opts: Optional[tqs_options],
                         level: int, node: int, sites: int) -> np.ndarray:
    out = np.zeros(max(sites, 1), dtype=np.uint8)
    _check(lib().tqs_debug_node_noise(c.ptr, nz.ptr, int(shots), int(seed), C.byref(opts) if opts else None,
                                      int(level), int(node), out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out[:sites]


def tqs_debug_plan_order(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options], n_gates: int):
    """Host only.  Returns (order, pass_of, tiles): the gate indices in the order
    the plan applies them, the pass applying each, and each pass's tile (mask of
    physical qubits)."""
    order = np.zeros(max(n_gates, 1), dtype=np.uint32)
    pas = np.zeros(max(n_gates, 1), dtype=np.uint32)
    tiles = np.zeros(max(n_gates, 1) + 64, dtype=np.uint32)
    npass = C.c_uint32()
    u32p = C.POINTER(C.c_uint32)
    _check(lib().tqs_debug_plan_order(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None,
                                      order.ctypes.data_as(u32p), pas.ctypes.data_as(u32p),
                                      tiles.ctypes.data_as(u32p), C.byref(npass)))
    return order[:n_gates], pas[:n_gates], tiles[:npass.value]


def tqs_debug_spec_check(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options]) -> Tuple[int, int]:
    """Host only.  Generates and compiles (NVRTC, not loaded) every specialised
    pass kernel of the plan; returns (kernels, generated source bytes)."""
    nk = C.c_uint32()
    nb = C.c_uint64()
    _check(lib().tqs_debug_spec_check(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None,
                                      C.byref(nk), C.byref(nb)))
    return nk.value, nb.value


def tqs_debug_spec_source(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options], pass_index: int,
                          mode: int) -> str:
    """Host only.  The generated source (layout constants and statements) of one
    pass's specialised kernel in mode 0 (store), 1 (sums) or 2 (sample)."""
    n = C.c_uint64()
    _check(lib().tqs_debug_spec_source(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None,
                                       int(pass_index), int(mode), None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(lib().tqs_debug_spec_source(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None,
                                       int(pass_index), int(mode), buf, n.value + 1, C.byref(n)))
    return buf.value.decode()


def tqs_simulate_static(c: Handle, nz: Handle, shots: int, seed: int, opts: Optional[tqs_options],
                        d_counts: int) -> None:
    """Simulation whose device scratch is the library's static array (no device
    allocation); d_counts is the device address of a 2^n uint64 histogram."""
    _check(lib().tqs_simulate_static(c.ptr, nz.ptr, int(shots), int(seed), C.byref(opts) if opts else None,
                                     C.c_void_p(int(d_counts))))


class Batch(Handle):
    """A tqs_batch plus the handles it was built from (kept alive)."""

    def __init__(self, ptr, keep, sizes):
        super().__init__(ptr, lib().tqs_batch_destroy)
        self._keep = keep
        self.sizes = sizes


def tqs_batch_create(circuits, noises, shots, opts: Optional[tqs_options] = None) -> Batch:
    """circuits, noises: sequences of Handles; shots: sequence of ints."""
    n = len(circuits)
    ca = (C.c_void_p * n)(*[c.ptr for c in circuits])
    na = (C.c_void_p * n)(*[z.ptr for z in noises])
    sa = np.ascontiguousarray(shots, dtype=np.uint64)
    out = C.c_void_p()
    _check(lib().tqs_batch_create(n, ca, na, sa.ctypes.data_as(C.POINTER(C.c_uint64)),
                                  C.byref(opts) if opts else None, C.byref(out)))
    return Batch(out.value, (list(circuits), list(noises)), None)


def tqs_batch_execute(b: Batch, seeds, report: bool = False):
    sa = np.ascontiguousarray(seeds, dtype=np.uint64)
    rep = tqs_report() if report else None
    _check(lib().tqs_batch_execute(b.ptr, sa.ctypes.data_as(C.POINTER(C.c_uint64)),
                                   C.byref(rep) if rep is not None else None))
    return rep.as_dict() if rep is not None else None


def tqs_batch_counts(b: Batch, i: int, n: int) -> np.ndarray:
    out = np.zeros(1 << n, dtype=np.uint64)
    _check(lib().tqs_batch_counts(b.ptr, int(i), out.ctypes.data_as(C.POINTER(C.c_uint64))))
    return out


def tqs_batch_device_counts(b: Batch, i: int) -> int:
    return int(lib().tqs_batch_device_counts(b.ptr, int(i)) or 0)


def tqs_batch_size(b: Batch) -> int:
    return int(lib().tqs_batch_size(b.ptr))


def tqs_batch_destroy(b: Batch) -> None:
    b.close()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def tqs_learned_param_count() -> int:
    return int(lib().tqs_learned_param_count())


def tqs_learned_features(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options] = None):
    """(features float32[40], allowed uint8[20])."""
    f = np.zeros(TQS_LEARNED_FEATURES, dtype=np.float32)
    a = np.zeros(TQS_LEARNED_CLASSES, dtype=np.uint8)
    _check(lib().tqs_learned_features(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None, _fp(f),
                                      a.ctypes.data_as(C.POINTER(C.c_uint8))))
    return f, a


def tqs_learned_candidate(c: Handle, nz: Handle, shots: int, opts: Optional[tqs_options], cls: int):
    L = C.c_uint32()
    a = (C.c_uint64 * TQS_MAX_LEVELS)()
    s = (C.c_uint32 * (TQS_MAX_LEVELS + 1))()
    _check(lib().tqs_learned_candidate(c.ptr, nz.ptr, int(shots), C.byref(opts) if opts else None, int(cls),
                                       C.byref(L), a, s))
    return list(a[:L.value]), list(s[:L.value + 1])


def tqs_learned_train(X, y, epochs: int, batch: int, lr: float, seed: int, init=None):
    X, y = _f32(X), np.ascontiguousarray(y, dtype=np.int32)
    w = np.zeros(tqs_learned_param_count(), dtype=np.float32)
    loss = C.c_float()
    ini = _f32(init) if init is not None else None
    _check(lib().tqs_learned_train(_fp(X), y.ctypes.data_as(C.POINTER(C.c_int32)), len(y), int(epochs), int(batch),
                                   float(lr), int(seed), _fp(ini) if ini is not None else None, _fp(w),
                                   C.byref(loss)))
    return w, float(loss.value)


def tqs_learned_loss_grad(w, X, y):
    w, X, y = _f32(w), _f32(X), np.ascontiguousarray(y, dtype=np.int32)
    g = np.zeros(tqs_learned_param_count(), dtype=np.float32)
    loss = C.c_float()
    _check(lib().tqs_learned_loss_grad(_fp(w), _fp(X), y.ctypes.data_as(C.POINTER(C.c_int32)), len(y),
                                       C.byref(loss), _fp(g)))
    return float(loss.value), g


def tqs_learned_predict(w, X):
    w, X = _f32(w), _f32(X)
    out = np.zeros((X.shape[0], TQS_LEARNED_CLASSES), dtype=np.float32)
    _check(lib().tqs_learned_predict(_fp(w), _fp(X), X.shape[0], _fp(out)))
    return out


def tqs_learned_set_model(w) -> None:
    if w is None:
        _check(lib().tqs_learned_set_model(None))
    else:
        w = _f32(w)
        _check(lib().tqs_learned_set_model(_fp(w)))
