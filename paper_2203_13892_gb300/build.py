"""Build libtqs.so in-tree with nvcc for sm_103a (no cmake, no torch extension).

Every translation unit under ``csrc/`` is compiled in parallel to an object in
``_build/`` and linked into ``_build/libtqs.so`` (CUDA runtime linked
statically).  Rebuilds only what is out of date.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtqs.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", OUT]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtqs")


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


# The headers the specialised pass kernels are compiled from at run time (NVRTC),
# embedded into the library as string literals.
JIT_HEADERS = ["internal.h", "device_common.cuh", "pass_kernel.h", "pass_kernel.cuh"]
JIT_INC = os.path.join(OUT, "tqs_jit_sources.inc")


def _write_jit_sources() -> None:
    delim = "tqsjit"
    names, texts = [], []
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if ")" + delim + '"' in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        names.append(f'"{h}"')
        texts.append(f'R"{delim}({text}){delim}"')
    body = ("// generated by build.py from the csrc headers the specialised pass kernels include\n"
            f"static const char *const kJitNames[] = {{{', '.join(names)}}};\n"
            f"static const char *const kJitTexts[] = {{\n" + ",\n".join(texts) + "};\n")
    if not os.path.exists(JIT_INC) or open(JIT_INC).read() != body:
        tmp = JIT_INC + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            f.write(body)
        os.replace(tmp, JIT_INC)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    _write_jit_sources()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_time = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    cc = nvcc()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(OUT, os.path.basename(s) + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            extra = ["-Xptxas", "-v"] if (ptxas_verbose and s.endswith(".cu")) else []
            jobs.append([cc] + ARCH + FLAGS + extra + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose or ptxas_verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return r

    if jobs:
        with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
            list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv))
