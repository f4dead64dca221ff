"""CPU oracle for the noisy tree Monte-Carlo hot path (TQSim, arXiv 2203.13892).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  Nothing on the CUDA product path imports,
links or runs anything in this package, and this package imports nothing from
the product package.

Contents
  * ``tqs_oracle.c`` -- FP64 state vector, Philox noise draws, sampling, tree MC
  * ``core``         -- ctypes wrapper around the C file
  * ``partition``    -- DCP / UCP / XCP partitioners and tree arithmetic (Sec. 3.1-3.2, 3.6)
  * ``density``      -- exact density-matrix simulation for n <= 6 (Sec. 2.3.1)
  * ``fidelity``     -- F_s and normalised fidelity F (Sec. 4.1)

Parity status per function is stated in each module header.
"""
from . import core, partition, density, fidelity  # noqa: F401
