"""Seeded synthetic workload generators shared by the CUDA path's tests/bench and the oracle.

This module only builds gate lists (data).  It holds none of the simulation
arithmetic: no gate matrices, no state vectors, no noise or sampling.  A circuit
is a ``Circuit(n, gates)`` where every gate is a plain tuple
``(name, q0, q1, theta, mat)``:

* ``name``  -- one of ``h x y z s sdg t tdg rx ry rz p cx cz cp swap u1 u2``
* ``q0,q1`` -- qubit indices (``q1 = -1`` for one-qubit gates); for ``cx`` q0 is
  the control, for ``cp``/``cz`` the two qubits are symmetric
* ``theta`` -- rotation / phase angle in radians (0.0 when unused)
* ``mat``   -- ``None`` or, for ``u1``/``u2``, a complex 2x2 / 4x4 numpy array
  in the local basis ``k = bit(q0) + 2*bit(q1)``

Qubit q is bit q of the amplitude index (little-endian).
"""
from .circuits import (  # noqa: F401
    Circuit,
    qft,
    qft_on_basis,
    inverse_qft_on_fourier_state,
    qpe,
    qaoa_maxcut,
    random_regular_graph,
    random_layers,
    ghz,
    batch_circuits_spec,
    splitmix64,
    write_text,
    read_text,
)
