"""GB300 (sm_103a) implementation of the axisymmetric (r,z) 2D3V
electrostatic particle-in-cell step with Monte-Carlo electron-neutral
collisions of arXiv 2206.14662 (Sec. II.A), behind the C ABI of
include/pic.h.

* ``paper_2206_14662_gb300.build``  -- nvcc build of libpic.so
* ``paper_2206_14662_gb300._capi``  -- ctypes binding (``Simulation``)
* ``paper_2206_14662_gb300.inputs`` -- seeded synthetic workloads

Nothing here loads the CUDA library at import time.
"""
from .inputs import WORKLOADS, seed_particles, workload  # noqa: F401


def Simulation(*args, **kwargs):
    """Create a simulation handle (see ``_capi.Simulation``)."""
    from ._capi import Simulation as _S
    return _S(*args, **kwargs)
