"""GB300-native Godunov hydrodynamics step (arXiv:2501.02317, Sec. 3).

* ``workloads`` -- seeded synthetic initial states (no method arithmetic)
* ``khydro``    -- ctypes binding of libkhydro.so (the CUDA library)
* ``build``     -- nvcc build of libkhydro.so for sm_103a
"""
from . import workloads  # noqa: F401

__all__ = ["workloads"]
