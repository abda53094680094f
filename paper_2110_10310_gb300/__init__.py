"""GB300 (sm_103a) implicit-midpoint Lindblad solver with discrete adjoint.

The compute path is the CUDA library in ``csrc/`` behind the C ABI of
``include/lindblad_gb300.h``; ``_lib`` binds it with ctypes and ``system``
marshals problems into it, with PyTorch supplying device memory and streams.
"""

from .build import LIB_PATH, build  # noqa: F401


def __getattr__(name):
    # lazy: importing the package does not import torch or load the library
    if name in ("LindbladSystem", "LindbladBatch", "LindbladObjective", "objective", "colmajor", "from_colmajor"):
        from . import system

        return getattr(system, name)
    raise AttributeError(name)
