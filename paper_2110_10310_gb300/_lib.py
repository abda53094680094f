"""ctypes binding of the C ABI in ``include/lindblad_gb300.h`` (same names).

Argument marshalling only: every step of the method runs in the CUDA library.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_void_p

import importlib

_build = importlib.import_module(__package__ + ".build")

LB_OK = 0
LB_EINVAL = 1
LB_ENOMEM = 2
LB_ECUDA = 3
LB_ENOTCONV = 4
LB_ENAN = 5

LB_J_FROB = 0
LB_J_TR = 1

LB_CKPT_AUTO = -1
LB_PRED_AUTO = -1
LB_PRED_NONE = -2
LB_PREC_F64 = 0
LB_PREC_F32X2 = 1

LB_SWEEP_AUTO = 0
LB_SWEEP_RESIDENT = 1
LB_SWEEP_GRID = 2
LB_SWEEP_CLUSTER = 3

LB_SOLVER_AUTO = 0
LB_SOLVER_JACOBI = 1
LB_SOLVER_NEUMANN = 2
LB_SOLVER_GMRES = 3
LB_J_NM = 2
LB_SYM_NONE = 0
LB_SYM_HERMITIAN = 1
LB_SYM_AUTO = 2

LB_MAX_SUBSYSTEMS = 8
LB_MAX_LEVELS = 64
LB_STATIC_SCRATCH_BYTES = 64 * 1024 * 1024

ERROR_NAMES = {1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ENOTCONV", 5: "LB_ENAN"}


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class lb_system_desc(ctypes.Structure):
    _fields_ = [
        ("Q", c_int32),
        ("levels", POINTER(c_int32)),
        ("essential", POINTER(c_int32)),
        ("detuning_ghz", POINTER(c_double)),
        ("selfkerr_ghz", POINTER(c_double)),
        ("crosskerr_ghz", POINTER(c_double)),
        ("t1_us", POINTER(c_double)),
        ("t2_us", POINTER(c_double)),
        ("T_ns", c_double),
        ("n_steps", c_int64),
    ]


class lb_stats(ctypes.Structure):
    _fields_ = [
        ("state_steps", c_int64),
        ("inner_iterations", c_int64),
        ("max_iterations", c_int32),
        ("kernel_launches", c_int32),
        ("phase_steps", c_int64 * 3),
        ("phase_iterations", c_int64 * 3),
        ("ms_forward", ctypes.c_float),
        ("ms_backward", ctypes.c_float),
        ("sweep", c_int32),
        ("solver", c_int32),
        ("ckpt_every", c_int32),
        ("symmetry", c_int32),
        ("states_integrated", c_int32),
        ("pad", c_int32),
        ("phase_diff_iterations", c_int64 * 3),
    ]


# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "lb_system_create": (c_int32, [POINTER(lb_system_desc), POINTER(c_void_p)]),
    "lb_system_destroy": (None, [c_void_p]),
    "lb_controls_define": (c_int32, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_double)]),
    "lb_controls_set": (c_int32, [c_void_p, POINTER(c_double), c_int64]),
    "lb_controls_set_horizon": (c_int32, [c_void_p, c_double]),
    "lb_states_set": (c_int32, [c_void_p, c_int32, c_void_p, POINTER(c_double)]),
    "lb_objective_set": (c_int32, [c_void_p, c_int32, c_void_p, c_double]),
    "lb_objective_set_gate": (c_int32, [c_void_p, c_int32, c_void_p, c_double]),
    "lb_objective_set_measure": (c_int32, [c_void_p, c_int32, c_double]),
    "lb_objective_set_penalty": (c_int32, [c_void_p, c_double, c_double]),
    "lb_solver_set": (c_int32, [c_void_p, c_int32, c_double, c_int32, c_int32]),
    "lb_set_sweep": (c_int32, [c_void_p, c_int32]),
    "lb_set_symmetry": (c_int32, [c_void_p, c_int32]),
    "lb_set_predictor": (c_int32, [c_void_p, c_int32, c_int32]),
    "lb_set_pairing": (c_int32, [c_void_p, c_int32]),
    "lb_get_predictor": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "lb_set_wait_limit": (c_int32, [c_void_p, c_int64]),
    "lb_set_difference_iterations": (c_int32, [c_void_p, c_int32]),
    "lb_set_precision": (c_int32, [c_void_p, c_int32]),
    "lb_system_set_coupling": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    "lb_workspace_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "lb_bind_workspace": (c_int32, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "lb_forward": (c_int32, [c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    "lb_gradient": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
    "lb_gradient_async": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "lb_optimize": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_double, c_double, POINTER(c_double),
                              POINTER(c_double), POINTER(c_int32), POINTER(c_int32), POINTER(c_double)]),
    "lb_gradient_static": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
    "lb_propagate": (c_int32, [c_void_p, c_void_p, c_int32, c_int64, c_int64, c_void_p, c_int32]),
    "lb_apply": (c_int32, [c_void_p, c_void_p, c_int32, c_int64, c_void_p, c_void_p, c_int32]),
    "lb_get_stats": (c_int32, [c_void_p, POINTER(lb_stats)]),
    "lb_set_timing": (c_int32, [c_void_p, c_int32]),
    "lb_autotune": (c_int32, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "lb_batch_create": (c_int32, [POINTER(c_void_p), c_int32, POINTER(c_void_p)]),
    "lb_batch_destroy": (None, [c_void_p]),
    "lb_batch_workspace_bytes": (c_int32, [c_void_p, POINTER(c_size_t)]),
    "lb_batch_bind_workspace": (c_int32, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "lb_batch_forward": (c_int32, [c_void_p, c_void_p, POINTER(c_double)]),
    "lb_batch_gradient": (c_int32, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
    "lb_batch_capture_graph": (c_int32, [c_void_p, c_void_p, c_int32]),
    "lb_batch_get_stats": (c_int32, [c_void_p, POINTER(lb_stats)]),
    "lb_last_error": (c_char_p, []),
    "lb_version": (c_char_p, []),
}

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load the shared library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(
                f"CUDA library not built ({path} missing); run paper_2110_10310_gb300.build.build() "
                "or __graft_entry__.build()"
            )
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != LB_OK:
        msg = _lib.lb_last_error().decode() if _lib is not None else ""
        raise LBError(rc, msg)


def __getattr__(name):
    # module-level access to the C functions by their ABI names: _lib.lb_forward(...)
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
