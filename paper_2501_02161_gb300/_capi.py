"""ctypes binding of liblbmadj.so: the C-ABI of include/lbmadj.h, same names.

Argument marshalling only; every step of the solve runs in the CUDA library.
Importing this module raises if the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbmadj.so")

LBM_OK, LBM_NOT_CONVERGED = 0, 1
LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA = -1, -2, -3
LBM_ERR_DIVERGED, LBM_ERR_ORDER, LBM_ERR_UNSUPPORTED = -4, -5, -6
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_NOT_CONVERGED", -1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM",
                -3: "LBM_ERR_CUDA", -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_ORDER",
                -6: "LBM_ERR_UNSUPPORTED"}
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16_OFS, LBM_BF16_OFS = 0, 1, 2, 3
LBM_DTYPE_F64, LBM_DTYPE_F32 = 0, 1
LBM_GAMMA_EQ12, LBM_GAMMA_LINEAR = 0, 1
LBM_VEL, LBM_PRES = 2, 3
LBM_ADJOINT_DISCRETE, LBM_ADJOINT_CONTINUOUS = 0, 1
LBM_PHASE_FLOW, LBM_PHASE_TEMPERATURE, LBM_PHASE_FLOW_ADJOINT, LBM_PHASE_TEMPERATURE_ADJOINT = 0, 1, 2, 3


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("gamma_model", ctypes.c_int), ("kappa_f", ctypes.c_double),
                ("k_ratio", ctypes.c_double), ("q_flux", ctypes.c_double),
                ("T0", ctypes.c_double), ("beta_max", ctypes.c_double)]


class lbm_objective(ctypes.Structure):
    _fields_ = [("w_pin", ctypes.c_double), ("w_tmean", ctypes.c_double),
                ("w_qgen", ctypes.c_double)]


class lbm_physics(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("u_ref", ctypes.c_double), ("l_ref", ctypes.c_double),
                ("dp", ctypes.c_double), ("pr", ctypes.c_double), ("rho0", ctypes.c_double),
                ("gamma_model", ctypes.c_int), ("k_ratio", ctypes.c_double),
                ("q_flux", ctypes.c_double), ("T0", ctypes.c_double),
                ("beta_max", ctypes.c_double)]


class lbm_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_steps", ctypes.c_longlong),
                ("check_every", ctypes.c_int), ("reset", ctypes.c_int)]


class lbm_report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("residual", ctypes.c_double),
                ("I", ctypes.c_double), ("J", ctypes.c_double), ("ms", ctypes.c_double),
                ("status", ctypes.c_int)]


class lbm_step_desc(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int), ("storage", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("stride", ctypes.c_longlong),
                ("f_in", ctypes.c_void_p), ("f_out", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("bc", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("sums", ctypes.c_void_p), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("gamma_model", ctypes.c_int)]


# every entry point declared in include/lbmadj.h, with its ctypes signature
_VP, _SZ, _I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
SIGNATURES = {
    "lbm_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, _I, _I, _I]),
    "lbm_destroy": (None, [_VP]),
    "lbm_set_stream": (_I, [_VP, _VP]),
    "lbm_set_flags": (_I, [_VP, _VP, _SZ, _I]),
    "lbm_set_gamma": (_I, [_VP, _VP, _SZ, _I, _I]),
    "lbm_set_bc_values": (_I, [_VP, _VP, _SZ, _I, _I]),
    "lbm_set_params": (_I, [_VP, ctypes.POINTER(lbm_params)]),
    "lbm_set_objective": (_I, [_VP, ctypes.POINTER(lbm_objective)]),
    "lbm_physics_to_params": (_I, [ctypes.POINTER(lbm_physics), ctypes.POINTER(lbm_params)]),
    "lbm_set_physics": (_I, [_VP, ctypes.POINTER(lbm_physics)]),
    "lbm_set_bc": (_I, [_VP, _I, _I, _VP, _SZ, _I, _I]),
    "lbm_set_symmetry": (_I, [_VP, _I]),
    "lbm_set_adjoint_scheme": (_I, [_VP, _I]),
    "lbm_forward": (_I, [_VP, ctypes.POINTER(lbm_solve_opts), ctypes.POINTER(lbm_report)]),
    "lbm_adjoint": (_I, [_VP, ctypes.POINTER(lbm_solve_opts), ctypes.POINTER(lbm_report)]),
    "lbm_solve_phase": (_I, [_VP, _I, ctypes.POINTER(lbm_solve_opts), ctypes.POINTER(lbm_report)]),
    "lbm_sensitivity": (_I, [_VP, _VP, _I, _I]),
    "lbm_get_fields": (_I, [_VP, _VP, _VP, _VP, _I, _I]),
    "lbm_get_objective": (_I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "lbm_get_adjoint": (_I, [_VP, _VP, _VP, _I, _I]),
    "lbm_time_steps": (_I, [_VP, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "lbm_flow_step_noalloc": (_I, [ctypes.POINTER(lbm_step_desc), _VP]),
    "lbm_footprint_bytes": (ctypes.c_size_t, [_I, _I, _I, _I, _I, _I]),
    "lbm_batch_create": (_I, [ctypes.POINTER(_VP), _I, _I, _I, _SZ]),
    "lbm_batch_release": (_I, [_VP, _VP]),
    "lbm_batch_memory": (_I, [_VP, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "lbm_batch_destroy": (None, [_VP]),
    "lbm_batch_admit": (_I, [_VP, _VP, ctypes.POINTER(lbm_solve_opts), ctypes.POINTER(_I)]),
    "lbm_state_bytes": (ctypes.c_size_t, [_VP]),
    "lbm_export_state": (_I, [_VP, _VP, ctypes.c_size_t]),
    "lbm_import_state": (_I, [_VP, _VP, ctypes.c_size_t]),
    "lbm_batch_step": (_I, [_VP, ctypes.POINTER(_I)]),
    "lbm_batch_set_solo_tiles": (_I, [_VP, ctypes.c_longlong]),
    "lbm_batch_poll": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_VP), ctypes.POINTER(lbm_report),
                            _I, ctypes.POINTER(_I)]),
    "lbm_check_addressing": (_I, [_I, _I, _I, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_version": (ctypes.c_char_p, []),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load liblbmadj.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2501_02161_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int, where: str) -> int:
    if code < 0:
        raise LBMError(code, where, lib().lbm_last_error().decode(errors="replace"))
    return code
