"""ctypes declarations of the C ABI in include/dmeig.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmeig.so")

DM_OK = 0
STATUS = {0: "DM_OK", 1: "DM_ERR_INVALID_ARG", 2: "DM_ERR_NO_CONVERGENCE", 3: "DM_ERR_TIMEOUT",
          4: "DM_ERR_CUDA", 5: "DM_ERR_OOM", 6: "DM_ERR_GEOMETRY"}
PREC = {"f64": 0, "f32": 1, "bf16": 2}


class MGParams(C.Structure):
    _fields_ = [("max_coarse", C.c_int), ("band_sweeps", C.c_int), ("band_brick", C.c_int), ("omega_scale", C.c_double),
                ("power_iters", C.c_int), ("precision", C.c_int), ("autotune", C.c_int),
                ("stencil_shape", C.c_int), ("band_sweeps_coarse", C.c_int), ("symmetric_transform", C.c_int),
                ("dense_coarse", C.c_int), ("krylov_ff", C.c_int), ("jacobi_sweeps", C.c_int)]


class EigParams(C.Structure):
    _fields_ = [("sigma", C.c_double), ("nev", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("proj_tol", C.c_double), ("basis", C.c_int), ("max_restarts", C.c_int),
                ("inner_restart", C.c_int), ("inner_maxit", C.c_int), ("seed", C.c_ulonglong),
                ("mg", MGParams), ("learned", C.c_void_p), ("max_seconds", C.c_double),
                ("rho_tol", C.c_double)]


class EigReport(C.Structure):
    _fields_ = [("n_converged", C.c_int), ("outer_iters", C.c_int), ("restarts", C.c_int),
                ("inner_iters", C.c_int), ("proj_iters", C.c_int), ("mg_levels", C.c_int),
                ("mg_complexity", C.c_double), ("rho_max", C.c_double), ("delta_max", C.c_double),
                ("setup_seconds", C.c_double), ("solve_seconds", C.c_double), ("kernel_launches", C.c_longlong),
                ("learned_applied", C.c_int), ("learned_fallbacks", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("params", EigParams), ("k2_out", C.POINTER(C.c_double)),
                ("b_out", C.c_void_p), ("b_on_device", C.c_int), ("report", EigReport), ("status", C.c_int)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "dm_context_create": (C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    "dm_context_destroy": (None, [_P]),
    "dm_last_error": (C.c_char_p, [_P]),
    "dm_context_launch_count": (C.c_longlong, [_P]),
    "dm_debug_allocation_count": (C.c_longlong, []),
    "dm_trace_enable": (C.c_int, [_P, C.c_int]),
    "dm_trace_count": (C.c_int, [_P]),
    "dm_trace_entry": (C.c_int, [_P, C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double)]),
    "dm_trace_entry_bytes": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "dm_measure_fma_rates": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dm_geometry_create": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     _D, _P, C.c_int, C.c_double, C.POINTER(_P)]),
    "dm_geometry_create_walls": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                           _D, _P, C.c_int, C.c_double, C.POINTER(C.c_int), C.POINTER(_P)]),
    "dm_geometry_create_from_fractions": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                                    C.c_double, _P, _P, _P, C.c_int, C.POINTER(_P)]),
    "dm_geometry_destroy": (None, [_P]),
    "dm_geometry_num_levels": (C.c_int, [_P]),
    "dm_geometry_level_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "dm_geometry_fractions": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int]),
    "dm_mg_params_default": (None, [C.POINTER(MGParams)]),
    "dm_operator_create": (C.c_int, [_P, _P, C.c_double, C.POINTER(MGParams), C.POINTER(_P)]),
    "dm_operator_destroy": (None, [_P]),
    "dm_operator_num_levels": (C.c_int, [_P]),
    "dm_operator_stencil_shape": (C.c_int, [_P, C.c_int]),
    "dm_operator_get_omega": (C.c_double, [_P, C.c_int, C.c_int]),
    "dm_operator_set_omega": (C.c_int, [_P, C.c_int, C.c_int, C.c_double]),
    "dm_operator_apply": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "dm_operator_apply_ff": (C.c_int, [_P, _P, _P, C.c_int]),
    "dm_operator_diagonal": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "dm_operator_apply_noalloc": (C.c_int, [_P, C.c_int, _P, _P]),
    "dm_operator_smooth": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "dm_operator_restrict": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "dm_operator_prolong": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "dm_operator_vcycle": (C.c_int, [_P, _P, _P, C.c_int]),
    "dm_operator_solve": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "dm_operator_project": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.POINTER(C.c_int)]),
    "dm_operator_scalar_vcycle": (C.c_int, [_P, _P, _P, C.c_int]),
    "dm_eig_params_default": (None, [C.POINTER(EigParams)]),
    "dm_eigensolve": (C.c_int, [_P, _P, C.POINTER(EigParams), _D, _P, C.c_int, C.POINTER(EigReport)]),
    "dm_certify": (C.c_int, [_P, _P, C.c_int, _D, _P, C.c_int, _D, _D, _D]),
    "dm_eigensolve_batched": (C.c_int, [_P, C.c_int, C.POINTER(BatchItem), C.c_int]),
    "dm_learned_create": (C.c_int, [_P, C.c_ulonglong, C.POINTER(_P)]),
    "dm_learned_destroy": (None, [_P]),
    "dm_learned_num_params": (C.c_longlong, []),
    "dm_learned_get_weights": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "dm_learned_set_weights": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "dm_learned_apply": (C.c_int, [_P, _P, _P, _P, C.c_int]),
    "dm_learned_loss_grad": (C.c_int, [_P, _P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_float)]),
    "dm_learned_train": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_float, C.c_ulonglong, C.POINTER(C.c_float)]),
    "dm_learned_train_step": (C.c_int, [_P, _P, _P, C.c_int, C.c_float, C.POINTER(C.c_float),
                                        C.POINTER(C.c_float)]),
    "dm_operator_set_learned": (C.c_int, [_P, _P]),
}


def header_symbols(header_path=None):
    """Function names declared in include/dmeig.h."""
    import re
    if header_path is None:
        header_path = os.path.join(os.path.dirname(_HERE), "include", "dmeig.h")
    text = open(header_path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z0-9_]+)\s*\(", text)))


_lib = None


def load(path=None):
    """Load libdmeig.so (fails loudly if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libdmeig.so not found at {p}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
