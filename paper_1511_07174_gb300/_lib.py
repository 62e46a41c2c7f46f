"""ctypes view of the C ABI in include/gbla.h (argument marshalling only).

The shared library is the in-tree build (paper_1511_07174_gb300/libgbla.so).
Loading fails loudly when it is missing: there is no fallback path.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbla.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbla.h")

GBLA_PREC = {"fp32": 1, "tf32": 2, "bf16": 3, "fp16": 4, "fp16x3": 5, "bf16x3": 6}
GBLA_INFO_TIMEOUT = -1000
KERNEL_KINDS = ["panel", "laswp", "trsm", "gemm_simt", "gemm_tc", "convert", "trsv", "matvec", "mgs",
                "gmres_update", "permute", "copy", "batched"]
GBLA_ERR_NOT_CONVERGED = 1004

_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
_d = ctypes.c_double


class GmresirOpts(ctypes.Structure):
    _fields_ = [("tol", _d), ("inner_tol", _d), ("max_outer", _i), ("restart_m", _i),
                ("restarts", _i)]


class GmresirStats(ctypes.Structure):
    _fields_ = [("outer", _i), ("inner", _i), ("converged", _i), ("beta", _d), ("beta0", _d)]


class KrylovOpts(ctypes.Structure):
    _fields_ = [("tol", _d), ("max_iter", _i), ("restart_m", _i)]


class KrylovStats(ctypes.Structure):
    _fields_ = [("iterations", _i), ("converged", _i), ("breakdown", _i), ("pad", _i),
                ("relres", _d)]


_SIGS = {
    "gbla_version": ([], ctypes.c_char_p),
    "gbla_status_string": ([_i], ctypes.c_char_p),
    "gbla_last_error": ([], ctypes.c_char_p),
    "gbla_set_wait_timeout_ns": ([ctypes.c_uint64], None),
    "gbla_launch_count": ([], ctypes.c_uint64),
    "gbla_kernel_kind_name": ([_i], ctypes.c_char_p),
    "gbla_prof_enable": ([ctypes.c_uint], None),
    "gbla_prof_reset": ([], None),
    "gbla_prof_read": ([_i, ctypes.POINTER(_i), ctypes.POINTER(_d)], _i),
    "gbla_get_wait_timeout_ns": ([], ctypes.c_uint64),
    "gbla_prof_list": ([_i, _i, ctypes.POINTER(_d)], _i),
    "gbla_fma_peak": ([_i, _i, ctypes.POINTER(_d), _vp], _i),
    "gbla_set_substitution_ctas": ([_i], _i),
    "gbla_get_substitution_ctas": ([], _i),
    "gbla_set_lookahead": ([_i], _i),
    "gbla_get_lookahead": ([], _i),
    "gbla_lu_factor_workspace": ([_i, _i], _sz),
    "gbla_lu_factor": ([_i, _vp, _i, _vp, _vp, _i, _vp, _sz, _vp], _i),
    "gbla_lu_factor_static": ([_i, _vp, _i, _vp, _vp, _i, _vp], _i),
    "gbla_lu_solve_workspace": ([_i, _i], _sz),
    "gbla_lu_solve": ([_i, _i, _i, _vp, _i, _vp, _vp, _i, _vp, _vp, _sz, _vp], _i),
    "gbla_chol_factor": ([_i, _vp, _i, _vp, _i, _vp], _i),
    "gbla_chol_solve_workspace": ([_i, _i], _sz),
    "gbla_chol_solve": ([_i, _i, _vp, _i, _vp, _i, _vp, _vp, _sz, _vp], _i),
    "gbla_lu_factor_mixed_workspace": ([_i, _i, _i], _sz),
    "gbla_lu_factor_mixed": ([_i, _vp, _i, _vp, _i, _vp, _vp, _i, _i, _vp, _sz, _vp], _i),
    "gbla_gmresir_workspace": ([_i, _i], _sz),
    "gbla_gmresir_solve": ([_i, _vp, _i, _vp, _i, _vp, _vp, _vp, ctypes.POINTER(GmresirOpts),
                            ctypes.POINTER(GmresirStats), _vp, _sz, _vp], _i),
    "gbla_gmresir_solve_nrhs": ([_i, _i, _vp, _i, _vp, _i, _vp, _vp, _i, _vp, _i,
                                 ctypes.POINTER(GmresirOpts), ctypes.POINTER(GmresirStats), _vp, _sz,
                                 _vp], _i),
    "gbla_chol_factor_mixed_workspace": ([_i, _i, _i], _sz),
    "gbla_chol_factor_mixed": ([_i, _vp, _i, _vp, _i, _vp, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_gmresir_solve_nrhs": ([_i, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _i,
                                      ctypes.POINTER(GmresirOpts), ctypes.POINTER(GmresirStats), _vp,
                                      _sz, _vp], _i),
    "gbla_krylov_workspace": ([_i, _i], _sz),
    "gbla_gmres_solve": ([_i, _vp, _i, _vp, _vp, _vp, _i, _vp, ctypes.POINTER(KrylovOpts),
                          ctypes.POINTER(KrylovStats), _vp, _sz, _vp], _i),
    "gbla_bicgstab_solve": ([_i, _vp, _i, _vp, _vp, _vp, _i, _vp, ctypes.POINTER(KrylovOpts),
                             ctypes.POINTER(KrylovStats), _vp, _sz, _vp], _i),
    "gbla_lu_batched_workspace": ([_i], _sz),
    "gbla_lu_solve_batched": ([_i] + [_vp] * 9 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_lu_solve_batched_f32": ([_i] + [_vp] * 9 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_lu_factor_batched": ([_i] + [_vp] * 6 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_lu_factor_batched_f32": ([_i] + [_vp] * 6 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_lu_solve_factored_batched": ([_i] + [_vp] * 8 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_lu_solve_factored_batched_f32": ([_i] + [_vp] * 8 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_factor_batched": ([_i] + [_vp] * 5 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_factor_batched_f32": ([_i] + [_vp] * 5 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_solve_factored_batched": ([_i] + [_vp] * 7 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_solve_factored_batched_f32": ([_i] + [_vp] * 7 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_batched_workspace": ([_i], _sz),
    "gbla_chol_solve_batched": ([_i] + [_vp] * 8 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_chol_solve_batched_f32": ([_i] + [_vp] * 8 + [_i, _i, _i, _vp, _sz, _vp], _i),
    "gbla_rank_k_update": ([_i, _i, _i, _d, _vp, _i, _vp, _i, _d, _vp, _i, _vp], _i),
    "gbla_backward_error_workspace": ([_i, _i], _sz),
    "gbla_backward_error": ([_i, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _vp, _sz, _vp], _i),
}

_lib = None


def header_symbols():
    """Names of the functions include/gbla.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbla_[a-z0-9_]+)\s*\(", text)))


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgbla.so is not built (python -m paper_1511_07174_gb300.build); "
                               "there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def status_string(rc):
    return load().gbla_status_string(int(rc)).decode()
