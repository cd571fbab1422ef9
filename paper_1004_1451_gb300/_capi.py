"""ctypes declarations of include/bamg.h.  Loading fails loudly when libbamg.so is
missing: there is no other implementation to fall back to."""

from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbamg.so")

BAMG_OK, BAMG_EINVAL, BAMG_ENOTSTOCH, BAMG_ECUDA, BAMG_ENOMEM, BAMG_ENOCONV, BAMG_ETIMEOUT, BAMG_ENUMERIC, \
    BAMG_ESIZE, BAMG_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
COARSEN_GRID, COARSEN_CR = 0, 1
X_GUESS, X_HOST, NORM_L2 = 1, 2, 4
INTERP_LS, INTERP_LEARNED = 0, 1
MLP_F, MLP_H, MLP_S = 112, 128, 16
EXPORT_B, EXPORT_T, EXPORT_P, EXPORT_CF, EXPORT_X, EXPORT_PINV, EXPORT_XINIT, EXPORT_LAMBDA = range(8)

ERROR_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOTSTOCH", -3: "ECUDA", -4: "ENOMEM", -5: "ENOCONV", -6: "ETIMEOUT",
               -7: "ENUMERIC", -8: "ESIZE", -9: "EOVERFLOW"}


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_host", C.c_int32)]


class Mat(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("omega", C.c_double), ("nu_tv", C.c_int32), ("nu_ev", C.c_int32), ("nu_pre", C.c_int32),
                ("nu_post", C.c_int32), ("caliber", C.c_int32), ("z", C.c_int32), ("mmax", C.c_int32),
                ("k_ev", C.c_int32), ("coarse_max", C.c_int32), ("gmres_m", C.c_int32), ("max_it", C.c_int32),
                ("precision", C.c_int32), ("coarsen", C.c_int32), ("grid_nx", C.c_int32), ("grid_ny", C.c_int32),
                ("seed", C.c_uint64), ("tv_lo", C.c_double), ("tv_hi", C.c_double), ("ev_change_tol", C.c_double),
                ("ridge", C.c_double), ("ridge32", C.c_double), ("weight_floor", C.c_double),
                ("cr_theta", C.c_double), ("cr_nu", C.c_int32), ("cr_max_rounds", C.c_int32),
                ("cr_omega", C.c_double), ("stream", C.c_void_p), ("interp", C.c_int32), ("learned_refit", C.c_int32),
                ("model", C.c_void_p), ("learned_rho_max", C.c_double),
                ("device_loop", C.c_int32), ("mle_restart", C.c_int32), ("setup_cycles", C.c_int32),
                ("mu", C.c_int32), ("smoother", C.c_int32), ("persistent", C.c_int32),
                ("coarse_tail", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("restarts", C.c_int32),
                ("true_checks", C.c_int32), ("residual_l1", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("host_waits", C.c_int32), ("mle_restarts", C.c_int32)]


class LevelIn(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("h_row_ptr", C.c_void_p), ("h_col", C.c_void_p),
                ("h_val", C.c_void_p), ("p_nnz", C.c_int32), ("h_p_row_ptr", C.c_void_p),
                ("h_p_col", C.c_void_p), ("h_p_val", C.c_void_p)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
# name -> (restype, argtypes); every symbol declared in include/bamg.h
SIGNATURES = {
    "bamg_default_opts": (_I, [C.POINTER(Opts)]),
    "bamg_setup": (_I, [C.POINTER(Csr), _I, _I, C.POINTER(Opts), C.POINTER(_P)]),
    "bamg_solve": (_I, [_P, _P, _I, _D, C.POINTER(Stats)]),
    "bamg_mle_solve": (_I, [C.POINTER(Csr), _I, _I, C.POINTER(Opts), _D, _I, _I, _P, C.POINTER(Stats), C.POINTER(_P)]),
    "bamg_parnoldi": (_I, [_P, _P, _I, _D, C.POINTER(Stats)]),
    "bamg_free": (None, [_P]),
    "bamg_solve_batch": (_I, [_I, C.POINTER(Csr), C.POINTER(_I), C.POINTER(_I), C.POINTER(Opts), C.POINTER(_P), _I,
                              _D, _I, C.POINTER(Stats)]),
    "bamg_last_error": (C.c_char_p, []),
    "bamg_launch_count": (C.c_uint64, []),
    "bamg_hierarchy_info": (_I, [_P, C.POINTER(_I), _P, _P, C.POINTER(_D)]),
    "bamg_level_export": (_I, [_P, _I, _I, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "bamg_hierarchy_layout": (_I, [_P, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "bamg_import": (_I, [_I, C.POINTER(LevelIn), _P, _P, C.POINTER(Opts), C.POINTER(_P)]),
    "bamg_vcycle_apply": (_I, [_P, _P, _P]),
    "bamg_hierarchy_precision": (_I, [_P]),
    "bamg_smooth_apply": (_I, [_P, _I, _I, _P, _P, _P]),
    "bamg_tv_init": (_I, [_I, _I, _I, _I, _I, C.c_uint64, _D, _D, _P, _P]),
    "bamg_relax": (_I, [_I, C.POINTER(Mat), _P, _P, _I, _I, _I, _D, _I, _P, _P, _P]),
    "bamg_relax_noalloc": (_I, [_I, C.POINTER(Mat), _P, _P, _I, _I, _I, _D, _I, _P, _P]),
    "bamg_tv_weights": (_I, [_I, C.POINTER(Mat), _I, _I, _I, _P, _D, _P, _P, _P]),
    "bamg_coarsen_grid": (_I, [_I, _I, _P, _P, _P]),
    "bamg_coarsen_cr": (_I, [C.POINTER(Mat), _I, C.c_uint64, _D, _I, _D, _I, _P, _P, C.POINTER(_I), C.POINTER(_I),
                             _P]),
    "bamg_interp_ls": (_I, [_I, C.POINTER(Mat), _P, _P, _P, _I, _I, _P, _I, _I, _I, _D, _P, _P, _P, _P]),
    "bamg_galerkin": (_I, [_I, C.POINTER(Mat), _P, _I, _P, _P, _P, _I, _P, _P, _P, _P, C.c_int64,
                           C.POINTER(C.c_int64), _P]),
    "bamg_autotune_report": (_I, [_P, _I]),
    "bamg_coarse_eig": (_I, [_I, _I, _P, _P, _I, _P, _P, _P, C.POINTER(_I), _P, _P]),
    "bamg_interp_features": (_I, [_I, C.POINTER(Mat), _P, _P, _P, _I, _I, _P, _I, _I, _I, _D, _P, _P, _P, _P]),
    "bamg_interp_learned": (_I, [_I, C.POINTER(Mat), _P, _P, _P, _I, _I, _P, _I, _I, _I, _D, _P, _I, _P, _P, _P,
                                 _P]),
    "bamg_model_create": (_I, [C.c_uint64, C.POINTER(_P)]),
    "bamg_model_free": (None, [_P]),
    "bamg_model_param_count": (C.c_int64, []),
    "bamg_model_set": (_I, [_P, _P, C.c_int64]),
    "bamg_model_get": (_I, [_P, _P, C.c_int64]),
    "bamg_model_forward": (_I, [_P, _P, C.c_int64, _P, _P]),
    "bamg_model_gradients": (_I, [_P, _P, _P, C.c_int64, _P, C.POINTER(_D), _P]),
    "bamg_model_train": (_I, [_P, _P, _P, C.c_int64, _I, _I, _D, _P, _P]),
    "bamg_interp_dataset": (_I, [C.POINTER(Csr), _I, _I, C.POINTER(Opts), _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "bamg_vcycle_factor": (_I, [_P, _I, C.POINTER(_D)]),
    "bamg_hierarchy_interp": (_I, [_P, C.POINTER(_D)]),
}

_lib = None


def load():
    """Loads libbamg.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with __graft_entry__.build() "
                           "or python paper_1004_1451_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class BamgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code):
    if code != BAMG_OK:
        raise BamgError(code, load().bamg_last_error().decode())
    return code
