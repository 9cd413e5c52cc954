"""ctypes loader of the in-tree C-ABI library ``libgbri.so`` (declared in include/gbri.h).

There is no fallback: if the library is missing or does not load, importing the
binding raises.  Build it with ``python -m paper_1903_04502_gb300.build`` or
``__graft_entry__.build()``.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GBRI_DEBUG_LIB=1 selects the bounds-checked build libgbri_debug.so (build(debug=True))
LIB_PATH = os.path.join(HERE, "libgbri_debug.so" if os.environ.get("GBRI_DEBUG_LIB") == "1" else "libgbri.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ECUFFT, ETIMEOUT, ENONFINITE = -1, -2, -3, -4, -5, -6
ENOTCONV = 1
F32, F64 = 0, 1
PLAN_ORDER = 1
ALGO_PD, ALGO_ADMM, ALGO_FISTA = 0, 1, 2
K_PAD, K_FFT_FWD, K_DEGRID, K_GRID, K_FFT_INV, K_CROP, K_PSI_ADJ, K_PSI, K_UPDATE, K_OTHER = range(10)
K_NAMES = ["pad", "fft_fwd", "degrid", "grid", "fft_inv", "crop", "psi_adjoint", "psi", "update", "other",
           "degrid_grid"]


class PlanDesc(C.Structure):
    _fields_ = [("n_side", C.c_int32), ("oversample", C.c_int32), ("J", C.c_int32),
                ("samples_per_unit", C.c_int32), ("kb_beta", C.c_double), ("M", C.c_int64),
                ("precision", C.c_int32), ("vis_per_run", C.c_int32), ("autotune", C.c_int32),
                ("interp_order", C.c_int32), ("deterministic", C.c_int32),
                ("layout", C.c_int32)]


class SolveParams(C.Structure):
    _fields_ = [("algo", C.c_int32), ("max_iter", C.c_int32), ("rel_tol", C.c_double), ("eps", C.c_double),
                ("gamma", C.c_double), ("op_norm_sq", C.c_double), ("tau", C.c_double), ("sigma1", C.c_double),
                ("sigma2", C.c_double), ("theta", C.c_double), ("rho", C.c_double), ("varrho", C.c_double),
                ("eta", C.c_double), ("dualfb_iters", C.c_int32), ("check_every", C.c_int32),
                ("seed", C.c_uint64), ("n_balls", C.c_int32), ("reserved", C.c_int32)]


class SolveReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("rel_change", C.c_double),
                ("residual_norm", C.c_double), ("op_norm_sq", C.c_double), ("gamma", C.c_double),
                ("ms_total", C.c_double)]


P = C.c_void_p
I32, I64, U32, U64, D = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double

# name -> (restype, argtypes): every symbol declared in include/gbri.h
SIGNATURES = {
    "gbri_plan_create": (I32, [C.POINTER(P), C.POINTER(PlanDesc), P, P]),
    "gbri_plan_destroy": (I32, [P]),
    "gbri_plan_info": (I32, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
    "gbri_plan_launch_config": (I32, [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]),
    "gbri_plan_tap_mode": (I32, [P, C.POINTER(I32)]),
    "gbri_solver_capture": (I32, [P]),
    "gbri_plan_debug_word": (I32, [P, C.POINTER(U32), C.POINTER(I64), I32, P]),
    "gbri_wstack_create": (I32, [P, P, P, I32, D, P]),
    "gbri_wstack_destroy": (I32, [P]),
    "gbri_wstack_info": (I32, [P, C.POINTER(I32), P, P]),
    "gbri_wstack_phi": (I32, [P, P, P, P]),
    "gbri_wstack_phi_adjoint": (I32, [P, P, P, P]),
    "gbri_debug_inject_alloc_failure": (I32, [I32]),
    "gbri_plan_permutation": (I32, [P, P, P]),
    "gbri_vis_reorder": (I32, [P, P, P, I32, P]),
    "gbri_phi": (I32, [P, P, P, U32, P]),
    "gbri_phi_adjoint": (I32, [P, P, P, U32, P]),
    "gbri_op_norm": (I32, [P, I32, D, U64, C.POINTER(D), C.POINTER(I32), P]),
    "gbri_wavelet_create": (I32, [C.POINTER(P), I32, I32, C.POINTER(I32), I32, I32]),
    "gbri_wavelet_destroy": (I32, [P]),
    "gbri_psi": (I32, [P, P, P, P]),
    "gbri_psi_adjoint": (I32, [P, P, P, P]),
    "gbri_prox_l1": (I32, [P, P, I64, D, I32, I32, P]),
    "gbri_prox_l1_weighted": (I32, [P, P, P, I64, D, I32, I32, P]),
    "gbri_proj_l2ball": (I32, [P, P, P, I64, D, P, I32, P]),
    "gbri_proj_l2ball_noalloc": (I32, [P, P, P, I64, D, P, P]),
    "gbri_solver_create": (I32, [C.POINTER(P), P, P, P, C.POINTER(SolveParams), U32, P]),
    "gbri_solver_destroy": (I32, [P]),
    "gbri_solver_step": (I32, [P, I32, P]),
    "gbri_solver_reweight": (I32, [P, D, P]),
    "gbri_solver_get_x": (I32, [P, P, P]),
    "gbri_solver_status": (I32, [P, C.POINTER(I32), C.POINTER(D), P]),
    "gbri_solver_report": (I32, [P, C.POINTER(SolveReport), P]),
    "gbri_solve": (I32, [P, P, P, C.POINTER(SolveParams), P, C.POINTER(SolveReport), U32, P]),
    "gbri_batch_create": (I32, [C.POINTER(P)]),
    "gbri_batch_destroy": (I32, [P]),
    "gbri_batch_add": (I32, [P, P]),
    "gbri_batch_remove": (I32, [P, P]),
    "gbri_batch_size": (I32, [P]),
    "gbri_batch_step": (I32, [P, I32, P]),
    "gbri_batch_set_shared_pass": (I32, [P, I32]),
    "gbri_batch_shared_members": (I32, [P]),
    "gbri_profile_enable": (I32, [I32]),
    "gbri_profile_read": (I32, [I32, C.POINTER(D), C.POINTER(I64)]),
    "gbri_launch_count": (I64, []),
    "gbri_launch_count_reset": (None, []),
    "gbri_last_error": (C.c_char_p, []),
    "gbri_version": (C.c_char_p, []),
}

_lib = None


class GbriError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gbri error %d: %s" % (code, msg))
        self.code = code


def load():
    """Load libgbri.so and bind every declared symbol; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built; run __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code):
    """Raise GbriError for a negative status; return the (non-negative) status otherwise."""
    if code < 0:
        raise GbriError(code, load().gbri_last_error().decode())
    return code
