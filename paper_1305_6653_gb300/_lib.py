"""ctypes binding of libfde.so (include/fde.h).  Argument marshalling only: every
numerical step runs in the library's CUDA kernels.  There is no CPU fallback; if
the library is missing, loading it raises."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfde.so")

FDE_OK = 0
FDE_ERR_ARG = -1
FDE_ERR_ALLOC = -2
FDE_ERR_CUDA = -3
FDE_ERR_SINGULAR = -4
FDE_ERR_NOT_CONVERGED = -5
FDE_ERR_NAN = -6
FDE_ERR_STATE = -7
FDE_ERR_TIMEOUT = -8

FDE_GBDF, FDE_GAM, FDE_ETR = 1, 2, 3
FDE_FP64, FDE_FP32, FDE_TF32, FDE_BF16, FDE_TF32X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FDE_FP64, "fp32": FDE_FP32, "tf32": FDE_TF32, "bf16": FDE_BF16, "tf32x3": FDE_TF32X3}
FAMILIES = {"GBDF": FDE_GBDF, "GAM": FDE_GAM, "ETR": FDE_ETR}

ERROR_NAMES = {
    FDE_ERR_ARG: "FDE_ERR_ARG", FDE_ERR_ALLOC: "FDE_ERR_ALLOC", FDE_ERR_CUDA: "FDE_ERR_CUDA",
    FDE_ERR_SINGULAR: "FDE_ERR_SINGULAR", FDE_ERR_NOT_CONVERGED: "FDE_ERR_NOT_CONVERGED",
    FDE_ERR_NAN: "FDE_ERR_NAN", FDE_ERR_STATE: "FDE_ERR_STATE", FDE_ERR_TIMEOUT: "FDE_ERR_TIMEOUT",
}

# Every symbol declared in include/fde.h (checked by the CPU tests).
EXPORTED = [
    "fde_problem_create", "bvm_assemble", "strang_precond_factor", "fde_factor_storage", "bccb_precond_setup",
    "fde_precond_none",
    "pgmres_solve",
    "fde_problem_destroy",
    "fde_last_error", "fde_matvec", "fde_matvec_fp32", "fde_precond_apply", "fde_get_rhs", "fde_get_factor_block",
    "fde_get_grunwald", "fde_problem_sizes", "fde_profile_enable", "fde_profile_select", "fde_profile_read", "fde_launch_count",
    "fde_release_cached_memory", "fde_tune_set", "fde_tune_cache", "fde_tune_query",
    "fde_precond_apply_noalloc", "fde_batch_create", "fde_batch_share_operator", "fde_batch_block_solver",
    "fde_batch_assemble",
    "fde_batch_factor",
    "fde_batch_solve", "fde_batch_size", "fde_batch_problem", "fde_batch_destroy",
    "fde_nop_create", "fde_nop_num_params", "fde_nop_in_channels", "fde_nop_set_params", "fde_nop_get_params",
    "fde_nop_forward", "fde_nop_loss_grad", "fde_nop_adam_step", "fde_nop_features", "fde_nop_warm_start",
    "fde_nop_destroy", "fde_nop_coefficients", "fde_nop_synthesize",
]
FDE_TUNE_MATVEC, FDE_TUNE_TRSV, FDE_TUNE_LU = 0, 1, 2
BLOCK_SOLVERS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}
STORAGES = {"fp32": 0, "bf16": 1}
STAGES = ["assemble", "form", "lu_diag", "lu_panel", "lu_update", "tfft_fwd", "trsv", "tfft_inv", "matvec",
          "krylov", "lu_tc", "lu_pack", "lu_panel_tc"]


class FdeProblemDesc(C.Structure):
    _fields_ = [
        ("m", C.c_int), ("s", C.c_int), ("alpha", C.c_double), ("xL", C.c_double), ("xR", C.c_double),
        ("t0", C.c_double), ("T", C.c_double), ("dplus", C.c_void_p), ("dminus", C.c_void_p),
        ("dplus_c", C.c_double), ("dminus_c", C.c_double), ("family", C.c_int), ("mu", C.c_int),
        ("u0", C.c_void_p), ("f", C.c_void_p), ("device_ptrs", C.c_int),
        ("dplus_t", C.c_void_p), ("dminus_t", C.c_void_p),
    ]


class FdePgmresOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int), ("reorth", C.c_int),
                ("matvec_precision", C.c_int), ("relax", C.c_double)]


class FdeStats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int), ("precision", C.c_int),
        ("rel_residual", C.c_double), ("rel_residual_estimate", C.c_double), ("ms_solve", C.c_double),
        ("x0_rejected", C.c_int), ("matvecs_fp32", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class FdeError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libfde.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, f64 = C.c_void_p, C.c_int, C.c_double
    sig = {
        "fde_problem_create": (i32, [C.POINTER(FdeProblemDesc), vp, C.POINTER(vp)]),
        "bvm_assemble": (i32, [vp]),
        "strang_precond_factor": (i32, [vp, i32]),
        "fde_factor_storage": (i32, [vp, i32]),
        "bccb_precond_setup": (i32, [vp, i32, i32]),
        "fde_precond_none": (i32, [vp]),
        "pgmres_solve": (i32, [vp, C.POINTER(FdePgmresOpts), vp, vp, C.POINTER(FdeStats)]),
        "fde_problem_destroy": (None, [vp]),
        "fde_last_error": (C.c_char_p, []),
        "fde_matvec": (i32, [vp, vp, vp]),
        "fde_matvec_fp32": (i32, [vp, vp, vp]),
        "fde_precond_apply": (i32, [vp, vp, vp]),
        "fde_get_rhs": (i32, [vp, vp]),
        "fde_get_factor_block": (i32, [vp, i32, vp, vp]),
        "fde_get_grunwald": (i32, [vp, vp]),
        "fde_problem_sizes": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "fde_profile_enable": (i32, [vp, i32]),
        "fde_profile_select": (i32, [vp, C.c_uint]),
        "fde_profile_read": (i32, [vp, i32, C.POINTER(f64), C.POINTER(i32)]),
        "fde_launch_count": (C.c_longlong, []),
        "fde_release_cached_memory": (C.c_int, []),
        "fde_tune_set": (i32, [i32, i32]),
        "fde_tune_cache": (i32, [C.c_char_p]),
        "fde_tune_query": (i32, [i32, i32, i32, i32, C.POINTER(i32)]),
        "fde_precond_apply_noalloc": (i32, [vp, vp, vp]),
        "fde_batch_create": (i32, [C.POINTER(FdeProblemDesc), i32, vp, C.POINTER(vp)]),
        "fde_batch_assemble": (i32, [vp]),
        "fde_batch_factor": (i32, [vp, i32]),
        "fde_batch_share_operator": (i32, [vp]),
        "fde_batch_block_solver": (i32, [vp, i32]),
        "fde_batch_solve": (i32, [vp, C.POINTER(FdePgmresOpts), C.POINTER(vp), C.POINTER(FdeStats)]),
        "fde_batch_size": (i32, [vp]),
        "fde_batch_problem": (vp, [vp, i32]),
        "fde_batch_destroy": (None, [vp]),
        "fde_nop_create": (i32, [i32, i32, i32, i32, i32, i32, C.c_ulonglong, vp, C.POINTER(vp)]),
        "fde_nop_num_params": (C.c_longlong, [vp]),
        "fde_nop_in_channels": (i32, [vp]),
        "fde_nop_set_params": (i32, [vp, vp]),
        "fde_nop_get_params": (i32, [vp, vp]),
        "fde_nop_forward": (i32, [vp, vp, vp, i32]),
        "fde_nop_loss_grad": (i32, [vp, vp, vp, i32, C.POINTER(f64), vp]),
        "fde_nop_adam_step": (i32, [vp, C.c_float]),
        "fde_nop_features": (i32, [vp, vp, vp]),
        "fde_nop_warm_start": (i32, [vp, vp, vp]),
        "fde_nop_destroy": (None, [vp]),
        "fde_nop_coefficients": (i32, [vp, vp, vp]),
        "fde_nop_synthesize": (i32, [vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().fde_last_error().decode()


def check(code: int, where: str) -> int:
    if code != FDE_OK:
        raise FdeError(code, where, last_error())
    return code
