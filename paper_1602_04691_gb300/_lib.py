"""ctypes declarations of the C ABI in include/ori.h (argument marshalling only).

The library is loaded from the package directory, where ``build.py`` puts it.
There is no fallback: if libori.so is missing or fails to load, every entry
point raises.
"""

from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libori.so")

ABI_VERSION = 6   # ORI_ABI_VERSION of include/ori.h that these declarations follow

ORI_OK = 0
ORI_ERR_INVALID_ARG = 1
ORI_ERR_CUDA = 2
ORI_ERR_OOM = 3
ORI_ERR_NOT_CONVERGED = 4
ORI_ERR_BREAKDOWN = 5
ORI_ERR_NONFINITE = 6
ORI_ERR_UNSUPPORTED = 7

ORI_FP64 = 0
ORI_FP32 = 1
ORI_MIXED = 2
ORI_DF = 3
ORI_FORM_A = 0
ORI_FORM_B = 1

# Every symbol include/ori.h declares.
EXPORTS = [
    "ori_default_solve_opts", "ori_default_plan_opts", "ori_plan", "ori_plan_set_medium",
    "ori_plan_destroy", "ori_plan_info", "ori_matvec", "ori_matvec32", "ori_cocg_solve",
    "ori_adjoint_solve", "ori_status_string", "ori_last_error", "ori_abi_version",
    "ori_plan_set_timing", "ori_plan_get_stats", "ori_plan_reset_stats", "ori_matvec_noalloc",
    "ori_cocg_solve_batch", "ori_plan_get_schedule", "ori_plan_set_schedule", "ori_plan_autotune",
    "ori_field", "ori_plan_spectrum_bytes", "ori_plan_save_spectrum", "ori_plan_from_spectrum",
    "ori_plan_residual_history",
]

ORI_SCHED_PERSISTENT = 0
ORI_SCHED_TILES = 1

PASS_NAMES = ["xfwd", "yfwd", "zconv", "yinv", "xinv", "update", "vector", "unused"]
PASS_NAMES = ([k + "_f32" for k in PASS_NAMES] + [k + "_f64" for k in PASS_NAMES]
              + [k + "_df" for k in PASS_NAMES])


class Domain(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("side", C.c_double)]


class PlanOpts(C.Structure):
    _fields_ = [("c_S", C.c_double), ("mem_cap", C.c_size_t), ("n_k", C.c_int),
                ("ks", C.POINTER(C.c_double)), ("min_L", C.c_int), ("lean", C.c_int), ("reserved", C.c_int * 2)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int), ("check_every", C.c_int),
                ("alpha", C.c_double * 3), ("use_graph", C.c_int), ("residual", C.c_int),
                ("resid_update", C.c_int), ("history", C.c_int), ("reserved", C.c_int * 4), ("x0", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("fp64_matvecs", C.c_int),
                ("relres", C.c_double), ("relres_recur", C.c_double), ("status", C.c_int),
                ("ms", C.c_float), ("resid_updates", C.c_int), ("relres_bound", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Schedule(C.Structure):
    _fields_ = [("yfwd", C.c_int), ("zconv", C.c_int), ("ctas_per_sm", C.c_int),
                ("vec_ctas_per_sm", C.c_int), ("yinv", C.c_int), ("yfwd_variant", C.c_int),
                ("zconv_variant", C.c_int), ("yinv_variant", C.c_int)]

    VARIANTS = ("yfwd_variant", "zconv_variant", "yinv_variant")

    def as_dict(self):
        d = {"yfwd": int(self.yfwd), "zconv": int(self.zconv), "yinv": int(self.yinv),
             "ctas_per_sm": int(self.ctas_per_sm), "vec_ctas_per_sm": int(self.vec_ctas_per_sm)}
        for k in self.VARIANTS:
            d[k] = int(getattr(self, k))
        return d

    @classmethod
    def from_dict(cls, d):
        s = cls()
        s.yfwd = int(d["yfwd"])
        s.zconv = int(d["zconv"])
        s.ctas_per_sm = int(d["ctas_per_sm"])
        s.vec_ctas_per_sm = int(d["vec_ctas_per_sm"])
        s.yinv = int(d.get("yinv", 0))
        for k in cls.VARIANTS:
            setattr(s, k, int(d.get(k, 0)))
        return s


class PlanStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("pass_ms", C.c_double * 24),
                ("pass_count", C.c_uint64 * 24), ("fp32_matvecs", C.c_uint64),
                ("fp64_matvecs", C.c_uint64), ("df_matvecs", C.c_uint64),
                ("fp32_bulk_matvecs", C.c_uint64)]

    def as_dict(self):
        return {
            "kernel_launches": int(self.kernel_launches),
            "pass_ms": {PASS_NAMES[i]: float(self.pass_ms[i]) for i in range(24) if self.pass_count[i]},
            "pass_count": {PASS_NAMES[i]: int(self.pass_count[i]) for i in range(24) if self.pass_count[i]},
            "fp32_matvecs": int(self.fp32_matvecs),
            "fp64_matvecs": int(self.fp64_matvecs),
            "df_matvecs": int(self.df_matvecs),
            "fp32_bulk_matvecs": int(self.fp32_bulk_matvecs),
        }


class OriError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def load():
    """Load libori.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    import torch  # noqa: F401  (loads the CUDA runtime first, so the library shares it)
    lib = C.CDLL(LIB_PATH)
    vp, d, i64, i = C.c_void_p, C.c_double, C.c_int64, C.c_int
    lib.ori_default_solve_opts.argtypes = [C.POINTER(SolveOpts)]
    lib.ori_default_solve_opts.restype = None
    lib.ori_default_plan_opts.argtypes = [C.POINTER(PlanOpts)]
    lib.ori_default_plan_opts.restype = None
    lib.ori_plan.argtypes = [i64, d, C.POINTER(Domain), vp, vp, C.POINTER(PlanOpts), vp, C.POINTER(vp)]
    lib.ori_plan.restype = i
    lib.ori_plan_set_medium.argtypes = [vp, vp, vp, vp]
    lib.ori_plan_set_medium.restype = i
    lib.ori_plan_destroy.argtypes = [vp]
    lib.ori_plan_destroy.restype = i
    lib.ori_plan_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_size_t)]
    lib.ori_plan_info.restype = i
    lib.ori_matvec.argtypes = [vp, vp, vp, i, i, vp]
    lib.ori_matvec.restype = i
    lib.ori_matvec32.argtypes = [vp, vp, vp, i, vp]
    lib.ori_matvec32.restype = i
    lib.ori_cocg_solve.argtypes = [vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
    lib.ori_cocg_solve.restype = i
    lib.ori_cocg_solve_batch.argtypes = [vp, i, vp, vp, vp, C.POINTER(SolveOpts), vp, vp]
    lib.ori_cocg_solve_batch.restype = i
    lib.ori_plan_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
    lib.ori_plan_get_schedule.restype = i
    lib.ori_plan_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
    lib.ori_plan_set_schedule.restype = i
    lib.ori_plan_autotune.argtypes = [vp, i, i, C.POINTER(Schedule), C.POINTER(C.c_float), vp]
    lib.ori_plan_autotune.restype = i
    lib.ori_field.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    lib.ori_field.restype = i
    lib.ori_adjoint_solve.argtypes = [vp, vp, vp, vp, vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo), vp]
    lib.ori_adjoint_solve.restype = i
    lib.ori_plan_set_timing.argtypes = [vp, i]
    lib.ori_plan_set_timing.restype = i
    lib.ori_plan_get_stats.argtypes = [vp, C.POINTER(PlanStats)]
    lib.ori_plan_get_stats.restype = i
    lib.ori_plan_reset_stats.argtypes = [vp]
    lib.ori_plan_reset_stats.restype = i
    lib.ori_plan_spectrum_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
    lib.ori_plan_spectrum_bytes.restype = i
    lib.ori_plan_save_spectrum.argtypes = [vp, vp, C.c_size_t, vp]
    lib.ori_plan_save_spectrum.restype = i
    lib.ori_plan_from_spectrum.argtypes = [i64, C.POINTER(Domain), vp, vp, C.POINTER(PlanOpts), vp, C.c_size_t, vp,
                                           C.POINTER(vp)]
    lib.ori_plan_from_spectrum.restype = i
    lib.ori_plan_residual_history.argtypes = [vp, i, vp, i, C.POINTER(i)]
    lib.ori_plan_residual_history.restype = i
    lib.ori_matvec_noalloc.argtypes = [i64, d, C.POINTER(Domain), d, vp, vp, vp, vp, vp]
    lib.ori_matvec_noalloc.restype = i
    lib.ori_status_string.argtypes = [i]
    lib.ori_status_string.restype = C.c_char_p
    lib.ori_last_error.argtypes = []
    lib.ori_last_error.restype = C.c_char_p
    lib.ori_abi_version.argtypes = []
    lib.ori_abi_version.restype = i
    if lib.ori_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{LIB_PATH} has ABI version {lib.ori_abi_version()}, the binding expects "
                           f"{ABI_VERSION}: rebuild it with __graft_entry__.build()")
    _lib = lib
    return lib


def check(status: int, what: str = "ori call"):
    if status != ORI_OK:
        lib = load()
        msg = lib.ori_last_error().decode() or lib.ori_status_string(status).decode()
        raise OriError(status, f"{what}: {msg}")
