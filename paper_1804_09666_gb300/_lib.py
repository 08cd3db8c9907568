"""ctypes declarations of libband's C ABI (include/band.h).

Argument marshalling only: every step of every solve runs in libband's CUDA kernels.
There is no fallback: if libband.so has not been built, loading raises.
"""
import ctypes as ct
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libband.so")

# band_status
OK, ERR_ARG, ERR_CUDA, ERR_ZERO_PIVOT, ERR_SINGULAR, ERR_NONFINITE, ERR_NOT_CONVERGED, \
    ERR_SYMBOLIC_RANGE, ERR_INTERNAL, ERR_WORKSPACE = range(10)
STATUS_NAMES = {OK: "OK", ERR_ARG: "ARG", ERR_CUDA: "CUDA", ERR_ZERO_PIVOT: "ZERO_PIVOT",
                ERR_SINGULAR: "SINGULAR", ERR_NONFINITE: "NONFINITE",
                ERR_NOT_CONVERGED: "NOT_CONVERGED", ERR_SYMBOLIC_RANGE: "SYMBOLIC_RANGE",
                ERR_INTERNAL: "INTERNAL", ERR_WORKSPACE: "WORKSPACE"}
# band_method
NTDM, NPDM, STDM, SPDM, AUTO_NUMERIC, AUTO_SYMBOLIC, MNPDM = range(7)
# band_dtype
F64, F32 = 0, 1
# band_schedule
SCHED_AUTO, SCHED_THREAD, SCHED_TWO_SIDED, SCHED_PARTITIONED, SCHED_GRID = 0, 1, 2, 3, 4
TUNE_JOINT = 1
REFINE_PAIRS = 1
# BAND_OP_*
OP_SOLVE, OP_FACTOR, OP_SIP, OP_REFINE, OP_ADJOINT, OP_DET, OP_ADI, OP_SIP2D = range(8)

EXPORTS = ("band_workspace_size", "band_solve", "band_factor", "band_sip", "band_refine_solve",
           "band_adjoint", "band_status_str", "band_version", "band_fp64_fma_rate",
           "band_solve_batch", "band_solve_static", "band_plan_ragged", "band_autotune",
           "band_autotune_reset", "band_batch_warps", "band_det", "band_adi_step", "band_sip2d",
           "band_refine_solve_ex")
MAX_BATCH = 64


class BandDesc(ct.Structure):
    _fields_ = [("half_bw", ct.c_int32), ("dtype", ct.c_int32), ("nsys", ct.c_int64),
                ("n", ct.c_int64), ("sys_stride", ct.c_int64), ("elem_stride", ct.c_int64),
                ("offsets", ct.c_void_p), ("hbw", ct.c_void_p), ("total_rows", ct.c_int64),
                ("schedule", ct.c_int32), ("chunks", ct.c_int32), ("systems", ct.c_void_p)]


_lib = None
P = ct.c_void_p
DIAG5 = ct.c_void_p * 5


class BandBucket(ct.Structure):
    _fields_ = [("first", ct.c_int64), ("count", ct.c_int64), ("n_max", ct.c_int64),
                ("half_bw", ct.c_int32), ("pad", ct.c_int32)]


class BandProblem(ct.Structure):
    _fields_ = [("op", ct.c_int32), ("method", ct.c_int32), ("desc", ct.POINTER(BandDesc)),
                ("diag", DIAG5), ("f", P), ("x", P), ("sys_status", P), ("ws", P),
                ("ws_bytes", ct.c_size_t), ("tol", ct.c_double), ("max_it", ct.c_int32),
                ("iters", P), ("resid", P)]


def load(path=None):
    """Load libband.so (built by paper_1804_09666_gb300/build.py)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libband.so is not built (%s); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ct.CDLL(path)
    D = ct.POINTER(BandDesc)
    i32, i64, sz, dbl = ct.c_int32, ct.c_int64, ct.c_size_t, ct.c_double
    lib.band_workspace_size.argtypes = [D, i32, i32, i32]
    lib.band_workspace_size.restype = sz
    lib.band_solve.argtypes = [D, i32, P, DIAG5, P, P, P, P, sz, P]
    lib.band_factor.argtypes = [D, i32, DIAG5, P, sz, P, P]
    lib.band_sip.argtypes = [D, DIAG5, P, P, dbl, i32, i32, i32, dbl, P, P, P, P, sz, P]
    lib.band_refine_solve.argtypes = [D, DIAG5, P, P, dbl, i32, P, P, P, sz, P]
    lib.band_refine_solve_ex.argtypes = [D, DIAG5, P, P, dbl, i32, i32, P, P, P, sz, P]
    lib.band_refine_solve_ex.restype = ct.c_int
    lib.band_adjoint.argtypes = [D, i32, P, DIAG5, P, P, DIAG5, P, P, P, sz, P]
    lib.band_det.argtypes = [D, DIAG5, P, P, P, P, sz, P]
    lib.band_adi_step.argtypes = [D, dbl, dbl, P, P, P, P, sz, P]
    lib.band_adi_step.restype = ct.c_int
    lib.band_sip2d.argtypes = [D, i64, DIAG5, P, P, dbl, i32, P, P, P, P, sz, P]
    lib.band_sip2d.restype = ct.c_int
    for name in ("band_solve", "band_factor", "band_sip", "band_refine_solve", "band_adjoint",
                 "band_det"):
        getattr(lib, name).restype = ct.c_int
    lib.band_status_str.argtypes = [i32]
    lib.band_status_str.restype = ct.c_char_p
    lib.band_solve_batch.argtypes = [ct.POINTER(BandProblem), i32, P]
    lib.band_solve_batch.restype = ct.c_int
    lib.band_solve_static.argtypes = [D, i32, DIAG5, P, P, P, P]
    lib.band_solve_static.restype = ct.c_int
    lib.band_plan_ragged.argtypes = [P, P, i32, i64, P, ct.POINTER(BandBucket), i32]
    lib.band_plan_ragged.restype = i32
    lib.band_autotune.argtypes = [ct.POINTER(BandProblem), i32, i32, i32, P, P, P]
    lib.band_autotune.restype = ct.c_int
    lib.band_autotune_reset.argtypes = []
    lib.band_autotune_reset.restype = None
    lib.band_batch_warps.argtypes = [i32]
    lib.band_batch_warps.restype = ct.c_int32
    lib.band_fp64_fma_rate.argtypes = [P, sz, P]
    lib.band_fp64_fma_rate.restype = ct.c_double
    lib.band_version.argtypes = []
    lib.band_version.restype = ct.c_char_p
    if path == LIB_PATH:
        _lib = lib
    return lib


class BandError(RuntimeError):
    pass


def check(code, what):
    if code != OK:
        raise BandError("%s failed: %s" % (what, STATUS_NAMES.get(code, str(code))))
