"""ctypes declarations of the C ABI in include/hoscf.h.

Loading fails loudly when the compiled library is missing: the package has
no CPU fallback.  Build it with ``paper_2403_01778_gb300.build.build()``."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_void_p, ctypes.c_size_t)

HOSCF_OK, HOSCF_EINVAL, HOSCF_ENOMEM, HOSCF_ECUDA = 0, 1, 2, 3
HOSCF_NOT_CONVERGED, HOSCF_NONFINITE, HOSCF_TIMEOUT, HOSCF_EUNSUPPORTED = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "NOT_CONVERGED",
                5: "NONFINITE", 6: "TIMEOUT", 7: "EUNSUPPORTED"}

HOSCF_F32, HOSCF_BF16, HOSCF_F8E4M3, HOSCF_F16 = 0, 1, 2, 3
VARIANTS = {"hoscf": 0, "ihoscf": 1, "ihoscf_prev": 2, "jacobi_hopm": 3, "asvd": 4}
MAX_ORDER = 8

# Every entry point the header declares (checked by the ABI test).
EXPORTS = ("hoscf_create", "hoscf_destroy", "hoscf_last_error", "hoscf_opts_default",
           "hoscf_workspace_size", "hoscf_ttvc_blocks", "hoscf_eig_step", "hoscf_rqi_step", "hoscf_solve",
           "hoscf_solve_batched", "hoscf_backward", "hoscf_quantize",
           "hoscf_ttvc_blocks_static", "hoscf_profile_enable", "hoscf_profile_read",
           "hoscf_selftest_timeout", "hoscf_solve_greedy", "hoscf_device_status",
           "hoscf_ttvc_blocks_slab", "hoscf_solve_sharded")


class TensorDesc(ctypes.Structure):
    _fields_ = [("order", c_int), ("dims", ctypes.POINTER(c_int64)), ("dtype", c_int),
                ("data", c_void_p), ("scales", c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("variant", c_int),
                ("eig_tol", c_double), ("eig_max_steps", c_int), ("eig_adapt", c_double),
                ("refine", ctypes.POINTER(TensorDesc)), ("switch_tol", c_double),
                ("timeout_ns", c_int64), ("batch_threads", c_int), ("batch_faces", c_int),
                ("switch_predict", c_int)]


# int reduce(float* H, int64_t count, void* stream, void* user)
REDUCE_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_int64, c_void_p, c_void_p)


class Shard(ctypes.Structure):
    _fields_ = [("row0", c_int64), ("dim0", c_int64), ("reduce", REDUCE_FN), ("user", c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("passes", c_int), ("passes_refine", c_int),
                ("rqi_accepts", c_int), ("resid", c_double), ("resid_4_1", c_double),
                ("sigma_raw", c_double)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libhoscf.so (no implicit build, no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"HOSCF CUDA library not built ({path} missing); "
                           "run paper_2403_01778_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.hoscf_create.argtypes = [P(c_void_p), c_int]
    lib.hoscf_destroy.argtypes = [c_void_p]
    lib.hoscf_last_error.argtypes = [c_void_p]
    lib.hoscf_last_error.restype = ctypes.c_char_p
    lib.hoscf_opts_default.argtypes = [P(Opts)]
    lib.hoscf_workspace_size.argtypes = [c_int, P(c_int64), c_int, P(c_size_t)]
    lib.hoscf_ttvc_blocks.argtypes = [c_void_p, P(TensorDesc), c_void_p, c_void_p, c_void_p]
    lib.hoscf_eig_step.argtypes = [c_void_p, c_int, P(c_int64), c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, P(Opts), c_void_p]
    lib.hoscf_rqi_step.argtypes = [c_void_p, c_int, P(c_int64), c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, P(Opts), c_void_p]
    lib.hoscf_solve.argtypes = [c_void_p, P(TensorDesc), c_void_p, P(Opts), c_void_p,
                                P(c_double), P(Info), c_void_p]
    lib.hoscf_solve_batched.argtypes = [c_void_p, c_int, P(TensorDesc), P(c_void_p), P(Opts),
                                        P(c_void_p), P(c_double), P(Info), c_void_p]
    lib.hoscf_backward.argtypes = [c_void_p, P(TensorDesc), c_void_p, c_double, c_double,
                                   c_void_p, c_void_p, c_void_p]
    lib.hoscf_quantize.argtypes = [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_void_p,
                                   c_void_p]
    lib.hoscf_ttvc_blocks_static.argtypes = [P(TensorDesc), c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hoscf_device_status.argtypes = [c_void_p, c_void_p]
    lib.hoscf_ttvc_blocks_slab.argtypes = [c_void_p, P(TensorDesc), c_int64, c_int64, c_void_p,
                                           c_void_p, c_void_p]
    lib.hoscf_solve_sharded.argtypes = [c_void_p, P(TensorDesc), P(Shard), c_void_p, P(Opts),
                                        c_void_p, P(c_double), P(Info), c_void_p]
    lib.hoscf_profile_enable.argtypes = [c_void_p, c_int]
    lib.hoscf_profile_read.argtypes = [c_void_p, c_int, P(c_int), P(c_double)]
    lib.hoscf_selftest_timeout.argtypes = [c_void_p, c_int, c_int64, c_void_p]
    lib.hoscf_solve_greedy.argtypes = [c_void_p, P(TensorDesc), c_int, c_void_p, P(Opts),
                                       c_void_p, P(c_double), P(Info), P(c_double), c_void_p]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name != "hoscf_last_error":
            f.restype = c_int
    _LIB = lib
    return lib
