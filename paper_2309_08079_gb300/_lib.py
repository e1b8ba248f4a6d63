"""ctypes declarations of the C ABI in include/mpcg.h (libmpcg.so).

Argument marshalling only: structs mirror the header field by field and
every entry point keeps its C name.  Loading fails loudly if the library has
not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpcg.so")

# return codes
MPCG_OK = 0
MPCG_EINVAL = -1
MPCG_ECUDA = -2
MPCG_EUNSUPPORTED = -3
MPCG_ETOOLARGE = -4
# status codes (mpcg_stats.status)
MPCG_CONVERGED = 0
MPCG_NOT_CONVERGED = 1
MPCG_BREAKDOWN = 2
MPCG_NONFINITE = 3
MPCG_BADINPUT = 4
MPCG_TIMEOUT = 5
MPCG_INFO_BADINPUT = 1

EXPORTS = (
    "mpcg_version", "mpcg_strerror", "mpcg_create", "mpcg_destroy", "mpcg_workspace_bytes",
    "mpcg_form_schur", "mpcg_form_precon", "mpcg_pcg_solve", "mpcg_recover_step",
    "mpcg_form_schur_batched", "mpcg_form_precon_batched", "mpcg_pcg_solve_batched",
    "mpcg_recover_step_batched", "mpcg_backward_batched", "mpcg_backward",
    "mpcg_backward_batched_noalloc", "mpcg_refine_step", "mpcg_refine_step_batched",
    "mpcg_linearize", "mpcg_linearize_batched", "mpcg_line_search", "mpcg_line_search_batched",
    "mpcg_form_schur_precon", "mpcg_form_schur_precon_batched", "mpcg_selftest_wait",
    "mpcg_selftest_drain", "mpcg_pcg_shape", "mpcg_bench_exchange",
)


class mpcg_dims(C.Structure):
    _fields_ = [("nx", C.c_int), ("nu", C.c_int), ("N", C.c_int), ("dtype", C.c_int)]


class mpcg_lq(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("A", "B", "Qd", "Rd", "q", "r", "c", "Q", "R")]


class mpcg_model(C.Structure):
    _fields_ = [("nx", C.c_int), ("nu", C.c_int), ("dt", C.c_double)] + \
        [(n, C.c_void_p) for n in ("P", "damp", "stiff", "wq", "wr", "wf")]


class mpcg_lq_out(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("A", "B", "Qd", "Rd", "q", "r", "c")]


class mpcg_schur(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Sd", "So", "Pd", "Po", "gamma")] + [("info", C.c_void_p)] + \
        [(n, C.c_void_p) for n in ("Sdp", "Pdp")]


class mpcg_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("tol_mode", C.c_int), ("max_iter", C.c_int),
                ("cluster", C.c_int), ("mode", C.c_int), ("instances", C.c_void_p),
                ("n_instances", C.c_int), ("precon", C.c_int), ("refine", C.c_int),
                ("dot", C.c_int), ("refine_tol", C.c_double)]


class mpcg_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("eta", C.c_double),
                ("relres", C.c_double)]


class mpcg_grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("A", "B", "Qd", "Rd", "q", "r", "c")]


STATS_BYTES = C.sizeof(mpcg_stats)

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libmpcg.so and declare every entry point; raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with paper_2309_08079_gb300.build.build() "
            "(the solve path has no CPU fallback)")
    lib = C.CDLL(path)
    P = C.POINTER
    vp, i32 = C.c_void_p, C.c_int
    lib.mpcg_version.restype = C.c_char_p
    lib.mpcg_version.argtypes = []
    lib.mpcg_strerror.restype = C.c_char_p
    lib.mpcg_strerror.argtypes = [i32]
    lib.mpcg_create.restype = i32
    lib.mpcg_create.argtypes = [P(vp)]
    lib.mpcg_destroy.restype = None
    lib.mpcg_destroy.argtypes = [vp]
    lib.mpcg_workspace_bytes.restype = C.c_size_t
    lib.mpcg_workspace_bytes.argtypes = [mpcg_dims, i32]
    lib.mpcg_form_schur.restype = i32
    lib.mpcg_form_schur.argtypes = [vp, mpcg_dims, P(mpcg_lq), P(mpcg_schur), vp]
    lib.mpcg_form_precon.restype = i32
    lib.mpcg_form_precon.argtypes = [vp, mpcg_dims, P(mpcg_schur), vp]
    lib.mpcg_pcg_solve.restype = i32
    lib.mpcg_pcg_solve.argtypes = [vp, mpcg_dims, P(mpcg_schur), vp, P(mpcg_opts), vp, vp]
    lib.mpcg_recover_step.restype = i32
    lib.mpcg_recover_step.argtypes = [vp, mpcg_dims, P(mpcg_lq), vp, vp, vp, vp]
    lib.mpcg_form_schur_batched.restype = i32
    lib.mpcg_form_schur_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), P(mpcg_schur), vp]
    lib.mpcg_form_precon_batched.restype = i32
    lib.mpcg_form_precon_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_schur), vp]
    lib.mpcg_pcg_solve_batched.restype = i32
    lib.mpcg_pcg_solve_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_schur), vp,
                                           P(mpcg_opts), vp, vp, vp]
    lib.mpcg_recover_step_batched.restype = i32
    lib.mpcg_recover_step_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), vp, vp, vp, vp]
    lib.mpcg_backward_batched.restype = i32
    lib.mpcg_backward_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), P(mpcg_schur), vp, vp,
                                          vp, vp, vp, vp, P(mpcg_grads), P(mpcg_opts), vp, vp, vp]
    lib.mpcg_backward.restype = i32
    lib.mpcg_backward.argtypes = [vp, mpcg_dims, P(mpcg_lq), P(mpcg_schur), vp, vp, vp, vp, vp,
                                  vp, P(mpcg_grads), P(mpcg_opts), vp, vp, vp]
    lib.mpcg_refine_step.restype = i32
    lib.mpcg_refine_step.argtypes = [vp, mpcg_dims, P(mpcg_lq), P(mpcg_schur), vp, P(mpcg_opts), vp,
                                     vp, vp]
    lib.mpcg_refine_step_batched.restype = i32
    lib.mpcg_refine_step_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), P(mpcg_schur), vp,
                                             P(mpcg_opts), vp, vp, vp]
    lib.mpcg_backward_batched_noalloc.restype = i32
    lib.mpcg_backward_batched_noalloc.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), P(mpcg_schur), vp,
                                                  vp, vp, vp, vp, vp, P(mpcg_grads), P(mpcg_opts), vp,
                                                  vp]
    lib.mpcg_form_schur_precon.restype = i32
    lib.mpcg_form_schur_precon.argtypes = [vp, mpcg_dims, P(mpcg_lq), P(mpcg_schur), vp]
    lib.mpcg_form_schur_precon_batched.restype = i32
    lib.mpcg_form_schur_precon_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_lq), P(mpcg_schur), vp]
    lib.mpcg_linearize.restype = i32
    lib.mpcg_linearize.argtypes = [vp, mpcg_dims, P(mpcg_model), vp, vp, vp, vp, P(mpcg_lq_out), vp]
    lib.mpcg_linearize_batched.restype = i32
    lib.mpcg_linearize_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_model), vp, vp, vp, vp,
                                           P(mpcg_lq_out), vp]
    lib.mpcg_line_search.restype = i32
    lib.mpcg_line_search.argtypes = [vp, mpcg_dims, P(mpcg_model), vp, vp, vp, vp, vp, vp, vp,
                                     C.c_double, i32, vp, vp, vp]
    lib.mpcg_line_search_batched.restype = i32
    lib.mpcg_line_search_batched.argtypes = [vp, mpcg_dims, i32, vp, P(mpcg_model), vp, vp, vp, vp,
                                             vp, vp, vp, C.c_double, i32, vp, vp, vp]
    lib.mpcg_selftest_wait.restype = i32
    lib.mpcg_selftest_wait.argtypes = [vp, i32, C.c_double, vp, vp]
    lib.mpcg_selftest_drain.restype = i32
    lib.mpcg_selftest_drain.argtypes = [vp, i32, C.c_double, vp, vp, vp]
    lib.mpcg_pcg_shape.restype = i32
    lib.mpcg_pcg_shape.argtypes = [vp, mpcg_dims, i32, P(mpcg_schur), P(mpcg_opts), P(i32)]
    lib.mpcg_bench_exchange.restype = i32
    lib.mpcg_bench_exchange.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    _lib = lib
    return lib


class MPCGError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = load().mpcg_strerror(code).decode()
        super().__init__(f"{fn} failed: {msg} ({code})")
        self.code = code


def check(fn: str, code: int) -> None:
    if code != MPCG_OK:
        raise MPCGError(fn, code)
