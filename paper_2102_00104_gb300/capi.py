"""ctypes binding of libttsvd.so: the C ABI of include/tt_svd.h, argument marshalling only.

Every function here has the name and argument order of the C entry point.  The
library is loaded on first use; if it is missing (not built) loading raises
RuntimeError -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libttsvd.so")

TT_MAX_D = 32
STATUS = {0: "TT_OK", 1: "TT_EINVAL", 2: "TT_ENOMEM", 3: "TT_ECUDA", 4: "TT_ETIMEOUT",
          5: "TT_ENOTIMPL", 6: "TT_ECANCELLED", 7: "TT_ENUMERIC", 8: "TT_EAGAIN"}
(TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_ETIMEOUT, TT_ENOTIMPL, TT_ECANCELLED, TT_ENUMERIC,
 TT_EAGAIN) = range(9)
TT_F64, TT_F32 = 0, 1
TT_ARITH_AUTO, TT_ARITH_DF, TT_ARITH_F64 = 0, 1, 2

# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ["tt_query", "tt_core_caps", "tt_svd", "tt_svd_ex", "tt_last_device_status",
            "tt_tsqr_query", "tt_tsqr", "tt_small_svd_query", "tt_small_svd", "tt_tsmm",
            "tt_gen_uniform", "tt_batched_query", "tt_svd_batched", "tt_serve_create",
            "tt_serve_submit", "tt_serve_poll", "tt_serve_release", "tt_serve_destroy", "tt_status_str",
            "tt_profile", "tt_profile_read", "tt_stats", "tt_last_error", "tt_small_svd_noalloc", "tt_tune_set",
            "tt_query_from_host", "tt_svd_from_host", "tt_query_ex", "tt_range_rule", "tt_fma_rate",
            "tt_wait_selftest", "tt_tsmm_ex", "tt_tsqr_ex"]


class tt_opts(C.Structure):
    _fields_ = [("arith", C.c_int), ("no_elide", C.c_int), ("tsqr_ctas", C.c_int),
                ("thick_m_min", C.c_int), ("thick_f1_min", C.c_double), ("thick_r_est", C.c_int),
                ("two_sided", C.c_int)]


class tt_job(C.Structure):
    _fields_ = [("X", C.c_void_p), ("dtype", C.c_int), ("d", C.c_int),
                ("n", C.c_int64 * TT_MAX_D), ("r_max", C.c_int), ("tol", C.c_double),
                ("cores_out", C.c_void_p * TT_MAX_D), ("ranks_out", C.c_void_p),
                ("sigma_out", C.c_void_p), ("err2_out", C.c_void_p), ("status_out", C.c_void_p)]


class tt_serve_opts(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("arena_bytes", C.c_size_t), ("timeout_s", C.c_double),
                ("policy", C.c_int), ("max_wait_s", C.c_double)]


class tt_job_result(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double)]


class TTError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


_lib = None

_SIGS = {
    "tt_query": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p]),
    "tt_core_caps": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tt_svd": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "tt_svd_ex": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                            C.c_void_p]),
    "tt_query_ex": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "tt_query_from_host": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int,
                                     C.c_void_p]),
    "tt_svd_from_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                   C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "tt_last_device_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tt_tsqr_query": (C.c_int, [C.c_int64, C.c_int, C.c_int, C.c_void_p]),
    "tt_tsqr": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_void_p,
                          C.c_size_t, C.c_void_p]),
    "tt_small_svd_query": (C.c_int, [C.c_int, C.c_void_p]),
    "tt_small_svd": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                               C.c_void_p]),
    "tt_tsmm": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_int,
                          C.c_void_p, C.c_int64, C.c_void_p]),
    "tt_gen_uniform": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_int64, C.c_void_p]),
    "tt_batched_query": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "tt_svd_batched": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "tt_serve_create": (C.c_int, [C.c_size_t, C.c_void_p, C.c_void_p]),
    "tt_serve_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tt_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p]),
    "tt_serve_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "tt_serve_destroy": (C.c_int, [C.c_void_p]),
    "tt_status_str": (C.c_char_p, [C.c_int]),
    "tt_profile": (C.c_int, [C.c_int]),
    "tt_profile_read": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "tt_stats": (C.c_int, [C.c_void_p]),
    "tt_last_error": (C.c_char_p, []),
    "tt_small_svd_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tt_tune_set": (C.c_int, [C.c_char_p, C.c_int]),
    "tt_range_rule": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tt_fma_rate": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "tt_wait_selftest": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "tt_tsqr_ex": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_void_p,
                             C.c_size_t, C.c_int, C.c_void_p]),
    "tt_tsmm_ex": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_int,
                             C.c_void_p, C.c_int64, C.c_int, C.c_void_p]),
}


def lib(path: str | None = None):
    """Load libttsvd.so once (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2102_00104_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    L = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    # layouts chosen by the autotuner on this kind of GPU (tune_table.json), if present,
    # then any overrides from the environment: TT_TUNE="key=value,key=value"
    from . import autotune
    autotune.load()
    for kv in filter(None, os.environ.get("TT_TUNE", "").split(",")):
        key, val = kv.split("=", 1)
        check(L.tt_tune_set(key.strip().encode(), int(val)), "tt_tune_set (TT_TUNE)")
    return L


def check(code: int, where: str) -> None:
    if code != TT_OK:
        detail = ""
        if code == TT_ECUDA and _lib is not None:
            detail = " [" + _lib.tt_last_error().decode() + "]"
        raise TTError(code, where + detail)


def i64_array(vals):
    arr = (C.c_int64 * max(1, len(vals)))(*[int(v) for v in vals])
    return arr


def ptr_array(ptrs):
    return (C.c_void_p * max(1, len(ptrs)))(*[C.c_void_p(int(p)) for p in ptrs])


# ---- same-name wrappers ------------------------------------------------------------------
def tt_query(d, n, r_max, tol, dt):
    cb, wb = C.c_size_t(0), C.c_size_t(0)
    check(lib().tt_query(d, i64_array(n), r_max, tol, dt, C.byref(cb), C.byref(wb)), "tt_query")
    return cb.value, wb.value


def tt_query_ex(d, n, r_max, tol, dt, opts: tt_opts | None = None):
    cb, wb = C.c_size_t(0), C.c_size_t(0)
    check(lib().tt_query_ex(d, i64_array(n), r_max, tol, dt, C.byref(opts) if opts is not None else None,
                            C.byref(cb), C.byref(wb)), "tt_query_ex")
    return cb.value, wb.value


def tt_core_caps(d, n, r_max):
    caps = (C.c_int64 * d)()
    ss, sc = C.c_int64(0), C.c_int64(0)
    check(lib().tt_core_caps(d, i64_array(n), r_max, caps, C.byref(ss), C.byref(sc)), "tt_core_caps")
    return list(caps), ss.value, sc.value


def tt_svd(X_ptr, dt, d, n, r_max, tol, core_ptrs, ranks_ptr, sigma_ptr, err2_ptr, work_ptr,
           work_bytes, stream=0, opts: tt_opts | None = None):
    code = lib().tt_svd_ex(X_ptr, dt, d, i64_array(n), r_max, tol, ptr_array(core_ptrs), ranks_ptr,
                           sigma_ptr, err2_ptr, work_ptr, work_bytes, stream,
                           C.byref(opts) if opts is not None else None)
    check(code, "tt_svd")


def tt_query_from_host(d, n, r_max, tol, dt, chunks=0):
    wb = C.c_size_t(0)
    check(lib().tt_query_from_host(d, i64_array(n), r_max, tol, dt, chunks, C.byref(wb)),
          "tt_query_from_host")
    return wb.value


def tt_svd_from_host(Xh_ptr, Xd_ptr, dt, d, n, r_max, tol, chunks, core_ptrs, ranks_ptr, sigma_ptr,
                     err2_ptr, work_ptr, work_bytes, stream=0, opts: tt_opts | None = None):
    code = lib().tt_svd_from_host(Xh_ptr, Xd_ptr, dt, d, i64_array(n), r_max, tol, chunks,
                                  ptr_array(core_ptrs), ranks_ptr, sigma_ptr, err2_ptr, work_ptr,
                                  work_bytes, stream, C.byref(opts) if opts is not None else None)
    check(code, "tt_svd_from_host")


def tt_last_device_status(work_ptr, stream=0):
    return lib().tt_last_device_status(work_ptr, stream)


def tt_tsqr_query(rows, m, dt):
    wb = C.c_size_t(0)
    check(lib().tt_tsqr_query(rows, m, dt, C.byref(wb)), "tt_tsqr_query")
    return wb.value


def tt_tsqr(W_ptr, dt, rows, m, ld, R_ptr, work_ptr, work_bytes, stream=0):
    check(lib().tt_tsqr(W_ptr, dt, rows, m, ld, R_ptr, work_ptr, work_bytes, stream), "tt_tsqr")


def tt_small_svd_query(m):
    wb = C.c_size_t(0)
    check(lib().tt_small_svd_query(m, C.byref(wb)), "tt_small_svd_query")
    return wb.value


def tt_small_svd(R_ptr, m, sigma_ptr, V_ptr, work_ptr, work_bytes, stream=0):
    check(lib().tt_small_svd(R_ptr, m, sigma_ptr, V_ptr, work_ptr, work_bytes, stream), "tt_small_svd")


def tt_small_svd_noalloc(R_ptr, m, sigma_ptr, V_ptr, stream=0):
    check(lib().tt_small_svd_noalloc(R_ptr, m, sigma_ptr, V_ptr, stream), "tt_small_svd_noalloc")


def tt_tsmm(W_ptr, dt, rows, m, ld, V_ptr, k, Y_ptr, ldy, stream=0):
    check(lib().tt_tsmm(W_ptr, dt, rows, m, ld, V_ptr, k, Y_ptr, ldy, stream), "tt_tsmm")


def tt_gen_uniform(out_ptr, dt, count, seed, start=0, stream=0):
    check(lib().tt_gen_uniform(out_ptr, dt, count, seed, start, stream), "tt_gen_uniform")


def tt_status_str(code):
    return lib().tt_status_str(code).decode()


PROFILE_KINDS = {0: "tsqr_first_level", 1: "tsqr_upper_levels", 2: "svd_of_R", 3: "rank_and_core", 4: "tsmm",
                 5: "input_range", 6: "tsmm_fused_tsqr_first_level"}


def tt_profile(enable: bool):
    check(lib().tt_profile(1 if enable else 0), "tt_profile")


def tt_profile_read(max_records: int = 100000):
    n = C.c_int(0)
    kinds = (C.c_int * max_records)()
    steps = (C.c_int * max_records)()
    ms = (C.c_double * max_records)()
    by = (C.c_double * max_records)()
    fl = (C.c_double * max_records)()
    info = (C.c_int * max_records)()
    check(lib().tt_profile_read(max_records, C.byref(n), kinds, steps, ms, by, fl, info), "tt_profile_read")
    k = min(n.value, max_records)
    return [dict(kind=PROFILE_KINDS[kinds[j]], step=steps[j], ms=ms[j], bytes=by[j], flops=fl[j],
                 info=info[j]) for j in range(k)]


def tt_stats() -> int:
    v = C.c_int64(0)
    check(lib().tt_stats(C.byref(v)), "tt_stats")
    return v.value


# ---- batched and serve forms -------------------------------------------------------------
def tt_batched_query(jobs) -> int:
    arr = (tt_job * max(1, len(jobs)))(*jobs)
    wb = C.c_size_t(0)
    check(lib().tt_batched_query(len(jobs), arr, C.byref(wb)), "tt_batched_query")
    return wb.value


def tt_svd_batched(jobs, work_ptr, work_bytes, stream=0):
    arr = (tt_job * max(1, len(jobs)))(*jobs)
    check(lib().tt_svd_batched(len(jobs), arr, work_ptr, work_bytes, stream), "tt_svd_batched")


TT_SERVE_FIFO, TT_SERVE_SHORTEST = 0, 1


def tt_serve_create(budget_bytes, max_inflight=8, arena_bytes=0, timeout_s=60.0, policy=TT_SERVE_FIFO,
                    max_wait_s=0.0):
    srv = C.c_void_p(0)
    opts = tt_serve_opts(max_inflight, arena_bytes, timeout_s, policy, max_wait_s)
    check(lib().tt_serve_create(budget_bytes, C.byref(opts), C.byref(srv)), "tt_serve_create")
    return srv


def tt_serve_submit(srv, job, ready_stream=0) -> int:
    """Queue a tt_job; its kernels wait for the work queued so far on ready_stream
    (a cudaStream_t as int, 0 = the legacy default stream)."""
    t = C.c_uint64(0)
    check(lib().tt_serve_submit(srv, C.byref(job), ready_stream or None, C.byref(t)), "tt_serve_submit")
    return t.value


def tt_serve_release(srv, ticket) -> int:
    """Forget a finished request; TT_OK, TT_EAGAIN (still running) or TT_EINVAL."""
    return lib().tt_serve_release(srv, ticket)


def tt_serve_poll(srv, ticket, wait=False):
    """(code, tt_job_result); code is TT_OK when done, TT_EAGAIN while running."""
    res = tt_job_result()
    code = lib().tt_serve_poll(srv, ticket, 1 if wait else 0, C.byref(res))
    return code, res


def tt_serve_destroy(srv):
    check(lib().tt_serve_destroy(srv), "tt_serve_destroy")


TT_RANGE_NONE = -100000
FMA_FP32, FMA_FP64, FMA_DF, MMA_FP64 = 0, 1, 2, 3


def tt_fma_rate(kind, stream=0) -> float:
    """Measured multiply-add rate of this GPU in flop/s (2 per multiply-add): FMA_FP32,
    FMA_FP64 or FMA_DF (the lazy float-float multiply-add, FP64-equivalent)."""
    v = C.c_double(0.0)
    check(lib().tt_fma_rate(kind, C.byref(v), stream or None), "tt_fma_rate")
    return v.value


def tt_range_rule(sample_exp, seen_exp):
    """(k_try, redo, k) of the FP64 form's exponent-range rule (see include/tt_svd.h)."""
    a, b, c = C.c_int(0), C.c_int(0), C.c_int(0)
    check(lib().tt_range_rule(sample_exp, seen_exp, C.byref(a), C.byref(b), C.byref(c)), "tt_range_rule")
    return a.value, b.value, c.value


def tt_tune_set(key: str, value: int):
    check(lib().tt_tune_set(key.encode(), int(value)), "tt_tune_set")
