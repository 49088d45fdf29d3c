"""The C-ABI library loads, exports every symbol include/*.h declares, and its
host-side sizing and argument checks behave (no GPU needed, no compute calls)."""
import ctypes as C
import glob
import math
import os
import re

import numpy as np
import pytest

from paper_2102_00104_gb300 import build as B
from paper_2102_00104_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:tt_status|const\s+char\s*\*)\s+(tt_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18, names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(capi.EXPORTED)


def test_status_strings(lib):
    for code in range(8):
        assert capi.tt_status_str(code)
    assert capi.tt_status_str(99) == "unknown status"


def test_query_rejects_bad_arguments(lib):
    n = capi.i64_array([4, 4, 4])
    cb, wb = C.c_size_t(0), C.c_size_t(0)
    assert lib.tt_query(0, n, 2, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query(33, n, 2, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query(3, n, 0, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query(3, n, 2, -1.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query(3, n, 2, 0.0, 7, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    bad = capi.i64_array([4, 0, 4])
    assert lib.tt_query(3, bad, 2, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query(3, n, 2, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_OK
    assert wb.value > 0 and cb.value == 8 * (1 * 4 * 2 + 2 * 4 * 2 + 2 * 4 * 1)


def test_svd_rejects_bad_pointers_before_launch(lib):
    n = capi.i64_array([4, 4])
    cores = capi.ptr_array([0, 0])
    code = lib.tt_svd(None, 0, 2, n, 2, 0.0, cores, None, None, None, None, 0, None)
    assert code == capi.TT_EINVAL
    # misaligned workspace is rejected on the host
    cores = capi.ptr_array([1024, 2048])
    code = lib.tt_svd(C.c_void_p(4096), 0, 2, n, 2, 0.0, cores, None, None, None, C.c_void_p(4097), 1 << 20, None)
    assert code == capi.TT_EINVAL
    # workspace too small
    code = lib.tt_svd(C.c_void_p(4096), 0, 2, n, 2, 0.0, cores, None, None, None, C.c_void_p(4096), 16, None)
    assert code == capi.TT_ENOMEM


def test_core_caps_are_worst_case_ranks(lib):
    caps, stride, count = capi.tt_core_caps(10, [8] * 10, 10)
    # r_k = min(10, 8^k, 8^(10-k)): 8, 10, ..., 10, 8
    r = [1, 8] + [10] * 7 + [8, 1]
    assert caps == [r[i] * 8 * r[i + 1] for i in range(10)]
    assert stride == 80 and count == 80 * 9
    caps, stride, count = capi.tt_core_caps(1, [7], 3)
    assert caps == [7] and count == 0


def test_block_queries(lib):
    assert capi.tt_tsqr_query(1000, 8, 0) > 0
    assert capi.tt_small_svd_query(64) > 0
    wb = C.c_size_t(0)
    assert lib.tt_tsqr_query(0, 8, 0, C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_tsqr_query(10, 513, 0, C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_small_svd_query(0, C.byref(wb)) == capi.TT_EINVAL
    # unfoldings wider than the engine's limit are refused up front
    cb = C.c_size_t(0)
    assert lib.tt_query(3, capi.i64_array([600, 600, 600]), 600, 0.0, 0, C.byref(cb), C.byref(wb)) == capi.TT_ENOTIMPL


def test_tsqr_plans_terminate_for_all_shapes(lib):
    # every (rows, m) the engine accepts gets a TSQR plan that ends in a single R
    for m in (1, 2, 5, 8, 13, 16, 17, 31, 33, 64, 100, 160, 200, 256, 320, 400, 512):
        for rows in (1, 3, 31, 100, 1000, 5000, 65537, 1 << 21, 1 << 27):
            for dt in (capi.TT_F64, capi.TT_F32):
                assert capi.tt_tsqr_query(rows, m, dt) > 0, (rows, m, dt)


def test_plans_survive_out_of_range_tuning_values(lib):
    # tuning keys are user input (TT_TUNE): values outside their range must fall back to a
    # valid plan, never divide by zero or produce an empty grid
    odd = {"tsqr.pcap_q": 0, "tsqr.narrow_cpsm": 0, "tsqr.narrow_k": 7, "tsqr.merge_m": 0,
           "svd.block_nc": 99, "tsqr.colcfg.1": 42, "batched.streams": 0}
    try:
        for k, v in odd.items():
            assert lib.tt_tune_set(k.encode(), v) == capi.TT_OK
        for m in (1, 8, 16, 17, 64, 100, 200, 400):
            for rows in (1, 100, 65537, 1 << 24):
                assert capi.tt_tsqr_query(rows, m, capi.TT_F64) > 0, (rows, m)
        _, wb = capi.tt_query(10, [8] * 10, 10, 0.0, capi.TT_F64)
        assert wb > 0
    finally:
        for k in odd:
            lib.tt_tune_set(k.encode(), -1)


def test_query_paper_configurations(lib):
    for r in (1, 5, 10, 20, 50):
        _, wb = capi.tt_query(10, [8] * 10, r, 0.0, capi.TT_F64)
        assert 0 < wb < 16 << 30
    _, wb = capi.tt_query(10, [8] * 10, 32, 0.0, capi.TT_F32)
    assert 0 < wb < 16 << 30
    _, wb = capi.tt_query(10, [4] * 10, 8, 0.0, capi.TT_F64)
    assert 0 < wb < 1 << 30


def test_batched_and_serve_argument_checks(lib):
    wb = C.c_size_t(0)
    assert lib.tt_batched_query(-1, None, C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_batched_query(0, None, C.byref(wb)) == capi.TT_OK and wb.value == 0
    bad = capi.tt_job()
    bad.d = 0
    assert lib.tt_batched_query(1, C.byref(bad), C.byref(wb)) == capi.TT_EINVAL
    job = capi.tt_job()
    job.d = 3
    for i, n in enumerate((4, 5, 6)):
        job.n[i] = n
    job.r_max = 3
    arr = (capi.tt_job * 2)(job, job)
    assert lib.tt_batched_query(2, arr, C.byref(wb)) == capi.TT_OK
    single = capi.tt_query(3, [4, 5, 6], 3, 0.0, capi.TT_F64)[1]
    assert wb.value >= 2 * single
    assert lib.tt_svd_batched(1, arr, C.c_void_p(4097), 1 << 30, None) == capi.TT_EINVAL
    srv = C.c_void_p(0)
    assert lib.tt_serve_create(0, None, C.byref(srv)) == capi.TT_EINVAL
    bad_policy = capi.tt_serve_opts(4, 0, 1.0, 7, 0.0)  # rejected before any CUDA call
    assert lib.tt_serve_create(1 << 30, C.byref(bad_policy), C.byref(srv)) == capi.TT_EINVAL
    res = capi.tt_job_result()
    assert lib.tt_serve_poll(None, 1, 0, C.byref(res)) == capi.TT_EINVAL
    assert lib.tt_serve_destroy(None) == capi.TT_EINVAL
    assert lib.tt_serve_release(None, 1) == capi.TT_EINVAL
    t = C.c_uint64(0)
    assert lib.tt_serve_submit(None, C.byref(job), None, C.byref(t)) == capi.TT_EINVAL


def test_from_host_argument_checks(lib):
    n = capi.i64_array([4, 5, 6])
    wb = C.c_size_t(0)
    assert lib.tt_query_from_host(3, n, 3, 0.0, capi.TT_F64, -1, C.byref(wb)) == capi.TT_EINVAL
    assert lib.tt_query_from_host(3, n, 3, 0.0, capi.TT_F64, 0, None) == capi.TT_EINVAL
    assert lib.tt_query_from_host(3, n, 3, 0.0, capi.TT_F64, 0, C.byref(wb)) == capi.TT_OK
    # the streamed plan keeps the partial R's of every row block: never smaller than tt_query's
    assert wb.value >= capi.tt_query(3, [4, 5, 6], 3, 0.0, capi.TT_F64)[1]
    cores = capi.ptr_array([4096, 4096, 4096])
    args = (capi.TT_F64, 3, n, 3, 0.0, 0, cores, None, None, None, C.c_void_p(4096), 1 << 20, None, None)
    assert lib.tt_svd_from_host(None, C.c_void_p(4096), *args) == capi.TT_EINVAL
    assert lib.tt_svd_from_host(C.c_void_p(4096), None, *args) == capi.TT_EINVAL
    bad_chunks = list(args)
    bad_chunks[5] = 5000
    assert lib.tt_svd_from_host(C.c_void_p(4096), C.c_void_p(4096), *bad_chunks) == capi.TT_EINVAL
    misaligned = list(args)
    misaligned[10] = C.c_void_p(4097)
    assert lib.tt_svd_from_host(C.c_void_p(4096), C.c_void_p(4096), *misaligned) == capi.TT_EINVAL


def test_tune_overrides_from_environment():
    # TT_TUNE="key=value,..." is applied when the binding loads the library
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2102_00104_gb300 import capi; capi.lib(); "
            "print(capi.lib().tt_tune_set(b'tsmm.oz', 1))")
    env = dict(os.environ, TT_TUNE="tsmm.oz=0, batched.streams=32")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env["TT_TUNE"] = "tsmm.oz"  # no value: refused loudly
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True)
    assert r.returncode != 0


def test_range_rule(lib):
    """The exponent shift of the float-float FP64 form (include/tt_svd.h, tt_range_rule):
    X is read as X 2^-k with max|x| 2^-k in [0.5, 1); the first TSQR level runs again when
    the largest entry it met lies more than 40 binades outside the sample's window."""
    NONE = capi.TT_RANGE_NONE
    # uniform[0,1) data: largest entry in [0.5, 1) -> no shift, no re-run
    assert capi.tt_range_rule(-1, -1) == (0, 0, 0)
    # the definition: 2^e <= max|x| < 2^(e+1)  ->  k = e + 1
    for x in (1.0, 3.0, 1e25, 1e-30, 2.0 ** -1060, 1.7e308):
        e = int(np.floor(np.log2(x)))
        k_try, redo, k = capi.tt_range_rule(e, e)
        assert (k_try, redo, k) == (e + 1, 0, e + 1)
        assert 0.5 <= math.ldexp(x, -k) < 1.0
    # an entry far above the sample: re-run with the shift of the largest entry
    assert capi.tt_range_rule(-1, 40 - 1) == (0, 0, 0)      # 2^39: inside the window
    assert capi.tt_range_rule(-1, 41) == (0, 1, 42)          # 2^41: above it
    assert capi.tt_range_rule(83, 100) == (84, 0, 84)
    # no sample (a strided matrix): tiny data is caught on the other side of the window
    assert capi.tt_range_rule(NONE, -100) == (0, 1, -99)
    assert capi.tt_range_rule(NONE, -30) == (0, 0, 0)
    # nothing nonzero: no shift
    assert capi.tt_range_rule(NONE, NONE) == (0, 0, 0)
    code = lib.tt_range_rule(5000, 0, C.byref(C.c_int()), C.byref(C.c_int()), C.byref(C.c_int()))
    assert code == capi.TT_EINVAL
