"""Failure detection on the GPU without a fault: a bounded device wait runs out on a flag
that nothing sets, the kernel records the timeout in the status word and returns, the host
reads TT_ETIMEOUT, and the context stays usable for the next TT-SVD."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import capi
from paper_2102_00104_gb300.inputs import uniform_tensor
from tests.gpu_common import ensure_lib
from tests.test_gpu_tt_svd import compare, run_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    ensure_lib()
    L = capi.lib()
    work = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) & ~255
    stream = int(torch.cuda.current_stream().cuda_stream)
    t0 = time.time()
    assert L.tt_wait_selftest(C.c_void_p(wp), 4_000_000, C.c_void_p(stream)) == capi.TT_OK  # ~2 ms
    assert capi.tt_last_device_status(wp, stream) == capi.TT_ETIMEOUT
    assert time.time() - t0 < 5.0
    # argument checks
    assert L.tt_wait_selftest(C.c_void_p(wp + 8), 4_000_000, None) == capi.TT_EINVAL
    assert L.tt_wait_selftest(C.c_void_p(wp), 10, None) == capi.TT_EINVAL
    # the context is still usable
    X = uniform_tensor((4,) * 7, seed=71)
    compare(X, run_gpu(X, 6), O.tt_svd(X, 6), 1e-10)
