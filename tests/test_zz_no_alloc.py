"""tt_small_svd_noalloc: the small SVD for callers that cannot allocate device memory.

Its scratch is a static device array inside the library instead of a caller
workspace.  This file is collected last on purpose.  The test runs through the
C ABI and compares two calls in a row with tt_small_svd, the entry point that
takes a workspace, at the tolerance of the other small-SVD tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2102_00104_gb300 import api, capi
from tests.gpu_common import ensure_lib

pytestmark = pytest.mark.gpu


def graded_r(m, seed):
    rng = np.random.default_rng(seed)
    U, _, Vt = np.linalg.svd(np.triu(rng.standard_normal((m, m))))
    return np.triu(np.linalg.qr((U * np.logspace(0, -9, m)) @ Vt, mode="r"))


def noalloc_svd(R):
    m = R.shape[0]
    Rc = torch.from_numpy(R.T.copy()).cuda()  # column-major storage of R
    sig = torch.empty(m, dtype=torch.float64, device="cuda")
    V = torch.empty(m, m, dtype=torch.float64, device="cuda")
    capi.tt_small_svd_noalloc(Rc.data_ptr(), m, sig.data_ptr(), V.data_ptr(),
                              int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return sig.cpu().numpy(), V.t().cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    ensure_lib()
    # two calls in a row share the static scratch; the second must not see the first
    for m, seed in ((80, 1), (37, 2)):
        R = graded_r(m, seed)
        sig, V = noalloc_svd(R)
        ref_sig, ref_V = api.small_svd(torch.from_numpy(R).cuda())
        ref_sig, ref_V = ref_sig.cpu().numpy(), ref_V.cpu().numpy()
        assert not np.isnan(sig[0])
        assert np.max(np.abs(sig - ref_sig)) <= 1e-12 * ref_sig[0]
        # same columns up to sign
        signs = np.sign(np.sum(V * ref_V, axis=0))
        assert np.max(np.abs(V * signs - ref_V)) <= 1e-12 * max(m, 10)


def test_noalloc_at_its_size_limit_against_lapack():
    ensure_lib()
    # m = 256 fills the Jacobi working copies of the static scratch exactly; 255 is odd
    for m, seed in ((256, 3), (255, 4)):
        R = graded_r(m, seed)
        ref = np.linalg.svd(R, compute_uv=False)
        for _ in range(2):
            sig, V = noalloc_svd(R)
            assert np.max(np.abs(sig - ref)) <= 1e-12 * ref[0]
            assert np.max(np.abs(V.T @ V - np.eye(m))) <= 1e-13 * m
            # R V has orthogonal columns of norms sigma
            assert np.max(np.abs(np.linalg.norm(R @ V, axis=0) - sig)) <= 1e-12 * ref[0]


def test_noalloc_reports_a_device_failure_as_nan():
    ensure_lib()
    # a non-finite entry cannot give finite singular values: the kernels finish (the
    # Jacobi sweeps are bounded) and the failure shows as sigma[0] = NaN
    R = graded_r(40, 5)
    R[3, 7] = np.nan
    sig, _ = noalloc_svd(R)
    assert np.isnan(sig[0])
    # the next call on a finite matrix is unaffected (the status word is cleared)
    R = graded_r(40, 6)
    sig, _ = noalloc_svd(R)
    assert np.max(np.abs(sig - np.linalg.svd(R, compute_uv=False))) <= 1e-12 * sig[0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    ensure_lib()
    L = capi.lib()
    code = L.tt_small_svd_noalloc(C.c_void_p(256), 257, C.c_void_p(256), C.c_void_p(256), None)
    assert code == capi.TT_EINVAL
    assert "256" in L.tt_last_error().decode()
