"""GPU parity of the building blocks (one step of the path each) against the oracle."""
import numpy as np
import pytest
import torch

from oracle.householder import tsqr_flat
from paper_2102_00104_gb300 import api, capi
from paper_2102_00104_gb300.inputs import uniform_f64
from tests.gpu_common import colmajor, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("count,start", [(1, 0), (7, 3), (1000, 0), (4097, 12345), (1 << 20, 1)])
def test_generator_bit_exact(dtype, count, start):
    ref = uniform_f64(11, count, start)
    got = api.gen_uniform(count, 11, dtype, start).cpu().numpy()
    if dtype == torch.float32:
        ref = ref.astype(np.float32)
    assert np.array_equal(got, ref)


def sv(M):
    return np.linalg.svd(M, compute_uv=False)


# m values cover the narrow kernel (<= 16) and the wide one, rows cover ragged
# tails, several panels per warp, several TSQR levels and wide (rows < m) cases
TSQR_CASES = [(1, 1), (37, 1), (1000, 3), (4096, 4), (5000, 5), (70000, 8), (9, 8), (12345, 13),
              (3000, 16), (2049, 17), (20000, 32), (6000, 40), (100000, 64), (3000, 80), (50, 100),
              (5000, 160), (700, 257), (1500, 400), (9, 64), (30, 80), (100, 128)]


@pytest.mark.parametrize("rows,m", TSQR_CASES)
def test_tsqr_fp64_form(rows, m):
    rng = np.random.default_rng(rows * 1000 + m)
    W = rng.standard_normal((rows, m))
    R = api.tsqr(colmajor(W)).cpu().numpy()
    assert np.allclose(np.tril(R, -1), 0)
    # backward error of Householder in ~48-bit arithmetic: singular values to 1e-12 ||W||
    s_ref = sv(W)
    s_got = sv(R)[: len(s_ref)]
    assert np.max(np.abs(s_got - s_ref)) <= 1e-12 * s_ref[0]
    # R^T R = W^T W (closed form) and |R| = |oracle R| up to row signs
    nw2 = np.linalg.norm(W) ** 2
    assert np.max(np.abs(R.T @ R - W.T @ W)) <= 1e-12 * nw2
    if rows <= 20000:
        Ro = tsqr_flat(W, 64)
        k = min(rows, m)
        diag_ok = np.abs(np.abs(np.diag(R)[:k]) - np.abs(np.diag(Ro)[:k])) <= 1e-10 * np.sqrt(nw2)
        assert np.all(diag_ok)


@pytest.mark.parametrize("rows,m", [(1000, 3), (70000, 8), (20000, 32), (100000, 64), (5000, 256)])
def test_tsqr_fp32_form(rows, m):
    rng = np.random.default_rng(rows + m)
    W = rng.standard_normal((rows, m)).astype(np.float32)
    R = api.tsqr(colmajor(W, torch.float32)).cpu().numpy()
    s_ref = sv(W.astype(np.float64))
    s_got = sv(R)[: len(s_ref)]
    assert np.max(np.abs(s_got - s_ref)) <= 2e-5 * s_ref[0]


def test_tsqr_rank_deficient_and_zero_columns():
    rng = np.random.default_rng(7)
    B = rng.standard_normal((30000, 3))
    W = np.hstack([B, np.zeros((30000, 1)), 2.0 * B[:, :1], np.zeros((30000, 1)), B[:, 1:2] - B[:, 2:3]])
    R = api.tsqr(colmajor(W)).cpu().numpy()
    assert np.all(np.isfinite(R))
    s = sv(R)
    s_ref = sv(W)
    assert np.max(np.abs(s - s_ref)) <= 1e-12 * s_ref[0]
    assert np.all(s[3:] <= 1e-12 * s[0])
    Z = api.tsqr(colmajor(np.zeros((1000, 5)))).cpu().numpy()
    assert np.all(np.isfinite(Z)) and np.max(np.abs(Z)) < 1e-15


def _row_signed(R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return R * d[:, None]


# Above the first level, m >= 96 runs the tree of pairwise triangle merges: many
# first-level R's (odd counts on the way up), m off a multiple of 32, FP32 panels
# below FP64-class merges, and the widest m.
@pytest.mark.parametrize("rows,m,dtype", [(30000, 96, torch.float64), (50000, 130, torch.float64),
                                          (120000, 200, torch.float64), (60000, 400, torch.float64),
                                          (20000, 257, torch.float64), (100000, 200, torch.float32),
                                          (12000, 512, torch.float64), (8000, 130, torch.float64),
                                          (6000, 200, torch.float64)])
def test_tsqr_merge_tree(rows, m, dtype):
    rng = np.random.default_rng(rows + 7 * m)
    W = rng.standard_normal((rows, m))
    if dtype == torch.float32:
        W = W.astype(np.float32).astype(np.float64)
    R = api.tsqr(colmajor(W, dtype)).cpu().numpy()
    assert np.all(np.isfinite(R)) and np.allclose(np.tril(R, -1), 0)
    nw2 = np.linalg.norm(W) ** 2
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    assert np.max(np.abs(R.T @ R - W.T @ W)) <= tol * nw2
    s_ref = sv(W)
    assert np.max(np.abs(sv(R) - s_ref)) <= tol * s_ref[0]
    if rows * m <= 1_200_000 and dtype == torch.float64:
        # the oracle's flat Householder R, rows normalised to a positive diagonal
        Ro = tsqr_flat(W, 64)
        assert np.max(np.abs(_row_signed(R) - _row_signed(Ro))) <= 1e-10 * np.sqrt(nw2)


@pytest.mark.parametrize("m,rank", [(64, 10), (80, 10), (128, 7), (32, 3), (200, 12), (400, 9)])
def test_tsqr_low_rank_wide_panels(m, rank):
    # exactly low-rank W: after `rank` reflectors the panel columns hold only rounding
    # noise, which the float-float updates must keep at noise level (no growth, no NaN)
    rng = np.random.default_rng(m + rank)
    W = rng.standard_normal((40000, rank)) @ rng.standard_normal((rank, m))
    R = api.tsqr(colmajor(W)).cpu().numpy()
    assert np.all(np.isfinite(R))
    s, s_ref = sv(R), sv(W)
    assert np.max(np.abs(s - s_ref)) <= 1e-12 * s_ref[0]
    assert np.all(s[rank:] <= 1e-12 * s[0])


@pytest.mark.parametrize("m", [1, 2, 3, 8, 17, 40, 64, 80, 131, 160, 257, 400, 450, 512])
def test_small_svd(m):
    rng = np.random.default_rng(m)
    R = np.triu(rng.standard_normal((m, m)))
    # graded spectrum: singular values from 1 down to 1e-9
    U, _, Vt = np.linalg.svd(R)
    s_planted = np.logspace(0, -9, m)
    R = np.triu(np.linalg.qr((U * s_planted) @ Vt, mode="r"))
    sig, V = api.small_svd(torch.from_numpy(R).cuda())
    sig = sig.cpu().numpy()
    V = V.cpu().numpy()
    s_ref = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(sig - s_ref)) <= 1e-12 * s_ref[0]
    assert np.all(np.diff(sig) <= 0)
    # float-float rotations: orthogonality to ~m * 2^-46
    assert np.max(np.abs(V.T @ V - np.eye(m))) <= 1e-13 * max(m, 10)
    # R V has orthogonal columns of norms sigma (R = U Sigma V^T)
    RV = R @ V
    G = RV.T @ RV
    assert np.max(np.abs(G - np.diag(sig ** 2))) <= 1e-13 * max(m, 10) * s_ref[0] ** 2


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("rows,m,k", [(1, 1, 1), (1000, 8, 1), (5000, 8, 5), (33333, 40, 5),
                                      (4096, 64, 20), (3000, 400, 50), (65536 + 192, 64, 10),
                                      (20001, 80, 10), (12800, 96, 32), (70000, 17, 9)])
def test_tsmm(dtype, tol, rows, m, k):
    rng = np.random.default_rng(rows + m + k)
    W = rng.standard_normal((rows, m))
    if dtype == torch.float32:
        W = W.astype(np.float32).astype(np.float64)
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Y = api.tsmm(colmajor(W, dtype), torch.from_numpy(V).cuda(), k).cpu().numpy().T
    ref = W @ V[:, :k]
    assert np.max(np.abs(Y - ref)) <= tol * np.max(np.abs(W)) * np.sqrt(m)


def test_block_argument_errors():
    with pytest.raises(capi.TTError):
        capi.tt_tsmm(0, 0, 10, 4, 10, 0, 2, 0, 10)
    with pytest.raises(capi.TTError):
        capi.tt_gen_uniform(0, 0, 10, 1)


@pytest.mark.parametrize("m,rank", [(80, 8), (42, 5), (64, 1), (9, 0)])
def test_small_svd_rank_deficient(m, rank):
    # R of a wide unfolding: only `rank` nonzero rows; the zero singular values
    # must not stop the sweeps from converging (device status is checked)
    rng = np.random.default_rng(m + rank)
    R = np.zeros((m, m))
    R[:rank] = np.triu(rng.standard_normal((rank, m)))
    sig, V = api.small_svd(torch.from_numpy(R).cuda())
    sig, V = sig.cpu().numpy(), V.cpu().numpy()
    s_ref = np.linalg.svd(R, compute_uv=False)
    scale = max(s_ref[0], 1.0)
    assert np.max(np.abs(sig - s_ref)) <= 1e-12 * scale
    assert np.max(np.abs(V.T @ V - np.eye(m))) <= 1e-13 * max(m, 10)


@pytest.mark.parametrize("rows,m,k", [(65536 + 128, 64, 10), (20001, 80, 10), (12800, 64, 16),
                                      (70000, 33, 9)])
def test_tsmm_tcgen05(rows, m, k):
    # the tcgen05 form of the tensor-core W V_r (opt-in tuning key "tsmm.tc")
    rng = np.random.default_rng(rows + 7 * m + k)
    W = rng.standard_normal((rows, m))
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    capi.tt_tune_set("tsmm.tc", 1)
    try:
        Y = api.tsmm(colmajor(W, torch.float64), torch.from_numpy(V).cuda(), k).cpu().numpy().T
    finally:
        capi.tt_tune_set("tsmm.tc", 0)
    ref = W @ V[:, :k]
    assert np.max(np.abs(Y - ref)) <= 1e-13 * np.max(np.abs(W)) * np.sqrt(m)
