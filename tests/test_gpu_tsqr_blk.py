"""The blocked native-FP64 TSQR kernel (compact-WY blocks of eight reflectors, trailing
updates on the tensor cores with FP64-accurate Ozaki splitting), switched on with the
tuning key tsqr.blk64 (on by default), against the oracle's flat-tree Householder TSQR and against what
the R factor must satisfy: R upper triangular, R^T R = W^T W, singular values of W.

Bar: FP64 Householder backward error, 1e-13 of ||W|| (the float-float form is held to
1e-12); column scaling by powers of two up to 2^+-300 commutes with QR."""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from oracle.householder import tsqr_flat
from paper_2102_00104_gb300 import api, capi
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor
from tests.gpu_common import colmajor, ensure_lib, fortran_flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _blk():
    ensure_lib()
    capi.tt_tune_set("tsqr.blk64", 1)  # the default; set in case TT_TUNE turned it off


def sign_fixed(R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return d[:, None] * R


# one panel, a ragged panel, several blocks with a partial last block, all CTAs busy,
# rows < m, and the 2^20 x 64 shape of the benchmark's first level at 1/16 scale
CASES = [(128, 17), (129, 20), (1000, 24), (4096, 33), (20000, 48), (12345, 63), (100000, 64),
         (9, 40), (64, 64), (1 << 20, 64),
         # the 96-row layout for 64 < m <= 80 (the m = 80 steps of an 8^d tensor at r_max = 10)
         (96, 80), (97, 65), (5000, 72), (100000, 80), (30, 80), (1 << 19, 80),
         # the wide layouts (R in a global slice per CTA): 64-row panels up to m = 160,
         # 32-row panels up to 256 and 512 (one CTA per SM)
         (64, 96), (20000, 120), (100000, 160), (65, 161), (3000, 200), (20000, 256),
         (4000, 300), (20000, 400), (2000, 512), (9, 300)]


@pytest.mark.parametrize("rows,m", CASES)
def test_blocked_tsqr_matches_oracle(rows, m):
    rng = np.random.default_rng(rows * 7 + m)
    W = rng.standard_normal((rows, m))
    R = api.tsqr(colmajor(W), arith="f64").cpu().numpy()
    assert np.all(np.tril(R, -1) == 0)
    nw = np.linalg.norm(W)
    assert np.max(np.abs(R.T @ R - W.T @ W)) <= 1e-13 * nw * nw
    s_ref = np.linalg.svd(W, compute_uv=False)
    s_got = np.linalg.svd(R, compute_uv=False)[: len(s_ref)]
    assert np.max(np.abs(s_got - s_ref)) <= 1e-13 * s_ref[0]
    if rows >= m and rows <= 100000:
        Ro = tsqr_flat(W, max(64, m))
        assert np.max(np.abs(sign_fixed(R) - sign_fixed(Ro))) <= 1e-12 * nw


@pytest.mark.parametrize("m,rows", [(64, 300000), (80, 300000), (160, 100000), (256, 30000), (400, 20000)])
def test_blocked_equals_column_kernel(m, rows):
    # the same FP64 Householder sequence with the block transformations on the tensor cores:
    # R agrees with the FP64 panel kernels' R (blocked kernel off) to FP64 rounding
    rng = np.random.default_rng(5)
    W = rng.standard_normal((rows, m)) + 3.0
    Rb = api.tsqr(colmajor(W), arith="f64").cpu().numpy()
    capi.tt_tune_set("tsqr.blk64", 0)
    try:
        Rc = api.tsqr(colmajor(W), arith="f64").cpu().numpy()
    finally:
        capi.tt_tune_set("tsqr.blk64", 1)
    assert np.max(np.abs(sign_fixed(Rb) - sign_fixed(Rc))) <= 1e-13 * np.linalg.norm(W)


@pytest.mark.parametrize("span,m", [(0, 64), (60, 64), (300, 64), (300, 80), (300, 160), (300, 256)])
def test_blocked_tsqr_column_scaling(span, m):
    # W = G 2^s_c: R(W) = R(G) 2^s_c up to row signs, whatever the exponents
    rng = np.random.default_rng(span + 11)
    G = rng.standard_normal((50000, m))
    s = rng.integers(-span, span + 1, size=m) if span else np.zeros(m, dtype=np.int64)
    W = np.ldexp(G, s[None, :])
    R = api.tsqr(colmajor(W), arith="f64").cpu().numpy()
    Rg = np.ldexp(R, -s[None, :])
    Ro = tsqr_flat(G, max(64, m))
    assert np.max(np.abs(sign_fixed(Rg) - sign_fixed(Ro))) <= 1e-12 * np.linalg.norm(G)


def test_blocked_tsqr_rank_deficient_and_zero_columns():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((40000, 64))
    W[:, 5] = 0.0
    W[:, 7] = W[:, 3]
    W[:, 40:48] = W[:, 0:8] @ rng.standard_normal((8, 8))
    W[1000:, 63] = 0.0
    R = api.tsqr(colmajor(W), arith="f64").cpu().numpy()
    assert np.all(np.isfinite(R)) and np.all(np.tril(R, -1) == 0)
    nw = np.linalg.norm(W)
    assert np.max(np.abs(R.T @ R - W.T @ W)) <= 1e-13 * nw * nw
    assert abs(R[5, 5]) <= 1e-13 * nw and abs(R[7, 7]) <= 1e-12 * nw


def test_blocked_tsqr_zero_matrix():
    # a zero column meets the eps_FP guard of Alg. 6 (t = DBL_MIN): |R_jj| = sqrt(2 DBL_MIN)
    R = api.tsqr(torch.zeros(48, 5000, dtype=torch.float64, device="cuda"), arith="f64").cpu().numpy()
    assert np.all(np.isfinite(R)) and np.max(np.abs(R)) <= 1e-150


def run_f64(X, r_max):
    plan = api.TTSVDPlan(X.shape, r_max, 0.0, torch.float64, "f64", want_sigma=True)
    plan.run(fortran_flat(X))
    return plan.result()


@pytest.mark.parametrize("dims,r_max", [((8,) * 7, 8), ((4,) * 9, 6), ((6, 7, 8, 9, 5), 20), ((8,) * 6, 10),
                                        ((8,) * 6, 20), ((8,) * 6, 32), ((8,) * 6, 50)])
def test_tt_svd_native_fp64_with_blocked_tsqr(dims, r_max):
    # the whole native FP64 path with the blocked first levels (unfoldings of 24..400
    # columns), against the Alg. 1 oracle at the FP64 form's bar
    X = uniform_tensor(dims, seed=sum(dims) * r_max)
    res = run_f64(X, r_max)
    ref = O.tt_svd(X, r_max)
    assert res.ranks == ref.ranks
    smax = max(s[0] for s in ref.sigmas.values())
    for i, s in ref.sigmas.items():
        g = res.sigma.get(i)
        if g is None or torch.isnan(g).any():
            continue
        k = ref.ranks[i - 1]
        assert np.max(np.abs(g.cpu().numpy()[:k] - s[:k])) <= 1e-12 * smax
    nx = np.linalg.norm(X)
    err = np.linalg.norm(O.tt_full(res.core_arrays()) - X) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
    assert abs(err - err_ref) <= 1e-12


def test_tt_svd_planted_noise_singular_values():
    # planted TT rank 5 plus 1e-7 noise: the noise singular values (~1e-8 of sigma_max) are
    # resolved by the blocked kernel to FP64 accuracy
    X = planted_tt((8,) * 6, 5, seed=4, noise_rel=1e-7)
    res = run_f64(X, 12)
    ref = O.tt_svd(X, 12)
    assert res.ranks == ref.ranks
    smax = max(s[0] for s in ref.sigmas.values())
    for i, s in ref.sigmas.items():
        g = res.sigma.get(i)
        if g is None or torch.isnan(g).any():
            continue
        k = ref.ranks[i - 1]
        assert np.max(np.abs(g.cpu().numpy()[:k] - s[:k])) <= 1e-13 * smax
