"""End-to-end GPU parity of tt_svd (Alg. 2 on the device) against the Alg. 1 oracle.

Bar (FP64 form): ranks bit-exact; kept singular values of every computed step
within 1e-10 * sigma_max; relative reconstruction error within 1e-10 of the
oracle's; discarded energy within 1e-10 ||X||^2; cores 2..d orthonormal.
FP32 form: the same at 1e-5, against the oracle run on the FP32 values widened
to FP64 (and the error against the FP64 tensor is reported by the bench).
"""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import api
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor
from tests.gpu_common import ensure_lib, fortran_flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def run_gpu(X, r_max, tol=0.0, dtype=torch.float64, arith="df", no_elide=False):
    dims = X.shape
    plan = api.TTSVDPlan(dims, r_max, tol, dtype, arith, want_sigma=True, no_elide=no_elide)
    plan.run(fortran_flat(X, dtype))
    return plan.result()


def compare(X, res, ref, tol_rel, check_err2=True):
    assert res.ranks == ref.ranks, (res.ranks, ref.ranks)
    smax = max(s[0] for s in ref.sigmas.values())
    for i, s in ref.sigmas.items():
        g = res.sigma.get(i)
        if g is None or torch.isnan(g).any():
            continue  # elided step: no singular values computed
        k = ref.ranks[i - 1]
        got = g.cpu().numpy()[:k]
        assert np.max(np.abs(got - s[:k])) <= tol_rel * smax, (i, got, s[:k])
    nx = np.linalg.norm(X)
    cores = res.core_arrays()
    err = np.linalg.norm(O.tt_full(cores) - X) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
    assert abs(err - err_ref) <= tol_rel, (err, err_ref)
    if check_err2:
        assert abs(res.err2 - ref.err2) <= tol_rel * nx * nx
    for c in cores[1:]:
        assert O.core_orthonormality_defect(c) <= max(1e-12, tol_rel * 10)
    return err


CASES = [
    ((4,) * 10, 8),          # 4^10, r_max = 8 (the small configuration)
    ((3, 4, 5, 6, 7), 3),
    ((2,) * 12, 5),
    ((5, 6, 7), 100),        # every step elided
    ((9, 7), 4),             # d = 2: a truncated matrix SVD
    ((1, 4, 1, 5, 1), 2),    # unit extents
    ((4, 4, 4, 4, 4), 1),    # r_max = 1
    ((6, 5, 4, 3, 2), 50),   # ranks capped by the rows (wide unfoldings at the left end)
    ((8, 8, 8, 8, 8), 10),   # 8^5, m = 80 steps (wide TSQR kernel)
    ((3, 3, 3, 3, 3, 3, 3, 3, 3), 7),
    ((17, 3, 11), 5),        # odd extents, ragged panels
]


@pytest.mark.parametrize("dims,r_max", CASES)
def test_fp64_form_parity(dims, r_max):
    X = uniform_tensor(dims, seed=sum(dims) + r_max)
    compare(X, run_gpu(X, r_max), O.tt_svd(X, r_max), 1e-10)


@pytest.mark.parametrize("seed", [0, 1])
def test_small_config_seeds(seed):
    X = uniform_tensor((4,) * 10, seed=seed)
    compare(X, run_gpu(X, 8), O.tt_svd(X, 8), 1e-10)


def test_d1_is_a_copy():
    X = uniform_tensor((7,), seed=3)
    res = run_gpu(X, 3)
    assert res.ranks == [1, 1]
    assert np.array_equal(res.core_arrays()[0].ravel(), X)


@pytest.mark.parametrize("dims,r_max", [((4,) * 8, 6), ((8, 8, 8, 8, 8), 10), ((3, 4, 5, 6, 7), 3),
                                        ((8,) * 7, 20)])
def test_native_f64_arith_parity(dims, r_max):
    X = uniform_tensor(dims, seed=5)
    compare(X, run_gpu(X, r_max, arith="f64"), O.tt_svd(X, r_max), 1e-10)


@pytest.mark.parametrize("dims,r_max", [((4,) * 8, 6), ((8, 8, 8, 8, 8), 10), ((4,) * 10, 8)])
def test_no_elide_matches(dims, r_max):
    X = uniform_tensor(dims, seed=6)
    compare(X, run_gpu(X, r_max, no_elide=True), O.tt_svd(X, r_max), 1e-10)


@pytest.mark.parametrize("dims,rank,tol", [((4,) * 8, 3, 1e-4), ((5, 4, 6, 3, 4), 2, 1e-3),
                                          ((3,) * 8, 4, 1e-2), ((4,) * 11, 3, 1e-4)])
def test_tolerance_truncation(dims, rank, tol):
    X = planted_tt(dims, rank, seed=7, noise_rel=1e-6)
    ref = O.tt_svd(X, r_max=100, tol=tol)
    res = run_gpu(X, 100, tol)
    for i, s in ref.sigmas.items():
        assert not O.rank_is_ambiguous(s, ref.delta, ref.ranks[i - 1])
    compare(X, res, ref, 1e-10)
    assert np.linalg.norm(O.tt_full(res.core_arrays()) - X) <= tol * np.linalg.norm(X)


@pytest.mark.parametrize("dims,rank,r_max", [((4,) * 6, 1, 4), ((3, 4, 5, 6, 3), 2, 6),
                                           ((8, 8, 8, 8), 3, 10)])
def test_exact_low_rank_wide_steps(dims, rank, r_max):
    # no noise: the wide unfoldings at the left end are rank-deficient, so some of the kept
    # right singular vectors belong to zero singular values (the orthonormal completion)
    X = planted_tt(dims, rank, seed=4, noise_rel=0.0)
    compare(X, run_gpu(X, r_max), O.tt_svd(X, r_max), 1e-10)
    compare(X, run_gpu(X, r_max, arith="f64"), O.tt_svd(X, r_max), 1e-10)


def test_planted_rank_fp64():
    X = planted_tt((8, 8, 8, 8, 8), 4, seed=9, noise_rel=1e-6)
    compare(X, run_gpu(X, 10), O.tt_svd(X, 10), 1e-10)


@pytest.mark.parametrize("dims,r_max", [((4,) * 10, 8), ((8, 8, 8, 8, 8), 10), ((2,) * 14, 32),
                                        ((6, 5, 4, 3, 2), 50), ((4,) * 10, 40)])
def test_fp32_form_parity(dims, r_max):
    X64 = uniform_tensor(dims, seed=8)
    X32 = X64.astype(np.float32).astype(np.float64)
    res = run_gpu(X32, r_max, dtype=torch.float32)
    compare(X32, res, O.tt_svd(X32, r_max), 1e-5)


# wide unfoldings whose one-sided Jacobi working copy (rows x m values) exceeds shared memory:
# (8, 8, 8, 4, 8, 8) at r_max = 64 has a 64 x 512 step (256 KB in float-float or FP64), whose
# copy then lives in the workspace
@pytest.mark.parametrize("dtype,arith", [(torch.float64, "df"), (torch.float64, "f64"), (torch.float32, "df")])
def test_wide_step_beyond_shared_memory(dtype, arith):
    dims = (8, 8, 8, 4, 8, 8)
    X = planted_tt(dims, 20, seed=7, noise_rel=1e-3)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    res = run_gpu(X, 64, dtype=dtype, arith=arith)
    ref = O.tt_svd(X, 64)
    assert max(ref.ranks) == 64
    compare(X, res, ref, 1e-10 if dtype == torch.float64 else 1e-5)


# an unfolding with m = 512 (n 8 x rank cap 64): its small SVD runs on a 16-CTA cluster with
# V in global memory (A and V of 512 columns do not both fit the cluster's shared memory)
@pytest.mark.parametrize("dtype,arith", [(torch.float64, "df"), (torch.float32, "df")])
def test_m512_small_svd_with_global_v(dtype, arith):
    dims = (8, 8, 8, 2, 8, 8, 3, 8)
    X = planted_tt(dims, 24, seed=9, noise_rel=1e-3)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    res = run_gpu(X, 64, dtype=dtype, arith=arith)
    ref = O.tt_svd(X, 64)
    assert max(ref.ranks) == 64
    compare(X, res, ref, 1e-10 if dtype == torch.float64 else 1e-5)


def test_repeated_runs_are_identical():
    X = uniform_tensor((4,) * 10, seed=2)
    plan = api.TTSVDPlan(X.shape, 8, 0.0, torch.float64, "df", want_sigma=True)
    Xd = fortran_flat(X)
    plan.run(Xd)
    a = plan.result()
    plan.run(Xd)
    b = plan.result()
    assert a.ranks == b.ranks
    for ca, cb in zip(a.cores, b.cores):
        assert torch.equal(ca, cb)


# X in pinned host memory, copied in row blocks that overlap the first TSQR level
HOST_CASES = [((4,) * 10, 8, 0), ((8, 8, 8, 8, 8), 10, 5), ((2,) * 12, 5, 3), ((5, 6, 7), 100, 0),
              ((17, 3, 11), 5, 4), ((4, 4, 4, 4, 4), 1, 7), ((8,) * 6, 4, 1), ((3, 4, 5, 6, 7), 3, 64)]


@pytest.mark.parametrize("dims,r_max,chunks", HOST_CASES)
def test_from_host_parity(dims, r_max, chunks):
    X = uniform_tensor(dims, seed=11)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "df", want_sigma=True)
    Xh = fortran_flat(X).cpu().pin_memory()
    plan.run_host(Xh, chunks=chunks)
    res = plan.result()
    # X arrived intact, and the result meets the same bar as the device-input call
    assert torch.equal(plan.X_dev.cpu(), Xh)
    compare(X, res, O.tt_svd(X, r_max), 1e-10)


def test_from_host_fp32_and_repeat():
    dims, r_max = (8, 8, 8, 8, 8), 16
    X64 = uniform_tensor(dims, seed=12)
    X32 = X64.astype(np.float32).astype(np.float64)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float32, "df", want_sigma=True)
    Xh = fortran_flat(X32, torch.float32).cpu().pin_memory()
    plan.run_host(Xh, chunks=6)
    a = plan.result()
    compare(X32, a, O.tt_svd(X32, r_max), 1e-5)
    # a second call on a new input reuses X_dev only after the first call has read it
    Xh2 = fortran_flat(uniform_tensor(dims, seed=13).astype(np.float32).astype(np.float64),
                       torch.float32).cpu().pin_memory()
    plan.run_host(Xh, chunks=6)
    plan.run_host(Xh2, chunks=6)
    b = plan.result()
    X2 = uniform_tensor(dims, seed=13).astype(np.float32).astype(np.float64)
    compare(X2, b, O.tt_svd(X2, r_max), 1e-5)


# thick-bounds variant (Alg. 3): parity with the oracle's Alg. 3
from oracle.thick_bounds import tt_svd_thick  # noqa: E402

THICK_CASES = [((2,) * 12, 1, 16, 0.5), ((2,) * 12, 5, 16, 0.5), ((2,) * 12, 16, 16, 0.5),
               ((4,) * 8, 6, 16, 0.5), ((3, 4, 2, 2, 2, 3), 4, 8, 0.5), ((8,) * 6, 10, 16, 0.5),
               ((5, 6, 40), 3, 16, 0.5)]


@pytest.mark.parametrize("dims,r_max,m_min,f1", THICK_CASES)
def test_thick_bounds_parity(dims, r_max, m_min, f1):
    X = uniform_tensor(dims, seed=21)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "df", thick=(m_min, f1))
    plan.run(fortran_flat(X))
    res = plan.result()
    ref = tt_svd_thick(X, r_max, m_min, f1)
    assert res.ranks == ref.ranks, (res.ranks, ref.ranks)
    nx = np.linalg.norm(X)
    cores = res.core_arrays()
    err = np.linalg.norm(O.tt_full(cores) - X) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
    assert abs(err - err_ref) <= 1e-10, (err, err_ref)
    assert abs(res.err2 - ref.err2) <= 1e-10 * max(1.0, nx * nx)
    d, k = len(dims), ref.k
    for c in cores[d - k:] if k >= 2 else cores[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-12


# two-sided variant (Alg. 4): parity with the oracle's Alg. 4
from oracle.two_sided import tt_svd_two_sided  # noqa: E402

TWO_SIDED_CASES = [((4,) * 7, 5), ((2,) * 12, 4), ((3, 4, 2, 5), 100), ((8,) * 6, 10), ((6, 5), 3),
                   ((17, 3, 11, 4), 5), ((8,) * 5, 3)]


def _left_defect(core):
    r0, ni, r1 = core.shape
    M = O.freshape(core, (r0 * ni, r1))
    return float(np.max(np.abs(M.T @ M - np.eye(r1))))


@pytest.mark.parametrize("dims,r_max", TWO_SIDED_CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_two_sided_parity(dims, r_max, dtype):
    X = uniform_tensor(dims, seed=41)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    plan = api.TTSVDPlan(dims, r_max, 0.0, dtype, "df", two_sided=True)
    plan.run(fortran_flat(X, dtype))
    res = plan.result()
    ref = tt_svd_two_sided(X, r_max)
    assert res.ranks == ref.ranks, (res.ranks, ref.ranks)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    nx = np.linalg.norm(X)
    cores = res.core_arrays()
    err = np.linalg.norm(O.tt_full(cores) - X) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
    assert abs(err - err_ref) <= tol, (err, err_ref)
    assert abs(res.err2 - ref.err2) <= tol * nx * nx
    # the order of the steps fixes which cores are left- and which right-orthonormal
    d = len(dims)
    a, b, t = 1, d, 0
    while a < b:
        if t % 2 == 0:
            assert O.core_orthonormality_defect(cores[b - 1]) <= max(1e-12, tol), b
            b -= 1
        else:
            assert _left_defect(cores[a - 1]) <= max(1e-12, tol), a
            a += 1
        t += 1
