"""Parity at the full size of the benchmark: an 8^10 FP64 tensor (2^30 entries, 8 GiB),
uniform[0,1) from the same seed and with the same plan as bench.py, r_max = 10.

The oracle cannot decompose 8 GiB in a test, so the run is checked against what holds
at any size:
* ranks: the tol = 0 rule of Alg. 1 (r_{i-1} = min(r_max, rows, cols)), bit-exact;
* the first computed step (i = 9; step 10 is elided, which is exact) returns the singular
  values of the unfolding X_(8) (2^24 x 64): compared with the square roots of the
  eigenvalues of its FP64 Gram matrix, formed on the host (LAPACK; accurate to ~1e-15
  relative here, the unfolding being well conditioned);
* the sum of that step's sigma^2 equals ||X||_F^2;
* cores 2..10 have orthonormal rows (to 1e-13 m, float-float rotations);
* ||X - X~||_F^2 equals the reported discarded energy (successive orthogonal projections),
  with X~ contracted on the host.
"""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import api
from paper_2102_00104_gb300 import inputs
from tests.gpu_common import ensure_lib, tt_full_dev

pytestmark = pytest.mark.gpu


def test_full_size_8p10_rmax10():
    ensure_lib()
    dims, r_max = (8,) * 10, 10
    nbar = 8 ** 10
    X = api.gen_uniform(nbar, 0, torch.float64)  # the bench's input (seed 0)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "df", want_sigma=True)
    plan.run(X)
    res = plan.result()
    assert res.ranks == O.planned_ranks(list(dims), r_max)

    Xh = X.cpu().numpy()
    del X
    W8 = Xh.reshape(64, 8 ** 8)  # row c = column c of the unfolding X_(8) (Fortran order)
    G = W8 @ W8.T
    ev = np.linalg.eigvalsh(G)[::-1]
    s_ref = np.sqrt(np.maximum(ev, 0.0))
    assert s_ref[-1] > 1e-3 * s_ref[0]  # well conditioned: the Gram route is accurate
    got = res.sigma[9].cpu().numpy()
    assert got.shape[0] >= 64
    assert np.max(np.abs(got[:64] - s_ref)) <= 1e-10 * s_ref[0], np.max(np.abs(got[:64] - s_ref))
    nx2 = float(np.trace(G))
    assert abs(float(np.sum(got[:64] ** 2)) - nx2) <= 1e-12 * nx2

    cores = res.core_arrays()
    for c in cores[1:]:
        # float-float rotations: orthogonality to ~m 2^-46 (the bound of the small-SVD tests)
        assert O.core_orthonormality_defect(c) <= 1e-13 * 80
    Xt = O.tt_full(cores).ravel(order="F")
    d = Xh - Xt
    err2 = float(np.dot(d, d))
    assert abs(err2 - res.err2) <= 1e-10 * nx2, (err2, res.err2, nx2)


def test_full_size_8p10_fp32_form_rmax32():
    # the precision form at full size: the same 2^30 entries stored FP32 (4 GiB), r_max = 32;
    # reference values from the FP32 values widened to FP64, bar 1e-5 (relative to sigma_max)
    ensure_lib()
    dims, r_max = (8,) * 10, 32
    X = api.gen_uniform(8 ** 10, 0, torch.float32)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float32, "df", want_sigma=True)
    plan.run(X)
    res = plan.result()
    assert res.ranks == O.planned_ranks(list(dims), r_max)
    Xh = X.cpu().numpy().astype(np.float64)
    del X
    W8 = Xh.reshape(64, 8 ** 8)
    G = W8 @ W8.T
    s_ref = np.sqrt(np.maximum(np.linalg.eigvalsh(G)[::-1], 0.0))
    got = res.sigma[9].cpu().numpy()
    assert np.max(np.abs(got[:64] - s_ref)) <= 1e-5 * s_ref[0]
    cores = res.core_arrays()
    for c in cores[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-5
    Xt = O.tt_full(cores).ravel(order="F")
    d = Xh - Xt
    nx2 = float(np.trace(G))
    assert abs(float(np.dot(d, d)) - res.err2) <= 1e-5 * nx2


@pytest.mark.parametrize("r_max,arith", [(20, "f64"), (50, "df")])
def test_full_size_8p10_planted_rank16(r_max, arith):
    # the second input of the 8^10 configuration: planted TT rank 16 (Gaussian cores,
    # ||X||_F = 1) plus Gaussian noise of norm 1e-6, built on the device with bench.py's seed.
    # References formed on the device with library routines (FP64 Householder QR of the
    # 2^24 x 64 unfolding, then the singular values of its R), which keep the small noise
    # singular values that a Gram matrix would lose
    ensure_lib()
    dims = (8,) * 10
    X = inputs.planted_tt_device(dims, 16, 1, noise_rel=1e-6)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, arith, want_sigma=True)
    plan.run(X)
    res = plan.result()
    assert res.ranks == O.planned_ranks(list(dims), r_max)

    M = X.view(64, 8 ** 8)  # row c = column c of the unfolding X_(8) (Fortran order)
    R = torch.linalg.qr(M.t(), mode="r").R
    del M
    s_ref = torch.linalg.svdvals(R).cpu().numpy()
    nx2 = float(torch.dot(X, X).item())
    # the planted structure: 16 values carry the tensor, the rest the noise
    assert s_ref[15] > 1e-3 * s_ref[0] and s_ref[16] < 1e-5 * s_ref[0]
    got = res.sigma[9].cpu().numpy()[:64]
    assert np.max(np.abs(got - s_ref)) <= 1e-12 * s_ref[0], np.max(np.abs(got - s_ref))
    assert abs(float(np.sum(got ** 2)) - nx2) <= 1e-12 * nx2

    for c in res.core_arrays()[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-13 * 80
    Xt = tt_full_dev([c.to(torch.float64) for c in res.cores], dims)
    d = X - Xt
    del Xt
    err2 = float(torch.dot(d, d).item())
    assert abs(err2 - res.err2) <= 1e-12 * nx2, (err2, res.err2, nx2)
    # rank >= 16 keeps the planted part: only noise is discarded, 9 steps at most 1e-12 each
    assert err2 <= 9e-12 * nx2, err2 / nx2


def test_full_size_8p10_rmax10_native_fp64():
    # the headline arithmetic at full size: the same 8^10 tensor in native FP64 (blocked
    # tensor-core TSQR, FP64-accurate W V_r), held to FP64 bars: sigma of step 9 against the
    # singular values of the R of a library Householder QR of the 2^24 x 64 unfolding (a Gram
    # spectrum would lose ~1e-12 of sigma_max on the smallest values) to 1e-12 sigma_max,
    # cores orthonormal to 1e-14 m, ||X - X~||^2 equal to the reported discarded energy to
    # 1e-12 ||X||^2 (X~ contracted on the device)
    ensure_lib()
    dims, r_max = (8,) * 10, 10
    X = api.gen_uniform(8 ** 10, 0, torch.float64)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "f64", want_sigma=True)
    plan.run(X)
    res = plan.result()
    assert res.ranks == O.planned_ranks(list(dims), r_max)
    M = X.view(64, 8 ** 8)
    R = torch.linalg.qr(M.t(), mode="r").R
    del M
    s_ref = torch.linalg.svdvals(R).cpu().numpy()
    got = res.sigma[9].cpu().numpy()[:64]
    assert np.max(np.abs(got - s_ref)) <= 1e-12 * s_ref[0], np.max(np.abs(got - s_ref)) / s_ref[0]
    nx2 = float(torch.dot(X, X).item())
    for c in res.core_arrays()[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-14 * 80
    Xt = tt_full_dev([c.to(torch.float64) for c in res.cores], dims)
    d = X - Xt
    del Xt
    err2 = float(torch.dot(d, d).item())
    assert abs(err2 - res.err2) <= 1e-12 * nx2, (err2, res.err2, nx2)
