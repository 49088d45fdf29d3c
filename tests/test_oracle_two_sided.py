"""Pins of the two-sided oracle (Alg. 4) against what the mathematics fixes."""
import numpy as np
import pytest

from oracle import tt_svd_oracle as O
from oracle.two_sided import tt_svd_two_sided
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor


def left_defect(core):
    # T^(i) reshaped (r_{i-1} n_i) x r_i has orthonormal columns
    r0, ni, r1 = core.shape
    M = O.freshape(core, (r0 * ni, r1))
    return float(np.max(np.abs(M.T @ M - np.eye(r1))))


@pytest.mark.parametrize("dims", [(2,) * 7, (3, 4, 2, 5), (4, 4, 4, 4, 4, 4), (6, 5)])
def test_exact_without_truncation(dims):
    X = uniform_tensor(dims, seed=31)
    res = tt_svd_two_sided(X, 1000)
    assert np.linalg.norm(O.tt_full(res.cores) - X) <= 1e-12 * np.linalg.norm(X)
    assert res.ranks[0] == 1 and res.ranks[-1] == 1


def test_first_two_spectra_are_unfolding_spectra():
    # step d (right) sees X's last unfolding; with it untruncated, step 1 (left) sees the
    # first unfolding of X (a right projection that keeps everything changes nothing)
    X = uniform_tensor((3, 4, 5, 2), seed=32)
    res = tt_svd_two_sided(X, 100)
    s_right = O.unfolding_singular_values(X, 3)
    s_left = O.unfolding_singular_values(X, 1)
    assert np.allclose(res.sigmas[("R", 4)], s_right, rtol=0, atol=1e-13 * s_right[0])
    assert np.allclose(res.sigmas[("L", 1)], s_left, rtol=0, atol=1e-13 * s_left[0])


def test_orthonormality_and_error():
    X = uniform_tensor((4,) * 7, seed=33)
    res = tt_svd_two_sided(X, 5)
    d = 7
    # steps: right 7, left 1, right 6, left 2, right 5, left 3; middle core 4 carries the norm
    for i in (1, 2, 3):
        assert left_defect(res.cores[i - 1]) <= 1e-12
    for i in (5, 6, 7):
        assert O.core_orthonormality_defect(res.cores[i - 1]) <= 1e-12
    # left and right projections act on different index groups: the error is exactly the
    # discarded energy (up to rounding), as for the one-sided algorithm
    e2 = np.linalg.norm(O.tt_full(res.cores) - X) ** 2
    assert abs(e2 - res.err2) <= 1e-10 * np.linalg.norm(X) ** 2
    assert len(res.discarded2) == d - 1


def test_planted_ranks():
    X = planted_tt((3,) * 8, 4, seed=34, noise_rel=0.0)
    res = tt_svd_two_sided(X, 6)
    # r_max = 6 above the planted rank 4: exact (with tol = 0 the ranks keep the zero
    # singular values, r = min(r_max, rows, columns), as in the one-sided algorithm)
    assert np.linalg.norm(O.tt_full(res.cores) - X) <= 1e-12 * np.linalg.norm(X)
    assert res.ranks == O.tt_svd(X, 6).ranks
    # the kept singular values beyond the planted rank are zero
    for key, s in res.sigmas.items():
        assert np.all(s[4:] <= 1e-12 * s[0]), key


def test_two_dimensions_is_a_matrix_svd():
    X = uniform_tensor((9, 7), seed=35)
    res, ref = tt_svd_two_sided(X, 4), O.tt_svd(X, 4)
    assert res.ranks == ref.ranks
    assert np.allclose(O.tt_full(res.cores), O.tt_full(ref.cores), atol=1e-12)
