"""Pins of the thick-bounds oracle (Alg. 3) against what the mathematics fixes."""
import numpy as np
import pytest

from oracle import tt_svd_oracle as O
from oracle.model import thick_bounds_k
from oracle.thick_bounds import tt_svd_thick
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor


def rel_err(X, cores):
    return np.linalg.norm(O.tt_full(cores) - X) / np.linalg.norm(X)


def test_no_combination_is_plain_tt_svd():
    # k = 1 (the last extent alone reaches the threshold): Alg. 3 reduces to Alg. 1
    X = uniform_tensor((3, 4, 40), seed=1)
    assert thick_bounds_k((3, 4, 40), 16, 0.5, 5) == 1
    a, b = tt_svd_thick(X, 5), O.tt_svd(X, 5)
    assert a.k == 1 and a.ranks == b.ranks
    for ca, cb in zip(a.cores, b.cores):
        assert np.array_equal(ca, cb)


def test_exact_without_truncation():
    # r_max above every rank: the thick train reproduces X (rounding only)
    for dims in [(2,) * 8, (3, 4, 2, 2, 2, 3), (5, 2, 2, 2, 2)]:
        X = uniform_tensor(dims, seed=2)
        res = tt_svd_thick(X, 1000)
        assert res.k >= 2, dims
        assert rel_err(X, res.cores) <= 1e-12
        assert res.ranks[0] == 1 and res.ranks[-1] == 1
        assert [c.shape[1] for c in res.cores] == list(dims)
    # with r_max = 1000 the threshold r / f1_min is never reached and Alg. 3 degenerates to
    # Alg. 1 (k = d); a rank estimate of 8 (threshold 16) makes it combine 2 <= k < d
    # right-most extents, all different, so the recovery of line 4 runs on a tensor whose
    # dimension order matters
    for dims, k in [((2, 3, 4, 3, 2, 5), 3), ((3, 2, 2, 7, 3), 2), ((2, 2, 5, 3, 2, 4), 3)]:
        X = uniform_tensor(dims, seed=12)
        res = tt_svd_thick(X, 1000, m_min=16, f1_min=0.5, r_est=8)
        assert res.k == k and res.m == int(np.prod(dims[len(dims) - k:])), (dims, res.k)
        assert rel_err(X, res.cores) <= 1e-12, dims
        assert [c.shape[1] for c in res.cores] == list(dims)
        assert res.ranks == O.planned_ranks(list(dims), 1000)


def test_planted_ranks_are_recovered():
    # an exact TT of rank <= r_max is found exactly, with ranks not above the planted ones
    X = planted_tt((2,) * 10, 3, seed=3, noise_rel=0.0)
    res = tt_svd_thick(X, 8)
    assert res.k >= 2
    assert rel_err(X, res.cores) <= 1e-12
    plain = O.tt_svd(X, 8)
    assert all(a <= b for a, b in zip(res.ranks, plain.ranks))


def test_recovery_without_truncation_keeps_the_reduced_approximation():
    # when line 4 truncates nothing, the recovered train is the reduced train (line 3)
    # written with more cores: same tensor, same error, orthonormal recovered cores
    X = uniform_tensor((2,) * 10, seed=4)
    # m = 16, reduced rank r = 8: the recovery ranks of the 8 x 2 x 2 x 2 x 2 core are at
    # most (8, 8, 4, 2), so line 4 is exact
    res = tt_svd_thick(X, 8)
    assert res.k == 4 and res.m == 16
    assert res.recovery.err2 <= 1e-24
    full_thick, full_red = O.tt_full(res.cores), O.tt_full(res.reduced.cores)
    assert np.max(np.abs(full_thick - full_red.reshape(full_thick.shape, order="F"))) <= 1e-12
    e2 = np.linalg.norm(full_thick - X) ** 2
    assert abs(e2 - res.reduced.err2) <= 1e-10 * np.linalg.norm(X) ** 2
    for c in res.cores[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-12


def test_recovered_cores_right_orthonormal_with_truncation():
    # the recovery may truncate (r_max below its ranks): cores d-k+1..d stay orthonormal,
    # and the error is at least the reduced TT-SVD's own
    X = uniform_tensor((4, 4, 4, 4, 4, 4), seed=5)
    res = tt_svd_thick(X, 3, m_min=16, f1_min=0.5)
    assert res.k == 2
    d, k = 6, res.k
    for c in res.cores[d - k:]:
        assert O.core_orthonormality_defect(c) <= 1e-12
    assert np.linalg.norm(O.tt_full(res.cores) - X) ** 2 >= res.reduced.err2 * (1 - 1e-12)


@pytest.mark.parametrize("r_max,merged", [(1, 16), (5, 16), (16, 32)])
def test_paper_table_merged_dimension(r_max, merged):
    # Table (variants, Sec. 5.2): 2^d tensor, m_min = 16, f1_min = 1/2
    X = uniform_tensor((2,) * 12, seed=6)
    res = tt_svd_thick(X, r_max)
    assert res.m == merged
    # the reduced TT-SVD's first step reduces the work array by r / m (the table's f_1)
    assert res.reduced.ranks[-2] == min(r_max, res.m)
