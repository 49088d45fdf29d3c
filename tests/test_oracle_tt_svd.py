"""Pins of the Alg. 1 oracle against mathematics and the paper (no GPU).

Each check is independent of the oracle's own code path: unfoldings are built
here by explicit index loops, spectra by a different LAPACK routine (symmetric
eigenvalues of the Gram matrix or scipy's gesvd driver), and integer ranks are
compared with the paper's table of TT-ranks.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import tt_svd_oracle as O
from oracle.tt_svd_tsqr import tt_svd_tsqr
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_unfolding(X, k):
    """(n_1..n_k) x (n_{k+1}..n_d) unfolding by explicit Fortran-order index loops."""
    n = X.shape
    rows = int(np.prod(n[:k]))
    cols = int(np.prod(n[k:]))
    M = np.empty((rows, cols))
    for idx in itertools.product(*[range(s) for s in n]):
        r = 0
        stride = 1
        for a in range(k):
            r += idx[a] * stride
            stride *= n[a]
        c = 0
        stride = 1
        for a in range(k, len(n)):
            c += idx[a] * stride
            stride *= n[a]
        M[r, c] = X[idx]
    return M


def gram_singular_values(M):
    """sigma from eigenvalues of the smaller Gram matrix (a different LAPACK routine)."""
    G = M.T @ M if M.shape[0] >= M.shape[1] else M @ M.T
    ev = np.clip(np.linalg.eigvalsh(G)[::-1], 0, None)
    return np.sqrt(ev)


def test_first_step_spectrum_is_last_unfolding():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 2, 5))
    res = O.tt_svd(X, r_max=100)
    ref = gram_singular_values(brute_unfolding(X, 3))
    got = res.sigmas[4]
    assert np.allclose(got, ref[: len(got)], rtol=1e-10, atol=1e-12)


def test_untruncated_steps_follow_unfoldings():
    # with r_max large nothing is truncated, so step i sees the (i-1)-th unfolding of X
    rng = np.random.default_rng(2)
    X = rng.standard_normal((2, 3, 4, 3))
    res = O.tt_svd(X, r_max=1000)
    for i in (4, 3, 2):
        ref = gram_singular_values(brute_unfolding(X, i - 1))
        got = res.sigmas[i]
        k = min(len(got), len(ref))
        assert np.allclose(got[:k], ref[:k], rtol=1e-9, atol=1e-11), i


def test_sigma_energy_closed_form():
    X = uniform_tensor((4, 4, 4, 4, 4), seed=3)
    res = O.tt_svd(X, r_max=3)
    assert math.isclose(float(np.sum(res.sigmas[5] ** 2)), float(np.sum(X * X)), rel_tol=1e-12)


def test_interlacing_after_truncation():
    # projection onto the kept subspace cannot raise singular values of later unfoldings
    X = uniform_tensor((3, 3, 3, 3, 3), seed=4)
    res = O.tt_svd(X, r_max=2)
    for i in (4, 3, 2):
        ref = gram_singular_values(brute_unfolding(X, i - 1))
        got = res.sigmas[i]
        k = min(len(got), len(ref))
        assert np.all(got[:k] <= ref[:k] * (1 + 1e-10) + 1e-12)


@pytest.mark.parametrize("dims,rank", [((4, 4, 4, 4, 4), 3), ((2, 3, 4, 3, 2), 2), ((5, 6, 7), 4)])
def test_planted_exact_ranks(dims, rank):
    X = planted_tt(dims, rank, seed=5, noise_rel=0.0)
    res = O.tt_svd(X, r_max=50)
    Xt = O.tt_full(res.cores)
    assert np.linalg.norm(Xt - X) <= 1e-12 * np.linalg.norm(X)
    for i, s in res.sigmas.items():
        planted = min(rank, int(np.prod(dims[: i - 1])), int(np.prod(dims[i - 1:])))
        if len(s) > planted:
            assert np.all(s[planted:] <= 1e-13 * s[0]), i
    res_tol = O.tt_svd(X, r_max=50, tol=1e-8)
    expect = [1] + [min(rank, int(np.prod(dims[:k])), int(np.prod(dims[k:]))) for k in range(1, len(dims))] + [1]
    assert res_tol.ranks == expect


def test_error_bound_and_equality():
    X = uniform_tensor((3, 4, 3, 4, 3), seed=6)
    for r_max in (1, 2, 5):
        res = O.tt_svd(X, r_max=r_max)
        err2 = float(np.sum((O.tt_full(res.cores) - X) ** 2))
        assert err2 <= res.err2 * (1 + 1e-10) + 1e-24
        # for TT-SVD the successive projections are orthogonal: equality up to rounding
        assert math.isclose(err2, res.err2, rel_tol=1e-9)


def test_tolerance_guarantee():
    X = uniform_tensor((4, 4, 4, 4), seed=7)
    for tol in (0.3, 0.1, 0.01):
        res = O.tt_svd(X, r_max=10**6, tol=tol)
        err = np.linalg.norm(O.tt_full(res.cores) - X)
        assert err <= tol * np.linalg.norm(X) * (1 + 1e-12)


def test_core_orthonormality():
    X = uniform_tensor((4, 3, 5, 4, 3), seed=8)
    res = O.tt_svd(X, r_max=4)
    for c in res.cores[1:]:
        assert O.core_orthonormality_defect(c) <= 1e-13


def test_rank_one_tensor():
    a, b, c, e = (np.arange(1, k + 1, dtype=float) for k in (3, 4, 5, 2))
    X = np.einsum("i,j,k,l->ijkl", a, b, c, e)
    res = O.tt_svd(X, r_max=1)
    assert math.isclose(res.sigmas[4][0], np.linalg.norm(X), rel_tol=1e-13)
    assert np.linalg.norm(O.tt_full(res.cores) - X) <= 1e-12 * np.linalg.norm(X)
    assert res.ranks == [1, 1, 1, 1, 1]


def test_d2_is_truncated_matrix_svd():
    # d = 2: TT-SVD is the truncated SVD of the matrix (Eckart-Young), checked with scipy's gesvd
    rng = np.random.default_rng(9)
    A = rng.standard_normal((7, 5))
    for r in (1, 2, 3):
        res = O.tt_svd(A, r_max=r)
        U, s, Vt = scipy.linalg.svd(A, lapack_driver="gesvd")
        best = (U[:, :r] * s[:r]) @ Vt[:r]
        assert np.allclose(O.tt_full(res.cores), best, atol=1e-12)
        assert res.ranks == [1, r, 1]


def test_full_contraction_definition():
    # tt_full against the elementwise definition of Sec. 2.1.2 on a tiny train
    rng = np.random.default_rng(10)
    r = [1, 2, 3, 1]
    n = [2, 3, 2]
    cores = [rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(3)]
    X = O.tt_full(cores)
    for i in itertools.product(*[range(s) for s in n]):
        v = cores[0][0, i[0], :] @ cores[1][:, i[1], :] @ cores[2][:, i[2], 0]
        assert math.isclose(X[i], v, rel_tol=1e-13, abs_tol=1e-14)


def test_planned_ranks_closed_form_and_alg1():
    # without tolerance truncation r_k = min(r_max, n_1...n_k, n_{k+1}...n_d): the rank of
    # the k-th unfolding is capped by both of its sides (the maximal TT ranks), then by r_max;
    # Alg. 1 on a generic tensor reaches exactly these ranks
    for dims in [(2, 3, 4, 5), (5, 4, 3, 2), (2, 2, 7), (4, 1, 3, 2), (3,), (6, 2), (2, 5, 2, 3, 2)]:
        d = len(dims)
        for r_max in (1, 2, 3, 6, 100):
            closed = [1] + [min(r_max, int(np.prod(dims[:k])), int(np.prod(dims[k:]))) for k in range(1, d)] + [1]
            assert O.planned_ranks(list(dims), r_max) == closed, (dims, r_max)
            assert O.tt_svd(uniform_tensor(dims, seed=13), r_max).ranks == closed, (dims, r_max)


def test_truncation_rule_hand_cases():
    s = np.array([3.0, 2.0, 1.0])
    # tails after j: j=0:14, j=1:5, j=2:1, j=3:0
    assert O.truncation_rank(s, math.sqrt(1.0), 10, 10, 10) == 2  # "<=" as printed
    assert O.truncation_rank(s, math.sqrt(0.999), 10, 10, 10) == 3
    assert O.truncation_rank(s, math.sqrt(5.0), 10, 10, 10) == 1
    assert O.truncation_rank(s, 100.0, 10, 10, 10) == 1  # clamp r >= 1
    assert O.truncation_rank(s, 0.0, 2, 10, 10) == 2  # r_max caps
    assert O.truncation_rank(s, 0.0, 10, 2, 10) == 2  # rows cap (wide unfolding)
    assert O.truncation_rank(s, 0.0, 10, 10, 10) == 3  # tol = 0: no tolerance truncation
    assert list(O.tail_sums(s)) == [14.0, 5.0, 1.0, 0.0]
    assert O.rank_is_ambiguous(s, 1.0, 2)
    assert not O.rank_is_ambiguous(s, math.sqrt(3.0), 2)
    # a tie on the other side: delta^2 just below the tail after sigma_1 (5) keeps r = 2, but
    # a sum rounded the other way would take r = 1
    d_low = math.sqrt(5.0 * (1 - 1e-14))
    assert O.truncation_rank(s, d_low, 10, 10, 10) == 2
    assert O.rank_is_ambiguous(s, d_low, 2)
    assert not O.rank_is_ambiguous(s, math.sqrt(4.0), 2)


def test_rank_table_plain():
    g = json.load(open(os.path.join(GOLDEN, "rank_table_2d.json")))
    X = uniform_tensor((2,) * 10, seed=11)
    for row in g["plain"]["rows"]:
        res = O.tt_svd(X, r_max=row["r_max"])
        k = len(row["ranks_right"])
        # ranks r_{d-k} .. r_{d-1}, listed left to right ending at the right boundary
        assert res.ranks[10 - k:10] == row["ranks_right"], row
        assert O.planned_ranks((2,) * 10, row["r_max"])[10 - k:10] == row["ranks_right"]
        # reduction factors f_j = r_{i-1} / (n_i r_i), j = 1 at the right boundary
        f = [res.ranks[i - 1] / (2 * res.ranks[i]) for i in range(10, 10 - len(row["f"]), -1)]
        expect = [float(eval(x)) for x in row["f"]]
        assert np.allclose(f, expect), row


def test_rank_table_thick_bounds_shapes():
    g = json.load(open(os.path.join(GOLDEN, "rank_table_2d.json")))
    tb = g["thick_bounds"]
    from oracle.model import thick_bounds_k
    for row in tb["rows"]:
        k = thick_bounds_k((2,) * 30, tb["m_min"], tb["f1_min"], row["r_max"])
        assert 2 ** k == row["merged_dim"], row
        dims = (2,) * (12 - k) + (2 ** k,)
        r = O.planned_ranks(dims, row["r_max"])
        d = len(dims)
        assert r[d - len(row["ranks_right"]):d] == row["ranks_right"]
        f = [r[i - 1] / (dims[i - 1] * r[i]) for i in range(d, d - len(row["f"]), -1)]
        assert np.allclose(f, [float(eval(x)) for x in row["f"]]), row


def test_alg1_equals_alg2():
    # Alg. 1 and Alg. 2 have the same numerical properties in exact arithmetic (Sec. 3.1.2)
    for dims, r_max, tol in [((4, 4, 4, 4, 4), 5, 0.0), ((3, 5, 2, 4, 3), 3, 0.0), ((4, 4, 4, 4), 100, 0.05)]:
        X = uniform_tensor(dims, seed=12)
        a = O.tt_svd(X, r_max, tol)
        b = tt_svd_tsqr(X, r_max, tol, nb=7)
        assert a.ranks == b.ranks
        for i in a.sigmas:
            k = a.ranks[i - 1]
            assert np.allclose(a.sigmas[i][:k], b.sigmas[i][:k], rtol=0, atol=1e-11 * a.sigmas[i][0])
        assert np.allclose(O.tt_full(a.cores), O.tt_full(b.cores), atol=1e-11)
        assert math.isclose(a.delta, b.delta, rel_tol=1e-12, abs_tol=0)
