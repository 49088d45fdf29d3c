"""Pins of the Alg. 6 / TSQR oracle (no GPU)."""
import numpy as np
import pytest

from oracle.householder import (EPS_FP64, qless_householder_block, reflector, tsqr_flat,
                                tsqr_tree)


def rows_equal_up_to_sign(A, B, tol):
    for a, b in zip(A, B):
        if not (np.allclose(a, b, atol=tol) or np.allclose(a, -b, atol=tol)):
            return False
    return True


@pytest.mark.parametrize("n,m,nb", [(100, 5, 16), (37, 8, 7), (9, 9, 4), (5, 12, 3), (64, 1, 64)])
def test_tsqr_gram_and_library_qr(n, m, nb):
    rng = np.random.default_rng(n + m)
    W = rng.standard_normal((n, m))
    R = tsqr_flat(W, nb)
    assert np.allclose(np.tril(R, -1), 0)
    # closed form: R^T R = W^T W
    assert np.allclose(R.T @ R, W.T @ W, rtol=0, atol=1e-12 * np.linalg.norm(W) ** 2)
    # special case that reduces to a library routine: R equals numpy's R up to row signs
    Rq = np.linalg.qr(W, mode="r")
    Rq_full = np.zeros((m, m))
    Rq_full[: Rq.shape[0], :] = Rq
    assert rows_equal_up_to_sign(R, Rq_full, 1e-11 * np.linalg.norm(W))


def test_tree_shapes_agree():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((300, 6))
    R1 = tsqr_flat(W, 32)
    for parts in (2, 3, 5, 8):
        R2 = tsqr_tree(W, 16, parts)
        assert rows_equal_up_to_sign(R1, R2, 1e-11)


def test_reflector_norm_is_two():
    rng = np.random.default_rng(4)
    for u in [rng.standard_normal(10), np.zeros(6), np.array([0.0, 1e-200, 0.0]),
              np.array([5.0]), np.array([-3.0, 4.0]), np.array([1e150, 1e150])]:
        v, alpha = reflector(u)
        assert abs(np.dot(v, v) - 2.0) <= 1e-14 * 2, u
        # the reflection I - v v^T maps u onto alpha e_1
        w = u - np.dot(v, u) * v
        assert np.allclose(w[1:], 0, atol=1e-12 * max(1.0, np.linalg.norm(u)))
        assert abs(w[0] - alpha) <= 1e-12 * max(1.0, abs(alpha)) + 1e-150


def test_sign_rule_is_branch_free_variant():
    # alpha takes the sign opposite to the pivot (no cancellation in u_1 - alpha)
    v, alpha = reflector(np.array([2.0, 1.0]))
    assert alpha < 0
    v, alpha = reflector(np.array([-2.0, 1.0]))
    assert alpha > 0
    v, alpha = reflector(np.array([0.0, 1.0]))
    assert alpha > 0


def test_block_does_not_modify_M_and_records_reflectors():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((8, 4))
    M0 = M.copy()
    R = np.triu(rng.standard_normal((4, 4)))
    rec = []
    Rb = qless_householder_block(M, R, record=rec)
    assert np.array_equal(M, M0)
    assert len(rec) == 4
    for v in rec:
        assert abs(np.dot(v, v) - 2.0) < 1e-13
    S = np.vstack([M, R])
    assert np.allclose(Rb.T @ Rb, S.T @ S, atol=1e-12)


def test_rank_deficient_and_zero_columns():
    rng = np.random.default_rng(6)
    W = rng.standard_normal((50, 3))
    W = np.hstack([W, np.zeros((50, 1)), W[:, :1] * 2.0, np.zeros((50, 1))])
    R = tsqr_flat(W, 16)
    assert np.all(np.isfinite(R))
    assert np.allclose(R.T @ R, W.T @ W, atol=1e-12 * np.linalg.norm(W) ** 2)
    s = np.linalg.svd(R, compute_uv=False)
    # numerical rank preserved: 3 nonzero singular values
    assert s[2] > 1e-3 * s[0] and np.all(s[3:] <= 1e-13 * s[0])
    # an all-zero matrix gives a finite R of tiny norm (eps trick, no division by zero)
    Z = tsqr_flat(np.zeros((10, 3)), 4)
    assert np.all(np.isfinite(Z)) and np.max(np.abs(Z)) < 1e-150
    assert EPS_FP64 == np.finfo(np.float64).tiny
