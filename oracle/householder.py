"""Alg. 6 (Q-less Householder QR of [M; R], Sec. 3.2) and the flat-tree TSQR built on it.

Test infrastructure only (see ``oracle/__init__.py``).

Alg. 6 transforms a rectangle M (n_b x m) stacked on an upper triangle R (m x m)
into a new triangle R_bar with [M; R] = Q R_bar, without forming or storing Q
and without modifying M.  The index windows printed in the paper are garbled;
the reading used here is the mathematical content: the
reflector of column j acts on all n_b rows of M and on row j of R, with the
pivot element R[j, j]; rows 0..j-1 of R are final and untouched, rows j+1..m-1
of R are zero in column j and therefore unaffected.

The reflector is the paper's scaled, branch-free variant (Alg. 6 lines 4-7):
  t     = ||u||^2 + eps
  alpha = sqrt(t + eps), negated when the pivot u_1 > 0
  t     = t - alpha * u_1 ;  u_1 = u_1 - alpha ;  beta = 1 / sqrt(t)
  v     = beta * u          (so ||v||_2^2 = 2 in exact arithmetic)
and each later column w is updated as w <- w - (v^T w) v  (lines 9-12).
eps is the smallest positive normalised number of the arithmetic type.
"""
from __future__ import annotations

import math

import numpy as np

EPS_FP64 = float(np.finfo(np.float64).tiny)  # 2.2250738585072014e-308


def reflector(u: np.ndarray, eps: float = EPS_FP64):
    """Alg. 6 lines 4-7 for one column: returns (v, alpha) with u_1 as the pivot.

    ``u`` is the active part of the column with the pivot element first.
    """
    u = np.array(u, dtype=np.float64)
    t = float(np.dot(u, u)) + eps
    alpha = math.sqrt(t + eps)
    if u[0] > 0:
        alpha = -alpha
    t = t - alpha * u[0]
    u[0] = u[0] - alpha
    beta = 1.0 / math.sqrt(t)
    return beta * u, alpha


def qless_householder_block(M: np.ndarray, R: np.ndarray, eps: float = EPS_FP64,
                            record=None) -> np.ndarray:
    """Alg. 6: R_bar with [M; R] = Q R_bar; M is not modified (a copy is worked on).

    ``record``, if a list, receives every reflector vector v (pivot first) so
    tests can check ||v||^2 = 2.
    """
    M = np.array(M, dtype=np.float64)  # working copy: the caller's M stays intact
    R = np.array(R, dtype=np.float64)
    nb, m = M.shape
    assert R.shape == (m, m)
    for j in range(m):
        # active part of column j: pivot R[j, j] first, then the n_b rows of M
        u = np.concatenate(([R[j, j]], M[:, j]))
        v, alpha = reflector(u, eps)
        if record is not None:
            record.append(v.copy())
        for k in range(j + 1, m):
            w = np.concatenate(([R[j, k]], M[:, k]))
            gamma = float(np.dot(v, w))
            w = w - gamma * v
            R[j, k] = w[0]
            M[:, k] = w[1:]
        R[j, j] = alpha
        M[:, j] = 0.0  # column j of the M rows is annihilated by the reflector
    return R


def tsqr_flat(W: np.ndarray, nb: int, eps: float = EPS_FP64) -> np.ndarray:
    """Flat-tree TSQR (Sec. 3.2 display): R <- R_bar([M_k; R]) over row blocks M_k of height nb."""
    W = np.asarray(W, dtype=np.float64)
    n, m = W.shape
    R = np.zeros((m, m))
    for s in range(0, n, nb):
        R = qless_householder_block(W[s:s + nb, :], R, eps)
    return R


def tsqr_tree(W: np.ndarray, nb: int, parts: int, eps: float = EPS_FP64) -> np.ndarray:
    """Two-level TSQR (Sec. 3.2): flat trees on ``parts`` row ranges, then a
    binary tree over the partial R's, each combine being Alg. 6 with M = R_a."""
    W = np.asarray(W, dtype=np.float64)
    n, m = W.shape
    bounds = [n * p // parts for p in range(parts + 1)]
    Rs = [tsqr_flat(W[bounds[p]:bounds[p + 1]], nb, eps) for p in range(parts)]
    while len(Rs) > 1:
        nxt = []
        for a in range(0, len(Rs) - 1, 2):
            nxt.append(qless_householder_block(Rs[a], Rs[a + 1], eps))
        if len(Rs) % 2:
            nxt.append(Rs[-1])
        Rs = nxt
    return Rs[0]
