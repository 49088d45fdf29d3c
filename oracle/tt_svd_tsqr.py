"""Alg. 2 (optimized TSQR TT-SVD, Sec. 3.1.2), step by step, in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

It differs from Alg. 1 exactly where the paper says it does:
* delta comes from the singular values of the first step (line 7) instead of
  ||X||_F (Alg. 1 line 1);
* the SVD of W is replaced by the QR trick, Eq. (QR_trick): R from a Q-less
  QR (line 5, here the Alg. 6 flat tree of ``householder.tsqr_flat``), then
  the small SVD of R (line 6);
* the next work matrix is W V_{:,1:r} (line 11) instead of U_r Sigma_r.
In exact arithmetic both algorithms give the same singular values, ranks and
approximation (the paragraph after Alg. 2).
"""
from __future__ import annotations

import math

import numpy as np

from .householder import tsqr_flat
from .tt_svd_oracle import TTResult, freshape, truncation_rank


def tt_svd_tsqr(X: np.ndarray, r_max: int, tol: float = 0.0, nb: int = 64) -> TTResult:
    X = np.asarray(X, dtype=np.float64)
    n = list(X.shape)
    d = len(n)
    nbar = int(np.prod(n))  # line 1
    r = [1] * (d + 1)  # line 2
    W = freshape(X, (nbar // n[-1], n[-1]))  # line 3
    cores = [None] * d
    res = TTResult(cores=cores, ranks=r)
    delta = None
    for i in range(d, 1, -1):  # line 4
        rows, cols = W.shape
        Rm = tsqr_flat(W, nb)  # line 5 (Q is never formed)
        _, S, Vt = np.linalg.svd(Rm)  # line 6
        S = S[: min(rows, cols)]  # a wide W has only `rows` singular values
        if delta is None:  # line 7
            delta = tol / math.sqrt(d - 1) * math.sqrt(float(np.sum(S ** 2))) if tol > 0 else 0.0
            res.delta = delta
        rr = truncation_rank(S, delta, r_max, rows, cols)  # line 8
        r[i - 1] = rr
        cores[i - 1] = freshape(Vt[:rr, :], (rr, n[i - 1], r[i]))  # line 9
        nbar = nbar * rr // cols  # line 10
        Y = W @ Vt[:rr, :].T  # line 11: W V_{:,1:r}, then reshape for the next step
        res.sigmas[i] = S
        res.discarded2[i] = float(np.sum(S[rr:] ** 2))
        if i > 2:
            W = freshape(Y, (nbar // (n[i - 2] * rr), n[i - 2] * rr))
        else:
            W = Y
    cores[0] = freshape(W, (1, n[0], r[1]))  # line 13
    return res
