"""Two-sided TT-SVD (Alg. 4, Sec. 3.1.3 "Two-sided variant"), plain numpy FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path; shares no
code with the CUDA engine.

Alg. 4 computes cores alternately at the right and at the left end of the train
(i = d, 1, d-1, 2, ...).  The remaining work tensor Z has the shape
(r_L, n_a, ..., n_b, r_R).  A right step takes the SVD of the unfolding
(r_L n_a ... n_{b-1}) x (n_b r_R), keeps V^T as T^(b) and continues with U Sigma;
a left step takes the SVD of the unfolding (r_L n_a) x (n_{a+1} ... n_b r_R) -- the
transpose of the tall matrix whose QR the algorithm computes -- keeps the left
singular vectors as T^(a) and continues with Sigma V^T.  When one dimension is left,
Z itself is the middle core, which carries the norm.  Only the r_max-prescribed form
is defined here (r = min(r_max, rows, columns) at every step).
"""
from __future__ import annotations

import numpy as np

from .tt_svd_oracle import TTResult, freshape


def tt_svd_two_sided(X: np.ndarray, r_max: int) -> TTResult:
    X = np.asarray(X, dtype=np.float64)
    n = list(X.shape)
    d = len(n)
    cores = [None] * d
    ranks = [1] * (d + 1)
    res = TTResult(cores=cores, ranks=ranks)
    a, b = 1, d          # remaining dimensions a..b (1-based)
    rL, rR = 1, 1
    Z = X
    t = 0
    while a < b:
        mid = [n[i - 1] for i in range(a, b + 1)]
        if t % 2 == 0:
            # right step on dimension b
            rows = rL * int(np.prod(mid[:-1]))
            cols = n[b - 1] * rR
            U, S, Vt = np.linalg.svd(freshape(Z, (rows, cols)), full_matrices=False)
            r = min(r_max, rows, cols)
            cores[b - 1] = freshape(Vt[:r, :], (r, n[b - 1], rR))
            Z = freshape(U[:, :r] * S[:r], [rL] + mid[:-1] + [r])
            res.sigmas[("R", b)] = S
            res.discarded2[("R", b)] = float(np.sum(S[r:] ** 2))
            ranks[b - 1] = r
            rR = r
            b -= 1
        else:
            # left step on dimension a
            rows = rL * n[a - 1]
            cols = int(np.prod(mid[1:])) * rR
            U, S, Vt = np.linalg.svd(freshape(Z, (rows, cols)), full_matrices=False)
            r = min(r_max, rows, cols)
            cores[a - 1] = freshape(U[:, :r], (rL, n[a - 1], r))
            Z = freshape(S[:r, None] * Vt[:r, :], [r] + mid[1:] + [rR])
            res.sigmas[("L", a)] = S
            res.discarded2[("L", a)] = float(np.sum(S[r:] ** 2))
            ranks[a] = r
            rL = r
            a += 1
        t += 1
    cores[a - 1] = freshape(Z, (rL, n[a - 1], rR))
    return res
