"""Alg. 1 (original TT-SVD, Sec. 3.1.1 of the paper), written out plainly in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Conventions (Sec. 2.1 and the memory-layout paragraph of Sec. 3.1.2): tensors
are Fortran ordered (n_1 fastest), every reshape is a Fortran-order reshape,
and cores are T^(i) in R^{r_{i-1} x n_i x r_i} with r_0 = r_d = 1 (Sec. 2.1.2).
Step ``i`` runs from d down to 2 (right to left), as in Alg. 1.

Readings of the paper used here (where it is silent or ambiguous):
* tol == 0 means "no tolerance truncation": r_delta = number of singular values.
* The tail test of Alg. 1 line 8 uses "<=" as printed; the tail runs over all
  min(rows, cols) singular values of the unfolding.
* The chosen rank is clamped to [1, min(rows, cols)].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def freshape(a: np.ndarray, shape) -> np.ndarray:
    """Fortran-order reshape (Sec. 2.1: neighbouring dimensions are combined)."""
    return np.reshape(a, shape, order="F")


def frobenius_norm(x: np.ndarray) -> float:
    """||X||_F computed directly from the entries (Alg. 1 line 1)."""
    x = np.asarray(x, dtype=np.float64).ravel(order="K")
    return float(math.sqrt(float(np.dot(x, x))))


def tail_sums(sigma: np.ndarray) -> np.ndarray:
    """tail[j] = sigma_{j+1}^2 + sigma_{j+2}^2 + ... for j = 0..len(sigma) (1-based sigma).

    Plain suffix summation from the smallest singular value upwards.
    """
    s = np.asarray(sigma, dtype=np.float64)
    tail = np.zeros(len(s) + 1)
    acc = 0.0
    for j in range(len(s) - 1, -1, -1):
        acc += s[j] * s[j]
        tail[j] = acc
    return tail


def truncation_rank(sigma, delta: float, r_max: int, rows: int, cols: int) -> int:
    """Rank choice of Alg. 1 line 8 (identical in Alg. 2 line 8).

    r = min(r_max, r_delta) with r_delta = min{ j : sigma_{j+1}^2 + ... <= delta^2 },
    clamped to 1 <= r <= min(rows, cols).  delta == 0 disables the tolerance
    test (r_delta = number of singular values).
    """
    s = np.asarray(sigma, dtype=np.float64)
    if delta > 0.0:
        tail = tail_sums(s)
        d2 = delta * delta
        r_delta = next(j for j in range(len(s) + 1) if tail[j] <= d2)
    else:
        r_delta = len(s)
    r = min(int(r_max), int(r_delta), int(rows), int(cols))
    return max(r, 1)


def rank_is_ambiguous(sigma, delta: float, r: int, rel: float = 1e-12) -> bool:
    """True when the tail test at the chosen rank is a near tie (|tail - delta^2| tiny).

    Two correct implementations that sum the tail in different orders may then
    pick ranks that differ by one; parity tests accept either.
    """
    if delta <= 0.0:
        return False
    tail = tail_sums(sigma)
    d2 = delta * delta
    for j in (r - 1, r):
        if 0 <= j < len(tail) and abs(tail[j] - d2) <= rel * max(d2, tail[0]):
            return True
    return False


@dataclass
class TTResult:
    """Output of a TT-SVD: cores T^(1..d), ranks r_0..r_d and per-step spectra."""

    cores: list
    ranks: list
    sigmas: dict = field(default_factory=dict)  # step i -> all singular values of W^(i)
    discarded2: dict = field(default_factory=dict)  # step i -> sum of discarded sigma^2
    delta: float = 0.0

    @property
    def err2(self) -> float:
        """Sum over all steps of the discarded sigma^2 (a-posteriori error bound squared)."""
        return float(sum(self.discarded2.values()))


def tt_svd(X: np.ndarray, r_max: int, tol: float = 0.0) -> TTResult:
    """Alg. 1: TT-SVD by explicit unfoldings and full SVDs (Sec. 3.1.1).

    Parameters
    ----------
    X : ndarray of shape (n_1, ..., n_d), float64, indexed X[i_1, ..., i_d]
        (the Fortran-order meaning of the paper; numpy's own memory order is
        irrelevant because every reshape below is Fortran order).
    r_max : maximal TT rank (>= 1).
    tol : epsilon of Alg. 1 (relative Frobenius tolerance); 0 disables it.
    """
    X = np.asarray(X, dtype=np.float64)
    n = list(X.shape)
    d = len(n)
    if r_max < 1:
        raise ValueError("r_max must be >= 1")
    # line 1: delta = eps / sqrt(d-1) * ||X||_F
    delta = tol / math.sqrt(d - 1) * frobenius_norm(X) if (d > 1 and tol > 0) else 0.0
    W = X  # line 2
    nbar = int(np.prod(n))  # line 3
    r = [1] * (d + 1)  # r[0] .. r[d]; line 4 sets r_d = 1
    cores = [None] * d
    res = TTResult(cores=cores, ranks=r, delta=delta)
    for i in range(d, 1, -1):  # line 5: i = d, ..., 2
        ni = n[i - 1]
        cols = ni * r[i]
        rows = nbar // cols
        Wm = freshape(W, (rows, cols))  # line 6
        U, S, Vt = np.linalg.svd(Wm, full_matrices=False)  # line 7
        rr = truncation_rank(S, delta, r_max, rows, cols)  # line 8
        r[i - 1] = rr
        cores[i - 1] = freshape(Vt[:rr, :], (rr, ni, r[i]))  # line 9
        nbar = nbar * rr // cols  # line 10
        W = U[:, :rr] * S[:rr]  # line 11: U_{:,1:r} diag(sigma_1..sigma_r)
        res.sigmas[i] = S
        res.discarded2[i] = float(np.sum(S[rr:] ** 2))
    cores[0] = freshape(W, (1, n[0], r[1]))  # line 13
    return res


def tt_full(cores) -> np.ndarray:
    """Contract a tensor train back to the full tensor X~ (Sec. 2.1.2 definition)."""
    n = [c.shape[1] for c in cores]
    A = freshape(cores[0], (n[0], cores[0].shape[2]))
    N = n[0]
    for k in range(1, len(cores)):
        rk, nk, rk1 = cores[k].shape
        A = A @ freshape(cores[k], (rk, nk * rk1))
        N *= nk
        A = freshape(A, (N, rk1))
    return freshape(A, tuple(n))


def unfolding_singular_values(X: np.ndarray, k: int) -> np.ndarray:
    """Singular values of the k-th unfolding (n_1...n_k) x (n_{k+1}...n_d), brute force."""
    n = X.shape
    rows = int(np.prod(n[:k]))
    return np.linalg.svd(freshape(np.asarray(X, np.float64), (rows, -1)), compute_uv=False)


def core_orthonormality_defect(core: np.ndarray) -> float:
    """max |T T^T - I| for the r_{i-1} x (n_i r_i) matricization of a core (Alg. 1 line 9)."""
    r0 = core.shape[0]
    T = freshape(core, (r0, -1))
    return float(np.max(np.abs(T @ T.T - np.eye(r0))))


def planned_ranks(n, r_max: int) -> list:
    """Ranks of Alg. 1 without tolerance truncation: r_{i-1} = min(r_max, rows_i, n_i r_i)."""
    d = len(n)
    r = [1] * (d + 1)
    for i in range(d, 1, -1):
        cols = n[i - 1] * r[i]
        rows = int(np.prod(n[: i - 1]))
        r[i - 1] = max(1, min(r_max, rows, cols))
    return r
