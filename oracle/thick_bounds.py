"""Thick-bounds TT-SVD (Alg. 3, Sec. 3.1.3 "Thick-bounds variant"), plain numpy FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and the benchmark's CPU baseline), never
by the product path; shares no code with the CUDA engine.

Alg. 3 combines the k right-most dimensions into one of size m = n_{d-k+1} ... n_d
(line 1: the smallest k with m >= max(m_min, r_est / f1_min), the reading of the
garbled threshold that reproduces the paper's rank table), runs the TT-SVD of the
reshaped (d-k+1)-way tensor (line 3), and recovers the cores of the combined
dimensions from a TT-SVD of the last core T_bar (line 4).  The recovery here, in the
paper's order: T_bar (r x m, orthonormal rows) is reshaped to (r, n_{d-k+1}, ..., n_d)
and decomposed by Alg. 1 with the same r_max; its first core S_0 (an r x rho_1
matrix) is absorbed into the core to its left, T^(d-k) <- T^(d-k) x_3 S_0, and its
other cores are T^(d-k+1) ... T^(d).  Only the r_max-prescribed form is defined (the
paper's experiments prescribe r_max; it gives no tolerance rule for the recovery).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .model import thick_bounds_k
from .tt_svd_oracle import TTResult, freshape, tt_svd


@dataclass
class ThickResult:
    cores: list
    ranks: list
    k: int                       # number of combined right-most dimensions
    m: int                       # their product
    reduced: TTResult | None = None   # TT-SVD of the reshaped tensor (line 3)
    recovery: TTResult | None = None  # TT-SVD of T_bar (line 4)
    notes: dict = field(default_factory=dict)

    @property
    def err2(self) -> float:
        """Discarded sigma^2 of the reduced decomposition plus that of the recovery (the
        latter measured on the orthonormal T_bar, so it is not scaled by X)."""
        return float(self.reduced.err2 + (self.recovery.err2 if self.recovery else 0.0))


def tt_svd_thick(X: np.ndarray, r_max: int, m_min: int = 16, f1_min: float = 0.5,
                 r_est: int | None = None) -> ThickResult:
    X = np.asarray(X, dtype=np.float64)
    n = list(X.shape)
    d = len(n)
    k = thick_bounds_k(n, m_min, f1_min, r_max if r_est is None else r_est)   # line 1
    if k <= 1 or k >= d:
        # nothing to combine (k = 1), or everything (k = d): Alg. 3 is Alg. 1
        res = tt_svd(X, r_max)
        return ThickResult(cores=res.cores, ranks=list(res.ranks), k=k, m=int(np.prod(n[d - k:])),
                           reduced=res)
    m = int(np.prod(n[d - k:]))
    Wt = freshape(X, n[: d - k] + [m])                        # line 2
    red = tt_svd(Wt, r_max)                                   # line 3
    Tbar = red.cores[d - k]                                   # (r, m, 1), orthonormal rows
    r = Tbar.shape[0]
    rec = tt_svd(freshape(Tbar, [r] + n[d - k:]), r_max)      # line 4: TT-SVD of T_bar
    S0 = freshape(rec.cores[0], (r, rec.ranks[1]))            # (1, r, rho_1) as r x rho_1
    Tl = red.cores[d - k - 1]                                 # (r_{d-k-1}, n_{d-k}, r)
    a, b, _ = Tl.shape
    Tl_new = freshape(freshape(Tl, (a * b, r)) @ S0, (a, b, S0.shape[1]))
    cores = list(red.cores[: d - k - 1]) + [Tl_new] + list(rec.cores[1:])
    ranks = list(red.ranks[: d - k]) + list(rec.ranks[1:])
    return ThickResult(cores=cores, ranks=ranks, k=k, m=m, reduced=red, recovery=rec)
