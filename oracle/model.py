"""Performance model of Sec. 4 (flops and bytes of TSQR, TSMM and the whole TT-SVD).

Test infrastructure only (see ``oracle/__init__.py``); the benchmark derives
its own algorithmic byte counts independently.

All byte counts are for an element size ``es`` (8 for double precision, the
paper's case).
"""
from __future__ import annotations

import numpy as np


def tsqr_flops(n: int, m: int, nb: int) -> float:
    """Sec. 4.1.1: (n / n_b) blocks, each m(m+1)(n_b+1) FMAs = 2 m (m+1)(n_b+1) flops."""
    return (n / nb) * 2.0 * m * (m + 1) * (nb + 1)


def tsqr_flops_approx(n: int, m: int, nb: int) -> float:
    """Sec. 4.1.1 simplified form used by the paper's estimates: (1 + 1/n_b) 2 n m^2."""
    return (1.0 + 1.0 / nb) * 2.0 * n * m * m


def tsqr_bytes(n: int, m: int, es: int = 8) -> float:
    """Sec. 4.1.1: a cache-friendly TSQR reads X once, V_read = es * n * m."""
    return float(es) * n * m


def tsqr_intensity(m: int, nb: int, es: int = 8) -> float:
    """Sec. 4.1.1: I_c ~ (1 + 1/n_b) m / 4 for doubles (general: (1+1/n_b) 2 m / es)."""
    return (1.0 + 1.0 / nb) * 2.0 * m / es


def tsmm_flops(n: int, m: int, k: int) -> float:
    """Sec. 4.1.2: Y = reshape(X M) costs 2 n m k flops."""
    return 2.0 * n * m * k


def tsmm_bytes(n: int, m: int, k: int, es: int = 8) -> float:
    """Sec. 4.1.2: reads X (es n m) and writes Y (es n k)."""
    return float(es) * n * (m + k)


def tsmm_intensity(m: int, k: int, es: int = 8) -> float:
    """Sec. 4.1.2: I_c = m k / (4 (m + k)) for doubles."""
    return 2.0 * m * k / (es * (m + k))


def ttsvd_volume_bound(nbar: float, fbar: float, es: int = 8) -> float:
    """Eq. (TT-SVD_data_volume): V <= 2 nbar/(1-f) + f nbar/(1-f) elements, times es bytes."""
    return es * (2.0 * nbar / (1.0 - fbar) + fbar * nbar / (1.0 - fbar))


def ttsvd_flops_bound(nbar: float, r_max: int, fbar: float) -> float:
    """Eq. (TT-SVD_operations): n_flops <= 2 nbar r_max (1/f + 2/(1-f))."""
    return 2.0 * nbar * r_max * (1.0 / fbar + 2.0 / (1.0 - fbar))


def ttsvd_step_counts(n, ranks, nb: int = 10**9, es: int = 8):
    """Per-step flops and bytes of the unfused Alg. 2 (TSQR then TSMM each step),
    with the TSQR flops in the paper's simplified (1 + 1/n_b) 2 n m^2 form.

    ``ranks`` = r_0..r_d.  Step i (d..2) works on rows_i x (n_i r_i) and
    produces r_{i-1} columns.  Returns a list of dicts, one per step.
    """
    d = len(n)
    out = []
    for i in range(d, 1, -1):
        rows = int(np.prod(n[: i - 1]))
        m = n[i - 1] * ranks[i]
        k = ranks[i - 1]
        out.append(dict(step=i, rows=rows, m=m, k=k,
                        flops=tsqr_flops_approx(rows, m, nb) + tsmm_flops(rows, m, k),
                        bytes=tsqr_bytes(rows, m, es) + tsmm_bytes(rows, m, k, es)))
    return out


def thick_bounds_k(n, m_min: int, f1_min: float, r_est: int) -> int:
    """Alg. 3 line 1 (reading of the garbled threshold): the smallest k such that
    m = n_{d-k+1} ... n_d satisfies m >= max(m_min, r_est / f1_min)."""
    d = len(n)
    m = 1
    for k in range(1, d + 1):
        m *= n[d - k]
        if m >= max(m_min, r_est / f1_min):
            return k
    return d
