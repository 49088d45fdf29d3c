"""Multi-process plumbing with torch.distributed (no TT-SVD arithmetic here).

* ``max_over_ranks``: the benchmark's multi-GPU mode runs one independent
  TT-SVD per rank (weak scaling, no collective on the data path) and reports
  the slowest rank's time.
* ``shard_first_dims`` / ``gather_R``: the data movement of the distributed
  TSQR TT-SVD (Alg. 5, Sec. 3.1.3).  Rank j owns the sub-tensor with the first
  k indices fixed to its multi-index, stored contiguously; the only exchange of
  a step is the all-gather of every rank's m x m partial R, in rank order, so
  that every rank then runs the same fixed-order reduction tree and the same
  small SVD (identical ranks everywhere).
* ``tt_svd_alg5``: Alg. 5 itself, a host loop over the steps whose local work is
  done by ``DeviceOps`` (one C-ABI call of the library per step and block: TSQR R,
  small SVD, W V_r) and whose exchange is a torch.distributed all-gather (NCCL between
  GPUs).  The CPU tests drive the same loop with world-size-2 gloo ranks and plain
  numpy local steps.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def max_over_ranks(value: float, group=None, device=None) -> float:
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def shard_first_dims(X_fortran: np.ndarray, dims, k: int, rank: int) -> np.ndarray:
    """Rank ``rank``'s part of X for Alg. 5: indices (i_1..i_k) fixed to the rank's
    Fortran-order multi-index; returned as a contiguous (n_{k+1}, ..., n_d) tensor."""
    X = np.asarray(X_fortran).reshape(tuple(dims), order="F")
    idx = np.unravel_index(rank, tuple(dims[:k]), order="F")
    return np.ascontiguousarray(X[idx])


def gather_R(R_local: torch.Tensor, group=None) -> torch.Tensor:
    """All-gather of the m x m partial R factors, stacked in rank order ((world*m) x m)."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return R_local.clone()
    parts = [torch.empty_like(R_local) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, R_local.contiguous(), group=group)
    return torch.cat(parts, dim=0)


# ---- Alg. 5: distributed TSQR TT-SVD ---------------------------------------------------------
class DeviceOps:
    """The local steps of Alg. 5 on this process's GPU, each one call of the C ABI (the
    library's kernels): TSQR R of a tall matrix, small SVD, W V_r, and a plain TT-SVD.
    Matrices are column-major: a rows x m matrix is an (m, rows) C-order torch tensor."""

    def __init__(self, device="cuda"):
        from . import api
        self.api = api
        self.device = torch.device(device)

    def tsqr(self, Wt):
        return self.api.tsqr(Wt)  # (m, m) R

    def svd(self, R):
        return self.api.small_svd(R)  # sigma (m,), V (m, m)

    def tsmm(self, Wt, V, r):
        return self.api.tsmm(Wt, V, r)  # (r, rows): the column-major rows x r product

    def tt_svd(self, flat, dims, r_max):
        """TT-SVD of a small tensor given as flat Fortran-order data."""
        X = flat.reshape(tuple(reversed(dims))).contiguous()
        res = self.api.tt_svd(X, r_max, dims=list(dims))
        return [c.contiguous() for c in res.cores], res.err2


def _gather_rows(parts, group):
    """All-gather across processes of the per-rank blocks this process holds (a list, one
    block per local rank, in rank order): every process gets all blocks of all ranks."""
    local = torch.stack([p.contiguous() for p in parts])
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return [local[i] for i in range(local.shape[0])]
    world = dist.get_world_size(group)
    out = torch.empty((world * local.shape[0],) + tuple(local.shape[1:]), dtype=local.dtype,
                      device=local.device)
    dist.all_gather_into_tensor(out, local, group=group)
    return [out[i] for i in range(out.shape[0])]


def tt_svd_alg5(local_parts, dims, k: int, r_max: int, ops, group=None):
    """Alg. 5 (distributed TSQR TT-SVD, Sec. 3.1.3) with tol = 0.

    X (dims n_1..n_d) is distributed along its first k dimensions onto m = n_1...n_k
    ranks; rank j holds X[i_1..i_k = j's Fortran-order multi-index, :, ..., :] as flat
    Fortran-order data of the (n_{k+1}, ..., n_d) sub-tensor.  `local_parts` lists the
    parts this process holds, in rank order (one in a multi-process run, all m when a
    single process stands in for every rank); the processes' lists, concatenated in
    process order, are the m parts.

    Steps i = d..k+1 are Alg. 2 on the local parts with a global QR: every rank's local
    TSQR R (m_i x m_i) is all-gathered in rank order and the stacked R's are reduced by
    the same TSQR on every rank (a fixed order, so every rank gets the same R, the same
    small SVD and the same rank r_{i-1} = min(r_max, m_i, global rows)); W V_r stays local.
    After step k+1 each rank holds one row of length r_k; those rows, gathered in rank
    order, form V of shape (n_1, ..., n_{k-1}, n_k r_k), whose TT-SVD gives T^(1..k)
    (Alg. 5 lines 3-4).  Returns (cores, ranks, err2), the same on every rank: core i has
    shape (r_{i-1}, n_i, r_i); err2 is the sum of the discarded sigma^2 of every step."""
    d = len(dims)
    if not 1 <= k < d:
        raise ValueError("Alg. 5 needs 1 <= k < d")
    m_ranks = int(np.prod(dims[:k]))
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if len(local_parts) * world != m_ranks:
        raise ValueError(f"{m_ranks} ranks expected (n_1...n_k), got {len(local_parts)} x {world}")
    Ws = [p.reshape(-1) for p in local_parts]  # W^(d) of each rank, column-major
    cores = [None] * d
    ranks = [1] * (d + 1)
    err2 = 0.0
    r_i = 1
    rows_loc = int(np.prod(dims[k:d - 1]))  # rows of the local unfolding at step d
    for i in range(d, k, -1):  # global step i (1-based), columns m_i = n_i r_i
        n_i = dims[i - 1]
        m_i = n_i * r_i
        Wt = [W.reshape(m_i, rows_loc) for W in Ws]          # (m_i, rows) = column-major
        Rs = _gather_rows([ops.tsqr(w) for w in Wt], group)  # every rank's R, rank order
        R = Rs[0] if len(Rs) == 1 else ops.tsqr(torch.cat([r.t() for r in Rs], dim=1))
        sigma, V = ops.svd(R)
        rows_glob = m_ranks * rows_loc
        r = min(r_max, m_i, rows_glob)
        err2 += float(torch.sum(sigma[r:] ** 2).item()) if r < sigma.shape[0] else 0.0
        # T^(i) = reshape(V_{:,1:r}^T, (r, n_i, r_i)) in Fortran order: entry (a, j) of
        # V_r^T sits at a + r j, the C order of V_{:,1:r}
        cores[i - 1] = V[:, :r].contiguous().reshape(-1)
        ranks[i - 1] = r
        Ws = [ops.tsmm(w, V, r).reshape(-1) for w in Wt]     # rows_loc x r, column-major
        r_i = r
        rows_loc //= dims[i - 2] if i - 2 >= k else 1
    # every rank now holds one row of length r_k: V = (n_1, ..., n_{k-1}, n_k r_k)
    rows = _gather_rows([w.reshape(r_i) for w in Ws], group)  # m_ranks rows, rank order
    Vmat = torch.stack(rows)                                  # (m_ranks, r_k), C order
    vdims = list(dims[:k - 1]) + [dims[k - 1] * r_i]
    vflat = Vmat.t().contiguous().reshape(-1)                 # Fortran order of (n_1..n_k, r_k)
    if k == 1:
        cores[0] = vflat
    else:
        vc, e2 = ops.tt_svd(vflat, vdims, r_max)
        err2 += float(e2)
        for a in range(k):
            cores[a] = _fortran_flat(vc[a])
            ranks[a] = int(vc[a].shape[0])
    out = []
    for i in range(d):
        out.append(_as_core(cores[i], ranks[i], dims[i], ranks[i + 1]))
    return out, ranks, err2


def _fortran_flat(core):
    """Flat Fortran-order data of a (r0, n, r1) core (a torch tensor or view)."""
    return core.permute(2, 1, 0).contiguous().reshape(-1)


def _as_core(flat, r0, n, r1):
    """A (r0, n, r1) core from flat Fortran-order data (a torch view)."""
    return flat.reshape(r1, n, r0).permute(2, 1, 0)
