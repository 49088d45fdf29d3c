"""Multi-process plumbing with torch.distributed (no TT-SVD arithmetic here).

* ``max_over_ranks``: the benchmark's multi-GPU mode runs one independent
  TT-SVD per rank (weak scaling, no collective on the data path) and reports
  the slowest rank's time.
* ``shard_first_dims`` / ``gather_R``: the data movement of the distributed
  TSQR TT-SVD (Alg. 5, Sec. 3.1.3).  Rank j owns the sub-tensor with the first
  k indices fixed to its multi-index, stored contiguously; the only exchange of
  a step is the all-gather of every rank's m x m partial R, in rank order, so
  that every rank then runs the same fixed-order reduction tree and the same
  small SVD (identical ranks everywhere).  With one GPU per run the
  multi-GPU TSQR is not launched; this host logic is tested with CPU ranks.
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
