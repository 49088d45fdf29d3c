"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no TT-SVD arithmetic.  It only makes input tensors:

* ``uniform_f64`` -- i.i.d. uniform[0, 1) doubles from the counter-based
  generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11).  The CUDA library implements the same
  generator independently (``tt_gen_uniform``); both are written from the
  published definition, so a tensor generated on the device is bit-identical
  to the one generated here.
* ``planted_tt`` -- a tensor with planted TT ranks: i.i.d. N(0,1) cores with
  ranks capped by the dimension products, contracted in FP64, scaled to
  ||X||_F = 1, plus i.i.d. Gaussian noise scaled to a relative Frobenius norm
  ``noise_rel`` (numpy's PCG64 generator; host only, copied to the device).

Entry e of a tensor (Fortran order, n_1 fastest) is the e-th uniform of the
stream: Philox block b = e // 2 gives two doubles, counter (b_lo, b_hi, 0, 0),
key (seed_lo, seed_hi).  A double is built from two 32-bit words x, y as
((x >> 5) * 2^26 + (y >> 6)) * 2^-53.
"""
from __future__ import annotations

import numpy as np

# Philox4x32 round multipliers and Weyl key increments (Salmon et al., SC'11)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (vectorised over the counters)."""
    c0 = np.asarray(c0, np.uint32)
    c1 = np.asarray(c1, np.uint32)
    c2 = np.asarray(c2, np.uint32)
    c3 = np.asarray(c3, np.uint32)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint32(k0 + PHILOX_W0)
                k1 = np.uint32(k1 + PHILOX_W1)
            p0 = PHILOX_M0 * c0.astype(np.uint64)
            p1 = PHILOX_M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _words_to_unit(x, y):
    a = (x >> np.uint32(5)).astype(np.float64)
    b = (y >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)


def uniform_f64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Entries start .. start+count-1 of the uniform[0,1) stream of ``seed``."""
    if count <= 0:
        return np.zeros(0)
    first_blk = start // 2
    last_blk = (start + count - 1) // 2
    blk = np.arange(first_blk, last_blk + 1, dtype=np.uint64)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    x0, x1, x2, x3 = philox4x32_10((blk & _MASK32).astype(np.uint32),
                                   (blk >> np.uint64(32)).astype(np.uint32),
                                   np.zeros(len(blk), np.uint32), np.zeros(len(blk), np.uint32),
                                   k0, k1)
    out = np.empty(2 * len(blk))
    out[0::2] = _words_to_unit(x0, x1)
    out[1::2] = _words_to_unit(x2, x3)
    off = start - 2 * first_blk
    return out[off:off + count]


def uniform_tensor(dims, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """An i.i.d. uniform[0,1) tensor of shape ``dims`` (indexed X[i_1..i_d], Fortran order)."""
    total = int(np.prod(dims))
    flat = np.empty(total)
    for s in range(0, total, chunk):
        flat[s:s + chunk] = uniform_f64(seed, min(chunk, total - s), s)
    return flat.reshape(tuple(dims), order="F")


def planted_tt(dims, rank: int, seed: int, noise_rel: float = 1e-6) -> np.ndarray:
    """A tensor with planted TT ranks plus relative Gaussian noise (relative noise level).

    Cores are i.i.d. N(0,1) with ranks r_k = min(rank, n_1..n_k, n_{k+1}..n_d);
    the contraction is done in FP64, scaled to ||X||_F = 1, and noise E with
    ||E||_F = noise_rel is added.
    """
    rng = np.random.default_rng(seed)
    d = len(dims)
    r = [1] * (d + 1)
    for k in range(1, d):
        r[k] = min(rank, int(np.prod(dims[:k])), int(np.prod(dims[k:])))
    A = rng.standard_normal((dims[0], r[1]))
    N = dims[0]
    for k in range(1, d):
        core = rng.standard_normal((r[k], dims[k] * r[k + 1]))
        A = A @ core  # (N, n_k r_{k+1}), column index i_k + n_k * a
        N *= dims[k]
        A = A.reshape((N, r[k + 1]), order="F")
    X = A.reshape(tuple(dims), order="F")
    X /= np.sqrt(np.sum(X * X))
    if noise_rel > 0:
        E = rng.standard_normal(X.shape)
        X += E * (noise_rel / np.sqrt(np.sum(E * E)))
    return X


def planted_tt_device(dims, rank: int, seed: int, noise_rel: float = 1e-6, device="cuda"):
    """planted_tt built on the device for tensors too large for the host: the same cores
    (numpy PCG64 from ``seed``, drawn in the same order), contracted in FP64 with torch on
    the device; the noise is N(0,1) from torch's generator seeded with ``seed`` (a different
    draw of the same distribution), scaled to ||E||_F = noise_rel ||X||_F.  Returns the flat
    Fortran-order FP64 tensor (n_1 fastest) as a device tensor."""
    import torch

    rng = np.random.default_rng(seed)
    d = len(dims)
    r = [1] * (d + 1)
    for k in range(1, d):
        r[k] = min(rank, int(np.prod(dims[:k])), int(np.prod(dims[k:])))
    A = torch.from_numpy(rng.standard_normal((dims[0], r[1]))).to(device)
    N = dims[0]
    for k in range(1, d):
        core = torch.from_numpy(rng.standard_normal((r[k], dims[k] * r[k + 1]))).to(device)
        A = A @ core  # (N, n_k r_{k+1}), column index i_k + n_k * a
        N *= dims[k]
        # Fortran-order reshape to (N n_k, r_{k+1}): column-major A is A^T in C order
        A = A.t().contiguous().view(r[k + 1], N).t()
    X = A.t().contiguous().view(-1)  # column-major (N, 1) data = Fortran order
    X /= torch.sqrt(torch.sum(X * X))
    if noise_rel > 0:
        g = torch.Generator(device=device).manual_seed(seed)
        E = torch.randn(X.numel(), dtype=torch.float64, device=device, generator=g)
        X += E * (noise_rel / torch.sqrt(torch.sum(E * E)))
        del E
    return X


def to_device_layout(X: np.ndarray) -> np.ndarray:
    """Flat Fortran-order copy of X (n_1 fastest): the memory layout the library expects."""
    return np.asarray(X).ravel(order="F")
