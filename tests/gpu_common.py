"""Helpers shared by the GPU tests (build once, move arrays, compare up to signs)."""
import numpy as np
import torch

from paper_2102_00104_gb300 import build as B
from paper_2102_00104_gb300 import capi

_built = False


def ensure_lib():
    global _built
    if not _built:
        B.build()
        capi.lib()
        _built = True


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def colmajor(W, dtype=torch.float64):
    """A rows x m numpy matrix as a (m, rows) CUDA tensor (= column-major storage)."""
    return dev(np.asarray(W).T.copy(), dtype)


def fortran_flat(X, dtype=torch.float64):
    return dev(np.asarray(X).ravel(order="F"), dtype)


def tt_full_dev(cores, dims):
    """X~ of a TT whose cores (r_{i-1}, n_i, r_i) are FP64 device tensors, as a flat
    Fortran-order device vector (n_1 fastest); plain torch matmuls, for the full-size checks
    the host cannot contract in reasonable time."""
    A = cores[0].reshape(dims[0], -1)  # (n_1, r_1)
    N = dims[0]
    for k in range(1, len(dims)):
        r0, nk, r1 = cores[k].shape
        # (N, r0) @ (r0, n_k r_k): column j r_k + b of the product is X~(i, j, b)
        A = (A @ cores[k].reshape(r0, nk * r1)).reshape(N, nk, r1)
        A = A.permute(1, 0, 2).reshape(N * nk, r1)  # row i + N j
        N *= nk
    return A.reshape(-1)
