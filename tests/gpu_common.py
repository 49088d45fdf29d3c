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
