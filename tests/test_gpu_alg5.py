"""Alg. 5 (distributed TSQR TT-SVD, Sec. 3.1.3) on the GPU: one process holds the parts of
all m = n_1...n_k ranks (the exchange is then a concatenation; the multi-process exchange
is tested with gloo ranks on the CPU), and every local step runs in the library's kernels
(tt_tsqr, tt_small_svd, tt_tsmm, tt_svd).  The result meets the FP64 bar of the other
parity tests against the Alg. 1 oracle on the whole tensor."""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300.distributed import DeviceOps, shard_first_dims, tt_svd_alg5
from paper_2102_00104_gb300.inputs import uniform_tensor
from tests.gpu_common import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,k,r_max", [((2, 2, 4, 4, 4, 4), 2, 5), ((4, 8, 8, 8, 8), 1, 10),
                                          ((2, 3, 4, 5, 6), 1, 100), ((3, 2, 4, 4, 2), 2, 3)])
def test_alg5_on_the_gpu(dims, k, r_max):
    ensure_lib()
    X = uniform_tensor(dims, seed=51).ravel(order="F")
    m = int(np.prod(dims[:k]))
    parts = [torch.from_numpy(shard_first_dims(X, dims, k, j).ravel(order="F").copy()).cuda()
             for j in range(m)]
    cores, ranks, err2 = tt_svd_alg5(parts, dims, k, r_max, DeviceOps())
    full = X.reshape(dims, order="F")
    ref = O.tt_svd(full, r_max)
    assert ranks == ref.ranks
    nx = np.linalg.norm(full)
    cs = [c.cpu().numpy() for c in cores]
    err = np.linalg.norm(O.tt_full(cs) - full) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - full) / nx
    assert abs(err - err_ref) <= 1e-10, (err, err_ref)
    assert abs(err2 - ref.err2) <= 1e-10 * nx * nx
    for c in cs[k:]:
        assert O.core_orthonormality_defect(c) <= 1e-12
