"""Alg. 5 (distributed TSQR TT-SVD, Sec. 3.1.3) with world-size-2 gloo ranks on the CPU.

The step loop and exchange of paper_2102_00104_gb300.distributed.tt_svd_alg5 run as in a
multi-GPU job; the local steps (TSQR R, small SVD, W V_r, the TT-SVD of the gathered V)
are plain numpy/LAPACK stand-ins here, since the library's kernels need a GPU (their own
parity is tested on the GPU, also through this loop: tests/test_gpu_alg5.py).  Every rank
must end with the oracle's ranks, its reconstruction error and its discarded energy."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300.distributed import shard_first_dims, tt_svd_alg5
from paper_2102_00104_gb300.inputs import uniform_tensor


class NumpyOps:
    """Local steps on the CPU (LAPACK through numpy), with the layouts of DeviceOps."""

    def tsqr(self, Wt):
        W = Wt.t().numpy()
        R = np.linalg.qr(W, mode="r")
        out = np.zeros((W.shape[1], W.shape[1]))
        out[:R.shape[0]] = R
        return torch.from_numpy(out)

    def svd(self, R):
        _, S, Vt = np.linalg.svd(R.numpy())
        return torch.from_numpy(S), torch.from_numpy(Vt.T.copy())

    def tsmm(self, Wt, V, r):
        return (Wt.t() @ V[:, :r]).t().contiguous()

    def tt_svd(self, flat, dims, r_max):
        res = O.tt_svd(flat.numpy().reshape(tuple(dims), order="F"), r_max)
        return [torch.from_numpy(c) for c in res.cores], res.err2


CASES = [((2, 3, 4, 5), 1, 3), ((2, 4, 3, 3, 2), 1, 4), ((2, 3, 4, 5, 3), 1, 100)]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for c, (dims, k, r_max) in enumerate(CASES):
            X = uniform_tensor(dims, seed=11 + c).ravel(order="F")
            local = torch.from_numpy(shard_first_dims(X, dims, k, rank).ravel(order="F").copy())
            cores, ranks, err2 = tt_svd_alg5([local], dims, k, r_max, NumpyOps())
            Xt = O.tt_full([cc.numpy() for cc in cores])
            full = X.reshape(dims, order="F")
            out[rank, c, 0] = np.linalg.norm(Xt - full) / np.linalg.norm(full)
            out[rank, c, 1] = err2
            out[rank, c, 2:2 + len(ranks)] = torch.tensor(ranks, dtype=torch.float64)
    finally:
        dist.destroy_process_group()


def test_alg5_two_cpu_ranks_matches_the_oracle():
    world = 2
    out = torch.zeros(world, len(CASES), 12, dtype=torch.float64).share_memory_()
    port = 29600 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert torch.equal(out[0], out[1])  # every rank holds the same decomposition
    for c, (dims, k, r_max) in enumerate(CASES):
        X = uniform_tensor(dims, seed=11 + c)
        ref = O.tt_svd(X, r_max)
        d = len(dims)
        assert [int(v) for v in out[0, c, 2:2 + d + 1]] == ref.ranks
        nx = np.linalg.norm(X)
        err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
        assert abs(float(out[0, c, 0]) - err_ref) <= 1e-12
        assert abs(float(out[0, c, 1]) - ref.err2) <= 1e-12 * nx * nx


def test_alg5_one_process_holding_every_rank():
    # a single process standing in for all m = n_1 n_2 ranks (k = 2), the layout the GPU
    # test uses: the same result as the oracle
    dims, k, r_max = (2, 2, 3, 4, 3), 2, 3
    X = uniform_tensor(dims, seed=5).ravel(order="F")
    parts = [torch.from_numpy(shard_first_dims(X, dims, k, j).ravel(order="F").copy()) for j in range(4)]
    cores, ranks, err2 = tt_svd_alg5(parts, dims, k, r_max, NumpyOps())
    full = X.reshape(dims, order="F")
    ref = O.tt_svd(full, r_max)
    assert ranks == ref.ranks
    nx = np.linalg.norm(full)
    err = np.linalg.norm(O.tt_full([c.numpy() for c in cores]) - full) / nx
    assert abs(err - np.linalg.norm(O.tt_full(ref.cores) - full) / nx) <= 1e-12
    assert abs(err2 - ref.err2) <= 1e-12 * nx * nx
