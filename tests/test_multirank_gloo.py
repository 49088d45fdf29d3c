"""World-size-2 gloo tests on CPU of the multi-process host logic: the benchmark's
max-over-ranks timing and the R exchange of the distributed TSQR (Alg. 5)."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.householder import qless_householder_block, tsqr_flat
from oracle.tt_svd_oracle import freshape
from paper_2102_00104_gb300.distributed import gather_R, max_over_ranks, shard_first_dims
from paper_2102_00104_gb300.inputs import uniform_tensor


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # max over ranks of a per-rank time
        out[rank, 0] = max_over_ranks(1.5 + rank)
        # Alg. 5: shard along n_1, local TSQR of the local last unfolding, gather, fixed-order tree
        dims = (2, 3, 4, 5)
        X = uniform_tensor(dims, seed=3).ravel(order="F")
        local = shard_first_dims(X, dims, 1, rank)            # (3, 4, 5) tensor
        W = freshape(local, (12, 5))
        R_local = torch.from_numpy(tsqr_flat(W, 4))
        stacked = gather_R(R_local)
        Rs = [stacked[5 * j:5 * (j + 1)].numpy() for j in range(world)]
        R = Rs[0]
        for Rb in Rs[1:]:
            R = qless_householder_block(Rb, R)
        out[rank, 1:] = torch.from_numpy(np.abs(R).ravel())
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    world = 2
    out = torch.zeros(world, 1 + 25, dtype=torch.float64).share_memory_()
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0, 0] == out[1, 0] == 2.5
    # every rank ends with the same R (fixed-order tree), equal up to row signs to the
    # R of the whole unfolding
    assert torch.equal(out[0, 1:], out[1, 1:])
    dims = (2, 3, 4, 5)
    X = uniform_tensor(dims, seed=3)
    Rfull = np.linalg.qr(freshape(X, (24, 5)), mode="r")
    assert np.allclose(out[0, 1:].numpy().reshape(5, 5), np.abs(Rfull), atol=1e-12)


def test_shard_is_a_partition():
    dims = (2, 3, 4)
    X = uniform_tensor(dims, seed=1).ravel(order="F")
    parts = [shard_first_dims(X, dims, 1, r) for r in range(2)]
    full = X.reshape(dims, order="F")
    for r in range(2):
        assert np.array_equal(parts[r], full[r])
