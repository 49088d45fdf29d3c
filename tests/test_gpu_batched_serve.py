"""Batched and serve forms on the GPU: every job's result equals the single-call
result (same kernels, same inputs: identical), a captured CUDA graph replays the
batch, and the server gives the same results alone and in a mix of requests."""
import time

import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import api, capi
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor
from tests.gpu_common import ensure_lib, fortran_flat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def draw_jobs(count, seed, max_log2=14):
    """Small mixed jobs in the spirit of the batched configuration: d in 4..8,
    n_j from {2,3,4,8}, FP64/FP32, r_max in 4..32."""
    rng = np.random.default_rng(seed)
    jobs = []
    for t in range(count):
        d = int(rng.integers(4, 9))
        target = 2 ** rng.uniform(8, max_log2)
        best = None
        for _ in range(200):
            dims = tuple(int(x) for x in rng.choice([2, 3, 4, 8], size=d))
            tot = int(np.prod(dims))
            if best is None or abs(np.log2(tot) - np.log2(target)) < abs(np.log2(np.prod(best)) - np.log2(target)):
                best = dims
        dtype = torch.float64 if rng.random() < 0.5 else torch.float32
        r_max = int(rng.integers(4, 33))
        X = uniform_tensor(best, seed=1000 + t)
        jobs.append((best, dtype, r_max, X))
    return jobs


def single(dims, dtype, r_max, X, tol=0.0):
    plan = api.TTSVDPlan(dims, r_max, tol, dtype, "df")
    plan.run(fortran_flat(X, dtype))
    return plan.result()


def same_result(a, b):
    assert a.ranks == b.ranks
    for ca, cb in zip(a.cores, b.cores):
        assert torch.equal(ca, cb)


def test_batched_equals_single_calls():
    specs = draw_jobs(24, seed=1)
    jobs = [api.Job(fortran_flat(X, dt), dims, r) for dims, dt, r, X in specs]
    work = api.svd_batched(jobs)
    torch.cuda.synchronize()
    for job, (dims, dt, r, X) in zip(jobs, specs):
        assert int(job.status.item()) == 0
        same_result(job.result(), single(dims, dt, r, X))
    del work


def test_batched_parity_with_oracle():
    specs = draw_jobs(6, seed=2)
    jobs = [api.Job(fortran_flat(X, dt), dims, r) for dims, dt, r, X in specs]
    work = api.svd_batched(jobs)
    torch.cuda.synchronize()
    for job, (dims, dt, r, X) in zip(jobs, specs):
        Xr = X if dt == torch.float64 else X.astype(np.float32).astype(np.float64)
        ref = O.tt_svd(Xr, r)
        res = job.result()
        assert res.ranks == ref.ranks
        tol = 1e-10 if dt == torch.float64 else 1e-5
        nx = np.linalg.norm(Xr)
        err = np.linalg.norm(O.tt_full(res.core_arrays()) - Xr) / nx
        err_ref = np.linalg.norm(O.tt_full(ref.cores) - Xr) / nx
        assert abs(err - err_ref) <= tol
    del work


def test_batched_parity_with_oracle_large_jobs():
    # jobs of 2^16..2^20 entries (the upper part of the batched configuration that the oracle
    # still decomposes in seconds), mixed FP64/FP32, in one batch with small ones
    specs = draw_jobs(4, seed=12, max_log2=20)
    rng = np.random.default_rng(13)
    for t in range(3):
        d = int(rng.integers(6, 9))
        dims = tuple(int(x) for x in rng.choice([2, 4, 8], size=d))
        while np.prod(dims) < 2 ** 16:
            dims = dims + (2,)
        while np.prod(dims) > 2 ** 20:
            dims = dims[:-1]
        specs.append((dims, torch.float64 if t % 2 == 0 else torch.float32, int(rng.integers(4, 33)),
                      uniform_tensor(dims, seed=2000 + t)))
    jobs = [api.Job(fortran_flat(X, dt), dims, r) for dims, dt, r, X in specs]
    work = api.svd_batched(jobs)
    torch.cuda.synchronize()
    assert max(int(np.prod(s[0])) for s in specs) >= 2 ** 16
    for job, (dims, dt, r, X) in zip(jobs, specs):
        assert int(job.status.item()) == 0
        Xr = X if dt == torch.float64 else X.astype(np.float32).astype(np.float64)
        ref = O.tt_svd(Xr, r)
        res = job.result()
        assert res.ranks == ref.ranks
        tol = 1e-10 if dt == torch.float64 else 1e-5
        nx = np.linalg.norm(Xr)
        err = np.linalg.norm(O.tt_full(res.core_arrays()) - Xr) / nx
        err_ref = np.linalg.norm(O.tt_full(ref.cores) - Xr) / nx
        assert abs(err - err_ref) <= tol
    del work


def test_batched_graph_capture_replays():
    specs = draw_jobs(8, seed=3)
    jobs = [api.Job(fortran_flat(X, dt), dims, r) for dims, dt, r, X in specs]
    api.svd_batched(jobs)  # first call creates the library's stream pool outside capture
    torch.cuda.synchronize()
    refs = [j.result() for j in jobs]
    cj = [j.c for j in jobs]
    wb = capi.tt_batched_query(cj)
    work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) & ~255
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            capi.tt_svd_batched(cj, wp, wb, int(s.cuda_stream))
    for j in jobs:
        for t in j.cores_buf:
            t.zero_()
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for j, ref in zip(jobs, refs):
        same_result(j.result(), ref)


def test_serve_same_alone_and_in_mix():
    specs = draw_jobs(20, seed=4)
    # half of the requests use a tolerance on planted-rank tensors
    mixed = []
    for t, (dims, dt, r, X) in enumerate(specs):
        if t % 2:
            X = planted_tt(dims, 3, seed=t, noise_rel=1e-3)
            mixed.append((dims, dt, 64, X, 1e-2))
        else:
            mixed.append((dims, dt, r, X, 0.0))
    alone = [single(dims, dt, r, X, tol) for dims, dt, r, X, tol in mixed]
    srv = capi.tt_serve_create(8 << 30, max_inflight=6)
    try:
        jobs, tickets = [], []
        # the first half is queued at once; the second half arrives while the first runs
        for k, (dims, dt, r, X, tol) in enumerate(mixed):
            if k == len(mixed) // 2:
                code, res = capi.tt_serve_poll(srv, tickets[0], wait=True)
                assert code == capi.TT_OK
            j = api.Job(fortran_flat(X, dt), dims, r, tol)
            jobs.append(j)
            tickets.append(api.serve_submit(srv, j))
        spans = []
        for t, j, ref in zip(tickets, jobs, alone):
            code, res = capi.tt_serve_poll(srv, t, wait=True)
            assert code == capi.TT_OK and res.status == capi.TT_OK
            assert res.t_submit <= res.t_start <= res.t_done
            spans.append((res.t_start, res.t_done))
            same_result(j.result(), ref)
        # continuous batching: requests ran on the device at the same time, and some of
        # the later arrivals were admitted while earlier requests were still running
        overlaps = sum(1 for a in range(len(spans)) for b in range(a + 1, len(spans))
                       if spans[a][0] < spans[b][1] and spans[b][0] < spans[a][1])
        assert overlaps >= 1
        late = spans[len(spans) // 2:]
        early = spans[:len(spans) // 2]
        assert any(s0 < max(d for _, d in early) for s0, _ in late)
        # finished requests can be released; a released ticket is unknown afterwards
        for t in tickets:
            assert capi.tt_serve_release(srv, t) == capi.TT_OK
            assert capi.tt_serve_poll(srv, t, wait=False)[0] == capi.TT_EINVAL
            assert capi.tt_serve_release(srv, t) == capi.TT_EINVAL
    finally:
        capi.tt_serve_destroy(srv)


def test_serve_waits_for_the_submitters_stream():
    """The input is written on a side stream that is still busy at submission; the
    request must read the written values, and its zeroed outputs must not be cleared
    again after it ran."""
    dims = (4,) * 7
    X = uniform_tensor(dims, seed=21)
    ref = single(dims, torch.float64, 8, X)
    Xd = torch.zeros(X.size, dtype=torch.float64, device="cuda")
    src = fortran_flat(X)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    srv = capi.tt_serve_create(2 << 30, max_inflight=2)
    try:
        with torch.cuda.stream(side):
            torch.cuda._sleep(50_000_000)          # keeps the side stream busy for ~25 ms
            Xd.copy_(src)
            job = api.Job(Xd, dims, 8)             # outputs cleared on the side stream too
            t = api.serve_submit(srv, job, side)
        code, res = capi.tt_serve_poll(srv, t, wait=True)
        assert code == capi.TT_OK and res.status == capi.TT_OK
        side.synchronize()
        same_result(job.result(), ref)
    finally:
        capi.tt_serve_destroy(srv)


def test_serve_admission_under_budget_and_cancel():
    # a budget that fits about one large request at a time: requests queue and are
    # admitted as memory frees up; nothing is lost
    dims = (8,) * 7
    X = fortran_flat(uniform_tensor(dims, seed=9))
    _, wb = capi.tt_query(7, list(dims), 16, 0.0, capi.TT_F64)
    per_req = wb + X.numel() * 8 + 8 * 16 * 16 * 8 * 7
    srv = capi.tt_serve_create(int(per_req * 1.5), max_inflight=4, arena_bytes=int(wb * 1.5) + 4096)
    try:
        jobs = [api.Job(X, dims, 16) for _ in range(5)]
        tickets = [api.serve_submit(srv, j) for j in jobs]
        code, _ = capi.tt_serve_poll(srv, tickets[-1], wait=False)
        assert code in (capi.TT_EAGAIN, capi.TT_OK)
        starts = []
        for t in tickets:
            code, res = capi.tt_serve_poll(srv, t, wait=True)
            assert code == capi.TT_OK and res.status == capi.TT_OK
            starts.append((res.t_start, res.t_done))
        # admitted one at a time: each start is after the previous finish
        for (s0, d0), (s1, d1) in zip(starts, starts[1:]):
            assert s1 >= d0 - 1e-3
        ref = jobs[0].result()
        for j in jobs[1:]:
            same_result(j.result(), ref)
        # a request that can never fit the budget is refused at submission
        Xbig = torch.zeros(8 ** 8, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.TTError):
            api.serve_submit(srv, api.Job(Xbig, (8,) * 8, 16))
    finally:
        capi.tt_serve_destroy(srv)
    # stopping a server with queued requests cancels them and returns promptly
    srv = capi.tt_serve_create(int(per_req * 1.5), max_inflight=1, arena_bytes=int(wb * 1.5) + 4096)
    jobs = [api.Job(X, dims, 16) for _ in range(6)]
    tickets = [api.serve_submit(srv, j) for j in jobs]
    t0 = time.time()
    assert capi.lib().tt_serve_destroy(srv) == capi.TT_OK
    assert time.time() - t0 < 30
    torch.cuda.synchronize()


@pytest.mark.parametrize("policy,max_wait,small_first", [(capi.TT_SERVE_SHORTEST, 30.0, True),
                                                         (capi.TT_SERVE_FIFO, 0.0, False),
                                                         (capi.TT_SERVE_SHORTEST, 1e-6, False)])
def test_serve_admission_order(policy, max_wait, small_first):
    # one slot: a long request holds it while a large and three small requests queue.
    # SHORTEST admits the small ones before the large one; FIFO, or SHORTEST once the
    # large one has waited max_wait_s, admits in arrival order
    srv = capi.tt_serve_create(32 << 30, max_inflight=1, policy=policy, max_wait_s=max_wait)
    try:
        blocker = api.Job(api.gen_uniform(8 ** 8, 1, torch.float64), (8,) * 8, 10)
        big = api.Job(api.gen_uniform(8 ** 7, 2, torch.float64), (8,) * 7, 10)
        small = [api.Job(api.gen_uniform(4 ** 6, 3 + k, torch.float64), (4,) * 6, 4) for k in range(3)]
        torch.cuda.synchronize()
        tickets = [api.serve_submit(srv, j) for j in [blocker, big] + small]
        res = []
        for t in tickets:
            code, r = capi.tt_serve_poll(srv, t, wait=True)
            assert code == capi.TT_OK and r.status == capi.TT_OK
            res.append(r)
        t_big = res[1].t_start
        t_small = [r.t_start for r in res[2:]]
        if small_first:
            assert all(t < t_big for t in t_small), (t_big, t_small)
        else:
            assert all(t > t_big for t in t_small), (t_big, t_small)
    finally:
        capi.tt_serve_destroy(srv)
