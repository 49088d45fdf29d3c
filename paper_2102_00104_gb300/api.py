"""Thin PyTorch-facing wrappers over the C ABI (device memory and streams only).

PyTorch provides allocations and the current CUDA stream; every step of the
TT-SVD runs in the CUDA kernels of libttsvd.so.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import capi

_DT = {torch.float64: capi.TT_F64, torch.float32: capi.TT_F32}
_ARITH = {"auto": capi.TT_ARITH_AUTO, "df": capi.TT_ARITH_DF, "f64": capi.TT_ARITH_F64}


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass
class TTResult:
    cores: list                   # core i: (r_{i-1}, n_i, r_i) float64 Fortran data, as torch tensors
    ranks: list                   # r_0 .. r_d
    sigma: dict = field(default_factory=dict)   # step i -> singular values (torch, float64)
    err2: float = 0.0             # sum of discarded sigma^2

    def core_arrays(self):
        """Cores as numpy arrays of shape (r_{i-1}, n_i, r_i)."""
        out = []
        for c in self.cores:
            r0, n, r1 = c.shape
            out.append(c.detach().cpu().numpy().reshape((r0, n, r1), order="C"))
        return out


class TTSVDPlan:
    """Buffers for repeated tt_svd calls on one shape (workspace, cores, ranks, sigma).

    ``run(X)`` only launches (asynchronous on the stream); ``result()`` waits and
    trims the cores to the ranks found.
    """

    def __init__(self, dims, r_max: int, tol: float = 0.0, dtype=torch.float64, arith: str = "df",
                 want_sigma: bool = False, no_elide: bool = False, device="cuda", tsqr_ctas: int = 0,
                 thick=None, two_sided: bool = False):
        """thick = (m_min, f1_min[, r_est]) selects the thick-bounds variant (Alg. 3);
        two_sided = True the two-sided variant (Alg. 4)."""
        self.dims = [int(x) for x in dims]
        self.d = len(self.dims)
        self.r_max = int(r_max)
        self.tol = float(tol)
        self.dtype = dtype
        self.dt = _DT[dtype]
        th = tuple(thick) if thick else (0, 0.0, 0)
        th = th + (0,) * (3 - len(th))
        self.opts = capi.tt_opts(_ARITH[arith], 1 if no_elide else 0, int(tsqr_ctas), int(th[0]),
                                 float(th[1]), int(th[2]), 1 if two_sided else 0)
        _, self.work_bytes = capi.tt_query_ex(self.d, self.dims, self.r_max, self.tol, self.dt, self.opts)
        # also large enough for run_host (first TSQR level in row blocks)
        self.work_bytes = max(self.work_bytes, capi.tt_query_from_host(
            self.d, self.dims, self.r_max, self.tol, self.dt, 0))
        self.X_dev = None
        self.caps, self.sig_stride, sig_count = capi.tt_core_caps(self.d, self.dims, self.r_max)
        dev = torch.device(device)
        self.work = torch.empty(max(256, self.work_bytes) + 256, dtype=torch.uint8, device=dev)
        base = self.work.data_ptr()
        self.work_ptr = (base + 255) & ~255
        self.cores_buf = [torch.empty(max(1, c), dtype=torch.float64, device=dev) for c in self.caps]
        self.ranks = torch.empty(self.d + 1, dtype=torch.int64, device=dev)
        self.err2 = torch.zeros(1, dtype=torch.float64, device=dev)
        self.sigma = torch.empty(max(1, sig_count), dtype=torch.float64, device=dev) if want_sigma else None
        self._core_ptrs = [t.data_ptr() for t in self.cores_buf]

    def run(self, X: torch.Tensor, stream=None) -> None:
        if not X.is_cuda or X.dtype != self.dtype or not X.is_contiguous():
            raise ValueError("X must be a contiguous CUDA tensor of the plan's dtype")
        if X.numel() != int(torch.tensor(self.dims).prod()):
            raise ValueError("X does not have prod(dims) entries")
        capi.tt_svd(X.data_ptr(), self.dt, self.d, self.dims, self.r_max, self.tol, self._core_ptrs,
                    self.ranks.data_ptr(), self.sigma.data_ptr() if self.sigma is not None else None,
                    self.err2.data_ptr(), self.work_ptr, self.work_bytes, _stream_ptr(stream), self.opts)

    def run_host(self, X_host: torch.Tensor, stream=None, chunks: int = 0) -> None:
        """Same TT-SVD with X in (pinned) host memory: the copy to the device overlaps the
        first TSQR level, block by block (tt_svd_from_host)."""
        if X_host.is_cuda or X_host.dtype != self.dtype or not X_host.is_contiguous():
            raise ValueError("X_host must be a contiguous CPU tensor of the plan's dtype")
        if X_host.numel() != int(torch.tensor(self.dims).prod()):
            raise ValueError("X_host does not have prod(dims) entries")
        if self.X_dev is None:
            self.X_dev = torch.empty(X_host.numel(), dtype=self.dtype, device=self.work.device)
        need = capi.tt_query_from_host(self.d, self.dims, self.r_max, self.tol, self.dt, int(chunks))
        if need > self.work_bytes:  # more row blocks keep more partial R's
            torch.cuda.current_stream(self.work.device).synchronize()
            self.work = torch.empty(need + 256, dtype=torch.uint8, device=self.work.device)
            self.work_ptr = (self.work.data_ptr() + 255) & ~255
            self.work_bytes = need
        capi.tt_svd_from_host(X_host.data_ptr(), self.X_dev.data_ptr(), self.dt, self.d, self.dims,
                              self.r_max, self.tol, int(chunks), self._core_ptrs, self.ranks.data_ptr(),
                              self.sigma.data_ptr() if self.sigma is not None else None,
                              self.err2.data_ptr(), self.work_ptr, self.work_bytes, _stream_ptr(stream),
                              self.opts)

    def device_status(self, stream=None) -> int:
        return capi.tt_last_device_status(self.work_ptr, _stream_ptr(stream))

    def result(self, stream=None, check: bool = True) -> TTResult:
        st = self.device_status(stream)
        if check and st != capi.TT_OK:
            raise capi.TTError(st, "tt_svd (device)")
        r = [int(x) for x in self.ranks.cpu().tolist()]
        cores = []
        for i in range(self.d):
            cnt = r[i] * self.dims[i] * r[i + 1]
            # Fortran (r_{i-1}, n_i, r_i) data viewed as a C tensor of shape (r_i, n_i, r_{i-1})
            flat = self.cores_buf[i][:cnt]
            cores.append(flat.view(r[i + 1], self.dims[i], r[i]).permute(2, 1, 0))
        sig = {}
        if self.sigma is not None:
            rows = 1
            for a in range(self.d - 1):
                rows *= self.dims[a]
            for i in range(self.d, 1, -1):
                m = self.dims[i - 1] * r[i]
                s = min(rows, m)
                off = (self.d - i) * self.sig_stride
                sig[i] = self.sigma[off:off + s].clone()
                rows //= self.dims[i - 2]
        return TTResult(cores=cores, ranks=r, sigma=sig, err2=float(self.err2.item()))


def tt_svd(X: torch.Tensor, r_max: int, tol: float = 0.0, dims=None, arith: str = "df",
           want_sigma: bool = False, no_elide: bool = False, stream=None) -> TTResult:
    """Truncated TT-SVD of X (Alg. 2).  X: CUDA (or host) tensor indexed X[i_d, ..., i_1]
    (C order = the paper's Fortran order of X[i_1, ..., i_d]); dims = (n_1, ..., n_d)
    defaults to reversed(X.shape).  Host tensors are copied to the device first."""
    if dims is None:
        dims = list(reversed(X.shape))
    if not X.is_cuda:
        X = X.contiguous().to("cuda", non_blocking=True)
    plan = TTSVDPlan(dims, r_max, tol, X.dtype, arith, want_sigma, no_elide, device=X.device)
    plan.run(X.contiguous(), stream)
    return plan.result(stream)


def gen_uniform(count: int, seed: int, dtype=torch.float64, start: int = 0, device="cuda", stream=None):
    """Entries start..start+count-1 of the Philox4x32-10 uniform stream of ``seed`` on the device."""
    out = torch.empty(count, dtype=dtype, device=device)
    capi.tt_gen_uniform(out.data_ptr(), _DT[dtype], count, seed, start, _stream_ptr(stream))
    return out


def tsqr(W: torch.Tensor, stream=None, arith: str = "df") -> torch.Tensor:
    """R (m x m, FP64, upper triangular) of the Q-less TSQR of W.
    W: CUDA tensor of shape (m, rows), i.e. the column-major rows x m matrix.  arith "f64"
    with an FP64 W: every level in native FP64 (tt_tsqr_ex)."""
    m, rows = W.shape
    dt = _DT[W.dtype]
    wb = capi.tt_tsqr_query(rows, m, dt)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=W.device)
    wp = (work.data_ptr() + 255) & ~255
    R = torch.empty(m, m, dtype=torch.float64, device=W.device)  # R^T in C order
    ar = capi.TT_ARITH_F64 if arith == "f64" else capi.TT_ARITH_DF
    capi.check(capi.lib().tt_tsqr_ex(W.data_ptr(), dt, rows, m, W.stride(0), R.data_ptr(), wp, wb, ar,
                                     _stream_ptr(stream)), "tt_tsqr_ex")
    capi.check(capi.tt_last_device_status(wp, _stream_ptr(stream)), "tt_tsqr (device)")
    return R.t()


def small_svd(R: torch.Tensor, stream=None):
    """sigma (descending) and V of a square FP64 matrix R (torch, any layout)."""
    m = R.shape[0]
    Rc = R.t().contiguous()  # column-major storage of R
    wb = capi.tt_small_svd_query(m)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=R.device)
    wp = (work.data_ptr() + 255) & ~255
    sig = torch.empty(m, dtype=torch.float64, device=R.device)
    V = torch.empty(m, m, dtype=torch.float64, device=R.device)
    capi.tt_small_svd(Rc.data_ptr(), m, sig.data_ptr(), V.data_ptr(), wp, wb, _stream_ptr(stream))
    capi.check(capi.tt_last_device_status(wp, _stream_ptr(stream)), "tt_small_svd (device)")
    return sig, V.t()


def tsmm(W: torch.Tensor, V: torch.Tensor, k: int, stream=None, arith: str = "df") -> torch.Tensor:
    """Y = W V[:, :k] for W given as a (m, rows) tensor (column-major rows x m) and V (m x m FP64).
    Returns Y as a (k, rows) FP64 tensor (column-major rows x k).  arith "f64" with an FP64 W:
    the native FP64 form's product (tt_tsmm_ex)."""
    m, rows = W.shape
    Vc = V.t().contiguous()
    Y = torch.empty(k, rows, dtype=torch.float64, device=W.device)
    if arith == "f64":
        capi.check(capi.lib().tt_tsmm_ex(W.data_ptr(), _DT[W.dtype], rows, m, W.stride(0), Vc.data_ptr(), k,
                                         Y.data_ptr(), rows, capi.TT_ARITH_F64, _stream_ptr(stream)),
                   "tt_tsmm_ex")
    else:
        capi.tt_tsmm(W.data_ptr(), _DT[W.dtype], rows, m, W.stride(0), Vc.data_ptr(), k, Y.data_ptr(),
                     rows, _stream_ptr(stream))
    torch.cuda.synchronize()
    return Y


class Job:
    """A tt_job (C struct) with its device output buffers kept alive."""

    def __init__(self, X: torch.Tensor, dims, r_max: int, tol: float = 0.0, want_sigma: bool = False):
        self.X = X
        self.dims = [int(x) for x in dims]
        self.d = len(self.dims)
        self.r_max = int(r_max)
        self.tol = float(tol)
        dev = X.device
        caps, self.sig_stride, sig_count = capi.tt_core_caps(self.d, self.dims, self.r_max)
        self.cores_buf = [torch.empty(max(1, c), dtype=torch.float64, device=dev) for c in caps]
        self.ranks = torch.empty(self.d + 1, dtype=torch.int64, device=dev)
        self.err2 = torch.zeros(1, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.sigma = torch.empty(max(1, sig_count), dtype=torch.float64, device=dev) if want_sigma else None
        j = capi.tt_job()
        j.X = X.data_ptr()
        j.dtype = _DT[X.dtype]
        j.d = self.d
        for i, n in enumerate(self.dims):
            j.n[i] = n
        j.r_max = self.r_max
        j.tol = self.tol
        for i, t in enumerate(self.cores_buf):
            j.cores_out[i] = t.data_ptr()
        j.ranks_out = self.ranks.data_ptr()
        j.sigma_out = self.sigma.data_ptr() if self.sigma is not None else None
        j.err2_out = self.err2.data_ptr()
        j.status_out = self.status.data_ptr()
        self.c = j

    def result(self) -> TTResult:
        """Call after the work is complete (stream synchronised / request done)."""
        r = [int(x) for x in self.ranks.cpu().tolist()]
        cores = []
        for i in range(self.d):
            cnt = r[i] * self.dims[i] * r[i + 1]
            cores.append(self.cores_buf[i][:cnt].view(r[i + 1], self.dims[i], r[i]).permute(2, 1, 0))
        return TTResult(cores=cores, ranks=r, err2=float(self.err2.item()))


def serve_submit(srv, job: "Job", stream=None) -> int:
    """Queue a Job on a tt_serve server, ordered after the work queued so far on the
    stream (torch's current stream by default) that filled its input and cleared its outputs."""
    return capi.tt_serve_submit(srv, job.c, _stream_ptr(stream))


def svd_batched(jobs, stream=None):
    """Runs tt_svd_batched over Job objects (asynchronous on the stream); returns the workspace."""
    cj = [j.c for j in jobs]
    wb = capi.tt_batched_query(cj)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=jobs[0].X.device)
    wp = (work.data_ptr() + 255) & ~255
    capi.tt_svd_batched(cj, wp, wb, _stream_ptr(stream))
    return work
