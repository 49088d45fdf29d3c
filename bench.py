#!/usr/bin/env python
"""TT-SVD benchmark: input GB/s of a 2^30-entry FP64 tensor (8^10, 8 GiB) on GB300.

One step = one truncated TT-SVD (Alg. 2: TSQR, small SVD, rank choice, core,
W*V_r for every step) of an i.i.d. uniform[0,1) 8^10 tensor resident in HBM,
r_max from --rmax (default 10), no tolerance truncation.  The input (8 GiB) is
larger than L2 (126 MB), so no flush is needed between steps.  The headline runs in
native FP64 arithmetic (--arith f64, the FP64-accurate form); the float-float form
(FP64 storage, ~48-bit arithmetic) is reported beside it with its own roofline.

value    = N * 8 GiB / (device time per step, CUDA events, max over ranks), GB/s
e2e      = the same metric when every step also copies X from pinned host
           memory and reads the cores, ranks and error back
roofline = the dominant kernel of the step, timed live with CUDA events inside
           the timed region by the library's profile mode; its ALU peak is this
           GPU's FMA rate measured at start-up by the library (tt_fma_rate)
Also reported: the float-float form, the planted TT-rank-16 input, the r_max sweep
{1,5,10,20,50} in both arithmetics, the FP32-storage form at r_max=32 with its error
against the FP64 form, the batched and serve forms, the oracle's throughput on host
cores (cpu_baseline) and SM clocks.

--impl reference times the CPU oracle (Alg. 1, numpy/LAPACK FP64) on the same
metric with a bounded sample of the workload.

Multi-GPU (torchrun): every rank decomposes its own tensor (independent
problems, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0
ARITH_LABEL = {"f64": "f64 (native FP64 arithmetic)",
               "df": "f64 storage, float-float (2xFP32, ~48-bit) arithmetic"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--rmax", type=int, default=10)
    p.add_argument("--n", type=int, default=8)
    p.add_argument("--d", type=int, default=10)
    p.add_argument("--arith", default="f64", choices=["df", "f64"],
                   help="arithmetic of the headline (f64: native FP64; df: float-float)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--alg5", action="store_true",
                   help="distributed TSQR TT-SVD (Alg. 5) instead of independent problems: the "
                        "tensor (N, n^d) is split along its first dimension over the N ranks, "
                        "one all-gather of the partial R's per step")
    p.add_argument("--no-extras", action="store_true", help="skip sweep, FP32 form, e2e, CPU baseline")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--serve-seconds", type=float, default=4.0)
    p.add_argument("--serve-only", action="store_true", help="only the serving leg (both admission orders)")
    p.add_argument("--case", default="", help="one building block for profiling instead of the bench: "
                   "tsqr:ROWS:M[:LAYOUT] (float-float TSQR of a uniform FP64 matrix), tsqr64:ROWS:M (native FP64), ttsvd32:N:D:RMAX (FP32 form), fma (ALU rate probes), "
                   "tsmm:ROWS:M:K (W V(:, 0:K) of a uniform FP64 W), tsmm64:ROWS:M:K (the same in native FP64) or svd:M (small SVD of a "
                   "uniform upper-triangular R) or ttsvd:N:D:RMAX:ARITH (a whole TT-SVD of a "
                   "uniform N^D FP64 tensor, ARITH f64 or df), each optionally followed by "
                   ":KEY=VALUE tuning keys; prints one JSON line")
    return p.parse_args()


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---- clocks during the timed region -------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- the metric and the workload, shared by both arms ---------------------------------------
METRIC = "TT-SVD input GB/s vs 2-read HBM roofline (FP64 form)"


# The paper's TT-SVD times for the 8^10 FP64 tensor on one 14-core Skylake socket (Sec. 5.2,
# the figure of TT-SVD variants on 8^10: the faster of the plain and thick-bounds
# algorithms), by r_max, in seconds.  Another machine's figure: context for vs_baseline.
PAPER_TIME_8P10_S = {1: 0.298, 5: 0.611, 10: 0.732, 20: 1.12, 50: 4.23}


def paper_input_gbs(n: int, d: int, r_max: int, dtype_bytes: int = 8):
    """The paper's input GB/s for the same metric and workload, or None when it has none."""
    if (n, d, dtype_bytes) != (8, 10, 8) or r_max not in PAPER_TIME_8P10_S:
        return None
    return dtype_bytes * n ** d / PAPER_TIME_8P10_S[r_max] / 1e9


def workload_config(n: int, d: int, r_max: int, ranks, world: int) -> dict:
    """The `config` of the JSON line: the same dict for the CUDA arm and the reference arm."""
    in_bytes = 8 * n ** d
    return {"workload": f"TT-SVD of a {n}^{d} FP64 tensor ({in_bytes / 2**30:.0f} GiB), r_max={r_max}, tol=0",
            "dims": [n] * d, "r_max": r_max, "ranks": list(ranks),
            "l2_flush": f"input {in_bytes / 2**30:.0f} GiB > L2 (129 MB), no flush",
            "parallelism": f"{world} independent problem(s), one per GPU"}


# ---- CPU oracle throughput ----------------------------------------------------------------
def cpu_oracle_rate(n: int, r_max: int, seconds: float, seed: int):
    """Times the oracle (Alg. 1, FP64) on a bounded sample: n^8 tensors, repeated."""
    import numpy as np  # noqa: F401

    from oracle import tt_svd_oracle as O
    from paper_2102_00104_gb300.inputs import uniform_tensor

    dims = (n,) * 8
    X = uniform_tensor(dims, seed=seed)
    reps, t0 = 0, time.perf_counter()
    while True:
        O.tt_svd(X, r_max)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 50:
            break
    cores = len(os.sched_getaffinity(0))
    gbs = reps * X.nbytes / el / 1e9
    return gbs, el / reps, cores, f"{reps} x Alg. 1 on a {n}^8 uniform FP64 tensor ({X.nbytes / 2**20:.0f} MiB), r_max={r_max}"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    K, W = max(1, args.steps), max(0, args.warmup)
    from oracle import tt_svd_oracle as O
    from paper_2102_00104_gb300.inputs import uniform_tensor
    dims = (args.n,) * 8
    X = uniform_tensor(dims, seed=args.seed)
    for _ in range(W):
        O.tt_svd(X, args.rmax)
    t0 = time.perf_counter()
    for _ in range(K):
        O.tt_svd(X, args.rmax)
    el = (time.perf_counter() - t0) / K
    gbs = X.nbytes / el / 1e9
    cores = len(os.sched_getaffinity(0))
    sample = f"Alg. 1 oracle on a {args.n}^8 uniform FP64 tensor ({X.nbytes / 2**20:.0f} MiB) per step, r_max={args.rmax}"
    config = workload_config(args.n, args.d, args.rmax, O.planned_ranks([args.n] * args.d, args.rmax), args.gpus)
    # each timed step of this arm is a bounded sample of the workload: name it
    config["sample_per_step"] = sample
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": el * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: i.i.d. uniform[0,1) from Philox4x32-10, generated on the host",
            "config": config,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- the GPU arm ------------------------------------------------------------------------------
def kernel_source_hash(files=None):
    """Hash of the CUDA sources a kernel is built from (all of csrc/ when files is None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2102_00104_gb300", "csrc")
    names = sorted(files) if files else sorted(os.listdir(csrc))
    for f in names:
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def lookup_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from an ncu capture, if the kernel's sources are unchanged since."""
    try:
        t = json.load(open(TRAFFIC_JSON))
    except Exception:
        return None
    e = t.get(f"{kernel}|{workload}")
    if not e or e.get("source_hash") != kernel_source_hash(e.get("source_files")):
        return None
    return e.get("bytes_per_launch")


def run_case(spec: str) -> int:
    """One building block, warmed up and run three times (for ncu captures of one kernel)."""
    import torch

    import __graft_entry__ as G
    from paper_2102_00104_gb300 import api, capi

    G.build()
    capi.lib()
    parts = [x for x in spec.split(":") if "=" not in x]
    for kv in (x for x in spec.split(":") if "=" in x):  # tuning keys, e.g. svd.block_nc=8
        key, val = kv.split("=", 1)
        capi.tt_tune_set(key, int(val))
    s = torch.cuda.current_stream()
    if parts[0] == "tsqr":
        rows, m = int(parts[1]), int(parts[2])
        if len(parts) > 3:
            bucket = 0 if m <= 32 else 1 if m <= 64 else 2 if m <= 80 else 3 if m <= 128 else 4
            capi.tt_tune_set(f"tsqr.colcfg.{bucket}", int(parts[3]))
        W = api.gen_uniform(rows * m, 3, torch.float64)
        R = torch.empty(m * m, dtype=torch.float64, device="cuda")
        wb = capi.tt_tsqr_query(rows, m, capi.TT_F64)
        work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
        wp = (work.data_ptr() + 255) & ~255
        call = lambda: capi.tt_tsqr(W.data_ptr(), capi.TT_F64, rows, m, rows, R.data_ptr(), wp, wb,
                                    int(s.cuda_stream))
    elif parts[0] == "tsqr64":
        # tsqr64:ROWS:M -- the native FP64 TSQR (tt_tsqr_ex) of a uniform FP64 matrix
        rows, m = int(parts[1]), int(parts[2])
        W = api.gen_uniform(rows * m, 3, torch.float64)
        R = torch.empty(m * m, dtype=torch.float64, device="cuda")
        wb = capi.tt_tsqr_query(rows, m, capi.TT_F64)
        work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
        wp = (work.data_ptr() + 255) & ~255
        call = lambda: capi.check(capi.lib().tt_tsqr_ex(W.data_ptr(), capi.TT_F64, rows, m, rows, R.data_ptr(),
                                                        wp, wb, capi.TT_ARITH_F64, int(s.cuda_stream)),
                                  "tt_tsqr_ex")
    elif parts[0] == "tsmm":
        rows, m, k = int(parts[1]), int(parts[2]), int(parts[3])
        W = api.gen_uniform(rows * m, 3, torch.float64)
        import numpy as np
        Vh = np.linalg.qr(np.random.default_rng(0).standard_normal((m, m)))[0]
        V = torch.from_numpy(np.asfortranarray(Vh).ravel(order="F").copy()).cuda()
        Y = torch.empty(rows * k, dtype=torch.float64, device="cuda")
        call = lambda: capi.tt_tsmm(W.data_ptr(), capi.TT_F64, rows, m, rows, V.data_ptr(), k,
                                    Y.data_ptr(), rows, int(s.cuda_stream))
    elif parts[0] == "tsmm64":
        # tsmm64:ROWS:M:K -- the native FP64 form's W V(:, 0:K) (tt_tsmm_ex)
        rows, m, k = int(parts[1]), int(parts[2]), int(parts[3])
        W = api.gen_uniform(rows * m, 3, torch.float64)
        import numpy as np
        Vh = np.linalg.qr(np.random.default_rng(0).standard_normal((m, m)))[0]
        V = torch.from_numpy(np.asfortranarray(Vh).ravel(order="F").copy()).cuda()
        Y = torch.empty(rows * k, dtype=torch.float64, device="cuda")
        call = lambda: capi.check(capi.lib().tt_tsmm_ex(W.data_ptr(), capi.TT_F64, rows, m, rows, V.data_ptr(), k,
                                                        Y.data_ptr(), rows, capi.TT_ARITH_F64,
                                                        int(s.cuda_stream)), "tt_tsmm_ex")
    elif parts[0] == "ttsvd":
        # ttsvd:N:D:RMAX:ARITH -- a whole TT-SVD of a uniform N^D FP64 tensor
        n, d, r, ar = int(parts[1]), int(parts[2]), int(parts[3]), parts[4]
        X = api.gen_uniform(n ** d, 3, torch.float64)
        plan = api.TTSVDPlan([n] * d, r, 0.0, torch.float64, ar)
        call = lambda: plan.run(X)
    elif parts[0] == "ttsvd32":
        # ttsvd32:N:D:RMAX -- the FP32 form (FP32 storage and panels) of a uniform N^D tensor
        n, d, r = int(parts[1]), int(parts[2]), int(parts[3])
        X = api.gen_uniform(n ** d, 3, torch.float32)
        plan = api.TTSVDPlan([n] * d, r, 0.0, torch.float32, "df")
        call = lambda: plan.run(X)
    elif parts[0] == "fma":
        # fma -- the library's multiply-add rate probes (the ALU peaks of the rooflines)
        rates = {"fp32_tflops": capi.tt_fma_rate(capi.FMA_FP32) / 1e12,
                 "fp64_tflops": capi.tt_fma_rate(capi.FMA_FP64) / 1e12,
                 "float_float_tflops_fp64eq": capi.tt_fma_rate(capi.FMA_DF) / 1e12,
                 "fp64_mma_tflops": capi.tt_fma_rate(capi.MMA_FP64) / 1e12}
        print(json.dumps({"case": spec, **rates}), flush=True)
        return 0
    elif parts[0] == "svd":
        m = int(parts[1])
        g = torch.Generator(device="cuda").manual_seed(0)
        Rm = torch.triu(torch.rand(m, m, dtype=torch.float64, device="cuda", generator=g)).contiguous()
        call = lambda: api.small_svd(Rm)
    else:
        raise SystemExit(f"unknown case {spec}")
    call()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(3):
        call()
    b.record(s)
    torch.cuda.synchronize()
    print(json.dumps({"case": spec, "ms": a.elapsed_time(b) / 3}), flush=True)
    return 0


def run_alg5(args):
    """Alg. 5 over the ranks of a torchrun launch: rank j holds the n^d part X[j, :, ..., :]
    of a (world, n, ..., n) tensor (its own Philox stream, generated on its GPU); every
    step's local TSQR, small SVD and W V_r run in the library's kernels and the partial R's
    are all-gathered over NCCL.  value = world * (part bytes) / (max over ranks of the time
    per decomposition)."""
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    from paper_2102_00104_gb300 import api, capi
    from paper_2102_00104_gb300.distributed import DeviceOps, max_over_ranks, tt_svd_alg5

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        G.build()
    if world > 1:
        dist.barrier()
    capi.lib()
    K, W = max(1, args.steps), max(3, args.warmup)
    dims = [world] + [args.n] * args.d
    nloc = args.n ** args.d
    part = api.gen_uniform(nloc, args.seed + 1000 * rank, torch.float64)
    ops = DeviceOps()
    for _ in range(W):
        cores, ranks, _ = tt_svd_alg5([part], dims, 1, args.rmax, ops)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = capi.tt_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        cores, ranks, _ = tt_svd_alg5([part], dims, 1, args.rmax, ops)
    e1.record()
    torch.cuda.synchronize()
    launches = (capi.tt_stats() - launches0) // K
    ms = max_over_ranks(e0.elapsed_time(e1) / K, device="cuda")
    value = world * nloc * 8 / (ms / 1e3) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ARITH_LABEL["df"], "data": "synthetic: i.i.d. uniform[0,1) from Philox4x32-10, per rank",
            "config": {"workload": f"Alg. 5: TT-SVD of a ({world}, {args.n}^{args.d}) FP64 tensor split "
                                   f"along its first dimension, r_max={args.rmax}, tol=0",
                       "ranks": ranks, "parallelism": f"alg5 over {world} GPU(s): all-gather of R per step",
                       "l2_flush": "input > L2, no flush"},
            "gpu_launches": int(launches)}), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def aggregate_profile(prof, ms_step):
    """Per-kernel records of the library's profile mode, averaged per (kernel, step)."""
    agg = {}
    for r in prof:
        key = (r["kind"], r["step"])
        a = agg.setdefault(key, {"ms": 0.0, "bytes": r["bytes"], "flops": r["flops"], "n": 0, "info": r["info"]})
        a["ms"] += r["ms"]
        a["n"] += 1
    out = []
    for (kind, step), a in agg.items():
        t = a["ms"] / a["n"]
        out.append({"kernel": kind, "step": step, "ms": t, "share": t / ms_step, "info": a["info"],
                    "gbs": a["bytes"] / (t / 1e3) / 1e9,
                    "tflops_fp64eq": a["flops"] / (t / 1e3) / 1e12, "bytes": a["bytes"], "flops": a["flops"]})
    out.sort(key=lambda e: -e["ms"])
    return out


def roofline_of(top, arith, alu_peaks, hbm_peak, peak_src, workload):
    """The roofline object of the dominant kernel: its ALU fraction against this GPU's
    measured FMA rate for the arithmetic, its HBM fraction against the measured copy
    bandwidth; `bound` is the larger of the two."""
    alu_peak = alu_peaks[arith]
    hbm_frac = top["gbs"] / hbm_peak
    alu_frac = top["tflops_fp64eq"] / alu_peak if top["flops"] > 0 else 0.0
    kname = f"{top['kernel']}@step{top['step']}"
    traffic = lookup_traffic(top["kernel"], f"{workload} step{top['step']}")
    src = {"f64": "FP64 FMA rate measured by tt_fma_rate in this run",
           "df": "float-float multiply-add rate measured by tt_fma_rate in this run (FP64-equivalent)",
           "f32": "FP32 FMA rate measured by tt_fma_rate in this run"}[arith]
    if alu_frac > hbm_frac:
        out = {"bound": "alu", "kernel": kname, "achieved": top["tflops_fp64eq"], "peak": alu_peak,
               "unit": "TFLOP/s" + (" (FP64-equivalent)" if arith == "df" else ""), "frac": alu_frac,
               "traffic": traffic, "peak_source": src,
               "hbm_view": {"achieved": top["gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
                            "peak_source": peak_src}}
        if arith == "f64" and top["kernel"] == "tsqr_first_level":
            out["note"] = ("achieved counts the level's algorithmic 2 rows m^2 FP64 flops; for m <= 80 "
                           "the blocked kernel runs 7/8 of its multiply-adds on the tensor cores (exact "
                           "Ozaki digit products) and keeps the reflector chain on the FP64 pipe, so the "
                           "fraction of the FP64 FMA rate can exceed 1")
        return out
    return {"bound": "hbm", "kernel": kname, "achieved": top["gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": hbm_frac, "traffic": traffic, "peak_source": peak_src,
            "alu_view": {"achieved": top["tflops_fp64eq"], "peak": alu_peak, "frac": alu_frac,
                         "peak_source": src}}


def time_plan(torch, plan, X, reps, stream, capi=None):
    """Device ms per TT-SVD over `reps` back-to-back runs (CUDA events on the stream), and
    the per-kernel profile records when capi is given."""
    plan.run(X, stream)
    torch.cuda.synchronize()
    if capi:
        capi.tt_profile(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        plan.run(X, stream)
    b.record(stream)
    torch.cuda.synchronize()
    prof = None
    if capi:
        prof = capi.tt_profile_read()
        capi.tt_profile(False)
    return a.elapsed_time(b) / reps, prof


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args.case)
    if args.alg5:
        return run_alg5(args)
    if args.serve_only:
        import torch

        import __graft_entry__ as G
        from paper_2102_00104_gb300 import api, capi
        G.build()
        capi.lib()
        out = {"serve": bench_serve(api, capi, torch, args.seed, args.serve_seconds, capi.TT_SERVE_SHORTEST, 10.0),
               "serve_fifo": bench_serve(api, capi, torch, args.seed, args.serve_seconds, capi.TT_SERVE_FIFO, 0.0)}
        print(json.dumps(out), flush=True)
        return 0

    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    from paper_2102_00104_gb300 import api, capi
    from paper_2102_00104_gb300.distributed import max_over_ranks

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        G.build()
    if world > 1:
        dist.barrier()
    capi.lib()

    K, W = max(1, args.steps), max(3, args.warmup)
    dims = [args.n] * args.d
    nbar = args.n ** args.d
    in_bytes = nbar * 8
    hbm_peak, peak_src = load_peaks()
    stream = torch.cuda.current_stream()
    # this GPU's arithmetic peaks, measured by the library (FP64-equivalent flop/s)
    alu_peaks = {"f64": capi.tt_fma_rate(capi.FMA_FP64) / 1e12, "df": capi.tt_fma_rate(capi.FMA_DF) / 1e12,
                 "f32": capi.tt_fma_rate(capi.FMA_FP32) / 1e12}

    X = api.gen_uniform(nbar, args.seed + 1000 * rank, torch.float64)
    plan = api.TTSVDPlan(dims, args.rmax, 0.0, torch.float64, args.arith)
    for _ in range(W):
        plan.run(X)
    res = plan.result()
    ranks = res.ranks

    def barrier():
        if world > 1:
            dist.barrier()

    launches0 = capi.tt_stats()
    capi.tt_profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        plan.run(X)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    prof = capi.tt_profile_read()
    capi.tt_profile(False)
    launches = (capi.tt_stats() - launches0) // K
    ms = e0.elapsed_time(e1) / K
    ms = max_over_ranks(ms, device="cuda")
    value = world * in_bytes / (ms / 1e3) / 1e9

    per_kernel = aggregate_profile(prof, ms)
    workload = f"{args.n}^{args.d} f64 r_max={args.rmax} {args.arith}"
    roof = roofline_of(per_kernel[0], args.arith, alu_peaks, hbm_peak, peak_src, workload)
    two_read_ms = 2 * in_bytes / (hbm_peak * 1e9) * 1e3

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(args, api, capi, torch, X, plan, dims, nbar, in_bytes, hbm_peak, peak_src,
                            stream, alu_peaks)

    paper = paper_input_gbs(args.n, args.d, args.rmax)
    out = {
        "metric": METRIC,
        "value": value, "unit": "GB/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / paper if paper else None,
        "vs_baseline_ref": ({"gbs": paper,
                             "source": "the paper's TT-SVD time for this tensor and r_max on one 14-core "
                                       "Skylake socket (Sec. 5.2), another machine: context, not the target"}
                            if paper else None),
        "dtype": ARITH_LABEL[args.arith],
        "data": "synthetic: i.i.d. uniform[0,1) from Philox4x32-10, generated on the device",
        "config": workload_config(args.n, args.d, args.rmax, ranks, world),
        "two_read_roofline": {"ms": two_read_ms, "frac": two_read_ms / ms, "hbm_gbs": hbm_peak, "source": peak_src},
        "roofline": roof,
        "alu_peaks_tflops": alu_peaks,
        "per_kernel": per_kernel,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    out.update(extras)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def tt_full_device(torch, cores, dims):
    """The full tensor of a TT (cores of shape (r_{i-1}, n_i, r_i), FP64, on the device) as
    a flat Fortran-order vector (n_1 fastest): measurement only, plain torch matmuls."""
    A = cores[0].reshape(dims[0], -1)  # (n_1, r_1): core 1 with r_0 = 1
    N = dims[0]
    for k in range(1, len(dims)):
        c = cores[k]  # (r_{k-1}, n_k, r_k) as a torch view
        r0, nk, r1 = c.shape
        A = A @ c.reshape(r0, nk * r1)  # (N, n_k r_k), column j r_k + b
        # (N, n_k, r_k) -> (N n_k, r_k) with row index i + N j (Fortran order)
        A = A.reshape(N, nk, r1).permute(1, 0, 2).reshape(N * nk, r1)
        N *= nk
    return A.reshape(-1)


def run_extras(args, api, capi, torch, X, plan, dims, nbar, in_bytes, hbm_peak, peak_src, stream,
               alu_peaks):
    out = {}
    two_read_ms = 2 * in_bytes / (hbm_peak * 1e9) * 1e3
    other = "df" if args.arith == "f64" else "f64"
    # e2e: host buffers through the public API, copies inside the timed region
    try:
        Xh = torch.empty(nbar, dtype=torch.float64, pin_memory=True)
        Xh.copy_(X)
        caps_bytes = sum(int(c.numel()) * 8 for c in plan.cores_buf)
        host_cores = [torch.empty(c.numel(), dtype=torch.float64, pin_memory=True) for c in plan.cores_buf]
        host_ranks = torch.empty(len(dims) + 1, dtype=torch.int64, pin_memory=True)
        host_err = torch.empty(1, dtype=torch.float64, pin_memory=True)
        K2 = 3
        for it in range(K2 + 1):
            if it == 1:
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            plan.run_host(Xh)  # tt_svd_from_host: the H2D copy overlaps the first TSQR level
            for hc, dc in zip(host_cores, plan.cores_buf):
                hc.copy_(dc, non_blocking=True)
            host_ranks.copy_(plan.ranks, non_blocking=True)
            host_err.copy_(plan.err2, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / K2
        out["e2e"] = {"value": in_bytes / (ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms,
                      "h2d_bytes_per_step": in_bytes,
                      "d2h_bytes_per_step": caps_bytes + host_ranks.numel() * 8 + 8,
                      "api": "tt_svd_from_host (pinned X, 16 row blocks) + D2H of cores, ranks, err2",
                      "arith": args.arith}
        del Xh
    except Exception as e:  # pinned 8 GiB may be refused on small hosts
        out["e2e"] = {"value": None, "unit": "GB/s", "error": str(e)[:200]}
    # the same workload in the other arithmetic, with its own per-kernel profile and roofline
    p = api.TTSVDPlan(dims, args.rmax, 0.0, torch.float64, other)
    ms, prof = time_plan(torch, p, X, 3, stream, capi)
    pk = aggregate_profile(prof, ms)
    key = "float_float_form" if other == "df" else "fp64_native_form"
    out[key] = {"dtype": ARITH_LABEL[other], "r_max": args.rmax, "ms": ms,
                "gbs": in_bytes / (ms / 1e3) / 1e9, "two_read_frac": two_read_ms / ms,
                "roofline": roofline_of(pk[0], other, alu_peaks, hbm_peak, peak_src,
                                        f"{args.n}^{args.d} f64 r_max={args.rmax} {other}"),
                "per_kernel": pk[:6], "ranks": p.result().ranks}
    del p
    # r_max sweep in both arithmetics (outside the timed region)
    for ar, reps in ((args.arith, 2), (other, 2)):
        sweep = {}
        for r in (1, 5, 10, 20, 50):
            p = api.TTSVDPlan(dims, r, 0.0, torch.float64, ar)
            ms, _ = time_plan(torch, p, X, reps if ar == "df" or r < 50 else 1, stream)
            sweep[str(r)] = {"ms": ms, "gbs": in_bytes / (ms / 1e3) / 1e9, "two_read_frac": two_read_ms / ms}
            del p
        out[f"rmax_sweep_{ar}"] = sweep
    out.update(bench_planted(args, api, torch, dims, nbar, in_bytes, stream, two_read_ms))
    # thick-bounds variant (Alg. 3, m_min = 16, f1_min = 1/2) and two-sided variant (Alg. 4)
    # beside the plain algorithm, float-float arithmetic
    thick, two = {}, {}
    for r in (1, 5, 10):
        p = api.TTSVDPlan(dims, r, 0.0, torch.float64, "df", thick=(16, 0.5))
        ms, _ = time_plan(torch, p, X, 2, stream)
        thick[str(r)] = {"ms": ms, "ranks": p.result().ranks}
        del p
    for r in (5, 10):
        p = api.TTSVDPlan(dims, r, 0.0, torch.float64, "df", two_sided=True)
        ms, _ = time_plan(torch, p, X, 2, stream)
        two[str(r)] = {"ms": ms, "ranks": p.result().ranks}
        del p
    out["thick_bounds_df"] = thick
    out["two_sided_df"] = two
    out["fp32_form"] = bench_fp32_form(args, api, torch, X, dims, nbar, stream, hbm_peak)
    out["batched"] = bench_batched(api, capi, torch, stream, args.seed)
    # shortest estimated work first (a request waiting 10 s goes first), then FIFO for comparison
    out["serve"] = bench_serve(api, capi, torch, args.seed, args.serve_seconds, capi.TT_SERVE_SHORTEST, 10.0)
    out["serve_fifo"] = bench_serve(api, capi, torch, args.seed, args.serve_seconds, capi.TT_SERVE_FIFO, 0.0)
    # oracle on the host cores
    gbs, sec, cores, sample = cpu_oracle_rate(args.n, args.rmax, args.cpu_seconds, args.seed)
    out["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                           "sample": sample, "seconds_per_sample": sec}
    return out


def bench_planted(args, api, torch, dims, nbar, in_bytes, stream, two_read_ms):
    """The second input of the 8^10 configuration: planted TT rank 16 (Gaussian cores,
    ||X||_F = 1) plus Gaussian noise with ||E||_F = 1e-6, built on the device; r_max in
    {10, 20, 50}, both arithmetics."""
    from paper_2102_00104_gb300.inputs import planted_tt_device
    Xp = planted_tt_device(dims, 16, args.seed + 1, noise_rel=1e-6)
    out = {"input": "planted TT rank 16 + 1e-6 relative Gaussian noise (reading c15), seed "
                    f"{args.seed + 1}, built on the device"}
    for ar in ("f64", "df"):
        leg = {}
        for r in (10, 20, 50):
            p = api.TTSVDPlan(dims, r, 0.0, torch.float64, ar)
            ms, _ = time_plan(torch, p, Xp, 1, stream)
            res = p.result()
            leg[str(r)] = {"ms": ms, "gbs": in_bytes / (ms / 1e3) / 1e9, "two_read_frac": two_read_ms / ms,
                           "ranks": res.ranks, "rel_err": (max(res.err2, 0.0) ** 0.5)}
            del p
        out[ar] = leg
    del Xp
    return {"planted_rank16": out}


def bench_fp32_form(args, api, torch, X, dims, nbar, stream, hbm_peak):
    """FP32-storage form (r_max = 32) against the FP64 form at the same r_max: time, and
    per tensor ||X~32 - X~64||_F / ||X||_F and ||X - X~||_F / ||X||_F, with X~ contracted
    on the device (X~64 from native FP64 arithmetic)."""
    X32 = api.gen_uniform(nbar, args.seed, torch.float32)  # the same values, rounded to FP32
    p32 = api.TTSVDPlan(dims, 32, 0.0, torch.float32, "df")
    ms32, _ = time_plan(torch, p32, X32, 3, stream)
    r32 = p32.result()
    out = {"r_max": 32, "ms": ms32, "gbs_fp32_input": nbar * 4 / (ms32 / 1e3) / 1e9,
           "entries_per_s": nbar / (ms32 / 1e3),
           "two_read_frac": (2 * nbar * 4 / (hbm_peak * 1e9) * 1e3) / ms32, "ranks": r32.ranks}
    nx = float(torch.linalg.vector_norm(X).item())
    T32 = tt_full_device(torch, r32.cores, dims)
    del p32, X32
    out["rel_err_vs_X"] = float(torch.linalg.vector_norm(X - T32).item()) / nx
    for ar in ("f64", "df"):
        p64 = api.TTSVDPlan(dims, 32, 0.0, torch.float64, ar)
        ms64, _ = time_plan(torch, p64, X, 1, stream)
        T64 = tt_full_device(torch, p64.result().cores, dims)
        out[f"fp64_form_{ar}"] = {"ms": ms64, "speedup_of_fp32_form": ms64 / ms32,
                                  "rel_err_vs_X": float(torch.linalg.vector_norm(X - T64).item()) / nx,
                                  "rel_diff_fp32_form": float(torch.linalg.vector_norm(T32 - T64).item()) / nx}
        del p64, T64
    del T32
    out["note"] = ("rel_diff_fp32_form = ||X~32 - X~64||_F / ||X||_F: the FP32 form against the FP64 "
                   "form on the same tensor (it includes the FP32 rounding of the input)")
    return out


def draw_shape(rng, lo_log2, hi_log2, d_lo, d_hi):
    """d ~ U{d_lo..d_hi}, target size 2^U(lo, hi), n_j from {2,3,4,8}: the draw whose
    log2 size is closest to the target (and inside [lo, hi]) out of 1000 tries."""
    import numpy as np
    d = int(rng.integers(d_lo, d_hi + 1))
    target = rng.uniform(lo_log2, hi_log2)
    best, best_gap = None, None
    for _ in range(1000):
        dims = [int(x) for x in rng.choice([2, 3, 4, 8], size=d)]
        l2 = float(np.log2(np.prod(dims, dtype=np.float64)))
        if l2 < lo_log2 or l2 > hi_log2:
            continue
        gap = abs(l2 - target)
        if best is None or gap < best_gap:
            best, best_gap = dims, gap
    if best is None:
        best = [2] * int(lo_log2)
    return best


def bench_batched(api, capi, torch, stream, seed, count=256):
    """256 tensors (d 6..12, n_j in {2,3,4,8}, 2^12..2^24 entries, FP64/FP32, r_max 4..32)
    in one tt_svd_batched call captured in a CUDA graph; replays are timed."""
    import numpy as np
    rng = np.random.default_rng(seed + 4)
    jobs, in_bytes = [], 0
    for t in range(count):
        dims = draw_shape(rng, 12, 24, 6, 12)
        dt = torch.float64 if rng.random() < 0.5 else torch.float32
        nent = int(np.prod(dims))
        X = api.gen_uniform(nent, seed + 10000 + t, dt)
        jobs.append(api.Job(X, dims, int(rng.integers(4, 33))))
        in_bytes += nent * (8 if dt == torch.float64 else 4)
    api.svd_batched(jobs)  # creates the stream pool, warms up
    torch.cuda.synchronize()
    cj = [j.c for j in jobs]
    wb = capi.tt_batched_query(cj)
    work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
    wp = (work.data_ptr() + 255) & ~255
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            capi.tt_svd_batched(cj, wp, wb, int(s.cuda_stream))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    reps = 5
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    a.record(cur)
    for _ in range(reps):
        g.replay()
    b.record(cur)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    bad = sum(int(j.status.item()) != 0 for j in jobs)
    return {"jobs": count, "ms": ms, "gbs": in_bytes / (ms / 1e3) / 1e9, "input_bytes": in_bytes,
            "graph": "one CUDA graph replay per batch", "jobs_with_device_errors": bad}


# requests on the device at once: small jobs are latency-bound chains of launches, so the
# device fills only with many of them in flight
SERVE_SLOTS = 64


def bench_serve(api, capi, torch, seed, seconds, policy, max_wait_s):
    """The serving configuration: Poisson arrivals at 200 req/s for `seconds`; requests with
    d in 6..14, n_j from {2,3,4,8} and 2^14..2^28 entries (log-uniform), 50/50 FP64/FP32;
    half use r_max in {4,8,16,32} on uniform inputs, half tol in {1e-2,1e-4} with an r_max
    cap of 64 on planted-rank inputs (ranks 4..32, 1e-3 relative noise).  Inputs come from a
    pool of 48 device-resident tensors made before the arrivals (not timed); the server
    admits requests under a 150 GB budget with SERVE_SLOTS slots, in the given admission
    order (TT_SERVE_SHORTEST with its aging bound, or TT_SERVE_FIFO)."""
    import numpy as np
    from paper_2102_00104_gb300.inputs import planted_tt_device
    rng = np.random.default_rng(seed + 5)
    pool = []
    for t in range(48):
        dt = torch.float64 if t % 2 == 0 else torch.float32
        dims = draw_shape(rng, 14, 28, 6, 14)
        if t % 4 < 2:
            X = api.gen_uniform(int(np.prod(dims)), seed + 20000 + t, dt)
            spec = (int(rng.choice([4, 8, 16, 32])), 0.0)
        else:
            X = planted_tt_device(dims, int(rng.integers(4, 33)), seed + 30000 + t, noise_rel=1e-3).to(dt)
            spec = (64, float(rng.choice([1e-2, 1e-4])))
        pool.append((dims, X, spec))
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # the server's arena is one allocation outside torch's cache
    srv = capi.tt_serve_create(150 << 30, max_inflight=SERVE_SLOTS, arena_bytes=96 << 30, policy=policy,
                               max_wait_s=max_wait_s)
    n_req = int(200 * seconds)
    gaps = rng.exponential(1.0 / 200.0, size=n_req)
    picks = rng.integers(0, len(pool), size=n_req)
    tickets, jobs, nbytes = [], [], 0
    t0 = time.perf_counter()
    due = t0
    for gap, pk in zip(gaps, picks):
        due += gap
        while time.perf_counter() < due:
            time.sleep(min(1e-4, max(0.0, due - time.perf_counter())))
        dims, X, (r, tol) = pool[int(pk)]
        j = api.Job(X, dims, r, tol)
        jobs.append(j)
        tickets.append(api.serve_submit(srv, j))
        nbytes += X.numel() * X.element_size()
    lat, bad = [], 0
    first_submit, last_done = None, None
    for t in tickets:
        code, res = capi.tt_serve_poll(srv, t, wait=True)
        if code != capi.TT_OK or res.status != capi.TT_OK:
            bad += 1
            continue
        capi.tt_serve_release(srv, t)
        lat.append(res.t_done - res.t_submit)
        first_submit = res.t_submit if first_submit is None else min(first_submit, res.t_submit)
        last_done = res.t_done if last_done is None else max(last_done, res.t_done)
    capi.tt_serve_destroy(srv)
    lat.sort()
    p50 = lat[len(lat) // 2] * 1e3 if lat else None
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))] * 1e3 if lat else None
    span = (last_done - first_submit) if lat else None
    sizes = sorted(int(np.prod(d)) for d, _, _ in pool)
    return {"requests": n_req, "seconds_of_arrivals": seconds, "rate_per_s": 200,
            "p50_ms": p50, "p99_ms": p99, "failed": bad, "input_bytes": nbytes,
            "gbs": nbytes / span / 1e9 if span else None,
            "offered_gbs": nbytes / seconds / 1e9,
            "sizes": "2^14..2^28 entries (log-uniform), d 6..14, n_j in {2,3,4,8}, 50/50 FP64/FP32; "
                     "r_max in {4,8,16,32} or tol in {1e-2,1e-4} (r_max cap 64); pool of 48 "
                     f"device-resident inputs, largest {sizes[-1]} entries",
            "budget_bytes": 150 << 30, "slots": SERVE_SLOTS, "arena_bytes": 96 << 30,
            "admission": ("shortest estimated work first, oldest first after %.0f s" % max_wait_s
                          if policy == capi.TT_SERVE_SHORTEST else "FIFO")}


if __name__ == "__main__":
    sys.exit(main())
