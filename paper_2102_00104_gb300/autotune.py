"""Autotuner for the CTA-cooperative TSQR layouts (rows per panel and lanes per
column group), per m-bucket, on the GPU at hand.

``run()`` times every candidate layout of a bucket with the tt_tsqr building block
on a representative tall matrix (CUDA events, after a warm-up) and returns the
fastest; ``save``/``load`` keep the table in ``tune_table.json`` beside this file,
and the binding applies that table when it loads the library.
"""
from __future__ import annotations

import json
import os

PKG = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(PKG, "tune_table.json")

# bucket id -> (m used for timing, candidate layouts; ids < 16 are the built-in defaults)
BUCKETS = {1: (64, [1, 16, 18, 19]), 2: (80, [2, 17, 20]), 3: (128, [3])}


def apply(table: dict) -> None:
    from . import capi
    for key, val in table.items():
        capi.tt_tune_set(key, int(val))


def load(path: str = TABLE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        table = json.load(f).get("table", {})
    apply(table)
    return table


def save(table: dict, timings: dict, path: str = TABLE, note: str = "") -> None:
    with open(path, "w") as f:
        json.dump({"table": table, "timings_ms": timings, "note": note}, f, indent=1, sort_keys=True)


def run(rows: int = 1 << 22, reps: int = 3) -> tuple[dict, dict]:
    import torch

    from . import capi
    from .api import gen_uniform

    table, timings = {}, {}
    stream = torch.cuda.current_stream()
    for b, (m, cands) in BUCKETS.items():
        W = gen_uniform(rows * m, 7, torch.float64)
        wb = max(capi.tt_tsqr_query(rows, m, capi.TT_F64), 256)
        work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
        wp = (work.data_ptr() + 255) & ~255
        R = torch.empty(m * m, dtype=torch.float64, device="cuda")
        best = None
        key = f"tsqr.cfg.{b}"
        for cand in cands:
            capi.tt_tune_set(key, cand if cand >= 16 else -1)
            wb_c = capi.tt_tsqr_query(rows, m, capi.TT_F64)
            if wb_c > wb:
                continue
            capi.tt_tsqr(W.data_ptr(), capi.TT_F64, rows, m, rows, R.data_ptr(), wp, wb, int(stream.cuda_stream))
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                capi.tt_tsqr(W.data_ptr(), capi.TT_F64, rows, m, rows, R.data_ptr(), wp, wb,
                             int(stream.cuda_stream))
            e.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(e) / reps
            timings[f"{key}={cand}"] = ms
            if best is None or ms < best[1]:
                best = (cand, ms)
        if best is not None and best[0] >= 16:
            table[key] = best[0]
        capi.tt_tune_set(key, table.get(key, -1))
        del W, work
    return table, timings


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(PKG))
    t, tm = run()
    save(t, tm, note="float-float TSQR, rows = 2^22, GB300")
    print(json.dumps({"table": t, "timings_ms": tm}, indent=1))
