"""Autotuner for the TSQR level kernels of the float-float first level, per
m-bucket, on the GPU at hand.

Each bucket has a list of candidates; a candidate is a set of tuning keys
(``tt_tune_set``): the column-owned kernel with its default or an alternative
layout (``tsqr.colcfg.<bucket>``), or the row-group CTA kernel
(``tsqr.col.<bucket>`` = 0) with its default or alternative layout
(``tsqr.cfg.<bucket>``).  ``run()`` times every candidate with the tt_tsqr
building block on a representative tall matrix (CUDA events, after a warm-up)
and keeps the fastest; ``save``/``load`` keep the table in ``tune_table.json``
beside this file, and the binding applies that table when it loads the library.
"""
from __future__ import annotations

import json
import os

PKG = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(PKG, "tune_table.json")

# bucket -> (m used for timing, candidates); the first candidate is the built-in default
BUCKETS = {
    0: (32, [{}, {"tsqr.colcfg.0": 9}, {"tsqr.col.0": 0}]),
    1: (64, [{}, {"tsqr.colcfg.1": 5}, {"tsqr.colcfg.1": 6}, {"tsqr.colcfg.1": 8},
             {"tsqr.col.1": 0}, {"tsqr.col.1": 0, "tsqr.cfg.1": 16}]),
    2: (80, [{}, {"tsqr.colcfg.2": 7}, {"tsqr.col.2": 0}, {"tsqr.col.2": 0, "tsqr.cfg.2": 17}]),
    3: (128, [{}, {"tsqr.col.3": 0}]),
}
# value of every key when it is not set
DEFAULTS = {"tsqr.colcfg": -1, "tsqr.col": 1, "tsqr.cfg": -1}


def _default(key: str) -> int:
    return DEFAULTS[key.rsplit(".", 1)[0]]


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
        keys = sorted({k for c in cands for k in c})
        W = gen_uniform(rows * m, 7, torch.float64)
        wb = 0
        for cand in cands:
            for k in keys:
                capi.tt_tune_set(k, cand.get(k, _default(k)))
            wb = max(wb, capi.tt_tsqr_query(rows, m, capi.TT_F64))
        work = torch.empty(wb + 256, dtype=torch.uint8, device="cuda")
        wp = (work.data_ptr() + 255) & ~255
        R = torch.empty(m * m, dtype=torch.float64, device="cuda")
        best = None
        for cand in cands:
            for k in keys:
                capi.tt_tune_set(k, cand.get(k, _default(k)))
            run1 = lambda: capi.tt_tsqr(W.data_ptr(), capi.TT_F64, rows, m, rows, R.data_ptr(), wp, wb,
                                        int(stream.cuda_stream))
            run1()
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                run1()
            e.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(e) / reps
            name = ",".join(f"{k}={v}" for k, v in sorted(cand.items())) or "default"
            timings[f"m={m}:{name}"] = ms
            if best is None or ms < best[1]:
                best = (cand, ms)
        for k in keys:
            capi.tt_tune_set(k, best[0].get(k, _default(k)))
        table.update(best[0])
        del W, work
    return table, timings


if __name__ == "__main__":
    import sys
    sys.path.insert(0, os.path.dirname(PKG))
    t, tm = run()
    save(t, tm, note="float-float TSQR, rows = 2^22, GB300")
    print(json.dumps({"table": t, "timings_ms": tm}, indent=1))
