"""The reference arm of bench.py (the CPU oracle, timed on the host cores) keeps the JSON
contract of the CUDA arm: one line, the same metric, unit, direction and config, plus a
cpu_baseline block and a host-only e2e block; under a multi-rank launch only rank 0 runs."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--n", "4", "--d", "10", "--rmax", "8",
           "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)


def test_reference_line_matches_the_cuda_arm_contract():
    bench = load_bench()
    p = run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GB/s" and d["higher_is_better"] is True
    # 4^10 without tolerance: ranks min(8, 4^k, 4^(10-k))
    ranks = [1, 4, 8, 8, 8, 8, 8, 8, 8, 4, 1]
    # the workload's config, plus the name of the bounded sample each timed step runs
    cfg = dict(d["config"])
    assert "4^8" in cfg.pop("sample_per_step")
    assert cfg == bench.workload_config(4, 10, 8, ranks, 1)
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_exit_quietly():
    p = run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_paper_figure_for_vs_baseline():
    # 8^10 FP64 = 8.59 GB; the paper's 0.732 s at r_max = 10 is 11.7 GB/s of input
    bench = load_bench()
    assert abs(bench.paper_input_gbs(8, 10, 10) - 8 * 8 ** 10 / 0.732 / 1e9) < 1e-9
    assert round(bench.paper_input_gbs(8, 10, 10), 1) == 11.7
    assert round(bench.paper_input_gbs(8, 10, 1), 1) == 28.8
    # no figure for other workloads or for the FP32 form
    assert bench.paper_input_gbs(4, 10, 8) is None
    assert bench.paper_input_gbs(8, 10, 32) is None
    assert bench.paper_input_gbs(8, 10, 10, dtype_bytes=4) is None
