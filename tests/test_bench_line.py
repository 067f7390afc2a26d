"""The bench's printed JSON line stays small enough for a reader that keeps
only the last ~3 KB of the output (under 2.5 KB), with every key of the contract."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2206_07732_gb300 import synth  # noqa: E402


def _fake_run(steps):
    return {"ms": [71.234567] * steps, "wall": [0.0712345] * steps, "iters": [9] * steps,
            "residual": 7.123456789e-9, "launches": 1234 * steps}


def test_tank3d_line_is_compact_and_complete():
    c = synth.tank3d(seed=0)
    steps = 500
    res = {k: _fake_run(steps) for k, _ in bench.PATHS3}
    t = {k: sum(v["ms"]) / 1e3 for k, v in res.items()}
    tw = {k: sum(v["wall"]) for k, v in res.items()}
    tuned = {k: {"mg_pre": 3, "mg_post": 3, "restart": 5} for k in res}
    ck = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 1234}
    roof = {"bound": "hbm", "kernel": "mg3_rbgs", "achieved": 4896.66331, "peak": 6763.3, "unit": "GB/s",
            "frac": 0.7240171, "traffic": 907652361.0, "avg_launch_us": 137.317866, "share_of_step_gpu_time": 0.317,
            "peak_source": "measured", "algorithmic_bytes_per_launch": 672399360.0, "launches_timed": 24}
    cpu = {"value": 3041890.8357416485, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
           "sample": "1 step of the same 512x256x256 tank, 16 threads, 11.0 s",
           "single_thread": {"value": 298945.9545892255, "sample": "2 steps on 128x64x64, 3.5 s"}}
    tank2d = {"workload": "2D 1024x256 tank, learned warm start trained in the run",
              "value": {k: 1.23456789123e8 for k in ("mixed+learned", "mixed", "mixed_mg", "fp64")},
              "e2e": 1.765432123e8, "conv_roofline_frac": 0.149428196309143}
    line = bench.make_line3(c, 0, 1, steps, 5, tuned, res, t, tw, ck, roof, cpu, tank2d)
    line["batch"] = bench.rnd({"workload": "64 uneven 2D tanks, one graph launch per batch step",
                               "value": 3.1412345678e8, "ms_per_step": 21.912345678, "fp64_value": 1.2123456789e8,
                               "speedup_vs_fp64": 2.5987654321})
    line["detail_file"] = "results/run-001/bench_detail.json"
    text = json.dumps(line)
    assert len(text) < 2500, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline", "cpu_baseline"):
        assert k in line, k
    assert "workload" in line["config"]
    assert line["value"] > 0 and line["gpu_launches"] > 0
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"]
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"]
    # one line, no newline inside
    assert "\n" not in text
