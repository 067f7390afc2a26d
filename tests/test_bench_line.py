"""The bench's printed JSON line stays small enough for a reader that keeps
only the tail of the output (a few KB), with every key of the contract."""
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
    cpu = {"value": 1234567.89, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
           "sample": "1 oracle step of the same 512x256x256 tank from its initial state on 16 host threads "
                     "(27.3 s, 9 FGMRES iterations)",
           "single_thread": {"value": 234567.8, "sample": "2 oracle steps of the same tank physics on a 128x64x64 "
                                                          "grid, 1 thread (12.3 s)"}}
    tank2d = {"workload": "2D tank 1024x256 (16 m x 4 m, JONSWAP Hs 0.15 m Tp 1.6 s, 64 components, box 1.0 x 0.8 m, "
                          "dt 5e-4 s, MPC PTO), learned warm start trained in the run",
              "steps": 100,
              "value": {k: 1.23456789e8 for k in ("mixed+learned", "mixed", "mixed_mg", "fp64")},
              "ms_per_step": {k: 1.23456789 for k in ("mixed+learned", "mixed", "mixed_mg", "fp64")},
              "speedup_vs_fp64": {k: 1.8456789 for k in ("mixed+learned", "mixed", "mixed_mg")},
              "fgmres_iters_per_step": {k: 6.3456789 for k in ("mixed+learned", "mixed", "mixed_mg", "fp64")},
              "guess_kept_steps": "104/110", "e2e_value": 1.76543e8,
              "roofline": {k: roof.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")}}
    line = bench.make_line3(c, 0, 1, steps, 5, tuned, res, t, tw, ck, roof, cpu, tank2d)
    line["detail_file"] = "bench_detail.json"
    text = json.dumps(line)
    assert len(text) < 6000, len(text)
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
