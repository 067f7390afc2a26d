"""Autotuning of the pressure solver's options (multigrid sweeps and FGMRES
restart length) per workload and precision.

The kernels' own launch shapes are tuned inside the library (multigrid tiles
and the bottom split, per solver shape); which (mg_pre, mg_post, restart) is
fastest depends on the precision as well: FP32 smoothing is cheap, so the
mixed path gains from more sweeps (fewer FP64 Krylov iterations), while the
Arnoldi work of each iteration -- FP64 dot products over j+1 basis vectors --
shrinks with a shorter restart.  Every candidate solves to the same FP64
relative residual, so the choice changes the time, not the tolerance.  Timing
is by CUDA events on the current stream; the candidates run on the caller's
own problem (a tank's first steps, or the caller's 3D system).
"""
from __future__ import annotations

import statistics

from . import wec

# (mg_pre, mg_post, restart)
CANDIDATES_2D = ((2, 2, 20), (2, 2, 8), (3, 3, 8), (4, 4, 8), (4, 4, 20))
CANDIDATES_3D = ((2, 2, 20), (2, 2, 5), (3, 3, 5), (4, 4, 5), (3, 3, 8))


def with_options(cfg, opts):
    """A copy of a tank workload dict with solver options (mg_pre, mg_post, restart)."""
    c = dict(cfg)
    c["solver"] = dict(cfg["solver"], mg_pre=opts[0], mg_post=opts[1], restart=opts[2])
    return c


def tune_tank(cfg, precision, candidates=CANDIDATES_2D, steps=20, warmup=5, net=None, pto=0.0):
    """Fastest (mg_pre, mg_post, restart) for a tank: each candidate steps a fresh
    tank from the workload's initial state (warm-up steps, then `steps` timed
    graph-replayed steps).  Returns (best, table)."""
    import torch
    stream = torch.cuda.current_stream()
    table = []
    for opts in candidates:
        t = wec.Tank(with_options(cfg, opts), precision=precision)
        if net is not None:
            t.set_net(net)
        for _ in range(warmup):
            t.step(cfg["dt"], pto)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record(stream)
        for _ in range(steps):
            its.append(t.step(cfg["dt"], pto)["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        t.close()
        table.append({"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2],
                      "ms_per_step": e0.elapsed_time(e1) / steps, "iters": statistics.mean(its)})
    best = min(table, key=lambda r: r["ms_per_step"])
    return (best["mg_pre"], best["mg_post"], best["restart"]), table


def tune_poisson3(shape, coef, b, precision, candidates=CANDIDATES_3D, rtol=1e-8, trials=2):
    """Fastest (mg_pre, mg_post, restart) for one 3D system (coef = device
    beta_x, beta_y, beta_z; b = device right-hand side): each candidate solves it
    from a zero guess `trials` times after one warm-up solve, the best time
    kept.  Returns (best, table)."""
    import torch
    stream = torch.cuda.current_stream()
    table = []
    x = torch.zeros_like(b)
    for opts in candidates:
        P = wec.Poisson3(*shape, precision=precision, restart=opts[2], mg_pre=opts[0], mg_post=opts[1])
        P.set_coefficients(*coef)
        ts, its = [], 0
        for r in range(trials + 1):
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = P.solve(b, x, rtol=rtol)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
            its = info["iters"]
        P.close()
        table.append({"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2], "ms_per_solve": min(ts),
                      "iters": its})
    best = min(table, key=lambda r: r["ms_per_solve"])
    return (best["mg_pre"], best["mg_post"], best["restart"]), table


CANDIDATES_TANK3 = ((2, 2, 20), (2, 2, 5), (3, 3, 5), (4, 4, 5))


def tune_tank3(cfg, precision, candidates=CANDIDATES_TANK3, steps=2, warmup=1):
    """Fastest (mg_pre, mg_post, restart) for a 3D tank (wec_tank3): each
    candidate steps a fresh tank from the workload's initial state.  Returns
    (best, table)."""
    import torch
    stream = torch.cuda.current_stream()
    table = []
    for opts in candidates:
        t = wec.Tank3(with_options(cfg, opts), precision=precision)
        for _ in range(warmup):
            t.step(cfg["dt"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record(stream)
        for _ in range(steps):
            its.append(t.step(cfg["dt"])["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        t.close()
        table.append({"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2],
                      "ms_per_step": e0.elapsed_time(e1) / steps, "iters": statistics.mean(its)})
    best = min(table, key=lambda r: r["ms_per_step"])
    return (best["mg_pre"], best["mg_post"], best["restart"]), table
