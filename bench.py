#!/usr/bin/env python
"""Benchmark: cell-steps/s of the wave-tank step at a 1e-8 FP64 pressure residual.

Default workload (the largest configuration that fits one GPU): the 3D tank,
8 m x 4 m x 4 m on a 512 x 256 x 256 grid (33.5 M cells), depth 2 m, JONSWAP
Hs 0.2 m, Tp 2.0 s, gamma 3.3, 128 seeded components, a heaving vertical
cylinder (R 0.5 m, draft 0.4 m), dt 1e-3 s.  A step is one wec_tank3_step:
heave force and update, level set, momentum, pressure solve, projection.  The
headline `value` is the mixed-precision path of the precision contract (FP32
multigrid V-cycles inside the FP64 FGMRES; every stencil, the residual, the
Krylov orthogonalisation, the force and the heave FP64); beside it the plain
FP64 path and the FP32-stencil path, same GPU, each at its autotuned solver
options.  The U-Net of the learned warm start is two-dimensional: this
configuration runs without it, and the 2D tank with the learned path is
reported under `tank2d`.  The printed line keeps the keys a reader needs;
breakdowns, tuning tables and per-step records go to the --detail file.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tank3d|tank|batch|poisson3d] [--detail PATH]

--workload tank: the 2D 1024 x 256 JONSWAP tank with the learned warm start.
--workload batch: the 64 uneven 2D tanks of the batched configuration.
--workload poisson3d: the 3D pressure solve alone (512 x 256 x 256).

N > 1 (under torchrun): independent replicas, one tank per rank (a tank is not
partitioned), value = all ranks' cell-steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s at 1e-8 pressure residual: mixed+learned vs plain FP64, same GB300"
UNIT = "cell-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget (2D tank)")
    ap.add_argument("--workload", default="tank3d", choices=["tank3d", "tank", "batch", "poisson3d", "learned"])
    ap.add_argument("--learned-seeds", type=int, default=10, help="learned: training seeds")
    ap.add_argument("--learned-steps", type=int, default=2000, help="learned: problems per training seed")
    ap.add_argument("--train-iters", type=int, default=6000, help="learned: Adam steps")
    ap.add_argument("--no-2d", action="store_true", help="tank3d: skip the 2D tank reported beside it")
    ap.add_argument("--no-batch", action="store_true", help="tank3d: skip the batched 2D tanks reported beside it")
    ap.add_argument("--steps2d", type=int, default=0, help="tank3d: timed steps of the 2D tank (default 100)")
    ap.add_argument("--detail", default="bench_detail.json",
                    help="file for the breakdowns, tuning tables and per-step records ('' = none)")
    ap.add_argument("--ncu-steps", type=int, default=0,
                    help="profiling helper: run warm-up + this many steps only, print nothing")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_mg", "fp64", "mixed_fp32_stencils"],
                    help="profiling helper (tank3d): the path of the --ncu-steps run")
    ap.add_argument("--shape3", default=None,
                    help="profiling helper (tank3d): grid 'nx,ny,nz' of the --ncu-steps run (default 512,256,256)")
    ap.add_argument("--mg-opts", default=None,
                    help="profiling helper: solver options 'mg_pre,mg_post,restart' of the --ncu-steps run "
                         "(default: the workload's own)")
    return ap.parse_args()


def workload(seed):
    from paper_2206_07732_gb300 import synth
    return synth.tank_large(seed=seed)


def config_dict(cfg, precision, l2_note):
    return {"workload": cfg["name"], "grid": f"{cfg['nx']}x{cfg['ny']}", "cells": cfg["nx"] * cfg["ny"],
            "dt": cfg["dt"], "rtol": cfg["solver"]["rtol"], "precision": precision,
            "wave": "JONSWAP Hs=0.15 Tp=1.6 gamma=3.3 N=64", "body": "box 1.0x0.8 m, heave",
            "l2": l2_note, "seed": 0}


# ----------------------------------------------------------------- oracle --
def run_oracle(cfg, steps, budget_s=None):
    """Time the CPU oracle on the same workload; returns (cell-steps/s, steps run)."""
    from oracle.tank import OracleTank
    T = OracleTank(cfg)
    n = cfg["nx"] * cfg["ny"]
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        T.step(cfg["dt"])
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return n * done / el, done, el


# ------------------------------------------------------------------ clocks --
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline --
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tensor_peak():
    """Dense BF16 tensor peak: the sustained measurement (kernels timed inside a
    long step), else the burst one, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        if d.get("bf16_tflops_sustained"):
            return float(d["bf16_tflops_sustained"]), "measured bf16_tflops_sustained"
        return float(d["bf16_tflops"]), "measured bf16_tflops (burst)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback 1.7 PFLOP/s sustained"


def source_sha(files=None):
    """Hash of the library's kernel sources: the listed files of csrc/ (the
    translation unit of a profiled kernel), or all of them."""
    csrc = os.path.join(ROOT, "paper_2206_07732_gb300", "csrc")
    paths = sorted(glob.glob(os.path.join(csrc, "*"))) if files is None else [os.path.join(csrc, f) for f in files]
    h = hashlib.sha256()
    for f in paths:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """dram bytes per launch of `kernel_key` from a committed ncu summary, if it
    was captured on the current sources of that kernel (the summary's
    source_files, hashed; else None)."""
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(f) as fh:
            text = fh.read()
        m_k = re.search(r"^roofline_kernel:\s*(\S+)", text, re.M)
        m_s = re.search(r"^source_sha:\s*(\S+)", text, re.M)
        m_t = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
        m_f = re.search(r"^source_files:\s*(.+)$", text, re.M)
        files = m_f.group(1).split() if m_f else None
        if m_k and m_s and m_t and m_k.group(1) == kernel_key and m_s.group(1) == source_sha(files):
            return float(m_t.group(1))
    return None


def setup_lib():
    from paper_2206_07732_gb300 import build as B
    from paper_2206_07732_gb300 import wec
    B.build()
    return wec.load(), wec


# ---------------------------------------------------------------- our arm --
def make_controller(wec, torch, cfg, steps=8000):
    """The host MPC of the PTO force (untimed set-up): the box's effective mass
    and radiation damping from a free-decay run of the same tank in still water
    (released 2 cm below its draft), then the controller with the paper's
    parameters: dt_p 0.05 s, horizon one peak period, lam1 2 s, lam2 0.2 s,
    |F_PTO| <= the configuration's force limit."""
    import copy
    from paper_2206_07732_gb300 import mpc
    c = copy.deepcopy(cfg)
    c["wave"] = {"kind": "regular", "H": 0.0, "T": 1.6, "phase": 0.0}
    c["body"]["yc"] -= 0.02
    tank = wec.Tank(c, precision=wec.PREC_MIXED)
    recs = tank.step_n(steps, c["dt"])
    tank.close()
    kh = mpc.hydrostatic_stiffness(cfg["rho_w"], cfg["g"], cfg["body"]["width"])
    m_eff, c_r, wn, zeta = mpc.identify_free_decay([r["t"] for r in recs], [r["z"] - 0.02 for r in recs], kh)
    dt_p = 0.05
    Np = math.ceil(cfg["wave"]["Tp"] / dt_p)
    ctl = mpc.MPC(m_eff, kh, c_r, dt_p, Np, lam1=2.0, lam2=0.2, f_max=cfg["pto_limit"])
    info = {"model": "FOH heave model, J_3 objective, box QP (projected Newton) on the force sequence",
            "dt_p_s": dt_p, "Np": Np, "lam1_s": 2.0, "lam2_s": 0.2, "f_max_N_per_m": cfg["pto_limit"],
            "identified": {"m_eff_kg_per_m": m_eff, "c_r_Ns_per_m2": c_r, "omega_n": wn, "zeta": zeta,
                           "free_decay_steps": steps},
            "excitation": "k_h eta(x_B, t) of the tank's incident components (analytic forecast)"}
    return ctl, info


def make_controller3(wec, cfg, f_max=2000.0, shape=(128, 64, 64), dt=2e-3, steps=2000):
    """The host MPC of the 3D buoy's PTO force (untimed set-up): effective mass
    and radiation damping from a free-decay run of the same tank physics in
    still water on a coarser grid (128 x 64 x 64, h = 1/16 m), the cylinder
    released 2 cm below its draft; k_h = rho_w g pi R^2; then the controller
    with the paper's parameters (dt_p 0.05 s, horizon one peak period, lam1 2 s,
    lam2 0.2 s) and |F_PTO| <= f_max."""
    from paper_2206_07732_gb300 import mpc, synth
    c = synth.tank3d(seed=0, nx=shape[0], ny=shape[1], nz=shape[2])
    c["wave"] = {"kind": "regular", "H": 0.0, "T": 2.0, "phase": 0.0}
    c["body"]["zc"] -= 0.02
    T = wec.Tank3(c, precision=wec.PREC_MIXED)
    recs = [T.step(dt) for _ in range(steps)]
    T.close()
    b = cfg["body"]
    kh = cfg["rho_w"] * cfg["g"] * math.pi * b["radius"] ** 2
    m_eff, c_r, wn, zeta = mpc.identify_free_decay([r["t"] for r in recs], [r["z"] - 0.02 for r in recs], kh)
    dt_p = 0.05
    Np = math.ceil(cfg["wave"]["Tp"] / dt_p)
    ctl = mpc.MPC(m_eff, kh, c_r, dt_p, Np, lam1=2.0, lam2=0.2, f_max=f_max)
    info = {"identified": {"m_eff_kg": m_eff, "body_mass_kg": b["mass"], "c_r_Ns_per_m": c_r, "omega_n": wn,
                           "zeta": zeta, "free_decay": f"{steps} steps of dt {dt} s on {shape}"},
            "dt_p_s": dt_p, "Np": Np, "f_max_N": f_max}
    return ctl, info


class PtoSchedule:
    """Per-step PTO force of the MPC: a QP every dt_p of simulated time, the
    first force reached by first-order hold over the solver steps in between."""

    def __init__(self, ctl, cfg, wec):
        self.ctl, self.dt = ctl, cfg["dt"]
        self.nsub = int(round(ctl.dt_p / cfg["dt"]))
        amp, om, ph = wec.wave_components(cfg["wave"])
        kw = np.array([wec.wave_number(w, cfg["depth"], cfg["g"]) for w in om])
        xb = cfg["body"]["xc"]
        self.fexc = lambda t: ctl.kh * float(np.sum(amp * np.cos(kw * xb - om * t + ph)))
        self.F_now, self.ramp, self.k = 0.0, None, 0
        self.solves, self.fmax = 0, 0.0

    def force(self, z, zd):
        """Force for the next step, given the body state after the last one."""
        if self.k % self.nsub == 0:
            t0 = self.k * self.dt
            fut = [self.fexc(t0 + (i + 1) * self.ctl.dt_p) for i in range(self.ctl.Np)]
            F_next = float(self.ctl.solve(z, zd, self.F_now, self.fexc(t0), fut)[0])
            self.ramp = self.ctl.ramp(self.F_now, F_next, self.nsub)
            self.F_now = F_next
            self.solves += 1
        f = float(self.ramp[self.k % self.nsub])
        self.fmax = max(self.fmax, abs(f))
        self.k += 1
        return f


def time_path(L, wec, torch, cfg, precision, steps, warmup, flush, graph=True, profile_kernel=None, net=None,
              ctl=None):
    """Time K steps (CUDA events per step on the caller's stream, L2 flushed in
    between).  graph=False with profile_kernel: the eager pass that times one
    kernel's launches with event pairs (graph bodies cannot hold events).
    net: the trained U-Net giving each solve its initial guess; ctl: the MPC
    setting each step's PTO force (its QP runs on the host between steps)."""
    sched = PtoSchedule(ctl, cfg, wec) if ctl is not None else None
    state = [0.0, 0.0]

    def pto():
        return sched.force(*state) if sched else 0.0

    tank = wec.Tank(cfg, precision=precision)
    tank.use_graph(graph)
    if net is not None:
        tank.set_net(net)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        r = tank.step(cfg["dt"], pto())
        state[:] = [r["z"], r["zdot"]]
    torch.cuda.synchronize()
    if profile_kernel:
        wec.profile_read()
        wec.profile_enable(2, profile_kernel)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its, res = [], []
    n0 = wec.launch_count()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(steps):
        f = pto()  # host QP (every dt_p) outside the timed events
        flush.zero_()  # evict the working set from L2 (outside the timed events)
        ev[k][0].record(stream)
        r = tank.step(cfg["dt"], f)
        ev[k][1].record(stream)
        state[:] = [r["z"], r["zdot"]]
        its.append(r["iters"])
        res.append(r["residual"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    launches = wec.launch_count() - n0
    prof = None
    if profile_kernel:
        wec.profile_enable(0)
        prof = wec.profile_read()
    ms = [a.elapsed_time(b) for a, b in ev]
    stats = tank.net_stats() if net is not None else None
    tank.close()
    return dict(ms=ms, iters=its, residual=max(res), launches=launches, wall=wall, prof=prof, net_stats=stats,
                qp_solves=sched.solves if sched else 0, max_pto=sched.fmax if sched else 0.0)


def profile_all(wec, torch, cfg, precision, steps=2, net=None):
    """Untimed eager pass with every launch timed: which kernel dominates."""
    tank = wec.Tank(cfg, precision=precision)
    tank.use_graph(False)
    if net is not None:
        tank.set_net(net)
    for _ in range(3):
        tank.step(cfg["dt"])
    torch.cuda.synchronize()
    wec.profile_read()
    wec.profile_enable(1)
    for _ in range(steps):
        tank.step(cfg["dt"])
    wec.profile_enable(0)
    p = wec.profile_read()
    tank.close()
    return p


def e2e_path(wec, torch, cfg, precision, steps, warmup, flush, net=None, ctl=None):
    """Through the public call with host buffers: wec_step takes the host PTO
    force and returns the host step record (synchronous D2H) every step; the
    MPC's host QP (every dt_p) is inside the timed region."""
    sched = PtoSchedule(ctl, cfg, wec) if ctl is not None else None
    tank = wec.Tank(cfg, precision=precision)
    if net is not None:
        tank.set_net(net)
    z = zd = 0.0
    for _ in range(warmup):
        r = tank.step(cfg["dt"], sched.force(z, zd) if sched else 0.0)
        z, zd = r["z"], r["zdot"]
    torch.cuda.synchronize()
    t = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = tank.step(cfg["dt"], sched.force(z, zd) if sched else 0.0)  # record read back inside the call
        z, zd = r["z"], r["zdot"]
        t.append(time.perf_counter() - t0)
    tank.close()
    return t


def time_batch(wec, torch, cfgs, precision, steps, warmup, flush):
    """K batch steps, CUDA events on the caller's stream around each (the batch
    orders itself after and before that stream), L2 flushed in between."""
    B = wec.Batch(cfgs, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    dts = [c["dt"] for c in cfgs]
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        B.step(dts)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its, res, wall = [], [], []
    n0 = wec.launch_count()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        t0 = time.perf_counter()
        r = B.step(dts)  # host dt / PTO in, host records out, inside the call
        wall.append(time.perf_counter() - t0)
        ev[k][1].record(stream)
        its += [x["iters"] for x in r]
        res += [x["residual"] for x in r]
    torch.cuda.synchronize()
    launches = wec.launch_count() - n0
    B.close()
    return dict(ms=[a.elapsed_time(b) for a, b in ev], iters=its, residual=max(res), launches=launches, wall=wall)


def run_batch_leg(wec, torch, seed, rank, world, steps=20, warmup=3):
    """The 64 uneven 2D tanks of the batched configuration, mixed and FP64,
    `steps` timed batch steps each (the tanks sharded over ranks, the slowest
    rank's time): a compact summary and the detail."""
    from paper_2206_07732_gb300 import synth
    allc = synth.batch_tanks(64, seed=seed)
    cfgs = [c for i, c in enumerate(allc) if i % world == rank]
    cells = sum(c["nx"] * c["ny"] for c in allc)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    mixed = time_batch(wec, torch, cfgs, wec.PREC_MIXED, steps, warmup, flush)
    fp64 = time_batch(wec, torch, cfgs, wec.PREC_FP64, steps, warmup, flush)
    del flush

    def slowest(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    tm, tf = slowest(sum(mixed["ms"]) / 1e3), slowest(sum(fp64["ms"]) / 1e3)
    summary = {"workload": "64 uneven 2D tanks, one graph launch per batch step", "value": cells * steps / tm,
               "ms_per_step": tm / steps * 1e3, "fp64_value": cells * steps / tf, "speedup_vs_fp64": tf / tm}
    detail = dict(summary, cells=cells, tanks=64, steps=steps, warmup=warmup, ms_all=mixed["ms"],
                  fp64_ms_all=fp64["ms"], fgmres_iters_mean=sum(mixed["iters"]) / max(1, len(mixed["iters"])),
                  launches=mixed["launches"])
    return summary, detail


def bench_poisson3d(wec, torch, seed, solves=5, warmup=3, shape=(512, 256, 256), cpu_seconds=10.0):
    """The 3D pressure solve (wec_poisson_create3) to a 1e-8 FP64 relative
    residual from a zero guess, FP64 and mixed precision: CUDA events around
    each solve on the solver's stream (inputs 268 MB per vector, larger than L2),
    then one eager solve with every launch timed (per-kernel breakdown and the
    HBM roofline of the dominant kernel).  cpu_seconds > 0: the oracle's solve of
    the same structure on a 128 x 64 x 64 grid as the CPU baseline."""
    from paper_2206_07732_gb300 import synth
    nx, ny, nz = shape
    n = nx * ny * nz
    bx, by, bz, b = synth.poisson3d_case(nx, ny, nz, seed=seed)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    cb = [dev(a) for a in (bx, by, bz)]
    bd = dev(b)
    del bx, by, bz, b
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    out = {"workload": f"3D pressure solve {nx}x{ny}x{nz} (8 m x 4 m x 4 m, h = 1/64 m): water/air coefficients "
                       "across a seeded irregular surface, cylinder buoy (R 0.5 m, L 0.8 m) at the Brinkman value, "
                       "standard-normal right-hand side; rtol 1e-8 from a zero guess",
           "cells": n, "l2": "inputs larger than L2 (268 MB per FP64 vector)"}
    from paper_2206_07732_gb300 import tune
    for name, prec in (("fp64", wec.PREC_FP64), ("mixed", wec.PREC_MIXED)):
        opts, table = tune.tune_poisson3((nx, ny, nz), cb, bd, prec)
        P = wec.Poisson3(nx, ny, nz, precision=prec, mg_pre=opts[0], mg_post=opts[1], restart=opts[2])
        P.set_coefficients(*cb)
        x = torch.zeros_like(bd)
        for _ in range(warmup):
            x.zero_()
            P.solve(bd, x, rtol=1e-8)
        ms, its, rr = [], [], []
        n0 = wec.launch_count()
        for _ in range(solves):
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            info = P.solve(bd, x, rtol=1e-8)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append(info["iters"])
            rr.append(info["relres"])
        launches = (wec.launch_count() - n0) / solves
        x.zero_()
        torch.cuda.synchronize()
        wec.profile_read()
        wec.profile_enable(1)
        P.solve(bd, x, rtol=1e-8)
        wec.profile_enable(0)
        prof = wec.profile_read()
        P.close()
        by_name = {}
        for q in prof:
            d = by_name.setdefault(q["name"], dict(ms=0.0, bytes=0.0, launches=0))
            d["ms"] += q["ms"]; d["bytes"] += q["bytes"]; d["launches"] += q["launches"]
        tot = sum(d["ms"] for d in by_name.values())
        top = max(by_name, key=lambda k: by_name[k]["ms"])
        lv = {str(q["level"]): {"launches": q["launches"], "avg_us": q["ms"] / q["launches"] * 1e3,
                                "GBps": q["bytes"] / (q["ms"] / 1e3) / 1e9 if q["ms"] > 0 else None}
              for q in prof if q["name"] == top}
        # roofline on the finest level's launches of the dominant kernel (the
        # level a 33.5 M-cell sweep runs at; coarser levels are latency-bound)
        d = by_name[top]
        l0 = [q for q in prof if q["name"] == top and q["level"] == 0]
        b0 = sum(q["bytes"] for q in l0)
        t0 = sum(q["ms"] for q in l0)
        n0 = sum(q["launches"] for q in l0)
        ach = b0 / (t0 / 1e3) / 1e9 if t0 > 0 else None
        t = statistics.median(ms)
        out[name] = {
            "solver_options_autotuned": {"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2],
                                         "candidates": table},
            "ms_per_solve": t, "ms_per_solve_all": ms, "cell_solves_per_s": n / (t / 1e3),
            "fgmres_iters": statistics.mean(its), "max_relative_residual": max(rr),
            "gpu_launches_per_solve": launches,
            "kernel_breakdown_eager": [{"kernel": k, "launches": v["launches"], "ms": v["ms"], "share": v["ms"] / tot}
                                       for k, v in sorted(by_name.items(), key=lambda kv: -kv[1]["ms"])[:8]],
            "roofline": {"bound": "hbm", "kernel": top, "level": 0, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak if ach else None,
                         "traffic": ncu_traffic(f"{top}_l0_{nx}x{ny}x{nz}_{name}"),
                         "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                         "algorithmic_bytes_per_launch": b0 / n0 if n0 else None, "launches_timed": n0,
                         "avg_launch_us": t0 / n0 * 1e3 if n0 else None,
                         "share_of_solve_gpu_time": d["ms"] / tot, "level0_share_of_kernel_time": t0 / d["ms"],
                         "per_level": lv,
                         "timing": "event pair per launch over one eager solve; achieved over the finest level's "
                                   "launches"},
        }
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_solve"] / out["mixed"]["ms_per_solve"]
    del cb, bd
    torch.cuda.empty_cache()
    out["levelset3d"] = bench_levelset3d(wec, torch, seed, shape, peak, peak_kind)
    out["cpu_baseline"] = None
    if cpu_seconds > 0:
        from oracle import build as ob
        from oracle import poisson3d as O3
        ob.build()
        sx, sy, sz = 128, 64, 64
        cx, cy, cz, cbv = synth.poisson3d_case(sx, sy, sz, seed=seed)
        k, t0 = 0, time.perf_counter()
        while True:
            _, io = O3.solve(cx, cy, cz, cbv, rtol=1e-8)
            k += 1
            el = time.perf_counter() - t0
            if el > cpu_seconds:
                break
        out["cpu_baseline"] = {"value": sx * sy * sz * k / el, "unit": "cell-solves/s", "cores": 1, "kind": "oracle",
                               "sample": f"{k} oracle FP64 solves of the same structure on a {sx}x{sy}x{sz} grid "
                                         f"({io['iters']} iterations each, {el:.1f} s, 1 thread)"}
    return out


def bench_levelset3d(wec, torch, seed, shape, peak, peak_kind, reps=3):
    """The 3D tank's level-set kernels (wec_tank3, FP64) on the same grid: the
    incident JONSWAP surface with a cylinder, 0.3 m/s random face velocities;
    CUDA events around each call (advection, 4 reinitialisation pseudo-steps,
    materials), best of `reps`; algorithmic bytes over the measured HBM peak."""
    from paper_2206_07732_gb300 import synth
    nx, ny, nz = shape
    c = synth.tank3d(seed=seed, nx=nx, ny=ny, nz=nz)
    h = c["lx"] / nx
    amp, om, ph = wec.wave_components(c["wave"])
    k = np.array([wec.wave_number(w, c["depth"], c["g"]) for w in om])
    x = (np.arange(nx) + 0.5) * h
    eta = np.sum(amp[:, None] * np.cos(k[:, None] * x[None, :] + ph[:, None]), axis=0)
    z = (np.arange(nz) + 0.5) * h
    sig = np.broadcast_to(z[:, None, None] - c["depth"] - eta[None, None, :], (nz, ny, nx))
    f = synth.random_fields3(nx, ny, nz, seed=seed + 1, scale=0.3)
    T = wec.Tank3(c)
    for fid, a in ((wec.F3_SIGMA, sig), (wec.F3_U, f["u"]), (wec.F3_V, f["v"]), (wec.F3_W, f["w"])):
        T.set(fid, a)
    del f
    n = nx * ny * nz
    nfs = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)
    calls = {"advect": (lambda: T.advect(c["dt"], 0.0), 8.0 * (2 * n + nfs)),
             "reinit_4": (lambda: T.reinit(4, 0.0), 4 * 56.0 * n),
             "materials": (lambda: wec._check(wec.load().wec_tank3_materials(T.h, c["body"]["zc"])), 40.0 * n)}
    stream = torch.cuda.current_stream()
    out = {"precision": "fp64", "cells": n}
    for name, (fn, nbytes) in calls.items():
        fn()
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        gbs = nbytes / (best / 1e3) / 1e9
        out[name] = {"ms": best, "algorithmic_bytes": nbytes, "achieved_GBps": gbs, "frac_of_hbm": gbs / peak}
    out["peak_source"] = f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
    out["note"] = ("the calls synchronise the stream (timed with it); FP64 PPM / ENO stencils do hundreds of FP64 "
                   "operations per cell, so on this GPU they are bound by the FP64 pipe, not by HBM")
    T.close()
    return out


def main_batch(args):
    import torch
    from paper_2206_07732_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    L, wec = setup_lib()
    allc = synth.batch_tanks(64, seed=args.seed)
    cfgs = [c for i, c in enumerate(allc) if i % world == rank]  # tanks sharded over ranks, no collective
    cells_all = sum(c["nx"] * c["ny"] for c in allc)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    steps, warmup = args.steps, max(args.warmup, 3)
    clocks = Clocks(local)
    clocks.start()
    mixed = time_batch(wec, torch, cfgs, wec.PREC_MIXED, steps, warmup, flush)
    ck = clocks.stop()
    fp64 = time_batch(wec, torch, cfgs, wec.PREC_FP64, steps, warmup, flush)

    def reduce_max(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    t_mixed = reduce_max(sum(mixed["ms"]) / 1e3)
    t_fp64 = reduce_max(sum(fp64["ms"]) / 1e3)
    t_e2e = reduce_max(sum(mixed["wall"]))
    value = cells_all * steps / t_mixed
    nt = len(cfgs)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": t_mixed / steps * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64+f32(stencils,multigrid)", "data": "synthetic (seeded grids, Airy waves, boxes)",
        "config": {"workload": "batch of 64 uneven 2D tanks (256x128 .. 768x256, regular Airy waves, boxes), "
                               "one CUDA graph launch per batch step",
                   "cells": cells_all, "tanks": 64, "tanks_per_rank": nt, "rtol": 1e-8,
                   "precision": "mixed: FP32 stencils and V-cycles, FP64 storage/FGMRES/force/heave",
                   "l2": "flushed between timed steps (256 MiB write)", "seed": args.seed},
        "fp64_value": cells_all * steps / t_fp64, "fp64_ms_per_step": t_fp64 / steps * 1e3,
        "speedup_mixed_vs_fp64": t_fp64 / t_mixed,
        "fgmres_iters_per_step": {"mixed": statistics.mean(mixed["iters"]), "fp64": statistics.mean(fp64["iters"])},
        "max_relative_residual": {"mixed": mixed["residual"], "fp64": fp64["residual"]},
        "e2e": {"value": cells_all * steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 16 * nt,
                "d2h_bytes_per_step": 72 * nt,
                "note": "wec_batch_step wall clock: host dt / PTO arrays in, host records out, per step"},
        "gpu_launches": mixed["launches"],
        "clocks": ck,
        "roofline": None,
        "roofline_note": "per-kernel rooflines are reported by the default (single-tank) workload",
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def train_learned(wec, torch, cfg, seed, per_seed=60, skip=40, nseeds=10, iters=3000, batch=4):
    """The learned warm start's network, trained (untimed) on the pressure
    problems of mixed-precision runs of the same tank with other wave phases
    (seeds seed+1 .. seed+nseeds): features and targets from wec_net_sample,
    Adam on batches of 4 drawn from them."""
    from paper_2206_07732_gb300 import synth
    t0 = time.perf_counter()
    ny, nx = cfg["ny"], cfg["nx"]
    seeds = tuple(seed + 1 + k for k in range(nseeds))
    xs = torch.zeros((per_seed * len(seeds), ny, nx, 2), dtype=torch.float32, device="cuda")
    ts = torch.zeros((per_seed * len(seeds), ny, nx), dtype=torch.float32, device="cuda")
    k = 0
    for s in seeds:
        c = workload(s)
        tank = wec.Tank(c, precision=wec.PREC_MIXED)
        tank.step_n(skip, c["dt"], records=False)
        for _ in range(per_seed):
            tank.step(c["dt"])
            wec.net_sample(tank, xs[k], ts[k])
            k += 1
        tank.close()
    t1 = time.perf_counter()
    net = wec.Net(ny, nx, max_batch=batch)
    net.set_params(synth.unet_weights(wec.net_param_shapes(), seed))
    import numpy as np
    rng = np.random.default_rng(seed)
    losses = [net.train_step(xs, ts, rng.integers(0, k, batch), 1e-3 if it < 0.7 * iters else 3e-4)
              for it in range(iters)]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del xs, ts
    info = {"samples": k, "sample_seeds": list(seeds), "iterations": iters, "batch": batch,
            "loss_first_50": float(np.mean(losses[:50])), "loss_last_50": float(np.mean(losses[-50:])),
            "sampling_s": t1 - t0, "training_s": t2 - t1, "ms_per_training_step": (t2 - t1) / iters * 1e3}
    return net, info


def run_tank2d(wec, torch, args, rank, world, cpu_baseline=True):
    """The 2D 1024 x 256 JONSWAP tank (configuration 2 with the learned warm
    start of configuration 4): the mixed + learned path, mixed (FP32 stencils),
    mixed_mg (FP32 V-cycles only) and FP64, each at its autotuned solver
    options, under the host MPC; returns (summary, detail)."""
    cfg = workload(args.seed)
    n = cfg["nx"] * cfg["ny"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    steps, warmup = args.steps2d, max(args.warmup, 3)
    ctl, ctl_info = make_controller(wec, torch, cfg)
    net, train_info = train_learned(wec, torch, cfg, args.seed)
    from paper_2206_07732_gb300 import tune
    tuned, cfgs = {}, {}
    for key, prec, use_net in (("mixed+learned", wec.PREC_MIXED, net), ("mixed", wec.PREC_MIXED, None),
                               ("fp64", wec.PREC_FP64, None), ("mixed_mg", wec.PREC_MIXED_MG, None)):
        opts, table = tune.tune_tank(cfg, prec, net=use_net)
        tuned[key] = {"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2], "candidates": table}
        cfgs[key] = tune.with_options(cfg, opts)
    prof_all = profile_all(wec, torch, cfgs["mixed+learned"], wec.PREC_MIXED, net=net)
    by_name = {}
    for p in prof_all:
        d = by_name.setdefault(p["name"], dict(ms=0.0, bytes=0.0, launches=0))
        d["ms"] += p["ms"]; d["bytes"] += p["bytes"]; d["launches"] += p["launches"]
    top = max(by_name, key=lambda k: by_name[k]["ms"])
    tot_prof = sum(d["ms"] for d in by_name.values())
    breakdown = [{"kernel": k, "launches_per_step": d["launches"] / 2, "us_per_step": d["ms"] / 2 * 1e3,
                  "share": d["ms"] / tot_prof}
                 for k, d in sorted(by_name.items(), key=lambda kv: -kv[1]["ms"])[:12]]
    res = {}
    for key, prec in (("mixed+learned", wec.PREC_MIXED), ("mixed", wec.PREC_MIXED), ("fp64", wec.PREC_FP64),
                      ("mixed_mg", wec.PREC_MIXED_MG)):
        res[key] = time_path(None, wec, torch, cfgs[key], prec, steps, warmup, flush,
                             net=net if key == "mixed+learned" else None, ctl=ctl)
    kpass = time_path(None, wec, torch, cfgs["mixed+learned"], wec.PREC_MIXED, max(steps // 4, 5), warmup, flush,
                      graph=False, profile_kernel=top, net=net, ctl=ctl)
    e2e = e2e_path(wec, torch, cfgs["mixed+learned"], wec.PREC_MIXED, max(steps // 2, 5), warmup, flush, net=net,
                   ctl=ctl)
    t = {k: reduce_max(torch, world, sum(v["ms"]) / 1e3) for k, v in res.items()}
    val = {k: world * n * steps / v for k, v in t.items()}
    t_e2e = reduce_max(torch, world, sum(e2e))
    pk = [p for p in (kpass["prof"] or []) if p["name"] == top]
    roof = None
    if top == "net_conv":
        fl = wec.net_layer_flops(cfg["ny"], cfg["nx"])
        tot_f = sum(fl[p["level"]] * p["launches"] for p in pk if p["level"] < 100)
        tot_fm = sum(p["ms"] for p in pk if p["level"] < 100)
        nf = sum(p["launches"] for p in pk if p["level"] < 100)
        ach = tot_f / (tot_fm / 1e3) / 1e12 if tot_fm > 0 else None
        tpeak, tkind = tensor_peak()
        roof = {"bound": "tensor", "kernel": top, "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
                "frac": ach / tpeak if ach else None, "traffic": ncu_traffic(top),
                "peak_source": f"{tkind} (MEASURED_PEAKS.json)",
                "algorithmic_flops_per_launch": tot_f / nf if nf else None,
                "avg_launch_us": tot_fm / nf * 1e3 if nf else None, "share_of_step_gpu_time": by_name[top]["ms"] / tot_prof}
    else:
        peak, kind = peaks()
        nl = sum(p["launches"] for p in pk)
        tb, tm = sum(p["bytes"] for p in pk), sum(p["ms"] for p in pk)
        ach = (tb / nl) / (tm / nl / 1e3) / 1e9 if nl and tm > 0 else None
        roof = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak if ach else None, "traffic": ncu_traffic(top),
                "peak_source": f"{kind} hbm_gbs (MEASURED_PEAKS.json)",
                "algorithmic_bytes_per_launch": tb / nl if nl else None,
                "avg_launch_us": tm / nl * 1e3 if nl else None, "share_of_step_gpu_time": by_name[top]["ms"] / tot_prof}
    cpu = None
    if cpu_baseline and rank == 0 and world == 1:
        v, k, el = run_oracle(cfg, 1000, budget_s=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{k} oracle steps of the 1024x256 tank from its initial state ({el:.1f} s, 1 thread)"}
    tried, kept = res["mixed+learned"]["net_stats"]
    summary = {
        "workload": "2D tank 1024x256 (16 m x 4 m, JONSWAP Hs 0.15 m Tp 1.6 s, 64 components, box 1.0 x 0.8 m, "
                    "dt 5e-4 s, MPC PTO), learned warm start trained in the run",
        "steps": steps,
        "value": {k: val[k] for k in ("mixed+learned", "mixed", "mixed_mg", "fp64")},
        "ms_per_step": {k: t[k] / steps * 1e3 for k in t},
        "speedup_vs_fp64": {k: val[k] / val["fp64"] for k in ("mixed+learned", "mixed", "mixed_mg")},
        "fgmres_iters_per_step": {k: statistics.mean(v["iters"]) for k, v in res.items()},
        "guess_kept_steps": f"{kept}/{tried}",
        "e2e_value": world * n * len(e2e) / t_e2e,
        "roofline": {k: roof[k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")},
    }
    detail = {"summary": summary, "config": config_dict(cfg, "see summary", "flushed between timed steps (256 MiB)"),
              "roofline": roof, "kernel_breakdown_eager": breakdown, "solver_options_autotuned": tuned,
              "learned_warm_start": {"training": train_info, "guess_kept_steps": kept, "steps_with_net": tried},
              "pto_control": ctl_info, "max_relative_residual": {k: v["residual"] for k, v in res.items()},
              "cpu_baseline": cpu, "gpu_launches": res["mixed+learned"]["launches"]}
    net.close()
    return summary, detail


def reduce_max(torch, world, x):
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    return torch, rank, world, local


def write_detail(path, obj):
    if not path:
        return None
    try:
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        with open(path, "w") as f:
            json.dump(obj, f, indent=1, default=float)
        return path
    except OSError:
        return None


def main_tank2d(args):
    torch, rank, world, local = dist_setup()
    L, wec = setup_lib()
    cfg = workload(args.seed)
    if args.ncu_steps:
        # one-by-one launches: ncu cannot profile kernel nodes of graphs with
        # conditional nodes (same kernels, same order as the graph); the
        # headline path's kernels: an untrained network runs the same work
        from paper_2206_07732_gb300 import synth
        net = wec.Net(cfg["ny"], cfg["nx"], max_batch=1)
        net.set_params(synth.unet_weights(wec.net_param_shapes(), args.seed))
        if args.mg_opts:
            from paper_2206_07732_gb300 import tune
            cfg = tune.with_options(cfg, [int(v) for v in args.mg_opts.split(",")])
        tank = wec.Tank(cfg, precision=wec.PREC_MIXED)
        tank.use_graph(False)
        tank.set_net(net)
        for _ in range(max(args.warmup, 1) + args.ncu_steps):
            tank.step(cfg["dt"])
        torch.cuda.synchronize()
        return
    args.steps2d = args.steps
    clocks = Clocks(local)
    clocks.start()
    summary, detail = run_tank2d(wec, torch, args, rank, world, cpu_baseline=not args.no_cpu_baseline)
    ck = clocks.stop()
    n = cfg["nx"] * cfg["ny"]
    v = summary["value"]
    line = {
        "metric": METRIC + " (2D tank)", "value": v["mixed+learned"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": summary["ms_per_step"]["mixed+learned"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32(stencils,multigrid)+bf16(U-Net)",
        "data": "synthetic (seeded JONSWAP phases)",
        "config": {"workload": summary["workload"], "cells": n, "l2": "flushed between timed steps (256 MiB write)"},
        "fp64_value": v["fp64"], "speedup_vs_fp64": summary["speedup_vs_fp64"],
        "paths": {k: v[k] for k in v},
        "e2e": {"value": summary["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": 16, "d2h_bytes_per_step": 72},
        "gpu_launches": detail["gpu_launches"], "clocks": ck, "roofline": summary["roofline"],
        "cpu_baseline": detail["cpu_baseline"],
        "detail_file": write_detail(args.detail, detail),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ the 3D tank --
# The paths of configuration 5's step, the credited one first.
PATHS3 = (("mixed", "PREC_MIXED_DF"), ("mixed_mg", "PREC_MIXED_MG"), ("fp64", "PREC_FP64"),
          ("mixed_fp32_stencils", "PREC_MIXED"))
PATH3_NOTE = {
    "mixed": "FP32 multigrid V-cycles inside the FP64 FGMRES outer iteration; the step stencils in double-float "
             "arithmetic (float pairs, ~48-bit significands, FP64-equivalent: within 1e-10 of the FP64 oracle per "
             "step); the residual, the Krylov orthogonalisation, the force integral, the heave update and all "
             "fields FP64",
    "mixed_mg": "FP32 multigrid V-cycles inside the FP64 FGMRES; every stencil and all the rest FP64",
    "fp64": "everything FP64",
    "mixed_fp32_stencils": "mixed plus FP32 stencil arithmetic (level set, materials, momentum, Jacobi) over FP32 "
                           "working copies: narrower than the FP64 stencils of the precision contract, reported "
                           "beside it with its error against the FP64 oracle",
}


def h2d_d2h_bytes3(nz, precision_key):
    """Host copies of one wec_tank3_step: the boundary tables in (FP64, plus an
    FP32 copy for the FP32-stencil path); the heave force, the divergence norm
    and the probe column out (the step record itself is returned by value)."""
    h2d = (5 * nz + 3) * 8 + ((5 * nz + 3) * 4 if precision_key == "mixed_fp32_stencils" else 0)
    d2h = 8 + 8 + nz * 8
    return h2d, d2h


def time_tank3(wec, torch, cfg, precision, steps, warmup, world, pto=None):
    """K steps of a fresh tank after W warm-up steps: a CUDA event pair on the
    tank's stream around each wec_tank3_step call (the call synchronises on its
    own), the K steps bracketed by a barrier and synchronize; host wall clock
    around each call for e2e; launches counted over the K steps."""
    sched = pto(cfg) if pto else None
    state = [0.0, 0.0]
    force = (lambda: sched.force(*state)) if sched else (lambda: 0.0)
    T = wec.Tank3(cfg, precision=precision)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        r = T.step(cfg["dt"], force())
        state[:] = [r["z"], r["zdot"]]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its, res, wall = [], [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n0 = wec.launch_count()
    for k in range(steps):
        f = force()  # host QP (every dt_p) before the step
        t0 = time.perf_counter()
        ev[k][0].record(stream)
        r = T.step(cfg["dt"], f)
        ev[k][1].record(stream)
        wall.append(time.perf_counter() - t0)
        state[:] = [r["z"], r["zdot"]]
        its.append(r["iters"])
        res.append(r["residual"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = wec.launch_count() - n0
    T.close()
    return dict(ms=[a.elapsed_time(b) for a, b in ev], wall=wall, iters=its, residual=max(res), launches=launches,
                z=state[0], qp_solves=sched.solves if sched else 0, max_pto=sched.fmax if sched else 0.0)


def profile_tank3(wec, torch, cfg, precision, steps=1, warmup=1):
    """Untimed eager steps with an event pair around every launch: per-kernel
    totals and the launch records (name, level, bytes, ms, launches)."""
    T = wec.Tank3(cfg, precision=precision)
    for _ in range(warmup):
        T.step(cfg["dt"])
    torch.cuda.synchronize()
    wec.profile_read()
    wec.profile_enable(1)
    for _ in range(steps):
        T.step(cfg["dt"])
    wec.profile_enable(0)
    prof = wec.profile_read()
    T.close()
    return prof


def roofline3(prof, steps, top=None, shape=(512, 256, 256)):
    """The dominant kernel's roofline from an eager profile: achieved =
    algorithmic bytes per launch / mean launch time (multigrid kernels: over
    their finest-level launches, the 33.5 M-cell sweeps; coarser levels are
    latency-bound), against the measured HBM copy bandwidth."""
    prof = [q for q in prof if q["name"] != "tank3_section"]  # phase spans, not kernels
    by = {}
    for q in prof:
        d = by.setdefault(q["name"], dict(ms=0.0, bytes=0.0, launches=0))
        d["ms"] += q["ms"]; d["bytes"] += q["bytes"]; d["launches"] += q["launches"]
    tot = sum(d["ms"] for d in by.values())
    top = top or max(by, key=lambda k: by[k]["ms"])
    sel = [q for q in prof if q["name"] == top and q["level"] == 0] or [q for q in prof if q["name"] == top]
    b0, t0, n0 = (sum(q[k] for q in sel) for k in ("bytes", "ms", "launches"))
    peak, kind = peaks()
    ach = b0 / (t0 / 1e3) / 1e9 if t0 > 0 and b0 > 0 else None
    roof = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if ach else None,
            "traffic": ncu_traffic(f"{top}_l0_{shape[0]}x{shape[1]}x{shape[2]}" if any(q["level"] == 0 for q in sel)
                                   else f"{top}_{shape[0]}x{shape[1]}x{shape[2]}"),
            "peak_source": f"{kind} hbm_gbs (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": b0 / n0 if n0 else None,
            "avg_launch_us": t0 / n0 * 1e3 if n0 else None, "launches_timed": n0,
            "share_of_step_gpu_time": by[top]["ms"] / tot if tot else None}
    breakdown = [{"kernel": k, "launches_per_step": v["launches"] / steps, "ms_per_step": v["ms"] / steps,
                  "share": v["ms"] / tot,
                  "GBps": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 and v["bytes"] > 0 else None,
                  "hbm_frac": v["bytes"] / (v["ms"] / 1e3) / 1e9 / peak if v["ms"] > 0 and v["bytes"] > 0 else None}
                 for k, v in sorted(by.items(), key=lambda kv: -kv[1]["ms"])]
    return roof, breakdown


def oracle_baseline3(cfg, threads, steps=1):
    """The oracle's 3D step on the given tank: `steps` steps from its initial
    state on `threads` host threads; returns (cell-steps/s, seconds, iters)."""
    from oracle import build as ob
    from oracle import tank as otank
    from oracle import tank3d as OT3
    ob.build()
    used = otank.lib().oracle_threads(threads)
    o = OT3.OracleTank3(cfg)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    t0 = time.perf_counter()
    its = []
    for _ in range(steps):
        its.append(o.step(cfg["dt"])["iters"])
    el = time.perf_counter() - t0
    del o
    return n * steps / el, el, its, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def rnd(x, sig=5):
    """x to `sig` significant digits (floats in nested dicts and lists too)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}") if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: rnd(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [rnd(v, sig) for v in x]
    return x


def make_line3(c, seed, world, steps, warmup, tuned, res, t, tw, ck, roof, cpu, tank2d):
    """The printed JSON line of the 3D tank: under 2.5 KB (a reader may keep
    only the last ~3 KB of the output); the rest is in the detail file."""
    n = c["nx"] * c["ny"] * c["nz"]
    val = {k: world * n * steps / t[k] for k in t}
    h2d, d2h = h2d_d2h_bytes3(c["nz"], "mixed")
    o = tuned["mixed"]
    line = {
        "metric": METRIC, "value": val["mixed"], "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": t["mixed"] / steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32x2(stencils,krylov)+f32(multigrid)", "data": "synthetic (seeded JONSWAP phases)",
        "config": {"workload": "configuration 5: 3D tank 512x256x256 (8x4x4 m, depth 2 m, JONSWAP Hs 0.2 m Tp 2 s "
                               "128 comps, heaving cylinder R 0.5 m, dt 1e-3 s, rtol 1e-8)",
                   "cells": n,
                   "precision": "FP32 V-cycles; double-float stencils and Arnoldi step (<=1e-10 of the FP64 "
                                "oracle); FP64 true residual, solution, force, heave, fields",
                   "learned": "not used in 3D (2D U-Net: see tank2d)", "pto": "host MPC, |F| <= 2 kN",
                   "mg_pre,mg_post,restart": f"{o['mg_pre']},{o['mg_post']},{o['restart']}",
                   "l2": "inputs > L2, no flush", "seed": seed},
        "fp64_value": val["fp64"], "speedup_vs_fp64": val["mixed"] / val["fp64"],
        "paths": {k: {"value": val[k], "ms": t[k] / steps * 1e3, "its": statistics.mean(res[k]["iters"])}
                  for k in res if k != "mixed"},
        "e2e": {"value": world * n * steps / tw["mixed"], "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": res["mixed"]["launches"],
        "clocks": {k: ck.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "roofline": {k: roof.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")},
        "cpu_baseline": cpu,
        "tank2d": tank2d,
    }
    return rnd(line)


def main_tank3d(args):
    torch, rank, world, local = dist_setup()
    L, wec = setup_lib()
    from paper_2206_07732_gb300 import synth, tune
    c = synth.tank3d(seed=args.seed)
    if args.ncu_steps:
        # profiling helper: warm-up + ncu_steps steps of the tank at the given
        # precision (--precision), grid (--shape3) and solver options (--mg-opts),
        # no output
        if args.shape3:
            nx, ny, nz = (int(v) for v in args.shape3.split(","))
            c = synth.tank3d(seed=args.seed, nx=nx, ny=ny, nz=nz)
        if args.mg_opts:
            c = tune.with_options(c, [int(v) for v in args.mg_opts.split(",")])
        prec = getattr(wec, dict(PATHS3)[args.precision])
        T = wec.Tank3(c, precision=prec)
        for _ in range(max(args.warmup, 1) + args.ncu_steps):
            T.step(c["dt"])
        torch.cuda.synchronize()
        T.close()
        return
    n = c["nx"] * c["ny"] * c["nz"]
    steps, warmup = args.steps, max(args.warmup, 3)
    detail = {"workload": c["name"]}
    # solver options per path, autotuned on the tank's first steps (untimed)
    tuned, cfgs = {}, {}
    for key, pname in PATHS3:
        opts, table = tune.tune_tank3(c, getattr(wec, pname))
        tuned[key] = {"mg_pre": opts[0], "mg_post": opts[1], "restart": opts[2]}
        detail.setdefault("tuning", {})[key] = table
        cfgs[key] = tune.with_options(c, opts)
    # the timed runs: the credited path with the clocks sampled, then the others
    # the PTO force of every path: the host MPC (its QP runs between steps)
    ctl, ctl_info = make_controller3(wec, c)
    detail["pto_control"] = ctl_info
    res = {}
    clocks = Clocks(local)
    for key, pname in PATHS3:
        if key == "mixed":
            clocks.start()
        res[key] = time_tank3(wec, torch, cfgs[key], getattr(wec, pname), steps, warmup, world,
                              pto=lambda cfg: PtoSchedule(ctl, cfg, wec))
        if key == "mixed":
            ck = clocks.stop()
    t = {k: reduce_max(torch, world, sum(v["ms"]) / 1e3) for k, v in res.items()}
    tw = {k: reduce_max(torch, world, sum(v["wall"])) for k, v in res.items()}
    val = {k: world * n * steps / t[k] for k in t}
    # where the credited path's time goes (untimed eager step, every launch timed)
    prof = profile_tank3(wec, torch, cfgs["mixed"], getattr(wec, dict(PATHS3)["mixed"]))
    roof, breakdown = roofline3(prof, 1)
    detail["kernel_breakdown_eager"] = {"mixed": breakdown}
    detail["roofline"] = {"mixed": roof}
    # the oracle on host cores: one step of the same 512 x 256 x 256 tank on all
    # cores, and a single-thread sample of the same tank physics
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        v_all, el_all, its_all, used = oracle_baseline3(cfgs["mixed"], cores, steps=1)
        sc = tune.with_options(synth.tank3d(seed=args.seed, nx=128, ny=64, nz=64),
                               (c["solver"]["mg_pre"], c["solver"]["mg_post"], c["solver"]["restart"]))
        v_1, el_1, its_1, _ = oracle_baseline3(sc, 1, steps=2)
        cpu = {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"1 step of the same 512x256x256 tank, {used} threads, {el_all:.1f} s",
               "single_thread": {"value": v_1, "sample": f"2 steps on 128x64x64, {el_1:.1f} s"}}
    # the 2D tank with the learned warm start (configuration 2 / 4), beside it
    tank2d = None
    if not args.no_2d:
        args.steps2d = args.steps2d or 100
        try:
            s2, d2 = run_tank2d(wec, torch, args, rank, world, cpu_baseline=False)
            detail["tank2d"] = d2
            tank2d = {"workload": "2D 1024x256 tank, learned warm start trained in the run",
                      "value": s2["value"], "e2e": s2["e2e_value"],
                      "conv_roofline_frac": s2["roofline"]["frac"]}
        except Exception as ex:  # reported, not fatal to the 3D line
            tank2d = {"error": f"{type(ex).__name__}: {ex}"[:200]}
    # the batched configuration (64 uneven 2D tanks, one graph launch per batch
    # step; tanks sharded over ranks, no collective), beside it
    batch = None
    if not args.no_2d and not args.no_batch:
        try:
            batch, detail["batch"] = run_batch_leg(wec, torch, args.seed, rank, world)
        except Exception as ex:  # reported, not fatal to the 3D line
            batch = {"error": f"{type(ex).__name__}: {ex}"[:200]}
    detail.update({"paths": {k: {"ms_per_step_all": res[k]["ms"], "wall_s_all": res[k]["wall"],
                                 "fgmres_iters": res[k]["iters"], "max_relative_residual": res[k]["residual"],
                                 "qp_solves": res[k]["qp_solves"], "max_abs_pto_force_N": res[k]["max_pto"],
                                 "heave_z_m": res[k]["z"]}
                             for k in res}, "solver_options_autotuned": tuned, "clocks": ck})
    line = make_line3(c, args.seed, world, steps, warmup, tuned, res, t, tw, ck, roof, cpu, tank2d)
    if batch is not None:
        line["batch"] = rnd(batch)
    line["detail_file"] = write_detail(args.detail, dict(detail, line=line)) if rank == 0 else None
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main_learned(args):
    """Configuration 4: the U-Net warm start trained on pressure problems that
    the method itself generates -- runs of the 512 x 256 tank with the
    configuration-2 physics and seeded sea states (synth.tank_learned), 2000
    steps from each of ten seeds (20k problems, FP32 features and targets held
    on the device) -- then evaluated on held-out seeds against plain multigrid
    by FGMRES iterations and time per step to the 1e-8 FP64 residual (the
    network's inference included), mixed precision (FP32 V-cycles, FP64 and
    FP32 stencils)."""
    torch, rank, world, local = dist_setup()
    L, wec = setup_lib()
    from paper_2206_07732_gb300 import synth
    ny, nx = 256, 512
    nseeds, per, skip = args.learned_seeds, args.learned_steps, 40
    seeds = [args.seed + 100 + k for k in range(nseeds)]
    N = nseeds * per
    xs = torch.zeros((N, ny, nx, 2), dtype=torch.float32, device="cuda")
    ts = torch.zeros((N, ny, nx), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    k = 0
    for s_ in seeds:
        c = synth.tank_learned(seed=s_)
        T = wec.Tank(c, precision=wec.PREC_MIXED_MG)
        T.step_n(skip, c["dt"], records=False)
        for _ in range(per):
            T.step(c["dt"])
            wec.net_sample(T, xs[k], ts[k])
            k += 1
        T.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = wec.Net(ny, nx, max_batch=4)
    net.set_params(synth.unet_weights(wec.net_param_shapes(), args.seed))
    rng = np.random.default_rng(args.seed)
    iters = args.train_iters
    losses = [net.train_step(xs, ts, rng.integers(0, N, 4), 1e-3 if it < 0.7 * iters else 3e-4)
              for it in range(iters)]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del xs, ts
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()

    def run(c, prec, use_net, n):
        T = wec.Tank(c, precision=prec)
        if use_net:
            T.set_net(net)
        T.step_n(5, c["dt"], records=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        its = []
        for q in range(n):
            ev[q][0].record(stream)
            r = T.step(c["dt"])
            ev[q][1].record(stream)
            its.append(r["iters"])
            assert r["residual"] <= c["solver"]["rtol"]
        torch.cuda.synchronize()
        st = T.net_stats() if use_net else (0, 0)
        T.close()
        return statistics.mean(its), statistics.mean(a.elapsed_time(b) for a, b in ev), st

    held = [args.seed + 900 + k for k in range(2)]
    ev_out = {}
    for name, prec in (("mixed_mg", wec.PREC_MIXED_MG), ("mixed_fp32_stencils", wec.PREC_MIXED)):
        rows = []
        for hs in held:
            c = synth.tank_learned(seed=hs)
            c["solver"]["rtol"] = 1e-8
            ip, tp, _ = run(c, prec, False, args.steps)
            il, tl, (tried, kept) = run(c, prec, True, args.steps)
            rows.append({"seed": hs, "iters_plain": ip, "iters_learned": il, "ms_plain": tp, "ms_learned": tl,
                         "guess_kept": f"{kept}/{tried}"})
        ev_out[name] = rows
    line = {"metric": "FGMRES iterations and ms per step to the 1e-8 FP64 residual, learned warm start vs plain "
                      "multigrid (held-out seeds)",
            "workload": f"512x256 tank_learned, {N} training problems from {nseeds} seeds x {per} steps, "
                        f"{iters} Adam steps of batch 4; held-out seeds {held}, {args.steps} steps each",
            "training": {"samples": N, "sampling_s": t1 - t0, "training_s": t2 - t1,
                         "loss_first_100": float(np.mean(losses[:100])), "loss_last_100": float(np.mean(losses[-100:]))},
            "evaluation": ev_out}
    if rank == 0:
        print(json.dumps(line))
    net.close()


def main_reference(args):
    """The reference arm: the oracle (plain FP64 C, all host cores) on the same
    3D tank physics, each step a bounded sample: a 192 x 96 x 96 grid of the
    8 m x 4 m x 4 m tank (h = 1/24 m), so that --steps K --warmup W stays within
    a few minutes; cell-steps/s over that grid's cells."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2206_07732_gb300 import synth
    from oracle import build as ob
    from oracle import tank as otank
    from oracle import tank3d as OT3
    ob.build()
    used = otank.lib().oracle_threads(host_cores())
    from paper_2206_07732_gb300 import tune
    c = tune.with_options(synth.tank3d(seed=args.seed, nx=192, ny=96, nz=96), (3, 3, 5))
    n = c["nx"] * c["ny"] * c["nz"]
    o = OT3.OracleTank3(c)
    for _ in range(max(args.warmup, 0)):
        o.step(c["dt"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(c["dt"])
    el = time.perf_counter() - t0
    v = n * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded JONSWAP phases)",
            "config": {"workload": "configuration 5's tank physics (8 m x 4 m x 4 m, JONSWAP, cylinder) on a "
                                   "192x96x96 sample grid", "cells": n, "l2": "n/a (CPU)", "seed": args.seed},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{args.steps} timed oracle steps of a 192x96x96 grid of the tank after "
                                       f"{args.warmup} warm-up steps, {used} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        main_reference(a)
    elif a.workload == "batch":
        main_batch(a)
    elif a.workload == "poisson3d":
        main_poisson3d(a)
    elif a.workload == "tank":
        main_tank2d(a)
    elif a.workload == "learned":
        main_learned(a)
    else:
        main_tank3d(a)
