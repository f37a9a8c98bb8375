#!/usr/bin/env python
"""Benchmark: active-cell RK4 steps per second of the adaptive wavelet TRiSK step,
chosen form against the plain form at equal error.

Workload (seeded, synthetic): zonal jet u = 80 exp(-((lat - lat0)/7 deg)^2) m/s
with gradient-wind balanced depth (mean 10 km) and three 120 m Gaussian bumps,
radius 6.371e6 m, Omega 7.292e-5 1/s, g 9.80616 m/s^2, adaptive levels
Jmin=4..Jmax=9, eps = 1e-2 relative, RK4, CFL 0.8.  A step is one RK4 step with
its partial transform and grid adaptation.

* plain form: FP64, one member, the exact threshold criterion;
* chosen form (default): FP32 fields and stencils, an ensemble of --members
  independent members (seeds) advanced together on shared grid tables: the time
  step, RK base, every phase of each RK stage, the partial transform and the
  ghosts as one launch per phase over all members, then each member's adaptation
  on its own stream; the learned refinement proposal, trained first on masks of
  two extra members.

value = (live nodes over all levels and members, averaged over each step's start
and end) x steps / seconds, with per-step CUDA-event times (the L2 cache is
flushed between steps with a 512 MiB write outside the timed events).
equal_error: relative l2 errors of the Jmin depth and velocity after one model
day (--err-days) of the same dt, plain and chosen, against a non-adaptive FP64
run (every point live).  learned_turbulence: the learned-mask configuration
(turbulence, Jmax=10) timed with and without the proposal.

--impl reference runs the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm).  With --gpus N under torchrun every
rank runs its own members (seeds offset by rank): weak scaling, no collective on
the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# the oracle's worker processes are single-threaded numpy (one per host core)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
# ensemble members run on their own streams: let them use separate hardware queues
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

METRIC = "active-cell RK4 steps/s, adaptive Jmax=9, chosen vs plain form, equal error"
UNIT = "active-cell steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--jmin", type=int, default=4)
    p.add_argument("--jmax", type=int, default=9)
    p.add_argument("--eps", type=float, default=1e-2)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--patch", type=int, default=8)
    p.add_argument("--form", default="chosen", choices=["chosen", "plain"],
                   help="chosen: FP32 ensemble with the learned proposal; plain: FP64, one member")
    p.add_argument("--members", type=int, default=64, help="ensemble members of the chosen form")
    p.add_argument("--plain-steps", type=int, default=10)
    p.add_argument("--train-steps", type=int, default=10)
    p.add_argument("--err-steps", type=int, default=-1,
                   help="steps of the equal-error runs (-1: --err-days model days; 0: skip)")
    p.add_argument("--err-days", type=float, default=1.0)
    p.add_argument("--turb-steps", type=int, default=5,
                   help="timed steps of the turbulence configuration with and without the proposal (0: skip)")
    p.add_argument("--tau", type=float, default=0.9, help="proposal threshold on the perceptron probability")
    p.add_argument("--no-learned", action="store_true", help="chosen form without the learned proposal")
    p.add_argument("--no-tune", action="store_true", help="chosen form without the autotuner (patch, 4 blocks/SM)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-jmax", type=int, default=8, help="finest level of the oracle's hierarchy")
    return p.parse_args()


def workload_name(a):
    form = ("FP32 ensemble of independent members, learned proposal" if a.form == "chosen"
            else "FP64 plain form, one member")
    return (f"adaptive zonal jet + 3 bumps, Jmin={a.jmin}..Jmax={a.jmax}, eps={a.eps:g} relative, "
            f"RK4, CFL 0.8, {form}")


def edge_geometry(xyz, en):
    a, b = xyz[en[:, 0]], xyz[en[:, 1]]
    m = a + b
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    t = b - a
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return m, t


# ----------------------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- oracle sample

def host_cpu():
    """Model name and logical core count of the host (context for the CPU figures)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "logical_cores": os.cpu_count()}


def member_seeds(seed, rank, n):
    """Workload seeds of the n members of one rank (ranks 1000 seeds apart)."""
    return [seed + 1000 * rank + k for k in range(n)]


def oracle_member(hy, eps, seed, jmax):
    """The oracle's member of the benchmark's workload: the jet of `seed` given on
    level jmax of the hierarchy, adapted (twice: the second pass sees the first's
    grid)."""
    import workloads
    from oracle import model
    M = model.Model(hy, eps=eps, rk="rk4", cfl=0.8)
    L = hy.levels[jmax]
    dh, u = workloads.Workload("jet", seed=seed).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    M.set_uniform(dh, u)
    M.adapt()
    M.adapt()
    return M


def oracle_steps(M, steps):
    """Active-cell steps (mean of each step's start and end) and seconds of `steps`
    CFL steps of an oracle member."""
    cells, t0 = 0.0, time.perf_counter()
    for _ in range(steps):
        act = M.active_nodes()
        M.step(M.dt_cfl())
        cells += (act + M.active_nodes()) / 2
    return cells, time.perf_counter() - t0


def _oracle_worker(hy, a, jmax, k, go, res, barrier):
    """One member of the benchmark's workload (seed + k) stepped by the oracle, in a
    worker forked before any CUDA call: waits for (steps, warmup), then adapts,
    takes the warm-up steps, meets the other workers, and times its steps."""
    steps, warmup = go.get()
    try:
        M = oracle_member(hy, a.eps, a.seed + k, jmax)
        for _ in range(warmup):
            M.step(M.dt_cfl())
        barrier.wait()
        cells, secs = oracle_steps(M, steps)
        res.put((k, cells, secs, steps))
    except Exception as e:   # reported to the parent, which then leaves the figure out
        try:
            barrier.abort()
        except Exception:
            pass
        res.put((k, None, repr(e), 0))


class OraclePool:
    """The FP64 CPU oracle on the host cores: the hierarchy of Jmin..jmax is built
    once here and shared (copy on write) by one worker process per core, forked
    before this process makes any CUDA call; worker k steps the member of seed
    seed + k of the same workload.  run() times them together."""

    def __init__(self, a, jmax, nproc):
        import multiprocessing as mp
        from oracle import grid
        t0 = time.perf_counter()
        self.jmax, self.nproc = jmax, nproc
        self.hy = grid.Hierarchy(a.jmin, jmax)
        self.setup_s = time.perf_counter() - t0
        ctx = mp.get_context("fork")
        self.go, self.res = ctx.Queue(), ctx.Queue()
        self.barrier = ctx.Barrier(nproc)
        self.procs = [ctx.Process(target=_oracle_worker, args=(self.hy, a, jmax, k, self.go, self.res, self.barrier),
                                  daemon=True) for k in range(nproc)]
        for p in self.procs:
            p.start()

    def run(self, steps, warmup, timeout=1200):
        """(rate over all workers, median single-worker rate, seconds of the slowest
        worker, steps per worker) or None when a worker failed."""
        for _ in self.procs:
            self.go.put((steps, warmup))
        out = [self.res.get(timeout=timeout) for _ in self.procs]
        for p in self.procs:
            p.join(timeout=60)
        if any(o[1] is None for o in out):
            return None
        secs = max(o[2] for o in out)
        return (sum(o[1] for o in out) / secs, statistics.median(o[1] / o[2] for o in out), secs, steps)

    def sample(self, a, steps, warmup):
        return (f"the benchmark's jet workload and eps with the finest level capped at Jmax={self.jmax} "
                f"(Jmin={a.jmin}; the GPU run's cap is {a.jmax}), "
                f"{self.nproc} members (seeds {a.seed}..{a.seed + self.nproc - 1}) in {self.nproc} forked "
                f"single-threaded numpy oracle processes, one per host core, {steps} RK4 step(s) each after "
                f"{warmup} warm-up step(s); grid setup and adaptation before the steps untimed")


def oracle_cores():
    """Host cores for the oracle workers."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


# ----------------------------------------------------------------------------- reference arm

def run_reference(a, rank):
    """The oracle arm: the same metric and config on the host cores, a member per
    core; the --steps K / --warmup W are spread over the workers (each takes
    ceil(K / cores) timed and ceil(W / cores) warm-up steps)."""
    if rank != 0:
        return
    cores = oracle_cores()
    pool = OraclePool(a, min(a.cpu_jmax, a.jmax), cores)
    steps = max(1, math.ceil(a.steps / cores))
    warm = math.ceil(a.warmup / cores)
    r = pool.run(steps, warm)
    if r is None:
        print(json.dumps({"impl": "reference", "unavailable": "an oracle worker failed"}), flush=True)
        return
    v, single, secs, _ = r
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": steps * cores, "warmup": warm * cores, "ms_per_step": 1e3 * secs / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": pool.sample(a, steps, warm), "single_process": single,
                             "host": host_cpu(), "setup_s": pool.setup_s},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- ranks

def combine_ranks(seconds, cells, device, world):
    """Whole-job figures of independent members, one per rank: the slowest rank's
    time and the sum of all ranks' active-cell steps."""
    if world <= 1:
        return float(seconds), float(cells)
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([cells], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(c[0])


# ----------------------------------------------------------------------------- our arm

# Algorithmic bytes per live cell (one node, three edges, two triangles) of one
# RK stage at the minimum a fused stage must move: the state read (dh, u: 32 B in
# FP64, 16 B in FP32), the RK base read and the new state written (64 B; 32 B),
# and the FP64 geometry in its minimal form (cell area, 3 d_e, 3 l_e, 6 kite
# areas, 2 dual areas, Coriolis at the 2 dual cells: 17 words, 136 B, FP64 in
# both forms) -- 232 B in FP64, 184 B in FP32.
STAGE_BYTES_PER_CELL = {"fp64": 232, "fp32": 184}

# Algorithmic bytes per available cell (live or ghost node, with its three edges
# and two triangles) of the structured trend kernel k_tile_trend: dh and u read
# (4 words), the flags (4 B), the 17 FP64 geometry words (136 B), and F, q, div F,
# B and q F^perp written (8 words) -- 12 words + 140 B: 188 B in FP32, 236 B in FP64.
TREND_BYTES_PER_CELL = {"fp64": 236, "fp32": 188}

# DRAM bytes (read + write) of k_tile_trend per available cell, from an ncu
# full-set capture of the same jet at Jmin=4..Jmax=8 with 16 members (42.6 MB for
# 495 961 cells), scaled to a launch by the cells it processes.  The geometry
# share falls as more members read the same blocks, so at 64 members this
# overstates the traffic.  Remove the entry when the kernel changes.
TREND_TRAFFIC_PER_CELL = {"fp32": 85.9}


def _live(m):
    # the count the last set_state, adapt or step brought back (no device work)
    return m.live_nodes()


def _avail_st(st):
    return sum(st["live_nodes"].values()) + sum(st["ghost_nodes"].values())


def _avail(m):
    return _avail_st(m.stats())


_SAMPLINGS = {}


def _sampling(workloads, base, jmax):
    """Latitudes and edge directions of the grid, shared by every member's fields."""
    if id(base) not in _SAMPLINGS:
        xyz, en = base.grid(jmax)
        _SAMPLINGS[id(base)] = (base, workloads.Sampling(xyz, *edge_geometry(xyz, en)))
    return _SAMPLINGS[id(base)][1]


def _members(sww, workloads, base, a, precision, seeds, learned=None, persistent=True, patch=None, bps=0):
    ms = []
    S = _sampling(workloads, base, a.jmax)
    for sd in seeds:
        m = sww.Model(a.jmin, a.jmax, patch=patch or a.patch, eps=a.eps, rk="rk4", cfl=0.8, precision=precision,
                      share=base, persistent=persistent, blocks_per_sm=bps)
        dh, u = workloads.Workload("jet", seed=sd).fields_on(S)
        m.set_state(dh, u)
        m.adapt()
        m.adapt()
        if learned is not None:
            m.set_learned(2, learned, a.tau)
        ms.append(m)
    return ms


def _timed(sww, ms, steps, flush, stream):
    """CUDA-event time of each ensemble step (L2 flushed before each, outside the
    events) and the live cells advanced (mean of the step's start and end)."""
    import torch
    times, cells = [], []
    for _ in range(steps):
        c0 = sum(_live(m) for m in ms)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sww.step_ensemble(ms, -1.0, 1, True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        cells.append(0.5 * (c0 + sum(_live(m) for m in ms)))
    return times, cells


def _equal_error(sww, workloads, base, cbase, cpatch, cbps, a, learned, seed, steps, days):
    """Relative l2 errors of the Jmin depth and velocity at the final time (after
    `steps` steps of a fixed dt, or `days` model days when steps < 0), for the plain
    form (FP64, exact mask) and the chosen form (FP32, learned proposal), against a
    non-adaptive FP64 run (eps = 0: every point live) substepped at its own CFL
    limit to the same final time."""
    import numpy as np

    def state(b):
        xyz, en = b.grid(a.jmax)
        mid, tan = edge_geometry(xyz, en)
        return workloads.Workload("jet", seed=seed).fields(xyz, mid, tan)

    s_plain = state(base)
    s_chosen = s_plain if cbase is base else state(cbase)

    def make(precision, eps, prop=None):
        chosen = precision == "fp32"
        b = cbase if chosen else base
        dh, u = s_chosen if chosen else s_plain
        m = sww.Model(a.jmin, a.jmax, patch=cpatch if chosen else a.patch, eps=eps, rk="rk4", cfl=0.8,
                      precision=precision, share=b, blocks_per_sm=cbps if chosen else 0)
        m.set_state(dh, u)
        if eps > 0:
            m.adapt()
            m.adapt()
        if prop is not None:
            m.set_learned(2, prop, a.tau)
        return m

    plain, chosen, ref = make("fp64", a.eps), make("fp32", a.eps, learned), make("fp64", 0.0)
    plain.step(-1.0, 1, True)
    dt = plain.stats()["dt"]
    plain.close()
    plain = make("fp64", a.eps)
    if steps < 0:
        steps = max(1, int(round(days * 86400.0 / dt)))
    ref.step(-1.0, 1, False)
    sub = max(1, math.ceil(dt / ref.stats()["dt"]))
    ref.close()
    ref = make("fp64", 0.0)
    t0 = time.perf_counter()
    for m in (plain, chosen):
        m.step(dt, steps, True)
    ref.step(dt / sub, steps * sub, False)
    r_h, r_u = ref.get(a.jmin, sww.DH), ref.get(a.jmin, sww.U)

    def err(m):
        return {"dh": float(np.linalg.norm(m.get(a.jmin, sww.DH) - r_h) / np.linalg.norm(r_h)),
                "u": float(np.linalg.norm(m.get(a.jmin, sww.U) - r_u) / np.linalg.norm(r_u))}

    ep, ec = err(plain), err(chosen)
    out = {"steps": steps, "dt_s": dt, "model_days": steps * dt / 86400.0, "reference_substeps": sub,
           "level": a.jmin, "plain_fp64": ep, "chosen": ec, "ratio": ec["dh"] / max(ep["dh"], 1e-300),
           "ratio_u": ec["u"] / max(ep["u"], 1e-300), "wall_s": time.perf_counter() - t0}
    for m in (plain, chosen, ref):
        m.close()
    return out


def _turbulence(sww, workloads, a, steps, flush, peak, prec_bytes):
    """The learned-mask configuration timed with and without the proposal:
    decaying turbulence at Jmin=5..Jmax=10, eps=5e-3, FP32, one member given on
    level 7 and stepped with one launch per phase; the proposal trained on
    turbulence of two other seeds at Jmax=8.
    From the same state (a checkpoint after 6 steps), `steps` steps each way:
    active-cell steps/s, late refinements (misses), over-refinement, live cells,
    and the structured trend kernel's roofline on this large grid."""
    import tempfile

    import numpy as np
    import torch
    from paper_1404_0405_gb300 import learn
    jmin, jmax, jset, eps = 5, 10, 7, 5e-3
    t_setup = time.perf_counter()

    def member(b, seed, j1=jmax):
        # one launch per phase (the structured trend is a launch of its own, timed)
        m = sww.Model(jmin, j1, eps=eps, precision="fp32", share=b, persistent=False)
        xyz, en = m.grid(jset)
        mid, tan = edge_geometry(xyz, en)
        m.set_state(*workloads.Workload("turbulence", seed=seed).fields(xyz, mid, tan), level=jset)
        m.adapt()
        return m

    Xs, ys = [], []
    tb = sww.Model(jmin, 8, eps=eps, precision="fp32")
    for sd in (1, 2):
        m = member(tb, sd, 8)
        X, y = learn.collect(m, 8)
        Xs.append(X), ys.append(y)
        m.close()
    params, _ = learn.train(np.concatenate(Xs), np.concatenate(ys), epochs=300)
    base = sww.Model(jmin, jmax, eps=eps, precision="fp32")
    m = member(base, 7)
    m.step(-1.0, 6, True)
    out = {"workload": "decaying rotating turbulence, Jmin=5..Jmax=10, eps=5e-3 relative, RK4, FP32, one member "
                       "(fields given on level 7, 6 steps of spin-up); proposal trained on two other seeds at Jmax=8",
           "setup_s": 0.0}
    with tempfile.TemporaryDirectory() as d:
        ck = os.path.join(d, "turb.ckpt")
        m.save(ck)
        stream = torch.cuda.current_stream()
        out["setup_s"] = time.perf_counter() - t_setup
        for name, mode in (("with_proposal", 2), ("without_proposal", 0)):
            m.load(ck)
            m.set_learned(mode, params if mode else None, 0.5)
            m.learn_stats(reset=True)
            times, cells = _timed_single(sww, m, steps, flush, stream)
            st = m.stats()
            ls = m.learn_stats(reset=True)
            rec = {"value": sum(cells) / sum(times), "ms_per_step": 1e3 * sum(times) / steps,
                   "live_cells_per_step": sum(cells) / steps, "misses": ls["misses"], "over": ls["over"],
                   "proposed": ls["proposed"], "top_level": max(j for j, n in st["live_nodes"].items() if n > 0)}
            out[name] = rec
        # roofline of the structured trend on this grid (the run without the proposal)
        m.load(ck)
        m.set_learned(0)
        m.profile(["trend"])
        tb_bytes = tb_patches = 0.0
        for _ in range(steps):
            st = m.stats()
            tb_bytes += prec_bytes * _avail_st(st) * 4
            tb_patches += sum(st["active_patches"].values()) * 4
            flush.zero_()
            m.step(-1.0, 1, True)
        t_ms, t_n = m.profile_read()["trend"]
        m.profile([])
        if t_n > 0:
            ach = tb_bytes / (t_ms / 1e3) / 1e9
            out["roofline_trend"] = {"kernel": "k_tile_trend", "achieved": ach, "peak": peak, "unit": "GB/s",
                                     "frac": ach / peak, "avg_launch_us": t_ms * 1e3 / t_n, "launches": t_n,
                                     "algorithmic_bytes_per_launch": tb_bytes / t_n,
                                     "available_cells_per_launch": tb_bytes / prec_bytes / t_n,
                                     "patches_per_launch": tb_patches / t_n,
                                     "patch_fill": tb_bytes / prec_bytes / max(tb_patches, 1.0) / m.cfg.patch ** 2}
    m.close()
    base.close()
    tb.close()
    return out


def _timed_single(sww, m, steps, flush, stream):
    """CUDA-event time of each step of one member (L2 flushed before each) and the
    live cells advanced."""
    import torch
    times, cells = [], []
    for _ in range(steps):
        c0 = _live(m)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.step(-1.0, 1, True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        cells.append(0.5 * (c0 + _live(m)))
    return times, cells


def run_ours(a, rank, world):
    import torch
    import paper_1404_0405_gb300 as sww
    from paper_1404_0405_gb300 import learn
    import workloads

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    seed = member_seeds(a.seed, rank, 1)[0]
    t_setup = time.perf_counter()
    free0 = torch.cuda.mem_get_info()[0]
    base = sww.Model(a.jmin, a.jmax, patch=a.patch, eps=a.eps, rk="rk4", cfl=0.8)
    grid_bytes = free0 - torch.cuda.mem_get_info()[0]   # the shared FP64 grid tables and one FP64 handle
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # plain form: FP64, one member, the exact criterion alone
    plain_m = _members(sww, workloads, base, a, "fp64", [seed])
    for _ in range(a.warmup):
        sww.step_ensemble(plain_m, -1.0, 1, True)
    pt, pc = _timed(sww, plain_m, a.plain_steps, flush, stream)
    plain_t, plain_c = combine_ranks(sum(pt), sum(pc), "cuda", world)
    plain = {"value": plain_c / plain_t, "ms_per_step": 1e3 * plain_t / len(pt), "members": 1, "dtype": "f64",
             "active_cells_per_step": plain_c / len(pc) / max(world, 1)}

    # chosen form: FP32, an ensemble of members in one concurrent step, learned
    # proposal; patch side and work-list grid from the autotuner
    learned = None
    lstats = None
    tuned = None
    cbase, cpatch, cbps = base, a.patch, 0
    if a.form == "chosen" and not a.no_tune:
        from paper_1404_0405_gb300 import autotune

        def fields_of(xyz, en):
            mid, tan = edge_geometry(xyz, en)
            return [workloads.Workload("jet", seed=seed + 900 + k).fields(xyz, mid, tan) for k in range(4)]

        best, trials = autotune.tune(a.jmin, a.jmax, a.eps, fields_of, members=4, key_extra="jet",
                                     persistent="phased")
        tuned = {"best": best, "trials": trials}
        cpatch, cbps = best["patch"], best["blocks_per_sm"]
        if cpatch != a.patch:
            cbase = sww.Model(a.jmin, a.jmax, patch=cpatch, eps=a.eps, rk="rk4", cfl=0.8)
    if a.form == "chosen" and a.no_learned:
        ms = _members(sww, workloads, cbase, a, "fp32", member_seeds(a.seed, rank, a.members), persistent="phased",
                      patch=cpatch, bps=cbps)
        dtype = "f32"
    elif a.form == "chosen":
        train_m = _members(sww, workloads, cbase, a, "fp32", [seed + 500 + k for k in range(2)], patch=cpatch,
                           bps=cbps)
        Xs, ys = zip(*[learn.collect(m, a.train_steps) for m in train_m])
        X, y = np.concatenate(Xs), np.concatenate(ys)
        learned, losses = learn.train(X, y, epochs=300)
        del train_m
        ms = _members(sww, workloads, cbase, a, "fp32", member_seeds(a.seed, rank, a.members), learned,
                      persistent="phased", patch=cpatch, bps=cbps)
        dtype = "f32"
    else:
        ms, dtype = plain_m, "f64"
    # device memory of one more member of the timed kind (its state, flags, lists
    # and work lists; the grid tables are shared)
    member_bytes = None
    if a.form == "chosen":
        free1 = torch.cuda.mem_get_info()[0]
        probe = _members(sww, workloads, cbase, a, "fp32", [seed + 777], persistent="phased", patch=cpatch, bps=cbps)
        member_bytes = free1 - torch.cuda.mem_get_info()[0]
        probe[0].close()
        del probe
    setup_s = time.perf_counter() - t_setup
    for _ in range(a.warmup):
        sww.step_ensemble(ms, -1.0, 1, True)
    for m in ms:
        if learned is not None:
            m.learn_stats(reset=True)
    # the library's launch counter is process-wide and read through stats(), which
    # launches kernels itself: its own launches are counted and taken out (the
    # live-cell counts around the timed steps launch nothing)
    k_stats = ms[0].stats()["kernel_launches"]
    k_stats = ms[0].stats()["kernel_launches"] - k_stats
    launches0 = ms[0].stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    torch.cuda.profiler.start()   # the timed steps are the profiler's range (ncu --profile-from-start off)
    times, cells = _timed(sww, ms, a.steps, flush, stream)
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    launches = ms[0].stats()["kernel_launches"] - launches0 - k_stats
    total_all, cells_all = combine_ranks(sum(times), sum(cells), "cuda", world)
    value = cells_all / total_all
    if learned is not None:
        lstats = {"misses": 0, "over": 0, "proposed": 0}
        for m in ms:
            for k, v in m.learn_stats(reset=True).items():
                lstats[k] += v
        lstats["train_samples"] = int(len(y))
        lstats["train_loss"] = [float(losses[0]), float(losses[-1])]
        # the same members without the proposal (the exact rules alone), for comparison
        for m in ms:
            m.set_learned(0)
        for _ in range(a.warmup):
            sww.step_ensemble(ms, -1.0, 1, True)
        for m in ms:
            m.learn_stats(reset=True)
        t2, c2 = _timed(sww, ms, a.steps, flush, stream)
        t2, c2 = combine_ranks(sum(t2), sum(c2), "cuda", world)
        plain_misses = sum(m.learn_stats(reset=True)["misses"] for m in ms)
        lstats["without_proposal"] = {"value": c2 / t2, "ms_per_step": 1e3 * t2 / a.steps,
                                      "active_cells_per_step": c2 / a.steps / max(world, 1) / len(ms),
                                      "misses": plain_misses}
        for m in ms:
            m.set_learned(2, learned, a.tau)

    # live timing of the dominant kernel of the timed steps, the structured trend
    # k_tile_trend (one launch per RK stage over all members), and of the whole
    # batched stage, from CUDA events the library records on the first member's
    # stream around each launch group, over the same number of ensemble steps (L2
    # flushed before each)
    prec = "fp32" if dtype == "f32" else "fp64"
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = peaks["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    roofline = roofline_stage = None
    if a.form == "chosen":
        m0 = ms[0]
        classes = ["trend", "irregular", "fill", "restrict", "update", "stage", "dt", "partial", "coeff", "mask",
                   "inverse"]
        m0.profile(classes)
        tbytes = sbytes = tpatches = 0.0
        for _ in range(a.steps):
            sts = [m.stats() for m in ms]
            tbytes += TREND_BYTES_PER_CELL[prec] * sum(_avail_st(st) for st in sts) * 4
            sbytes += STAGE_BYTES_PER_CELL[prec] * sum(sum(st["live_nodes"].values()) for st in sts) * 4
            tpatches += sum(sum(st["active_patches"].values()) for st in sts) * 4
            flush.zero_()
            sww.step_ensemble(ms, -1.0, 1, True)
        prof = m0.profile_read()
        m0.profile([])
        t_ms, t_n = prof["trend"]
        s_ms, s_n = prof["stage"]
        if t_n > 0:
            achieved = tbytes / (t_ms / 1e3) / 1e9
            roofline = {"bound": "hbm", "kernel": "k_tile_trend (structured trend of every active patch, all members)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": f"{peak_src} (burst copy)",
                        "traffic": (TREND_TRAFFIC_PER_CELL[prec] * tbytes / TREND_BYTES_PER_CELL[prec] / t_n
                                    if prec in TREND_TRAFFIC_PER_CELL else None),
                        "avg_launch_us": t_ms * 1e3 / t_n, "launches": t_n,
                        "algorithmic_bytes_per_launch": tbytes / t_n,
                        "available_cells_per_launch": tbytes / TREND_BYTES_PER_CELL[prec] / t_n,
                        "patches_per_launch": tpatches / t_n,
                        "patch_fill": tbytes / TREND_BYTES_PER_CELL[prec] / max(tpatches, 1.0) / cpatch ** 2,
                        "bytes_per_available_cell": TREND_BYTES_PER_CELL[prec],
                        "share_of_step": (t_ms / 1e3) / max(sum(times), 1e-30)}
        if s_n > 0:
            nst = 4 * a.steps
            ach = sbytes / (s_ms / 1e3) / 1e9
            roofline_stage = {"kernels": "every launch of the RK stages (ghosts, trend, irregular patches, "
                                         "restrictions, update)",
                              "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "stage_us": s_ms * 1e3 / nst, "launches_per_stage": s_n / nst,
                              "bytes_per_live_cell_per_stage": STAGE_BYTES_PER_CELL[prec],
                              "share_of_step": (s_ms / 1e3) / max(sum(times), 1e-30),
                              "part_us_per_stage": {k: prof[k][0] * 1e3 / nst for k in
                                                    ("fill", "trend", "irregular", "restrict", "update")},
                              "step_us": {k: prof[k][0] * 1e3 / a.steps for k in
                                          ("dt", "stage", "partial", "coeff", "mask", "inverse")},
                              "step_launches": {k: prof[k][1] / a.steps for k in
                                                ("dt", "stage", "partial", "coeff", "mask", "inverse")}}
    # the persistent RK stage of the plain form's single member (fused trend + update)
    pm = plain_m[0]
    pm.profile(["stage"])
    pcells = 0.0
    for _ in range(a.plain_steps):
        flush.zero_()
        pcells += _live(pm)
        pm.step(-1.0, 1, adapt=True)
    sprof = pm.profile_read()["stage"]
    pm.profile([])
    stage_roof = None
    if sprof[1] > 0:
        ach = STAGE_BYTES_PER_CELL["fp64"] * pcells * 4 / (sprof[0] / 1e3) / 1e9
        stage_roof = {"kernel": "k_stage (plain form, FP64)", "achieved": ach, "peak": peak, "unit": "GB/s",
                      "frac": ach / peak, "avg_launch_us": sprof[0] * 1e3 / sprof[1],
                      "bytes_per_live_cell": STAGE_BYTES_PER_CELL["fp64"]}

    # equal error: chosen vs plain against a non-adaptive run of the same workload
    err = (_equal_error(sww, workloads, base, cbase, cpatch, cbps, a, learned, seed, a.err_steps, a.err_days)
           if a.err_steps != 0 else None)
    turb = (_turbulence(sww, workloads, a, a.turb_steps, flush, peak, TREND_BYTES_PER_CELL["fp32"])
            if a.turb_steps > 0 and a.form == "chosen" else None)

    # end to end through the public API from pinned host buffers
    S = _sampling(workloads, cbase, a.jmax)
    host = []
    for k, m in enumerate(ms):
        dh, u = workloads.Workload("jet", seed=seed + k).fields_on(S)
        host.append((torch.from_numpy(dh).pin_memory().numpy(), torch.from_numpy(u).pin_memory().numpy()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_set = t_adapt = 0.0   # host time in the calls (each returns after its work)
    for m, (dh, u) in zip(ms, host):
        t1 = time.perf_counter()
        m.set_state(dh, u)
        t2 = time.perf_counter()
        m.adapt()
        t_set, t_adapt = t_set + (t2 - t1), t_adapt + (time.perf_counter() - t2)
    t_steps = time.perf_counter()
    ecells = 0.0
    for _ in range(a.steps):
        sww.step_ensemble(ms, -1.0, 1, True)
        ecells += sum(_live(m) for m in ms)
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    e2e_s, ecells = combine_ranks(t_end - t0, ecells, "cuda", world)
    N, E, _, _ = base.sizes(a.jmax)
    e2e = {"value": ecells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(8 * (N + E) * len(ms) / a.steps),
           "d2h_bytes_per_step": int(len(ms) * sww.BATCH_OUT_BYTES),
           "breakdown_ms": {"set_state": 1e3 * t_set, "adapt": 1e3 * t_adapt, "steps": 1e3 * (t_end - t_steps)},
           "set_state_h2d_gbs": 8 * (N + E) * len(ms) / max(t_set, 1e-9) / 1e9,
           "note": "per member sww_set_state from pinned host arrays and sww_adapt once, then per step "
                   "sww_step_ensemble (its read-back: each member's dt, error flag, patch and live "
                   "counts) and sww_live_nodes of every member; breakdown_ms on rank 0's host clock"}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": 1e3 * total_all / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": workload_name(a), "form": a.form, "members": len(ms) * max(world, 1),
                           "l2": "flushed between steps (512 MiB write)", "patch": cpatch,
                           "blocks_per_sm": cbps or 4, "autotune": tuned,
                           "active_cells_per_step": cells_all / a.steps / max(world, 1) / len(ms),
                           "compression": (10 * 4 ** a.jmax + 2) / (cells_all / a.steps / max(world, 1) / len(ms)),
                           "setup_s": setup_s,
                           "device_bytes": {"grid_and_fp64_handle": grid_bytes, "per_member": member_bytes}},
                "plain": plain, "chosen_vs_plain": value / plain["value"], "equal_error": err,
                "learned_proposal": lstats, "learned_turbulence": turb, "clocks": clk, "e2e": e2e,
                "gpu_launches": int(launches),
                "roofline": roofline, "roofline_stage": roofline_stage, "roofline_persistent_stage": stage_roof}
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return line


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        run_reference(a, rank)
        return
    # the oracle's workers are forked before any CUDA call, and run after the GPU part
    pool = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        pool = OraclePool(a, min(a.cpu_jmax, a.jmax), oracle_cores())
    line = run_ours(a, rank, world)
    if rank == 0:
        if pool is not None:
            r = pool.run(1, 1)
            if r is not None:
                v, single, secs, steps = r
                line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": pool.nproc, "kind": "oracle",
                                        "sample": pool.sample(a, 1, 1), "single_process": single,
                                        "host": host_cpu(), "setup_s": pool.setup_s}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
