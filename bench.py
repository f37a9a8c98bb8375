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
equal_error: relative l2 error of the Jmin depth after --err-steps steps of the
same dt, plain and chosen, against a non-adaptive FP64 run (every point live).

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
    p.add_argument("--err-steps", type=int, default=20)
    p.add_argument("--tau", type=float, default=0.9, help="proposal threshold on the perceptron probability")
    p.add_argument("--no-learned", action="store_true", help="chosen form without the learned proposal")
    p.add_argument("--no-tune", action="store_true", help="chosen form without the autotuner (patch, 4 blocks/SM)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-jmax", type=int, default=6, help="finest level of the oracle sample")
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


def oracle_rate(a, steps, warmup, seed):
    """Active-cell steps/s of the FP64 CPU oracle on the same workload at
    Jmin..cpu_jmax (grid setup untimed)."""
    import workloads
    from oracle import grid, model
    jmax = min(a.cpu_jmax, a.jmax)
    Hy = grid.Hierarchy(a.jmin, jmax)
    M = model.Model(Hy, eps=a.eps, rk="rk4", cfl=0.8)
    L = Hy.levels[jmax]
    dh, u = workloads.Workload("jet", seed=seed).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    M.set_uniform(dh, u)
    M.adapt()
    M.adapt()
    for _ in range(warmup):
        M.step(M.dt_cfl())
    cells, t = 0, 0.0
    for _ in range(steps):
        act = M.active_nodes()
        t0 = time.perf_counter()
        M.step(M.dt_cfl())
        t += time.perf_counter() - t0
        cells += (act + M.active_nodes()) / 2
    sample = (f"same jet workload and eps at Jmin={a.jmin}..Jmax={jmax} ({steps} RK4 steps after {warmup} warm-up, "
              f"grid setup untimed), single-threaded numpy oracle")
    return cells / t, sample, t / steps


# ----------------------------------------------------------------------------- reference arm

def run_reference(a, rank):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    steps = max(1, min(a.steps, 6))
    warm = min(a.warmup, 2)
    v, sample, per_step = oracle_rate(a, steps, warm, a.seed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": 1e3 * per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
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
# persistent RK stage at the minimum a fused stage must move: the state read
# (dh, u: 32 B), the RK base read and the new state written (64 B), and the
# geometry in its minimal form (cell and dual areas, 3 d_e, 3 l_e, kite fractions,
# Coriolis at the dual cells: 17 words, 136 B) -- 232 B in FP64; the FP32 form
# halves every term (its state and stencil weights are FP32).
STAGE_BYTES_PER_CELL = {"fp64": 232, "fp32": 116}

# DRAM bytes (read + write) of the batched RK stage (the k_phase_batch launches of
# one stage) per live member-cell, from one ncu capture of the same jet at
# Jmin=4..Jmax=8 with 16 members (203.8 MB per stage over 302 856 member-cells,
# cold cache per launch; profiles/k_phase_batch_jet_J4-8_16members.md), scaled to a
# launch by the member-cells it processes; remove the entry when the kernel changes.
PHASE_TRAFFIC_PER_CELL_STAGE = {"fp32": 673.0}


def _live(m):
    return sum(m.stats()["live_nodes"].values())


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


def _equal_error(sww, workloads, base, cbase, cpatch, cbps, a, learned, seed, steps):
    """Relative l2 error of the Jmin depth after `steps` steps of a fixed dt, for the
    plain form (FP64, exact mask) and the chosen form (FP32, learned proposal),
    against a non-adaptive FP64 run (eps = 0: every point live) substepped at its own
    CFL limit to the same final time."""
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
    dt = plain.stats()["dt"] or 0.0
    if dt <= 0:
        plain.step(-1.0, 1, True)
        dt = plain.stats()["dt"]
        plain = make("fp64", a.eps)
    ref.step(-1.0, 1, False)
    sub = max(1, math.ceil(dt / ref.stats()["dt"]))
    ref = make("fp64", 0.0)
    for m in (plain, chosen):
        m.step(dt, steps, True)
    ref.step(dt / sub, steps * sub, False)
    r = ref.get(a.jmin, sww.DH)
    err = lambda m: float(np.linalg.norm(m.get(a.jmin, sww.DH) - r) / np.linalg.norm(r))
    out = {"steps": steps, "dt_s": dt, "reference_substeps": sub, "plain_fp64": err(plain),
           "chosen": err(chosen)}
    out["ratio"] = out["chosen"] / max(out["plain_fp64"], 1e-300)
    return out


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
    seed = a.seed + 1000 * rank
    t_setup = time.perf_counter()
    base = sww.Model(a.jmin, a.jmax, patch=a.patch, eps=a.eps, rk="rk4", cfl=0.8)
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
        ms = _members(sww, workloads, cbase, a, "fp32", [seed + k for k in range(a.members)], persistent="phased",
                      patch=cpatch, bps=cbps)
        dtype = "f32"
    elif a.form == "chosen":
        train_m = _members(sww, workloads, cbase, a, "fp32", [seed + 500 + k for k in range(2)], patch=cpatch,
                           bps=cbps)
        Xs, ys = zip(*[learn.collect(m, a.train_steps) for m in train_m])
        X, y = np.concatenate(Xs), np.concatenate(ys)
        learned, losses = learn.train(X, y, epochs=300)
        del train_m
        ms = _members(sww, workloads, cbase, a, "fp32", [seed + k for k in range(a.members)], learned,
                      persistent="phased", patch=cpatch, bps=cbps)
        dtype = "f32"
    else:
        ms, dtype = plain_m, "f64"
    setup_s = time.perf_counter() - t_setup
    for _ in range(a.warmup):
        sww.step_ensemble(ms, -1.0, 1, True)
    for m in ms:
        if learned is not None:
            m.learn_stats(reset=True)
    launches0 = ms[0].stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    times, cells = _timed(sww, ms, a.steps, flush, stream)
    clk = clocks.stop()
    launches = ms[0].stats()["kernel_launches"] - launches0   # process-wide counter: every member
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
        t2, c2 = _timed(sww, ms, a.steps, flush, stream)
        t2, c2 = combine_ranks(sum(t2), sum(c2), "cuda", world)
        lstats["without_proposal"] = {"value": c2 / t2, "ms_per_step": 1e3 * t2 / a.steps,
                                      "active_cells_per_step": c2 / a.steps / max(world, 1) / len(ms)}
        for m in ms:
            m.set_learned(2, learned, a.tau)

    # live timing of the dominant kernel of the timed steps: the batched RK stage
    # (k_phase_batch, one launch per phase over all members), from CUDA events the
    # library records on the first member's stream around each RK stage, over the
    # same number of ensemble steps (L2 flushed before each)
    prec = "fp32" if dtype == "f32" else "fp64"
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = peaks["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    roofline = None
    if a.form == "chosen":
        m0 = ms[0]
        m0.profile(["stage"])
        sbytes = 0.0
        for _ in range(a.steps):
            c = sum(_live(m) for m in ms)
            sbytes += STAGE_BYTES_PER_CELL[prec] * c * 4
            flush.zero_()
            sww.step_ensemble(ms, -1.0, 1, True)
        s_ms, s_n = m0.profile_read()["stage"]
        m0.profile([])
        if s_n > 0:
            achieved = sbytes / (s_ms / 1e3) / 1e9
            roofline = {"bound": "hbm", "kernel": "k_phase_batch (RK stage phases, all members)",
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_source": f"{peak_src} (burst copy)",
                        "traffic": (PHASE_TRAFFIC_PER_CELL_STAGE[prec] * sbytes / STAGE_BYTES_PER_CELL[prec] / s_n
                                    if prec in PHASE_TRAFFIC_PER_CELL_STAGE else None),
                        "avg_launch_us": s_ms * 1e3 / s_n,
                        "launches": s_n, "algorithmic_bytes_per_launch": sbytes / s_n,
                        "bytes_per_live_cell_per_stage": STAGE_BYTES_PER_CELL[prec],
                        "stage_share_of_step": (s_ms / 1e3) / max(sum(times), 1e-30)}
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
    err = (_equal_error(sww, workloads, base, cbase, cpatch, cbps, a, learned, seed, a.err_steps)
           if a.err_steps > 0 else None)

    # end to end through the public API from pinned host buffers
    S = _sampling(workloads, cbase, a.jmax)
    host = []
    for k, m in enumerate(ms):
        dh, u = workloads.Workload("jet", seed=seed + k).fields_on(S)
        host.append((torch.from_numpy(dh).pin_memory().numpy(), torch.from_numpy(u).pin_memory().numpy()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, (dh, u) in zip(ms, host):
        m.set_state(dh, u)
        m.adapt()
    ecells = 0.0
    for _ in range(a.steps):
        sww.step_ensemble(ms, -1.0, 1, True)
        ecells += sum(_live(m) for m in ms)
    torch.cuda.synchronize()
    e2e_s, ecells = combine_ranks(time.perf_counter() - t0, ecells, "cuda", world)
    N, E, _, _ = base.sizes(a.jmax)
    e2e = {"value": ecells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(8 * (N + E) * len(ms) / a.steps),
           "d2h_bytes_per_step": int(len(ms) * (8 + 8 * 70)),
           "note": "per member sww_set_state from pinned host arrays and sww_adapt once, then per step "
                   "sww_step_ensemble and sww_stats_get of every member"}

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
                           "setup_s": setup_s},
                "plain": plain, "chosen_vs_plain": value / plain["value"], "equal_error": err,
                "learned_proposal": lstats, "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
                "roofline": roofline, "roofline_persistent_stage": stage_roof}
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
    line = run_ours(a, rank, world)
    if rank == 0:
        if world == 1 and not a.no_cpu_baseline:
            v, sample, _ = oracle_rate(a, 2, 1, a.seed)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                    "host": host_cpu()}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
