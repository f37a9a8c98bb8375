#!/usr/bin/env python
"""Benchmark: active-cell RK4 steps per second of the adaptive wavelet TRiSK step.

Workload (seeded, synthetic): zonal jet u = 80 exp(-((lat - lat0)/7 deg)^2) m/s
with gradient-wind balanced depth (mean 10 km) and three 120 m Gaussian bumps,
radius 6.371e6 m, Omega 7.292e-5 1/s, g 9.80616 m/s^2, adaptive levels
Jmin=4..Jmax=9, eps = 1e-2 relative, RK4, CFL 0.8, FP64 throughout (the plain
form).  A step is one RK4 step with its partial transform and grid adaptation.
Value = (live nodes over all levels, averaged over the timed steps) x steps /
seconds, with per-step CUDA-event times (the L2 cache is flushed between steps
with a 512 MiB write outside the timed events).

--impl reference runs the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm for this build).  With --gpus N under torchrun every
rank runs an independent ensemble member (seed + rank): weak scaling, no
collective on the data path.
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
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-jmax", type=int, default=6, help="finest level of the oracle sample")
    return p.parse_args()


def workload_name(a):
    return (f"adaptive zonal jet + 3 bumps, Jmin={a.jmin}..Jmax={a.jmax}, eps={a.eps:g} relative, "
            f"FP64 plain form, RK4, CFL 0.8")


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
    return cells / t, sample


# ----------------------------------------------------------------------------- reference arm

def run_reference(a, rank):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    steps = max(1, min(a.steps, 6))
    warm = min(a.warmup, 2)
    v, sample = oracle_rate(a, steps, warm, a.seed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": steps,
            "warmup": warm, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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

# Algorithmic bytes per live edge of one launch of the second trend pass
# (k_node_coriolis, FP64).  Coriolis part, per live edge: the ten reconstruction
# weights and edge ids (10 x 12 B), the edge's own flux, its two triangle ids and
# potential vorticities (8 + 8 + 16 B), and the tendency it writes (8 B).  Node
# part, per node (three edges per node on the grid): area, depth, degree, six
# ring-edge codes, face and edge lengths already counted with the edges, and the
# divergence and Bernoulli function written (8 + 8 + 1 + 24 + 16 B = 57 B), i.e.
# 19 B per edge.  Values shared with neighbours are counted once, with their owner.
CORIOLIS_BYTES_PER_EDGE = 10 * 12 + 8 + 8 + 16 + 8 + 19
# DRAM bytes (read + write) per launch of k_node_coriolis from one ncu capture of
# the jet at Jmin=4..Jmax=8, eps=1e-2 (the same active set and launches as
# Jmax=9); None once the kernel changes.
CORIOLIS_TRAFFIC_PER_LAUNCH = 15.933184e6 + 0.344064e6


def run_ours(a, rank, world):
    import torch
    import paper_1404_0405_gb300 as sww
    import workloads

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    seed = a.seed + rank
    t_setup = time.perf_counter()
    m = sww.Model(a.jmin, a.jmax, patch=a.patch, eps=a.eps, rk="rk4", cfl=0.8, precision=a.precision)
    xyz, en = m.grid(a.jmax)
    mid, tan = edge_geometry(xyz, en)
    dh0, u0 = workloads.Workload("jet", seed=seed).fields(xyz, mid, tan)
    setup_s = time.perf_counter() - t_setup

    def active():
        return sum(m.stats()["live_nodes"].values())

    m.set_state(dh0, u0)
    m.adapt()
    m.adapt()
    for _ in range(a.warmup):
        m.step(-1.0, 1, adapt=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    clocks = Clocks(dev)
    times, cells = [], []
    launches0 = m.stats()["kernel_launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(a.steps):
        act0 = active()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.step(-1.0, 1, adapt=True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        cells.append(0.5 * (act0 + active()))
    clk = clocks.stop()
    launches = m.stats()["kernel_launches"] - launches0
    total = sum(times)
    total_all, cells_all = combine_ranks(total, sum(cells), "cuda", world)
    value = cells_all / total_all

    # live per-launch timing of the dominant kernel (Coriolis) over the same number of steps
    st = m.stats()
    m.profile(["coriolis"])
    live_edges = st["live_edges"]
    for _ in range(a.steps):
        flush.zero_()
        m.step(-1.0, 1, adapt=True)
    prof = m.profile_read()
    m.profile([])
    cor_ms, cor_n = prof["coriolis"]
    # one launch per RK stage covers every level; bytes use the live edges
    per_step_bytes = 4 * sum(live_edges.values()) * CORIOLIS_BYTES_PER_EDGE
    achieved = per_step_bytes * a.steps / (cor_ms / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = peaks["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    roofline = {"bound": "hbm", "kernel": "k_node_coriolis", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} (burst copy)",
                "traffic": CORIOLIS_TRAFFIC_PER_LAUNCH if a.jmax >= 8 and a.eps == 1e-2 else None,
                "avg_launch_us": cor_ms * 1e3 / max(cor_n, 1), "launches": cor_n,
                "bytes_per_live_edge": CORIOLIS_BYTES_PER_EDGE}

    # end to end through the public API from pinned host buffers
    dh_h = torch.from_numpy(dh0).pin_memory().numpy()
    u_h = torch.from_numpy(u0).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.set_state(dh_h, u_h)
    m.adapt()
    ecells = 0.0
    for _ in range(a.steps):
        m.step(-1.0, 1, adapt=True)
        s = m.stats()
        ecells += sum(s["live_nodes"].values())
    torch.cuda.synchronize()
    e2e_s, ecells = combine_ranks(time.perf_counter() - t0, ecells, "cuda", world)
    N, E, _, _ = m.sizes(a.jmax)
    e2e = {"value": ecells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(8 * (N + E) / a.steps),
           "d2h_bytes_per_step": int(8 + 8 * 70), "note": "sww_set_state from pinned host arrays + adapt + "
                                                         "per step sww_step and sww_stats_get"}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": 1e3 * total_all / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(a), "l2": "flushed between steps (512 MiB write)",
                           "members": world, "patch": a.patch,
                           "active_cells_per_step": cells_all / a.steps / max(world, 1),
                           "compression": (10 * 4 ** a.jmax + 2) / (cells_all / a.steps / max(world, 1)),
                           "grid_setup_s": setup_s},
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline}
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
            v, sample = oracle_rate(a, 2, 1, a.seed)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
