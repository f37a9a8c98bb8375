"""The workload configurations at their own sizes (the benchmark runs the jet at
Jmax=9; these are the other configurations):

* uniform J=5, harmonic depth with geostrophic velocity, FP64, RK4, CFL 0.8,
  100 steps: every field against the oracle after the 100 steps;
* adaptive FP64 jet, Jmin=4..Jmax=8, eps=1e-2, two model days: mass conserved
  to rounding (measured: unchanged), energy within 1 % (measured -2.4e-3: RK4
  and the adaptation are not energy-conserving), the state finite and the grid
  compressed throughout (at least 4x; measured 7.4x at the most refined step);
* the FP32 form of the jet at Jmax=9 against the FP64 form after one model day,
  per field on Jmin (measured: depth 2.5e-2, velocity 1.3e-2, mass 8.5e-9).  The
  two forms take different threshold decisions where a coefficient lies within
  FP32 rounding of eps, and the jet is unstable, so after a day they differ by
  the adaptation error (eps = 1e-2), not by FP32 rounding;
* an ensemble of members with uneven Jmax (6..9) and eps (1e-2, 3e-3), stepped
  with the batched phases: bit for bit the members stepped alone.
"""
import math

import numpy as np
import pytest

import workloads
from lib_mapping import LevelMap, lib_edge_geometry
from oracle import grid, model

pytestmark = pytest.mark.gpu

DAY = 86400.0


def _fields(m, level, kind, seed):
    xyz, en = m.grid(level)
    mid, tan = lib_edge_geometry(xyz, en)
    return workloads.Workload(kind, seed=seed).fields(xyz, mid, tan)


def test_uniform_j5_hundred_steps_match_oracle():
    import paper_1404_0405_gb300 as sww
    J = 5
    Hy = grid.Hierarchy(J, J)
    L = Hy.levels[J]
    W = workloads.Workload("harmonic", seed=1)
    dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    ora = model.Model(Hy, eps=0.0)
    ora.set_uniform(dh, u)
    ora.adapt()
    lib = sww.Model(J, J, eps=0.0)
    xyz, en = lib.grid(J)
    M = LevelMap(xyz, en, L)
    lib.set_state(M.nodes_to_lib(dh), M.edges_to_lib(u))
    lib.adapt()
    m0 = lib.stats()["mass"]
    worst_dt = 0.0
    for _ in range(100):
        dt = ora.dt_cfl()
        ora.step(dt, adapt_after=False)
        lib.step(-1.0, 1, adapt=False)
        worst_dt = max(worst_dt, abs(lib.stats()["dt"] / dt - 1))
    assert worst_dt < 1e-12
    h_l, u_l = M.nodes_to_ora(lib.get(J, sww.DH)), M.edges_to_ora(lib.get(J, sww.U))
    eh = np.abs(h_l - ora.dh[J]).max() / np.abs(ora.dh[J]).max()
    eu = np.abs(u_l - ora.u[J]).max() / np.abs(ora.u[J]).max()
    print(f"after 100 steps: dh {eh:.2e}, u {eu:.2e}, dt {worst_dt:.1e}")
    assert eh < 1e-12 and eu < 1e-12   # measured 6.8e-14 and 2.4e-14
    assert abs(lib.stats()["mass"] / m0 - 1) < 1e-14


def _run_days(m, days):
    """CFL steps until `days` model days; returns (steps, max live cells, min live cells)."""
    n, hi, lo = 0, 0, 1 << 62
    while m.stats()["t"] < days * DAY:
        m.step(-1.0, 50, True)
        n += 50
        live = sum(m.stats()["live_nodes"].values())
        hi, lo = max(hi, live), min(lo, live)
    return n, hi, lo


def test_adaptive_jet_two_days():
    import paper_1404_0405_gb300 as sww
    m = sww.Model(4, 8, eps=1e-2)
    m.set_state(*_fields(m, 8, "jet", 0))
    m.adapt()
    s0 = m.stats()
    n, hi, lo = _run_days(m, 2.0)
    s1 = m.stats()
    print(f"{n} steps, dt {s1['dt']:.1f} s, live cells {lo}..{hi}, mass drift {s1['mass'] / s0['mass'] - 1:.1e}, "
          f"energy drift {s1['energy'] / s0['energy'] - 1:.1e}")
    assert abs(s1["mass"] / s0["mass"] - 1) < 1e-12
    assert math.isfinite(s1["energy"]) and abs(s1["energy"] / s0["energy"] - 1) < 1e-2
    assert hi < sum(10 * 4 ** j + 2 for j in range(4, 9)) / 4   # compressed throughout
    for j in range(4, 9):
        assert np.isfinite(m.get(j, sww.DH)[(m.get(j, sww.NODE_FLAGS) & 1) > 0]).all()


def test_fp32_form_at_jmax9_one_day():
    import paper_1404_0405_gb300 as sww
    base = sww.Model(4, 9, eps=1e-2)
    dh, u = _fields(base, 9, "jet", 0)
    out = {}
    for prec in ("fp64", "fp32"):
        m = sww.Model(4, 9, eps=1e-2, share=base, precision=prec)
        m.set_state(dh, u)
        m.adapt()
        # a fixed time step (half the FP64 form's first CFL step, room for finer
        # levels to appear) so that both forms reach the same times
        if prec == "fp64":
            m.step(-1.0, 1, True)
            dt = 0.5 * m.stats()["dt"]
            m.set_state(dh, u)
            m.adapt()
        steps = int(round(DAY / dt))
        m.step(dt, steps, True)
        out[prec] = (m.get(4, sww.DH), m.get(4, sww.U), m.stats())
    eh = np.abs(out["fp32"][0] - out["fp64"][0]).max() / np.abs(out["fp64"][0]).max()
    eu = np.abs(out["fp32"][1] - out["fp64"][1]).max() / np.abs(out["fp64"][1]).max()
    dm = abs(out["fp32"][2]["mass"] / out["fp64"][2]["mass"] - 1)
    print(f"FP32 vs FP64 after one day ({steps} steps of {dt:.2f} s) on Jmin: dh {eh:.2e}, u {eu:.2e}, mass {dm:.1e}")
    assert eh < 5e-2 and eu < 5e-2 and dm < 1e-7


def test_uneven_ensemble_batched_matches_members_alone():
    import paper_1404_0405_gb300 as sww
    rng = np.random.default_rng(4)
    specs = [(int(rng.integers(6, 10)), [1e-2, 3e-3][k % 2], 40 + k) for k in range(8)]
    top = max(j for j, _, _ in specs)
    base = sww.Model(4, top, patch=8)
    ens, alone = [], []
    for jmax, eps, seed in specs:
        for group in (ens, alone):
            m = sww.Model(4, jmax, patch=8, eps=eps, share=base, precision="fp32", persistent="phased")
            m.set_state(*_fields(m, jmax, "jet", seed))
            m.adapt()
            group.append(m)
    sww.step_ensemble(ens, -1.0, 3, True)
    for m in alone:
        m.step(-1.0, 3, True)
    for a, b in zip(ens, alone):
        assert a.stats()["t"] == b.stats()["t"] and a.stats()["mass"] == b.stats()["mass"]
        for j in range(4, a.jmax + 1):
            for what in (sww.DH, sww.U, sww.NODE_FLAGS, sww.EDGE_FLAGS):
                assert np.array_equal(a.get(j, what), b.get(j, what))
