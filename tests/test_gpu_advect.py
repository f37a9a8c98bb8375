"""The advection test of Sec. 7.1 on the GPU over one full rotation (12 days):
the bell carried by the tilted solid-body rotation on the adaptive grid, with
the finest level left to the threshold (Sec. 2.3: Jmax may be set by eps).

* mass is conserved to rounding over the whole rotation;
* the error against the exact solution (the bell back at its start) falls as
  eps falls and, for small eps, reaches the error of the uniform grid of the
  finest level while holding fewer points;
* with a high level cap the finest level used is set by eps, not by the cap.
"""
import math

import numpy as np
import pytest

import workloads
from lib_mapping import lib_edge_geometry

pytestmark = pytest.mark.gpu

DAY = 86400.0
ALPHA = 0.05          # tilt of the rotation axis (rad)


def leaf_error(m, W, t, grids):
    """max |dh - exact| / bell height over live nodes that are not covered."""
    import paper_1404_0405_gb300 as sww
    e = 0.0
    for j, xyz in grids.items():
        nf = m.get(j, sww.NODE_FLAGS)
        leaf = ((nf & 1) > 0) & ((nf & 4) == 0)
        if leaf.any():
            e = max(e, float(np.abs(m.get(j, sww.DH)[leaf] - W.exact(xyz[leaf], t)).max()))
    return e / W.bell_h


def one_rotation(m, jmin, jmax):
    """Adaptive CFL steps until t >= 12 days; returns (steps, finest level used,
    mean live nodes)."""
    t, n, top, live = 0.0, 0, jmin, 0.0
    while t < 12 * DAY:
        st = m.stats()
        top = max([top] + [j for j in range(jmin, jmax + 1) if st["live_nodes"][j] > 0])
        live += sum(st["live_nodes"].values())
        m.step(-1.0, 1, adapt=True)
        t = m.stats()["t"]
        n += 1
        assert n < 20000
    return n, top, live / n


def _setup(jmin, jmax, kind):
    import paper_1404_0405_gb300 as sww
    W = workloads.Workload(kind, alpha=ALPHA)
    base = sww.Model(jmin, jmax, H=0.0, eps=0.0, advect=True)
    grids = {j: base.grid(j)[0] for j in range(jmin, jmax + 1)}
    xyz, en = base.grid(jmax)
    mid, tan = lib_edge_geometry(xyz, en)
    return sww, W, base, grids, W.fields(xyz, mid, tan)


def test_rotation_error_falls_with_eps_to_the_uniform_error():
    jmin, jmax = 4, 7
    sww, W, base, grids, (dh, u) = _setup(jmin, jmax, "tc1_smooth")
    uni = sww.Model(jmax, jmax, H=0.0, eps=0.0, advect=True)
    xyz, en = uni.grid(jmax)
    mid, tan = lib_edge_geometry(xyz, en)
    uni.set_state(*W.fields(xyz, mid, tan))
    uni.adapt()
    one_rotation(uni, jmax, jmax)
    e_uni = leaf_error(uni, W, uni.stats()["t"], {jmax: xyz})
    errs, lives = [], []
    for eps in (0.02, 0.002, 0.0002):
        m = sww.Model(jmin, jmax, H=0.0, eps=eps, advect=True, share=base)
        m.set_state(dh, u)
        m.adapt()
        m0 = m.stats()["mass"]
        _, _, live = one_rotation(m, jmin, jmax)
        assert abs(m.stats()["mass"] / m0 - 1) < 1e-13
        errs.append(leaf_error(m, W, m.stats()["t"], grids))
        lives.append(live)
        m.close()
    print("uniform", e_uni, "adaptive", errs, "live", lives)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1.2 * e_uni
    assert lives[2] < sum(grids[j].shape[0] for j in grids)


def test_finest_level_set_by_eps():
    jmin, jmax = 4, 9
    sww, W, base, grids, (dh, u) = _setup(jmin, jmax, "tc1_smooth")
    tops = {}
    for eps in (0.04, 0.02):
        m = sww.Model(jmin, jmax, H=0.0, eps=eps, advect=True, share=base)
        m.set_state(dh, u)
        m.adapt()
        _, tops[eps], _ = one_rotation(m, jmin, jmax)
        m.close()
    print("finest level used", tops)
    assert jmin < tops[0.04] < jmax
    assert tops[0.02] > tops[0.04]
