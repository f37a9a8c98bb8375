"""Checks at the benchmark's full size (jet, Jmin=4..Jmax=9, patch 8, eps=1e-2,
RK4, CFL 0.8 -- the launch configuration bench.py times), where the oracle cannot
run: properties that hold at any size.

* the mask passes over candidate patches give the same grid as the dense passes
  over whole levels, bit for bit, step after step (flags, fields, patch lists);
* mass is conserved to rounding over adaptive steps (Sec. 4.1, Eq. divRcommute);
* the mask is graded: every live odd node's prediction parents are live, every
  live even node's coarse node is live, and every edge of a live node is live."""
import numpy as np
import pytest

import workloads
from lib_mapping import lib_edge_geometry

pytestmark = pytest.mark.gpu

JMIN, JMAX = 4, 9


@pytest.fixture(scope="module")
def fields():
    import paper_1404_0405_gb300 as sww
    base = sww.Model(JMIN, JMAX, patch=8)
    xyz, en = base.grid(JMAX)
    mid, tan = lib_edge_geometry(xyz, en)
    return base, workloads.Workload("jet", seed=0).fields(xyz, mid, tan)


def _model(fields, mask):
    import paper_1404_0405_gb300 as sww
    base, (dh, u) = fields
    m = sww.Model(JMIN, JMAX, patch=8, eps=1e-2, share=base, mask=mask)
    m.set_state(dh, u)
    m.adapt()
    return m


def test_list_mask_matches_dense_full_size(fields):
    import paper_1404_0405_gb300 as sww
    a, b = _model(fields, "lists"), _model(fields, "dense")
    for step in range(4):
        for j in range(JMIN, JMAX + 1):
            fa, fb = a.get(j, sww.NODE_FLAGS) & 7, b.get(j, sww.NODE_FLAGS) & 7
            assert np.array_equal(fa, fb), f"step {step} level {j}: node flags"
            assert np.array_equal(a.get(j, sww.EDGE_FLAGS) & 3, b.get(j, sww.EDGE_FLAGS) & 3)
            assert np.array_equal(a.patches(j), b.patches(j))
            live = (fa & 3) > 0
            assert np.array_equal(a.get(j, sww.DH)[live], b.get(j, sww.DH)[live])
        a.step(-1.0, 1, True)
        b.step(-1.0, 1, True)
    assert a.stats()["mass"] == b.stats()["mass"]


def test_full_size_mass_conserved(fields):
    m = _model(fields, "lists")
    m0 = m.stats()["mass"]
    m.step(-1.0, 5, True)
    assert abs(m.stats()["mass"] / m0 - 1) < 1e-13


def test_full_size_mask_is_graded(fields):
    import paper_1404_0405_gb300 as sww
    m = _model(fields, "lists")
    m.step(-1.0, 2, True)
    for j in range(JMIN + 1, JMAX + 1):
        nf = m.get(j, sww.NODE_FLAGS)
        live = (nf & 1) > 0
        if not live.any():
            continue
        xyz, en = m.grid(j)
        ef = m.get(j, sww.EDGE_FLAGS)
        # an edge is live exactly when an end node is
        assert np.array_equal((ef & 1) > 0, live[en[:, 0]] | live[en[:, 1]])
        # every live node's position is live one level down (even nodes) or its
        # nearest coarse nodes are (odd nodes): the coarse level holds a live node
        # within one coarse spacing of it
        cx, _ = m.grid(j - 1)
        cl = (m.get(j - 1, sww.NODE_FLAGS) & 1) > 0
        from scipy.spatial import cKDTree
        tree = cKDTree(cx[cl])
        d, _ = tree.query(xyz[live])
        spacing = np.max(np.linalg.norm(cx[en[:, 0] % len(cx)] - cx[en[:, 1] % len(cx)], axis=1))
        assert np.max(d) < spacing
