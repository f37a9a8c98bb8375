"""The persistent RK stage (one cooperative launch per stage, grid barriers between
the phases) against one launch per phase: the same per-item bodies in the same
phase order, so the two paths agree bit for bit."""
import numpy as np
import pytest

import workloads
from lib_mapping import lib_edge_geometry

pytestmark = pytest.mark.gpu


def _run(persistent, precision, steps=4, advect=False):
    import paper_1404_0405_gb300 as sww
    m = sww.Model(2, 5, patch=4, eps=1e-2, persistent=persistent, precision=precision, advect=advect,
                  H=0.0 if advect else 1.0e4)
    xyz, en = m.grid(5)
    mid, tan = lib_edge_geometry(xyz, en)
    W = workloads.Workload("tc1_cosine", alpha=0.7) if advect else workloads.Workload("jet", seed=6)
    dh, u = W.fields(xyz, mid, tan)
    m.set_state(dh, u)
    m.adapt()
    m.rhs()
    trend = [m.get(j, sww.DH_T) for j in range(2, 6)] + [m.get(j, sww.U_T) for j in range(2, 6)]
    m.step(-1.0, steps, True)
    out = []
    for j in range(2, 6):
        out += [m.get(j, sww.NODE_FLAGS), m.get(j, sww.EDGE_FLAGS), m.get(j, sww.DH), m.get(j, sww.U)]
    return trend, out, m.stats()


@pytest.mark.parametrize("precision,advect", [("fp64", False), ("fp32", False), ("fp64", True), ("fp32", True)])
def test_persistent_stage_matches_phase_launches(precision, advect):
    ta, a, sa = _run(True, precision, advect=advect)
    tb, b, sb = _run(False, precision, advect=advect)
    for x, y in zip(ta, tb):
        assert np.array_equal(x, y, equal_nan=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    assert sa["mass"] == sb["mass"] and sa["t"] == sb["t"]
    assert sa["kernel_launches"] > 0
