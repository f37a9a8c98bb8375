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


def test_barrier_wait_runs_out_and_recovers():
    """The bounded grid barrier: with a short spin limit and one block told (on
    the host) not to arrive, every other block's wait runs out, the kernel
    returns, the step reports SWW_E_TIMEOUT without advancing t, and after the
    fault is cleared the next step equals a step of a handle that never failed.
    No wait outlasts the limit (about 1 ms here), so nothing hangs."""
    import paper_1404_0405_gb300 as sww

    def fresh():
        m = sww.Model(2, 5, patch=4, eps=1e-2, persistent=True)
        xyz, en = m.grid(5)
        mid, tan = lib_edge_geometry(xyz, en)
        dh, u = workloads.Workload("jet", seed=6).fields(xyz, mid, tan)
        m.set_state(dh, u)
        m.adapt()
        return m

    m = fresh()
    t0 = m.stats()["t"]
    m.barrier_fault(spin_cycles=2_000_000, skip_block=0)
    with pytest.raises(sww.SwwError) as ei:
        m.step(-1.0, 1, True)
    assert ei.value.code == sww.E_TIMEOUT
    assert m.stats()["t"] == t0 and m.stats()["steps"] == 0
    # a second failing step: the reset barrier state times out the same way
    with pytest.raises(sww.SwwError) as ei:
        m.step(-1.0, 1, True)
    assert ei.value.code == sww.E_TIMEOUT
    m.barrier_fault(0, -1)
    m.step(-1.0, 1, True)
    ref = fresh()
    ref.step(-1.0, 1, True)
    sm, sr = m.stats(), ref.stats()
    assert sm["steps"] == 1 and sm["t"] == sr["t"]
    for j in range(2, 6):
        for what in (sww.NODE_FLAGS, sww.EDGE_FLAGS):
            assert np.array_equal(m.get(j, what), ref.get(j, what)), (j, what)
        for what in (sww.DH, sww.U):
            x, y = m.get(j, what), ref.get(j, what)
            live = (m.get(j, sww.NODE_FLAGS if what == sww.DH else sww.EDGE_FLAGS) & sww.LIVE) > 0
            scale = max(np.abs(y[live]).max(), 1e-300)
            assert np.abs(x[live] - y[live]).max() <= 1e-12 * scale, (j, what)
