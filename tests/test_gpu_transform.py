"""Boundary calls around the transforms and the state, through the C ABI:

* sww_forward gives the oracle's wavelet coefficients (Eqs. 1-2, Sec. 4.1);
* sww_inverse after sww_forward returns the state to rounding, and the inverse
  of modified coefficients (sww_set_coeffs) matches the oracle's inverse of
  the same coefficients;
* sww_get_state (the full level from zero coefficients away from live points,
  Sec. 2.2) matches the oracle's reconstruction on every level;
* sww_save / sww_load resume a run bit for bit, and refuse foreign or
  truncated files and other grids with SWW_E_ARG.
"""
import math
import os

import numpy as np
import pytest

import workloads
from lib_mapping import lib_edge_geometry
from test_gpu_parity import Pair, rel_err

pytestmark = pytest.mark.gpu


def _live(P, j):
    return P.ora.live_n[j], P.ora.live_e[j]


def test_forward_matches_oracle_details():
    P = Pair(2, 4, kind="jet", seed=1)
    P.adapt()
    P.ora.step(P.ora.dt_cfl())
    P.lib.step(-1.0, 1, adapt=True)
    hdet, ue, ui = P.ora.details()
    P.lib.forward()
    hscale = max(np.nanmax(np.abs(P.ora.dh[j])) for j in P.ora.levels)
    uscale = max(np.nanmax(np.abs(P.ora.u[j])) for j in P.ora.levels)
    for j in (3, 4):
        Mf, Mc = P.maps[j], P.maps[j - 1]
        lh, le, li = P.lib.coeffs(j)
        odd = P.Hy.odd[j]
        h = Mf.nodes_to_ora(lh)[odd]
        ok = ~np.isnan(hdet[j])
        assert ok.any() and np.abs(h[ok] - hdet[j][ok]).max() < 1e-12 * hscale
        e = le[Mc.inv_edge]
        ok = ~np.isnan(ue[j])
        assert ok.any() and np.abs(e[ok] - ue[j][ok]).max() < 1e-12 * uscale
        i = Mf.edges_to_ora(li)[P.ora.VS[j].int_edge]
        ok = ~np.isnan(ui[j])
        assert ok.any() and np.abs(i[ok] - ui[j][ok]).max() < 1e-12 * uscale


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_forward_inverse_roundtrip(precision, tol):
    P = Pair(2, 4, kind="jet", seed=2, precision=precision)
    P.adapt()
    P.lib.step(-1.0, 2, adapt=True)
    before = {j: (P.lib.get(j, P.sww.DH), P.lib.get(j, P.sww.U)) for j in range(2, 5)}
    P.lib.forward()
    P.lib.inverse()
    for j in range(2, 5):
        nf, ef = P.lib.get(j, P.sww.NODE_FLAGS), P.lib.get(j, P.sww.EDGE_FLAGS)
        mn, me = (nf & 3) > 0, (ef & 3) > 0
        h, u = P.lib.get(j, P.sww.DH), P.lib.get(j, P.sww.U)
        assert rel_err(h[mn], before[j][0][mn]) < tol
        assert rel_err(u[me], before[j][1][me]) < tol


def test_inverse_of_modified_coefficients_matches_oracle():
    P = Pair(2, 4, kind="jet", seed=3)
    P.adapt()
    hdet, ue, ui = P.ora.details()
    P.lib.forward()
    # halve every coefficient of level 4 on both sides, then invert
    hdet[4], ue[4], ui[4] = 0.5 * hdet[4], 0.5 * ue[4], 0.5 * ui[4]
    P.ora.apply_mask(P.ora.live_n, P.ora.live_e, hdet, ue, ui)
    lh, le, li = P.lib.coeffs(4)
    P.lib.set_coeffs(4, 0.5 * lh, 0.5 * le, 0.5 * li)
    P.lib.inverse()
    P.check_masks()
    P.check_fields()


@pytest.mark.parametrize("advect", [False, True])
def test_full_level_state_matches_oracle(advect):
    kw = dict(kind="tc1_cosine", eps=0.02, advect=True, alpha=0.7) if advect else dict(kind="jet", seed=4)
    P = Pair(2, 4, **kw)
    P.adapt()
    for _ in range(2):
        P.ora.step(P.ora.dt_cfl())
        P.lib.step(-1.0, 1, adapt=True)
    assert P.ora.live_n[4].sum() < P.Hy.levels[4].N     # the fine level is partly live
    for j in range(2, 5):
        h_o, u_o = P.ora.get_uniform(j)
        h_l, u_l = P.lib.get_state(j)
        M = P.maps[j]
        assert rel_err(M.nodes_to_ora(h_l), h_o) < 1e-12, j
        assert rel_err(M.edges_to_ora(u_l), u_o) < 1e-12, j
    # the FP32 form to its stated bound
    P32 = Pair(2, 4, precision="fp32", **kw)
    P32.adapt()
    h_o, u_o = P32.ora.get_uniform(4)
    h_l, u_l = P32.lib.get_state(4)
    assert rel_err(P32.maps[4].nodes_to_ora(h_l), h_o) < 2e-6
    assert rel_err(P32.maps[4].edges_to_ora(u_l), u_o) < 2e-6


def _member(sww, precision, advect=False, jmax=5):
    m = sww.Model(2, jmax, patch=8, eps=1e-2, precision=precision, advect=advect, H=0.0 if advect else 1.0e4)
    xyz, en = m.grid(jmax)
    mid, tan = lib_edge_geometry(xyz, en)
    W = workloads.Workload("tc1_smooth", alpha=0.3) if advect else workloads.Workload("jet", seed=9)
    return m, W.fields(xyz, mid, tan)


def _snapshot(sww, m):
    out = []
    for j in range(m.jmin, m.jmax + 1):
        out += [m.get(j, sww.DH), m.get(j, sww.U), m.get(j, sww.NODE_FLAGS), m.get(j, sww.EDGE_FLAGS)]
        out.append(m.patches(j))
    st = m.stats()
    return out, (st["t"], st["steps"], st["mass"], st["dt"], st["eps_h"])


@pytest.mark.parametrize("precision,advect", [("fp64", False), ("fp32", False), ("fp64", True)])
def test_checkpoint_resumes_bit_for_bit(tmp_path, precision, advect):
    import paper_1404_0405_gb300 as sww
    path = str(tmp_path / "run.ckpt")
    a, (dh, u) = _member(sww, precision, advect)
    a.set_state(dh, u)
    a.adapt()
    a.step(-1.0, 3, True)
    a.save(path)
    a.step(-1.0, 4, True)
    b, _ = _member(sww, precision, advect)
    b.load(path)
    assert b.stats()["steps"] == 3
    b.step(-1.0, 4, True)
    xa, sa = _snapshot(sww, a)
    xb, sb = _snapshot(sww, b)
    for p, q in zip(xa, xb):
        assert np.array_equal(p, q)
    assert sa == sb


def test_checkpoint_refuses_foreign_truncated_and_other_grids(tmp_path):
    import paper_1404_0405_gb300 as sww
    path = str(tmp_path / "run.ckpt")
    a, (dh, u) = _member(sww, "fp64")
    a.set_state(dh, u)
    a.adapt()
    a.save(path)
    data = open(path, "rb").read()
    bad = str(tmp_path / "bad.ckpt")
    b, _ = _member(sww, "fp64")
    for blob in (data[: len(data) // 2], b"not a checkpoint" * 8, data[:-1]):
        open(bad, "wb").write(blob)
        with pytest.raises(sww.SwwError):
            b.load(bad)
    with pytest.raises(sww.SwwError):
        b.step(-1.0, 1, True)           # still without state: nothing was loaded
    other, _ = _member(sww, "fp64", jmax=4)
    with pytest.raises(sww.SwwError):
        other.load(path)
    fp32, _ = _member(sww, "fp32")
    with pytest.raises(sww.SwwError):
        fp32.load(path)
    b.load(path)                        # the good file still loads
    assert np.array_equal(b.get(5, sww.DH), a.get(5, sww.DH))


def test_state_level_error_paths():
    """A level out of range, and a prescribed velocity set below Jmax, are
    refused (SWW_E_ARG) and leave the handle usable."""
    import paper_1404_0405_gb300 as sww
    m = sww.Model(2, 4, patch=4, eps=1e-2)
    N3, E3, _, _ = m.sizes(3)
    with pytest.raises(sww.SwwError):
        m.set_state(np.zeros(N3), np.zeros(E3), level=5)
    adv = sww.Model(2, 4, patch=4, eps=1e-2, advect=True, H=0.0)
    with pytest.raises(sww.SwwError):
        adv.set_state(np.zeros(N3), np.zeros(E3), level=3)
    m.set_state(np.full(N3, 3.0), np.zeros(E3), level=3)
    m.adapt()
    h4, u4 = m.get_state(4)
    assert np.abs(h4 - 3.0).max() < 1e-12 and np.abs(u4).max() == 0.0


def test_non_finite_initial_fields_are_refused():
    """A NaN or an infinity in host initial fields is refused (SWW_E_NUMERIC)
    before the handle's state changes, wherever it sits (the first, middle and
    last value of either field); valid fields then load as usual."""
    import paper_1404_0405_gb300 as sww
    m, (dh, u) = _member(sww, "fp32", jmax=4)
    n, total = len(dh), len(dh) + len(u)
    for i in (0, n // 2, n - 1, n, n + len(u) // 2, total - 1):
        bad_dh, bad_u = (dh.copy(), u) if i < n else (dh, u.copy())
        if i < n:
            bad_dh[i] = np.nan
        else:
            bad_u[i - n] = np.inf
        with pytest.raises(sww.SwwError, match="non-finite"):
            m.set_state(bad_dh, bad_u)
    with pytest.raises(sww.SwwError):
        m.step(-1.0, 1, True)            # nothing was loaded
    m.set_state(dh, u)
    m.adapt()
    m.step(-1.0, 1, True)
    assert np.isfinite(m.stats()["mass"])


def test_mask_call_matches_level_flags():
    import paper_1404_0405_gb300 as sww
    P = Pair(2, 4, kind="jet", seed=6)
    P.adapt()
    for j in range(2, 5):
        nodes, edges = P.lib.mask(j)
        assert np.array_equal(nodes, P.lib.get(j, sww.NODE_FLAGS))
        assert np.array_equal(edges, P.lib.get(j, sww.EDGE_FLAGS))
    P.check_masks()


def test_host_fields_load_alike_from_pageable_pinned_and_device_memory():
    """The same fields from pageable host arrays, pinned host arrays and CUDA
    tensors give the same state, bit for bit, on every level."""
    import torch
    import paper_1404_0405_gb300 as sww
    got = []
    for kind in ("pageable", "pinned", "device"):
        m, (dh, u) = _member(sww, "fp64", jmax=5)
        if kind == "pinned":
            dh, u = (torch.from_numpy(x).pin_memory().numpy() for x in (dh, u))
        elif kind == "device":
            dh, u = (torch.from_numpy(x).cuda() for x in (dh, u))
        m.set_state(dh, u)
        m.adapt()
        got.append(_snapshot(sww, m))
    for other in got[1:]:
        assert other[1] == got[0][1]
        for x, y in zip(got[0][0], other[0]):
            assert np.array_equal(x, y)
