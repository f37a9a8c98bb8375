"""Ensemble members (shared grid, concurrent steps) against the same members
stepped one at a time: the library's kernels are deterministic (exact min/max
atomics, fixed reduction trees), so a member advanced by sww_step_ensemble must
equal, bit for bit, the same member advanced alone by sww_step on the same grid.

A member with a smaller jmax than the shared grid uses that grid's hierarchical
areas (Sec. 4.1: coarse areas are built up from the finest level), which differ
from a grid built to the member's own jmax by rounding only."""
import numpy as np
import pytest

import workloads
from lib_mapping import lib_edge_geometry

pytestmark = pytest.mark.gpu

MEMBERS = [  # (jmax, eps, seed)
    (4, 1e-2, 0),
    (3, 3e-3, 1),
    (4, 3e-3, 2),
]


def _fields(m, seed):
    xyz, en = m.grid(m.jmax)
    mid, tan = lib_edge_geometry(xyz, en)
    return workloads.Workload("jet", seed=seed).fields(xyz, mid, tan)


def _snapshot(sww, m):
    """Live and ghost values and flags of every level (values elsewhere are
    scratch that no live result reads)."""
    out = {}
    for j in range(m.jmin, m.jmax + 1):
        nf, ef = m.get(j, sww.NODE_FLAGS), m.get(j, sww.EDGE_FLAGS)
        na, ea = (nf & 3) > 0, (ef & 3) > 0
        out[f"nflag{j}"] = nf & 7
        out[f"eflag{j}"] = ef & 7
        out[f"dh{j}"] = m.get(j, sww.DH)[na]
        out[f"u{j}"] = m.get(j, sww.U)[ea]
    st = m.stats()
    return out, (st["t"], st["mass"], st["energy"], st["steps"])


@pytest.mark.parametrize("precision,persistent", [("fp64", "auto"), ("fp32", "auto"), ("fp64", "phased"),
                                                  ("fp32", "phased")])
def test_shared_members_match_single_runs(precision, persistent):
    """persistent "auto": the members' steps overlap on their streams; "phased":
    one regular launch per phase of a stage over all members."""
    import paper_1404_0405_gb300 as sww
    jmin, top = 2, max(j for j, _, _ in MEMBERS)
    base = sww.Model(jmin, top, patch=4)
    ens, alone = [], []
    for jmax, eps, seed in MEMBERS:
        for group in (ens, alone):
            m = sww.Model(jmin, jmax, patch=4, eps=eps, share=base, precision=precision, persistent=persistent)
            dh, u = _fields(m, seed)
            m.set_state(dh, u)
            m.adapt()
            group.append(m)
    sww.step_ensemble(ens, -1.0, 5, True)
    for m in alone:
        m.step(-1.0, 5, True)
    for i, (a, b) in enumerate(zip(ens, alone)):
        fa, sa = _snapshot(sww, a)
        fb, sb = _snapshot(sww, b)
        assert sa == sb, f"member {i}"
        for k in fa:
            x, y = fa[k], fb[k]
            assert x.shape == y.shape, f"member {i} {k}: {x.shape} vs {y.shape}"
            bad = np.flatnonzero(x != y)
            assert bad.size == 0, f"member {i} {k}: {bad.size} differ, first {bad[:5]}, {x[bad[:3]]} vs {y[bad[:3]]}"


@pytest.mark.parametrize("persistent", ["auto", "phased"])
def test_batched_members_with_given_time_step(persistent):
    """A given time step (the same for every member) through the batched stages."""
    import paper_1404_0405_gb300 as sww
    jmin, top = 2, max(j for j, _, _ in MEMBERS)
    base = sww.Model(jmin, top, patch=4)
    ens, alone = [], []
    for jmax, eps, seed in MEMBERS:
        for group in (ens, alone):
            m = sww.Model(jmin, jmax, patch=4, eps=eps, share=base, precision="fp32", persistent=persistent)
            m.set_state(*_fields(m, seed))
            m.adapt()
            group.append(m)
    sww.step_ensemble(ens, 120.0, 3, True)
    for m in alone:
        m.step(120.0, 3, True)
    for a, b in zip(ens, alone):
        fa, sa = _snapshot(sww, a)
        fb, sb = _snapshot(sww, b)
        assert sa == sb
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k


def test_shared_grid_matches_own_grid_to_rounding():
    """jmax=3 member on a jmax=4 grid against a jmax=3 grid of its own."""
    import paper_1404_0405_gb300 as sww
    base = sww.Model(2, 4, patch=4)
    a = sww.Model(2, 3, patch=4, eps=3e-3, share=base)
    b = sww.Model(2, 3, patch=4, eps=3e-3)
    for m in (a, b):
        dh, u = _fields(m, 1)
        m.set_state(dh, u)
        m.adapt()
        m.step(-1.0, 3, True)
    for j in (2, 3):
        assert np.array_equal(a.get(j, sww.NODE_FLAGS) & 7, b.get(j, sww.NODE_FLAGS) & 7)
        for q in (sww.DH, sww.U):
            x, y = a.get(j, q), b.get(j, q)
            live = (a.get(j, sww.NODE_FLAGS if q == sww.DH else sww.EDGE_FLAGS) & 1) > 0
            assert np.abs(x[live] - y[live]).max() <= 1e-12 * np.abs(y[live]).max()


def test_shared_grid_rules():
    import paper_1404_0405_gb300 as sww
    base = sww.Model(2, 3, patch=4)
    with pytest.raises(sww.SwwError):
        sww.Model(2, 4, patch=4, share=base)          # more levels than the shared grid
    with pytest.raises(sww.SwwError):
        sww.Model(2, 3, patch=2, share=base)          # another patch layout
    m = sww.Model(2, 2, patch=4, share=base)
    assert m.sizes(2) == base.sizes(2)
    del base                                          # the tables outlive the first handle
    xyz, _ = m.grid(2)
    assert np.allclose(np.linalg.norm(xyz, axis=1), 1.0)


def test_autotuner_picks_the_fastest_trial(tmp_path, monkeypatch):
    import paper_1404_0405_gb300 as sww
    from paper_1404_0405_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))

    def fields_of(xyz, en):
        mid, tan = lib_edge_geometry(xyz, en)
        return [workloads.Workload("jet", seed=s).fields(xyz, mid, tan) for s in (1, 2)]

    best, trials = autotune.tune(2, 4, 1e-2, fields_of, members=2, patches=(4, 8), blocks=(2, 4), steps=2,
                                 warmup=1, key_extra="test")
    assert len(trials) == 4
    assert best == max(trials, key=lambda t: t["rate"])
    assert all(t["rate"] > 0 for t in trials)
    again, _ = autotune.tune(2, 4, 1e-2, fields_of, members=2, patches=(4, 8), blocks=(2, 4), key_extra="test")
    assert again == best                              # cached


@pytest.mark.parametrize("adapt", [True, False])
def test_phased_members_with_proposal_match_single_runs(adapt):
    """The batched step with each member's learned proposal on (random perceptron
    weights, so that patches get proposed), and without adaptation: bit for bit
    the members stepped alone."""
    import paper_1404_0405_gb300 as sww
    rng = np.random.default_rng(5)
    params = rng.normal(0.0, 0.5, sww.MLP_PARAMS).astype(np.float32)
    jmin, top = 2, max(j for j, _, _ in MEMBERS)
    base = sww.Model(jmin, top, patch=4)
    ens, alone = [], []
    for jmax, eps, seed in MEMBERS:
        for group in (ens, alone):
            m = sww.Model(jmin, jmax, patch=4, eps=eps, share=base, precision="fp32", persistent="phased")
            m.set_state(*_fields(m, seed))
            m.adapt()
            m.set_learned(2, params, 0.5)
            group.append(m)
    sww.step_ensemble(ens, -1.0, 3, adapt)
    for m in alone:
        m.step(-1.0, 3, adapt)
    for a, b in zip(ens, alone):
        fa, sa = _snapshot(sww, a)
        fb, sb = _snapshot(sww, b)
        assert sa == sb
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        assert a.learn_stats() == b.learn_stats()


@pytest.mark.parametrize("persistent", ["auto", "phased"])
def test_live_node_count_follows_the_mask(persistent):
    """sww_live_nodes (the count the last set_state, adapt or step brought back)
    equals the live nodes counted from the flags by sww_stats_get, after every
    call that changes the mask, for single and ensemble steps."""
    import paper_1404_0405_gb300 as sww
    jmin, top = 2, max(j for j, _, _ in MEMBERS)
    base = sww.Model(jmin, top, patch=4)
    ms = []
    for jmax, eps, seed in MEMBERS:
        m = sww.Model(jmin, jmax, patch=4, eps=eps, share=base, precision="fp32", persistent=persistent)
        assert m.live_nodes() == 0
        m.set_state(*_fields(m, seed))
        ms.append(m)

    def check(where):
        for i, m in enumerate(ms):
            want = sum(m.stats()["live_nodes"].values())
            assert want > 0
            assert m.live_nodes() == want, f"{where}, member {i}"

    check("set_state")
    for m in ms:
        m.adapt()
    check("adapt")
    ms[0].step(-1.0, 2, True)
    ms[1].step(-1.0, 1, False)
    check("single steps")
    sww.step_ensemble(ms, -1.0, 3, True)
    check("ensemble steps")
    sww.step_ensemble(ms, 120.0, 1, False)
    check("ensemble step without adaptation")
