"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the
same seeded inputs, element by element after mapping the two grid orders.

Bar: integer flags, masks and patch lists bit-exact; FP64 fields within 1e-12
of the field's maximum per step (the oracle and the library build their
geometry independently; those differ by ~1e-14 relative at these levels, and
each RK step adds rounding of the same order)."""
import math

import numpy as np
import pytest

import workloads
from lib_mapping import LevelMap, lib_edge_geometry
from oracle import grid, model

pytestmark = pytest.mark.gpu

TOL = 1e-12
# Trends are differences of fluxes ~1e4 times larger than the result (div F, grad B
# against q F^perp in geostrophic balance), so two independent FP64 geometries
# agree on them to ~1e-12 relative to the terms, not to the trend itself; the
# fields, which change by dt * trend per step, keep the 1e-12 bar.
TREND_TOL = 1e-10


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


class Pair:
    """An oracle model and a library model on the same grid and initial state."""

    def __init__(self, jmin, jmax, kind="jet", seed=0, eps=1e-2, rk="rk4", patch=4, precision="fp64", nu=0.0,
                 advect=False, alpha=0.0, persistent=True, regime=0, share=None):
        import paper_1404_0405_gb300 as sww
        self.sww = sww
        self.Hy = grid.Hierarchy(jmin, jmax)
        H = 0.0 if advect else 1.0e4       # the advection test carries the bell itself
        self.ora = model.Model(self.Hy, H=H, eps=eps, rk=rk, nu=nu, advect=advect, regime=regime)
        self.lib = sww.Model(jmin, jmax, H=H, patch=patch, eps=eps, rk=rk, precision=precision, nu=nu,
                             advect=advect, persistent=persistent, regime=regime, share=share)
        self.maps = {}
        for j in range(jmin, jmax + 1):
            xyz, en = self.lib.grid(j)
            self.maps[j] = LevelMap(xyz, en, self.Hy.levels[j])
        L = self.Hy.levels[jmax]
        W = workloads.Workload(kind, seed=seed, alpha=alpha)
        dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
        self.ora.set_uniform(dh, u)
        M = self.maps[jmax]
        self.lib.set_state(M.nodes_to_lib(dh), M.edges_to_lib(u))
        self.jmin, self.jmax = jmin, jmax

    def flags(self, j):
        M = self.maps[j]
        nf = M.nodes_to_ora(self.lib.get(j, self.sww.NODE_FLAGS))
        ef = self.lib.get(j, self.sww.EDGE_FLAGS)[M.inv_edge]
        return nf, ef

    def check_masks(self):
        for j in range(self.jmin, self.jmax + 1):
            nf, ef = self.flags(j)
            assert np.array_equal((nf & 1) > 0, self.ora.live_n[j]), f"live nodes differ at level {j}"
            assert np.array_equal((nf & 2) > 0, self.ora.ghost_n[j]), f"ghost nodes differ at level {j}"
            assert np.array_equal((ef & 1) > 0, self.ora.live_e[j]), f"live edges differ at level {j}"
            assert np.array_equal((ef & 2) > 0, self.ora.ghost_e[j]), f"ghost edges differ at level {j}"
            if j < self.jmax:
                assert np.array_equal((nf & 4) > 0, self.ora.covered(j)), f"covered nodes differ at level {j}"

    def check_fields(self, tol=None, which="state"):
        tol = tol if tol is not None else (TOL if which == "state" else TREND_TOL)
        for j in range(self.jmin, self.jmax + 1):
            M = self.maps[j]
            if which == "state":
                a = M.nodes_to_ora(self.lib.get(j, self.sww.DH))
                b = M.edges_to_ora(self.lib.get(j, self.sww.U))
                ra, rb = self.ora.dh[j], self.ora.u[j]
                mn = self.ora.live_n[j] | self.ora.ghost_n[j]
                me = self.ora.live_e[j] | self.ora.ghost_e[j]
            else:
                a = M.nodes_to_ora(self.lib.get(j, self.sww.DH_T))
                b = M.edges_to_ora(self.lib.get(j, self.sww.U_T))
                ra, rb = self.trend
                ra, rb = ra[j], rb[j]
                mn, me = self.ora.live_n[j], self.ora.live_e[j]
            if mn.any():
                assert rel_err(a[mn], ra[mn]) < tol, f"{which} dh level {j}: {rel_err(a[mn], ra[mn]):.3e}"
            if me.any():
                assert rel_err(b[me], rb[me]) < tol, f"{which} u level {j}: {rel_err(b[me], rb[me]):.3e}"

    def adapt(self):
        self.ora.adapt()
        self.lib.adapt()

    def rhs(self):
        self.trend = self.ora.rhs(self.ora._copy(self.ora.dh), self.ora._copy(self.ora.u))
        self.lib.rhs()


@pytest.fixture(scope="module")
def built():
    import paper_1404_0405_gb300 as sww
    sww.build()
    return sww


def test_library_exports(built):
    lib = built.load()
    for name in built.EXPORTS:
        assert hasattr(lib, name)


def test_initial_restriction_matches(built):
    P = Pair(2, 4)
    P.check_fields()
    P.check_masks()


def test_trend_full_grid_matches(built):
    """Trend on the full (every point live) hierarchy: TRiSK on every level with
    restricted B, F and q F^perp (Sec. 3.1)."""
    P = Pair(2, 4)
    P.rhs()
    P.check_fields(which="trend")


def test_uniform_level_step_matches(built):
    """Plain method on one uniform level (no transforms): RK4 steps."""
    P = Pair(3, 3, kind="harmonic", seed=1)
    for _ in range(3):
        P.ora.step(200.0, adapt_after=False)
        P.lib.step(200.0, 1, adapt=False)
        P.check_fields()


@pytest.mark.parametrize("kind,seed", [("jet", 0), ("harmonic", 3)])
def test_adapt_masks_bit_exact(built, kind, seed):
    P = Pair(2, 4, kind=kind, seed=seed)
    P.adapt()
    # thresholds agree to rounding and no coefficient sits within 1e-10 of one
    st = P.lib.stats()
    assert abs(st["eps_h"] / P.ora.eps_h - 1) < 1e-12 and abs(st["eps_u"] / P.ora.eps_u - 1) < 1e-12
    P.check_masks()
    P.check_fields()
    # the jet grid is genuinely adapted (the global harmonic field keeps most points)
    if kind == "jet":
        live = sum(P.ora.live_n[j].sum() for j in P.ora.levels)
        assert live < sum(P.Hy.levels[j].N for j in P.ora.levels)


def test_trend_tolerance_regime(built):
    """regime 1: thresholds from eps^{3/2} (eps = 0.05 gives about 0.0112 relative)."""
    P = Pair(2, 4, kind="jet", seed=2, eps=0.05, regime=1)
    P.adapt()
    st = P.lib.stats()
    assert abs(st["eps_h"] / P.ora.eps_h - 1) < 1e-12 and abs(st["eps_u"] / P.ora.eps_u - 1) < 1e-12
    assert abs(P.ora.eps_h / (0.05 * math.sqrt(0.05) * np.nanmax(np.abs(P.ora.dh[2]))) - 1) < 0.2
    P.check_masks()
    P.check_fields()


def test_mask_from_identical_coefficients(built):
    """Same coefficients and thresholds in, bit-identical mask out."""
    P = Pair(2, 4, kind="jet", seed=5)
    hdet, ue, ui = P.ora.details()
    rng = np.random.default_rng(11)
    lib_h, lib_e, lib_i = {}, {}, {}
    for j in range(3, 5):
        Mf, Mc = P.maps[j], P.maps[j - 1]
        VS = P.ora.VS[j]
        full_h = np.zeros(P.Hy.levels[j].N)
        full_h[P.Hy.odd[j]] = np.nan_to_num(hdet[j])
        lib_h[j] = Mf.nodes_to_lib(full_h)
        # the coarse-edge coefficient ((u_h0 - P_h0) - (u_h1 - P_h1))/2 is unchanged when the
        # edge is reversed (halves swap and velocities change sign), so it maps without sign
        lib_e[j] = np.nan_to_num(ue[j])[Mc.edge]
        full_i = np.zeros(P.Hy.levels[j].E)
        full_i[VS.int_edge.ravel()] = np.nan_to_num(ui[j]).ravel()
        lib_i[j] = Mf.edges_to_lib(full_i)
    eh, eu = 4.0, 0.3
    sig = P.ora.significance(hdet, ue, ui, eh, eu)
    from oracle import adapt
    live_n, live_e = adapt.build_mask(P.Hy, sig)
    P.ora.apply_mask(live_n, live_e, hdet, ue, ui)
    P.lib.mask_from_coeffs(lib_h, lib_e, lib_i, eh, eu)
    for j in range(3, 5):
        s = P.maps[j].nodes_to_ora(P.lib.get(j, P.sww.SIG))
        assert np.array_equal(s > 0, sig[j])
    P.check_masks()
    P.check_fields()


def test_adaptive_trend_matches(built):
    P = Pair(2, 4)
    P.adapt()
    P.rhs()
    P.check_fields(which="trend")


@pytest.mark.parametrize("rk", ["rk4", "ssp43"])
def test_adaptive_steps_match(built, rk):
    P = Pair(2, 4, rk=rk)
    P.adapt()
    m0 = P.lib.stats()["mass"]
    for _ in range(3):
        dt_o = P.ora.dt_cfl()
        P.ora.step(dt_o)
        P.lib.step(-1.0, 1, adapt=True)
        st = P.lib.stats()
        assert abs(st["dt"] / dt_o - 1) < 1e-12
        P.check_masks()
        P.check_fields()
    assert abs(P.lib.stats()["mass"] / m0 - 1) < 1e-14


def test_patch_lists(built):
    P = Pair(2, 4, patch=4)
    P.adapt()
    for j in range(2, 5):
        nf = P.lib.get(j, P.sww.NODE_FLAGS)
        ef = P.lib.get(j, P.sww.EDGE_FLAGS)
        N, E, T, npatch = P.lib.sizes(j)
        nelem = E // 3
        pp = nelem // npatch
        act = ((nf[:nelem] | ef[:nelem] | ef[nelem:2 * nelem] | ef[2 * nelem:]) & 3) > 0
        expect = np.nonzero(act.reshape(npatch, pp).any(axis=1))[0]
        assert np.array_equal(P.lib.patches(j), expect)


def test_diagnostics_match(built):
    P = Pair(2, 4)
    P.adapt()
    st = P.lib.stats()
    assert abs(st["mass"] / P.ora.mass() - 1) < 1e-14
    assert abs(st["energy"] / P.ora.energy() - 1) < 1e-9
    for j in P.ora.levels:
        assert st["live_nodes"][j] == P.ora.live_n[j].sum()
        assert st["ghost_nodes"][j] == P.ora.ghost_n[j].sum()


# ----------------------------------------------------------------------------- viscous form (Sec. 3.1)

NU = 2e5   # m^2/s: the diffusion number nu dt / dx^2 stays below 0.05 on these grids


def test_viscous_trend_matches(built):
    P = Pair(2, 4, nu=NU)
    P.rhs()
    P.check_fields(which="trend")
    P2 = Pair(2, 4, nu=NU)
    P2.adapt()
    P2.rhs()
    P2.check_fields(which="trend")


def test_viscous_adaptive_steps_match(built):
    P = Pair(2, 4, nu=NU)
    P.adapt()
    m0 = P.lib.stats()["mass"]
    for _ in range(3):
        dt = P.ora.dt_cfl()
        P.ora.step(dt)
        P.lib.step(dt, 1, adapt=True)
        P.check_masks()
        P.check_fields()
    assert abs(P.lib.stats()["mass"] / m0 - 1) < 1e-14


# ----------------------------------------------------------------------------- prescribed velocity (Sec. 7.1)


@pytest.mark.parametrize("persistent", [True, False])
def test_advect_trend_matches(built, persistent):
    """Advection of the cosine bell by the tilted rotation: depth trend through the
    flux restriction, zero velocity trend on both sides."""
    P = Pair(2, 4, kind="tc1_cosine", eps=0.02, advect=True, alpha=math.pi / 4, persistent=persistent)
    P.adapt()
    assert P.lib.stats()["eps_u"] == math.inf and P.ora.eps_u == math.inf
    P.check_masks()
    P.rhs()
    P.check_fields(which="trend")
    for j in range(2, 5):
        assert np.all(P.maps[j].edges_to_ora(P.lib.get(j, P.sww.U_T))[P.ora.live_e[j]] == 0.0)


@pytest.mark.parametrize("kind,rk", [("tc1_cosine", "rk4"), ("tc1_smooth", "ssp43")])
def test_advect_adaptive_steps_match(built, kind, rk):
    P = Pair(2, 4, kind=kind, rk=rk, eps=0.02, advect=True, alpha=math.pi / 4)
    P.adapt()
    u_set = {j: P.lib.get(j, P.sww.U).copy() for j in range(2, 5)}
    m0 = P.lib.stats()["mass"]
    for _ in range(4):
        dt_o = P.ora.dt_cfl()
        P.ora.step(dt_o)
        P.lib.step(-1.0, 1, adapt=True)
        assert abs(P.lib.stats()["dt"] / dt_o - 1) < 1e-12
        P.check_masks()
        P.check_fields()
    for j in range(2, 5):
        assert np.array_equal(P.lib.get(j, P.sww.U), u_set[j])   # never written
    assert abs(P.lib.stats()["mass"] / m0 - 1) < 1e-14


# ----------------------------------------------------------------------------- state on a coarser level


def test_state_set_on_a_coarser_level_matches(built):
    """Fields given on level 3 of 2..5: levels above start empty and adaptation
    refines into them (one level per adaptation by the adjacent-in-scale rule)."""
    import paper_1404_0405_gb300 as sww
    Hy = grid.Hierarchy(2, 5)
    ora = model.Model(Hy, eps=1e-2)
    lib = sww.Model(2, 5, patch=4, eps=1e-2)
    maps = {j: LevelMap(*lib.grid(j), Hy.levels[j]) for j in range(2, 6)}
    L = Hy.levels[3]
    dh, u = workloads.Workload("jet", seed=0).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    ora.set_uniform(dh, u, level=3)
    lib.set_state(maps[3].nodes_to_lib(dh), maps[3].edges_to_lib(u), level=3)
    assert lib.stats()["live_nodes"][4] == 0 and lib.stats()["live_nodes"][5] == 0
    ora.adapt()
    lib.adapt()
    for _ in range(3):
        dt = ora.dt_cfl()
        ora.step(dt)
        lib.step(-1.0, 1, True)
        assert abs(lib.stats()["dt"] / dt - 1) < 1e-12
    assert ora.live_n[5].sum() > 0
    for j in range(2, 6):
        M = maps[j]
        nf = M.nodes_to_ora(lib.get(j, sww.NODE_FLAGS))
        assert np.array_equal((nf & 1) > 0, ora.live_n[j]) and np.array_equal((nf & 2) > 0, ora.ghost_n[j])
        mn = ora.live_n[j] | ora.ghost_n[j]
        if mn.any():
            assert rel_err(M.nodes_to_ora(lib.get(j, sww.DH))[mn], ora.dh[j][mn]) < TOL
        me = ora.live_e[j] | ora.ghost_e[j]
        if me.any():
            assert rel_err(M.edges_to_ora(lib.get(j, sww.U))[me], ora.u[j][me]) < TOL
