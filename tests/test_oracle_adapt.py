"""Pins for the oracle's adapted grid and adaptive step (Sec. 2.3, Sec. 3.1).

* the mask equals a literal set construction written with Python sets and
  loops (one rule at a time, as the rules are stated), and so does the
  significance step;
* the ghost band equals breadth-first distances, and the ghost values equal
  the inverse transform of the full levels with zero coefficients away from
  live points;
* the thresholds read live points only; Delta t equals a brute-force CFL
  minimum over every live point;
* mass is conserved to roundoff over adaptive steps (Sec. 4.1, Eq. divRcommute);
* trends at covered coarse nodes are the restriction of the fine trends;
* the adapted solution tracks the uniform fine solution with an error that
  shrinks with eps (error control, Sec. 6.2).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import adapt, grid, model, transform


def brute_mask(Hy, sig_sets):
    """Rules of Sec. 2.3 / 3.1 applied literally with sets of node ids."""
    jmin, jmax = Hy.jmin, Hy.jmax
    nbrs = {j: [set(int(x) for x in Hy.levels[j].nbr_nodes[i] if x >= 0) for i in range(Hy.levels[j].N)]
            for j in range(jmin, jmax + 1)}
    T = {j: set() for j in range(jmin, jmax + 1)}
    for j in range(jmin + 1, jmax + 1):
        for x in sig_sets[j]:
            T[j].add(x)
            T[j] |= nbrs[j][x]                                 # adjacent in space
            if j + 1 <= jmax:
                T[j + 1].add(x)                                # adjacent in scale: same place
                T[j + 1] |= nbrs[j + 1][x]                     # and its fine neighbours
    for j in range(jmax, jmin, -1):
        n0 = Hy.levels[j - 1].N
        for x in list(T[j]):
            if x >= n0:
                T[j] |= set(int(k) for k in Hy.K[j][x - n0])    # prediction parents
        if j - 1 > jmin:
            for x in T[j]:
                if x < n0:
                    T[j - 1].add(x)                            # coarse node of a live even node
    return T


def test_mask_matches_literal_rules():
    Hy = grid.Hierarchy(2, 4)
    rng = np.random.default_rng(0)
    sig = {}
    sig_sets = {}
    for j in range(3, 5):
        N = Hy.levels[j].N
        s = rng.random(N) < 0.02
        sig[j] = s
        sig_sets[j] = set(np.nonzero(s)[0].tolist())
    live_n, live_e = adapt.build_mask(Hy, sig)
    T = brute_mask(Hy, sig_sets)
    for j in range(3, 5):
        assert set(np.nonzero(live_n[j])[0].tolist()) == T[j]
        L = Hy.levels[j]
        for e in range(L.E):
            a, b = L.edges[e]
            assert live_e[j][e] == (a in T[j] or b in T[j])
    assert live_n[2].all()


def test_ghost_band_is_bfs_distance():
    Hy = grid.Hierarchy(2, 4)
    rng = np.random.default_rng(1)
    live = {2: np.ones(Hy.levels[2].N, bool)}
    live_e = {}
    for j in (3, 4):
        live[j] = rng.random(Hy.levels[j].N) < 0.01
    for j in (2, 3, 4):
        live_e[j] = adapt.edges_touching(Hy.levels[j], live[j])
    gn, ge = adapt.ghost_band(Hy, live, live_e)
    L = Hy.levels[4]
    dist = np.full(L.N, 99)
    frontier = list(np.nonzero(live[4])[0])
    dist[frontier] = 0
    d = 0
    while frontier and d < adapt.GHOST_HOPS:
        d += 1
        nxt = []
        for x in frontier:
            for y in L.nbr_nodes[x]:
                if y >= 0 and dist[y] > d:
                    dist[y] = d
                    nxt.append(y)
        frontier = nxt
    assert np.array_equal(gn[4], (dist >= 1) & (dist <= adapt.GHOST_HOPS))


def make_model(jmin=2, jmax=4, kind="jet", eps=1e-2, seed=0, rk="rk4", nu=0.0):
    Hy = grid.Hierarchy(jmin, jmax)
    M = model.Model(Hy, eps=eps, rk=rk, nu=nu)
    W = workloads.Workload(kind, seed=seed)
    L = Hy.levels[jmax]
    dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    M.set_uniform(dh, u)
    M.adapt()
    return M


@pytest.mark.parametrize("rk,nu", [("rk4", 0.0), ("ssp43", 0.0), ("rk4", 2e5)])
def test_adaptive_mass_conserved(rk, nu):
    """With nu > 0 the diffusive height flux goes through the conservative flux
    restriction with the mass flux, so the viscous form conserves mass too."""
    M = make_model(rk=rk, nu=nu)
    assert 0 < M.active_nodes() < sum(M.Hy.levels[j].N for j in M.levels)
    m0 = M.mass()
    dt = M.dt_cfl()
    for _ in range(8):
        M.step(dt)
    assert abs(M.mass() / m0 - 1) < 1e-15


def test_covered_trends_are_restrictions():
    M = make_model()
    dht, _ = M.rhs(M._copy(M.dh), M._copy(M.u))
    Hy = M.Hy
    checked = 0
    for j in range(M.jmin, M.jmax):
        cov = M.covered(j)
        odd = Hy.odd[j + 1]
        fine = np.nan_to_num(dht[j + 1])
        d = np.where(M.live_n[j + 1][odd], transform.height_detail(Hy, j + 1, fine), 0.0)
        full = np.zeros(Hy.levels[j + 1].N)
        full[: Hy.levels[j].N] = np.where(cov, fine[: Hy.levels[j].N], 0.0)
        hc = transform.height_update(Hy, j + 1, full, d)
        if cov.any():
            assert np.abs(hc[cov] - dht[j][cov]).max() < 1e-12 * np.abs(dht[j][cov]).max()
            checked += 1
    assert checked >= 1


def test_velocity_stays_consistent_across_levels():
    """On coarse edges whose two ends are covered, u^j = R_u(u^{j+1}) after steps."""
    M = make_model()
    dt = M.dt_cfl()
    for _ in range(3):
        M.step(dt, adapt_after=False)
    Hy = M.Hy
    for j in range(M.jmin, M.jmax):
        cov = M.covered(j)
        C = Hy.levels[j]
        e = cov[C.edges[:, 0]] & cov[C.edges[:, 1]]
        if e.any():
            r = transform.restrict_velocity(Hy, j + 1, M.u[j + 1])
            assert np.abs(r[e] - M.u[j][e]).max() < 1e-12 * np.nanmax(np.abs(M.u[j]))


def test_uniform_field_is_reproduced_exactly():
    """A constant depth perturbation has zero coefficients everywhere: thresholding
    keeps only Jmin, and prolongation onto any mask reproduces the constant."""
    Hy = grid.Hierarchy(2, 4)
    M = model.Model(Hy)
    L = Hy.levels[4]
    M.set_uniform(np.full(L.N, 5.0), np.zeros(L.E))
    M.adapt(eps_h=1e-9, eps_u=1e-9)
    assert M.live_n[3].sum() == 0 and M.live_n[4].sum() == 0
    rng = np.random.default_rng(7)
    sig = {j: rng.random(Hy.levels[j].N) < 0.01 for j in (3, 4)}
    live_n, live_e = adapt.build_mask(Hy, sig)
    zeros = {j: np.zeros(Hy.odd[j].size) for j in (3, 4)}
    ue = {j: np.zeros(Hy.levels[j - 1].E) for j in (3, 4)}
    ui = {j: np.zeros((Hy.levels[j - 1].T, 3)) for j in (3, 4)}
    M.apply_mask(live_n, live_e, zeros, ue, ui)
    assert M.live_n[4].sum() > 0 and M.ghost_n[4].sum() > 0
    for j in M.levels:
        v = M.dh[j][~np.isnan(M.dh[j])]
        assert v.size > 0 and np.abs(v - 5.0).max() < 1e-12
        w = M.u[j][~np.isnan(M.u[j])]
        assert np.abs(w).max() == 0.0


def test_dt_is_cfl_minimum():
    """Delta t = CFL min(1/omega_max, min dx/|u|) over the live points (Sec. 3.1,
    reading 2: omega = sqrt(f^2 + g h (pi/dx)^2), f = 2 Omega sin(latitude), dx the
    level's Table 1 spacing), by brute force over every live node and edge."""
    M = make_model()
    M.step(200.0)
    best = math.inf
    for j in M.levels:
        L = M.Hy.levels[j]
        dx = grid.nominal_spacing(j, L.radius)
        for i in np.nonzero(M.live_n[j])[0]:
            x, y, z = (float(v) for v in L.xyz[i])
            f = 2.0 * M.Hy.omega * z / math.sqrt(x * x + y * y + z * z)
            w = math.sqrt(f * f + M.g * (M.H + float(M.dh[j][i])) * (math.pi / dx) ** 2)
            best = min(best, 1.0 / w)
        for e in np.nonzero(M.live_e[j])[0]:
            a = abs(float(M.u[j][e]))
            if a > 0:
                best = min(best, dx / a)
    assert abs(M.dt_cfl() - M.cfl * best) <= 1e-14 * M.cfl * best


def test_error_controlled_by_eps():
    """Against the uniform Jmax solution, the adapted solution's error drops as
    eps drops (Sec. 6.2, Fig. 10 right)."""
    jmin, jmax = 2, 4
    Hy = grid.Hierarchy(jmin, jmax)
    W = workloads.Workload("jet", seed=0)
    L = Hy.levels[jmax]
    dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    ref = model.Model(grid.Hierarchy(jmax, jmax))
    ref.set_uniform(dh, u)
    dt = 300.0
    nsteps = 6
    for _ in range(nsteps):
        ref.step(dt)
    errs = []
    for eps in (3e-2, 1e-2, 3e-3):
        M = model.Model(Hy, eps=eps)
        M.set_uniform(dh, u)
        M.adapt()
        for _ in range(nsteps):
            M.step(dt)
        # compare on Jmin, where both solutions are complete
        jm = M.jmin
        r = ref.dh[jmax]
        for j in range(jmax, jm, -1):
            r = transform.restrict_height(Hy, j, r)
        errs.append(np.abs(M.dh[jm] - r).max())
    assert errs[2] < errs[0]


def test_uniform_reconstruction_exact_on_full_grid():
    """With every point live, the full level is the stored level itself: the
    input, to the rounding of the inverse transform that adaptation applies."""
    Hy = grid.Hierarchy(2, 4)
    M = model.Model(Hy, eps=0.0)
    L = Hy.levels[4]
    dh, u = workloads.Workload("jet", seed=4).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    M.set_uniform(dh, u)
    M.adapt()
    h4, u4 = M.get_uniform(4)
    assert np.array_equal(h4, M.dh[4]) and np.array_equal(u4, M.u[4])
    assert np.abs(h4 - dh).max() < 1e-12 * np.abs(dh).max() and np.abs(u4 - u).max() < 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("kind,seed", [("jet", 0), ("harmonic", 3)])
def test_uniform_reconstruction_error_bounded_by_threshold(kind, seed):
    """Dropping coefficients below eps (Sec. 2.3) perturbs the reconstructed
    field by a small multiple of the thresholds (measured at most 0.61 eps_h and
    0.41 eps_u on J2..5); a constant depth is reproduced exactly."""
    Hy = grid.Hierarchy(2, 5)
    L = Hy.levels[5]
    W = workloads.Workload(kind, seed=seed)
    dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    for eps in (3e-2, 1e-2):
        M = model.Model(Hy, eps=eps)
        M.set_uniform(dh, u)
        M.adapt()
        h5, u5 = M.get_uniform(5)
        assert np.abs(h5 - dh).max() <= 1.0 * M.eps_h
        assert np.abs(u5 - u).max() <= 1.0 * M.eps_u
    M = model.Model(Hy, eps=1e-2)
    M.set_uniform(np.full(L.N, 7.0), np.zeros(L.E))
    M.adapt(eps_h=1e-9, eps_u=1e-9)
    h5, u5 = M.get_uniform(5)
    assert M.live_n[5].sum() == 0
    assert np.abs(h5 - 7.0).max() < 1e-12 and np.abs(u5).max() == 0.0


def test_significance_matches_literal_rules():
    """Step 1 of the mask (Sec. 2.3, reading 1) by loops over the points: an odd
    node with a significant height coefficient; both ends and the midpoint of a
    coarse edge with a significant velocity coefficient; both ends of an interior
    fine edge with a significant one; only live points carry coefficients."""
    M = make_model(2, 4)
    Hy = M.Hy
    rng = np.random.default_rng(3)
    for j in (3, 4):
        C, F = Hy.levels[j - 1], Hy.levels[j]
        VS = M.VS[j]
        odd = Hy.odd[j]
        hdet = np.where(M.live_n[j][odd], rng.standard_normal(odd.size), np.nan)
        any_half = M.live_e[j][VS.half[:, 0]] | M.live_e[j][VS.half[:, 1]]
        ue = np.where(any_half, rng.standard_normal(C.E), np.nan)
        ui = np.where(M.live_e[j][VS.int_edge], rng.standard_normal(VS.int_edge.shape), np.nan)
        eps_h, eps_u = 1.2, 1.5
        S = adapt.significance(Hy, j, M.live_n[j], M.live_e[j], hdet, ue, ui, VS, eps_h, eps_u)
        want = set()
        for r, m in enumerate(odd):
            if M.live_n[j][m] and abs(hdet[r]) >= eps_h:
                want.add(int(m))
        for E in range(C.E):
            if not np.isnan(ue[E]) and abs(ue[E]) >= eps_u:
                want |= {int(C.edges[E, 0]), int(C.edges[E, 1]), int(Hy.mid[j - 1][E])}
        for t in range(C.T):
            for c in range(3):
                fe = VS.int_edge[t, c]
                if M.live_e[j][fe] and abs(ui[t, c]) >= eps_u:
                    want |= {int(F.edges[fe, 0]), int(F.edges[fe, 1])}
        assert set(np.nonzero(S)[0].tolist()) == want


def test_ghost_values_are_the_zero_detail_inverse():
    """Ghost values (reading, step 5) are the inverse transform (Eqs. 1-2) of the
    full levels with every coefficient away from live points set to zero: build
    the full levels from Jmin up with the transforms alone, then compare the live
    and ghost values of every level after an adaptive step."""
    M = make_model(2, 5)
    M.step(200.0)
    Hy = M.Hy
    hfull, ufull = M.dh[2].copy(), M.u[2].copy()
    for j in range(3, 6):
        C, F = Hy.levels[j - 1], Hy.levels[j]
        VS = M.VS[j]
        odd = Hy.odd[j]
        with np.errstate(invalid="ignore"):
            d = transform.height_detail(Hy, j, M.dh[j])
            de, di = transform.velocity_detail(VS, ufull, M.u[j])
        d = np.where(M.live_n[j][odd], d, 0.0)
        any_half = M.live_e[j][VS.half[:, 0]] | M.live_e[j][VS.half[:, 1]]
        de = np.where(any_half, de, 0.0)
        di = np.where(M.live_e[j][VS.int_edge], di, 0.0)
        assert np.isfinite(d).all() and np.isfinite(de).all() and np.isfinite(di).all()
        hfull = transform.inverse_height(Hy, j, hfull, d)
        ufull = transform.inverse_velocity(VS, ufull, de, di, F.E)
        for name, full, got, live, ghost in (("dh", hfull, M.dh[j], M.live_n[j], M.ghost_n[j]),
                                             ("u", ufull, M.u[j], M.live_e[j], M.ghost_e[j])):
            scale = np.abs(full).max()
            assert ghost.sum() > 0
            assert np.abs(got[live] - full[live]).max() <= 1e-12 * scale, (name, j, "live")
            assert np.abs(got[ghost] - full[ghost]).max() <= 1e-12 * scale, (name, j, "ghost")


def test_thresholds_read_live_points_only():
    """eps_h = eps max|dh| and eps_u = eps max|u| over the live points (reading 11):
    a large ghost value leaves them alone, a large live value sets them; with eps
    read as the trend tolerance (regime 1) both scale by eps^{3/2}, i.e. by
    sqrt(eps) against regime 0 (reading 22)."""
    M = make_model(2, 4)
    th = M.thresholds()
    j = 4
    gn, ge = np.nonzero(M.ghost_n[j])[0], np.nonzero(M.ghost_e[j])[0]
    assert gn.size and ge.size
    M.dh[j][gn[0]], M.u[j][ge[0]] = 1e9, 1e9
    assert M.thresholds() == th
    M.regime = 1
    r = M.thresholds()
    assert math.isclose(r[0], th[0] * math.sqrt(M.eps), rel_tol=1e-14)
    assert math.isclose(r[1], th[1] * math.sqrt(M.eps), rel_tol=1e-14)
    M.regime = 0
    ln, le = np.nonzero(M.live_n[j])[0], np.nonzero(M.live_e[j])[0]
    M.dh[j][ln[0]], M.u[j][le[0]] = -1e9, 1e9
    assert M.thresholds() == (M.eps * 1e9, M.eps * 1e9)
