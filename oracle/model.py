"""Oracle: the adaptive time step (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

One trend evaluation (Sec. 3.1): q and K everywhere; B, F and q F^perp on every
level; then, from Jmax-1 down to Jmin, B, F and q F^perp are replaced at coarse
points covered by live fine points by their restrictions of the finer level
(B by injection, q F^perp by R_u, F by R_F); finally div and grad on every level
give the trends of all live points.  After the last RK stage the partial height
transform R_h refreshes the covered coarse heights, then the grid is adapted.

Readings: a coarse node k is covered when its whole restriction stencil is live
one level up (the fine node at the same place and the 2N odd nodes M_k); then
every odd node that R_F on a face of k reads lies in M_k, and
sum_faces R_F = A_k R_h(div F) holds exactly.  Covered nodes get B by injection
and R_h in the partial transform; a coarse edge gets its flux by R_F when an end
node is covered (commutation at a covered node needs all of its faces) and its
q F^perp by R_u when both end nodes are covered.  Live fine points of a coarse
region that is not covered evolve on both levels; adaptation rebuilds them from
the coarse values and their retained coefficients.  B restriction is injection (with R_u of the mean of
the two halves this makes R_u(grad B) = grad(R B) exactly).  Time scheme:
classical RK4 ("rk4") or the 4-stage 3rd-order SSP scheme of Spiteri & Ruuth
("ssp43", Sec. 3.1).  dt = cfl * min(1/omega_max, min dx/|u|) with
omega = sqrt(f^2 + g h (pi/dx)^2) (the printed omega is dimensionally
inconsistent; this reading restores pi/dx squared) and dx the Table 1 spacing of
each point's level.  Thresholds: eps_h = eps max|dh|, eps_u = eps max|u| over live
points (the printed formulas are dimensionally inconsistent; this relative
reading keeps their eps^{3/2} scaling as an option, ``regime=1``, which puts
eps^{3/2} in place of eps).  Diagnostics: mass = sum_{Jmin} A_k h_k (Jmin is always
full); energy of Sec. 7.2 evaluated on Jmin with the TRiSK kinetic energy.

Prescribed-velocity mode (``advect=True``, the advection test case of Sec. 7.1):
the velocity is the field given to ``set_uniform`` and its restrictions R_u on
every coarser level, at every point of every level, for all time; only the
depth evolves, d h/dt = -div(h_e u_e) with the same flux restriction, partial
transform and adaptation.  Readings (the paper gives the test, not the mode's
details): the velocity takes no part in the significance test (eps_u infinite),
newly active edges take the prescribed value rather than a prediction, and
dt = cfl * min dx/|u| (no gravity waves to resolve).
"""
from __future__ import annotations

import math
import numpy as np

from . import adapt, grid, transform, trisk


class Model:
    def __init__(self, Hy, H=1.0e4, g=9.80616, eps=1e-2, rk="rk4", cfl=0.8, nu=0.0, advect=False, regime=0):
        self.Hy, self.H, self.g, self.eps, self.rk, self.cfl = Hy, H, g, eps, rk, cfl
        self.nu, self.advect, self.regime = nu, advect, regime
        self.jmin, self.jmax = Hy.jmin, Hy.jmax
        self.VS = {j: transform.VelocityStencils(Hy, j) for j in range(self.jmin + 1, self.jmax + 1)}
        self.FS = {j: transform.FluxStencils(Hy, j) for j in range(self.jmin + 1, self.jmax + 1)}
        self.levels = range(self.jmin, self.jmax + 1)
        self.dh, self.u = {}, {}
        self.eps_h = self.eps_u = None

    # ------------------------------------------------------------------ state
    def set_uniform(self, dh_f, u_f, level=None):
        """Fields on the full level Jmax (or `level`); every coarser level gets
        their restriction (R_h, R_u) and every point up to that level is live;
        the levels above it hold no point."""
        Hy = self.Hy
        J = self.jmax if level is None else level
        self.dh[J], self.u[J] = dh_f.astype(np.float64).copy(), u_f.astype(np.float64).copy()
        for j in range(J, self.jmin, -1):
            self.dh[j - 1] = transform.restrict_height(Hy, j, self.dh[j])
            self.u[j - 1] = transform.restrict_velocity(Hy, j, self.u[j])
        for j in range(J + 1, self.jmax + 1):
            self.dh[j] = np.full(Hy.levels[j].N, np.nan)
            self.u[j] = np.full(Hy.levels[j].E, np.nan)
        self.u_set = {j: self.u[j].copy() for j in self.levels}
        self.live_n = {j: np.full(Hy.levels[j].N, j <= J) for j in self.levels}
        self.live_e = {j: np.full(Hy.levels[j].E, j <= J) for j in self.levels}
        self.ghost_n = {j: np.zeros(Hy.levels[j].N, dtype=bool) for j in self.levels}
        self.ghost_e = {j: np.zeros(Hy.levels[j].E, dtype=bool) for j in self.levels}

    def _mask_values(self):
        """Put NaN at every point that is neither live nor ghost."""
        for j in self.levels:
            av_n = self.live_n[j] | self.ghost_n[j]
            av_e = self.live_e[j] | self.ghost_e[j]
            self.dh[j][~av_n] = np.nan
            self.u[j][~av_e] = np.nan
        self._prescribe(self.u)

    def _prescribe(self, u):
        """Prescribed-velocity mode: the set velocity at every live or ghost edge."""
        if not self.advect:
            return
        for j in self.levels:
            av_e = self.live_e[j] | self.ghost_e[j]
            u[j] = np.where(av_e, self.u_set[j], np.nan)

    def fill_ghosts(self, dh=None, u=None):
        dh = self.dh if dh is None else dh
        u = self.u if u is None else u
        for j in range(self.jmin + 1, self.jmax + 1):
            adapt.prolong_level(self.Hy, self.VS[j], j, dh, u, self.live_n[j], self.live_e[j],
                                self.ghost_n[j], self.ghost_e[j])
        self._prescribe(u)

    # ------------------------------------------------------------------ wavelet coefficients
    def details(self):
        """Wavelet coefficients at live points: hdet[j] over odd nodes, udet_e[j]
        over coarse edges, udet_i[j][T_{j-1},3] over interior fine edges (NaN
        where the point is not live)."""
        Hy = self.Hy
        hdet, ue, ui = {}, {}, {}
        for j in range(self.jmin + 1, self.jmax + 1):
            VS = self.VS[j]
            odd = Hy.odd[j]
            with np.errstate(invalid="ignore"):
                d = transform.height_detail(Hy, j, self.dh[j])
            hdet[j] = np.where(self.live_n[j][odd], d, np.nan)
            with np.errstate(invalid="ignore"):
                de, di = transform.velocity_detail(VS, self.u[j - 1], self.u[j])
            any_half = self.live_e[j][VS.half[:, 0]] | self.live_e[j][VS.half[:, 1]]
            ue[j] = np.where(any_half, de, np.nan)
            ui[j] = np.where(self.live_e[j][VS.int_edge], di, np.nan)
        return hdet, ue, ui

    def thresholds(self):
        # regime 1: eps is the trend tolerance of Sec. 2.3 and the coefficient
        # thresholds scale as eps^{3/2} (the factor both of the paper's regimes share)
        e = self.eps * math.sqrt(self.eps) if self.regime == 1 else self.eps
        # levels without live points contribute nothing
        mh = max(float(np.nanmax(np.abs(self.dh[j][self.live_n[j]]), initial=0.0)) for j in self.levels)
        if self.advect:
            return e * mh, math.inf
        mu = max(float(np.nanmax(np.abs(self.u[j][self.live_e[j]]), initial=0.0)) for j in self.levels)
        return e * mh, e * mu

    def significance(self, hdet, ue, ui, eps_h, eps_u):
        sig = {}
        for j in range(self.jmin + 1, self.jmax + 1):
            sig[j] = adapt.significance(self.Hy, j, self.live_n[j], self.live_e[j], hdet[j], ue[j], ui[j],
                                        self.VS[j], eps_h, eps_u)
        return sig

    def adapt(self, eps_h=None, eps_u=None, extra=None):
        """Coefficients -> thresholds -> mask -> inverse transform of the retained
        coefficients onto the new live set -> ghosts.  extra[j]: nodes of level j
        joining the set T before the closure (an external refinement proposal).

        Reading: the adapted field is the inverse wavelet transform of the
        coefficients kept (Sec. 2.3: dropping a coefficient sets it to zero), so the
        coarse scaling coefficients -- and with them the mass -- never change in
        adaptation; new points get zero coefficients (prolongation)."""
        hdet, ue, ui = self.details()
        if eps_h is None:
            eps_h, eps_u = self.thresholds()
        self.eps_h, self.eps_u = eps_h, eps_u
        sig = self.significance(hdet, ue, ui, eps_h, eps_u)
        live_n, live_e = adapt.build_mask(self.Hy, sig, extra)
        self.apply_mask(live_n, live_e, hdet, ue, ui)
        return hdet, ue, ui

    def apply_mask(self, live_n, live_e, hdet, ue, ui):
        Hy = self.Hy
        ghost_n, ghost_e = adapt.ghost_band(Hy, live_n, live_e)
        self.live_n, self.live_e, self.ghost_n, self.ghost_e = live_n, live_e, ghost_n, ghost_e
        for j in range(self.jmin + 1, self.jmax + 1):
            C, F = Hy.levels[j - 1], Hy.levels[j]
            VS = self.VS[j]
            odd = Hy.odd[j]
            hd = np.where(live_n[j][odd], np.nan_to_num(hdet[j], nan=0.0), 0.0)
            anyh = live_e[j][VS.half[:, 0]] | live_e[j][VS.half[:, 1]]
            de = np.where(anyh, np.nan_to_num(ue[j], nan=0.0), 0.0)
            di = np.where(live_e[j][VS.int_edge], np.nan_to_num(ui[j], nan=0.0), 0.0)
            with np.errstate(invalid="ignore"):
                hf = transform.inverse_height(Hy, j, self.dh[j - 1], hd)
                uf = transform.inverse_velocity(VS, self.u[j - 1], de, di, F.E)
            self.dh[j] = np.where(live_n[j], hf, np.nan)
            self.u[j] = np.where(live_e[j], uf, np.nan)
            # ghosts of this level before the next finer level reads them
            adapt.prolong_level(Hy, VS, j, self.dh, self.u, live_n[j], live_e[j], ghost_n[j], ghost_e[j])
        self._mask_values()

    def get_uniform(self, J):
        """Fields of the full level J (Sec. 2.2): live points keep their values,
        every other point takes the inverse transform with zero coefficients of
        the full level J-1, from Jmin (always full) up.  A prescribed velocity is
        returned as set."""
        dh = {self.jmin: self.dh[self.jmin].copy()}
        u = {self.jmin: self.u[self.jmin].copy()}
        for j in range(self.jmin + 1, J + 1):
            dh[j] = np.where(self.live_n[j], self.dh[j], 0.0)
            u[j] = np.where(self.live_e[j], self.u[j], 0.0)
            adapt.prolong_level(self.Hy, self.VS[j], j, dh, u, self.live_n[j], self.live_e[j],
                                ~self.live_n[j], ~self.live_e[j])
            if self.advect:
                u[j] = self.u_set[j].copy()
        return dh[J], u[J]

    # ------------------------------------------------------------------ trend
    def covered(self, j):
        """Coarse nodes of level j whose restriction stencil is complete at j+1: the
        fine node at the same place and every odd node m of M_k (the 2N fine nodes
        whose hexagons overlap hexagon k, Sec. 4.3) are live."""
        Hy = self.Hy
        C = Hy.levels[j]
        odd = Hy.odd[j + 1]
        dead = ~self.live_n[j + 1][odd]
        bad = np.zeros(C.N, dtype=bool)
        bad[Hy.K[j + 1][dead].ravel()] = True
        return self.live_n[j + 1][: C.N] & ~bad

    def rhs(self, dh, u):
        """Trends (d dh/dt, du/dt) at live points of every level; ghosts of (dh, u)
        are refreshed first.  Returns dicts of arrays (NaN away from live points)."""
        Hy, H, g = self.Hy, self.H, self.g
        self.fill_ghosts(dh, u)
        F, q, B, c, Q = {}, {}, {}, {}, {}
        with np.errstate(invalid="ignore"):
            nu = self.nu
            for j in self.levels:
                L = Hy.levels[j]
                F[j] = trisk.thickness_flux(L, dh[j], u[j], H)
                if self.advect:
                    # prescribed velocity: the height flux alone (plus diffusion)
                    if nu:
                        F[j] = F[j] - nu * trisk.gradient(L, dh[j])
                    c[j] = trisk.divergence(L, F[j])
                    continue
                q[j] = trisk.potential_vorticity(L, dh[j], u[j], H)
                B[j] = trisk.bernoulli(L, dh[j], u[j], g)
                Q[j] = -trisk.coriolis_tendency(L, F[j], q[j])
                if nu:
                    # viscous form: the diffusive height flux joins F after the Coriolis
                    # term (which takes the mass flux), -nu div u joins B, and
                    # nu grad^perp curl u joins Q; the restriction then carries them
                    F[j] = F[j] - nu * trisk.gradient(L, dh[j])
                    B[j] = B[j] - nu * trisk.divergence(L, u[j])
                    Q[j] = Q[j] + nu * trisk.perp_gradient(L, trisk.vorticity(L, u[j]))
                c[j] = trisk.divergence(L, F[j])
            for j in range(self.jmax - 1, self.jmin - 1, -1):
                C, Fl = Hy.levels[j], Hy.levels[j + 1]
                cov_n = self.covered(j)
                if not self.advect:
                    B[j][cov_n] = B[j + 1][: C.N][cov_n]
                    VS = self.VS[j + 1]
                    h0, h1 = VS.half[:, 0], VS.half[:, 1]
                    s0, s1 = VS.half_sign[:, 0], VS.half_sign[:, 1]
                    cov_e = cov_n[C.edges[:, 0]] & cov_n[C.edges[:, 1]]
                    Q[j][cov_e] = 0.5 * (s0[cov_e] * Q[j + 1][h0[cov_e]] + s1[cov_e] * Q[j + 1][h1[cov_e]])
                rf = cov_n[C.edges[:, 0]] | cov_n[C.edges[:, 1]]
                Fint = transform.restrict_flux(self.FS[j + 1], F[j + 1], Fl.l_e, c[j + 1])
                F[j][rf] = Fint[rf] / C.l_e[rf]
                c[j] = trisk.divergence(C, F[j])
        dht, dut = {}, {}
        for j in self.levels:
            L = Hy.levels[j]
            with np.errstate(invalid="ignore"):
                a = -c[j]
                b = np.zeros(L.E) if self.advect else -Q[j] - trisk.gradient(L, B[j])
            a[~self.live_n[j]] = np.nan
            b[~self.live_e[j]] = np.nan
            assert not np.isnan(a[self.live_n[j]]).any(), f"incomplete stencil for a live node at level {j}"
            assert not np.isnan(b[self.live_e[j]]).any(), f"incomplete stencil for a live edge at level {j}"
            dht[j], dut[j] = a, b
        self.last = dict(F=F, q=q, B=B, c=c, Q=Q)
        return dht, dut

    # ------------------------------------------------------------------ time step
    def _axpy(self, x, a, y):
        return {j: x[j] + a * y[j] for j in self.levels}

    def _copy(self, x):
        return {j: x[j].copy() for j in self.levels}

    def step(self, dt, adapt_after=True):
        h0, u0 = self._copy(self.dh), self._copy(self.u)
        if self.rk == "rk4":
            k1 = self.rhs(self._copy(h0), self._copy(u0))
            h1, u1 = self._axpy(h0, 0.5 * dt, k1[0]), self._axpy(u0, 0.5 * dt, k1[1])
            k2 = self.rhs(h1, u1)
            h2, u2 = self._axpy(h0, 0.5 * dt, k2[0]), self._axpy(u0, 0.5 * dt, k2[1])
            k3 = self.rhs(h2, u2)
            h3, u3 = self._axpy(h0, dt, k3[0]), self._axpy(u0, dt, k3[1])
            k4 = self.rhs(h3, u3)
            hn = {j: h0[j] + dt / 6.0 * (k1[0][j] + 2.0 * k2[0][j] + 2.0 * k3[0][j] + k4[0][j]) for j in self.levels}
            un = {j: u0[j] + dt / 6.0 * (k1[1][j] + 2.0 * k2[1][j] + 2.0 * k3[1][j] + k4[1][j]) for j in self.levels}
        elif self.rk == "ssp43":
            k = self.rhs(self._copy(h0), self._copy(u0))
            h1, u1 = self._axpy(h0, 0.5 * dt, k[0]), self._axpy(u0, 0.5 * dt, k[1])
            k = self.rhs(h1, u1)
            h2, u2 = self._axpy(h1, 0.5 * dt, k[0]), self._axpy(u1, 0.5 * dt, k[1])
            k = self.rhs(h2, u2)
            h3 = {j: 2.0 / 3.0 * h0[j] + 1.0 / 3.0 * h2[j] + dt / 6.0 * k[0][j] for j in self.levels}
            u3 = {j: 2.0 / 3.0 * u0[j] + 1.0 / 3.0 * u2[j] + dt / 6.0 * k[1][j] for j in self.levels}
            k = self.rhs(h3, u3)
            hn, un = self._axpy(h3, 0.5 * dt, k[0]), self._axpy(u3, 0.5 * dt, k[1])
        else:
            raise ValueError(self.rk)
        for j in self.levels:
            hn[j][~self.live_n[j]] = np.nan
            un[j][~self.live_e[j]] = np.nan
        self.dh, self.u = hn, un
        self.partial_transform()
        self.fill_ghosts()
        if adapt_after:
            self.adapt()
        else:
            self.fill_ghosts()
            self._mask_values()

    def partial_transform(self):
        """R_h at covered coarse nodes, from Jmax-1 down (Sec. 3.1)."""
        Hy = self.Hy
        for j in range(self.jmax, self.jmin, -1):
            C = Hy.levels[j - 1]
            odd = Hy.odd[j]
            with np.errstate(invalid="ignore"):
                d = transform.height_detail(Hy, j, self.dh[j])
            d = np.where(self.live_n[j][odd], d, 0.0)
            cov = self.covered(j - 1)
            hf = np.where(cov, self.dh[j][: C.N], 0.0)
            full = np.zeros(Hy.levels[j].N)
            full[: C.N] = hf
            hc = transform.height_update(Hy, j, full, d)
            self.dh[j - 1][cov] = hc[cov]

    def dt_cfl(self):
        wmax, rmin = 0.0, math.inf
        for j in self.levels:
            L = self.Hy.levels[j]
            dx = grid.nominal_spacing(j, L.radius)
            f = 2.0 * self.Hy.omega * L.xyz[:, 2]
            h = self.H + self.dh[j]
            ln = self.live_n[j]
            if not self.advect:
                w = np.sqrt(f[ln] ** 2 + self.g * h[ln] * (math.pi / dx) ** 2)
                wmax = max(wmax, float(w.max(initial=0.0)))
            au = np.abs(self.u[j][self.live_e[j]])
            au = au[au > 0]
            if au.size:
                rmin = min(rmin, float((dx / au).min()))
        return self.cfl * min(1.0 / wmax if wmax > 0 else math.inf, rmin)

    # ------------------------------------------------------------------ diagnostics
    def mass(self):
        L = self.Hy.levels[self.jmin]
        return math.fsum((L.A_i * (self.H + self.dh[self.jmin])).tolist())

    def energy(self):
        L = self.Hy.levels[self.jmin]
        h = self.H + self.dh[self.jmin]
        K = trisk.kinetic_energy(L, self.u[self.jmin])
        g = self.g
        AS = 4.0 * math.pi * L.radius ** 2
        c2 = g * math.fsum((L.A_i * h).tolist()) / AS
        return math.fsum((L.A_i * g * h * (0.5 * g * h + K)).tolist()) - 0.5 * c2 * c2 * AS

    def active_nodes(self):
        return sum(int(self.live_n[j].sum()) for j in self.levels)
