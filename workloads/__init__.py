"""Seeded synthetic initial conditions for the shallow-water workloads.

This module evaluates analytic fields at points the caller supplies (node
positions, edge midpoints and edge tangents on the unit sphere).  It holds
none of the discretisation: no grid, no operator, no transform.  Both the
CUDA library's tests and the oracle's tests draw their inputs from here.

Workloads (all seeded; numpy PCG64):
  * ``harmonic``: mean depth 10 km plus 100 m of random real spherical
    harmonics of degree 1..8 (coefficients N(0,1), field scaled to max 100 m);
    velocity from the geostrophic stream function psi = g*dh/f0 with
    f0 = 2*Omega*sin(45 deg).
  * ``jet``: zonal jet u = 80 exp(-((lat-lat0)/7deg)^2) m/s, lat0 ~ U[20,60] deg,
    depth from zonal gradient-wind balance (mean 10 km), plus three Gaussian
    height bumps of 120 m (e-folding radius 500 km) at seeded sites.
  * ``tc2``: Williamson test case 2 (solid-body zonal flow, u0 = 2 pi R / 12 d,
    g*H = 2.94e4 m^2/s^2), depth from the same gradient-wind balance.
  * ``turbulence``: random-phase vorticity with energy spectrum (l/32)^2 below
    degree 32 and (l/32)^-3 above (degrees 1..96), rms velocity 20 m/s, depth in
    geostrophic balance with f0 = 2 Omega sin 45 deg about a 10 km mean (the
    spectrum's shape and the balance are readings).
  * ``tc1_cosine`` / ``tc1_smooth``: the advection test of Sec. 7.1 -- a bell
    of height 1000 m and radius L = R/3 centred at lat 0, lon 0 (the cosine
    bell (H/2)(1 + cos(pi r/L)) for r < L, or the smooth bell
    H exp(r^2/(r^2 - 2 L^2)) for r < sqrt(2) L; zero outside, the reading of
    both), carried by solid-body rotation of speed U = 2 pi R / 12 d about an
    axis tilted by ``alpha`` from the pole.  The depth is the bell itself
    (``mean_depth`` 0); ``exact(xyz, t)`` is the bell rotated by U t / R.
"""
from __future__ import annotations

import math
import numpy as np

DAY = 86400.0


def _latlon(xyz):
    xyz = np.asarray(xyz, dtype=np.float64)
    r = np.linalg.norm(xyz, axis=-1)
    lat = np.arcsin(np.clip(xyz[..., 2] / r, -1.0, 1.0))
    lon = np.arctan2(xyz[..., 1], xyz[..., 0])
    return lat, lon


def _east_north(xyz):
    """Unit east and north vectors at unit-sphere points."""
    xyz = np.asarray(xyz, dtype=np.float64)
    lat, lon = _latlon(xyz)
    east = np.stack([-np.sin(lon), np.cos(lon), np.zeros_like(lon)], axis=-1)
    north = np.stack([-np.sin(lat) * np.cos(lon), -np.sin(lat) * np.sin(lon), np.cos(lat)], axis=-1)
    return east, north


def _legendre_all(lmax, x):
    """Fully normalised associated Legendre functions P[l][m](x), 0<=m<=l<=lmax
    (orthonormal on the sphere together with the 1/sqrt(2 pi) azimuthal factor)."""
    P = {}
    s = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    P[(0, 0)] = np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))
    for m in range(1, lmax + 1):
        P[(m, m)] = -math.sqrt((2 * m + 1) / (2.0 * m)) * s * P[(m - 1, m - 1)]
    for m in range(0, lmax):
        P[(m + 1, m)] = math.sqrt(2 * m + 3) * x * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[(l, m)] = a * (x * P[(l - 1, m)] - b * P[(l - 2, m)])
    return P


class _Harmonic:
    def __init__(self, seed, lmax=8, lmin=1):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.lmax = lmax
        self.coef = []
        for l in range(lmin, lmax + 1):
            for m in range(0, l + 1):
                a = rng.standard_normal()
                b = rng.standard_normal() if m > 0 else 0.0
                self.coef.append((l, m, a, b))

    def __call__(self, xyz):
        lat, lon = _latlon(xyz)
        P = _legendre_all(self.lmax, np.sin(lat))
        out = np.zeros_like(lat)
        for l, m, a, b in self.coef:
            if m == 0:
                out += a * P[(l, 0)]
            else:
                out += math.sqrt(2.0) * P[(l, m)] * (a * np.cos(m * lon) + b * np.sin(m * lon))
        return out


class _Spectral:
    """A real spherical-harmonic series sum_{l,m} (a_lm cos(m lon) + b_lm sin(m lon))
    P_lm(sin lat) of degrees 1..lmax (fully normalised), evaluated at arbitrary
    points one order m at a time (the Legendre recurrence runs over the points,
    so memory stays a few arrays of the point count)."""

    def __init__(self, lmax, a, b):
        self.lmax, self.a, self.b = lmax, a, b   # a[l, m], b[l, m]

    def __call__(self, xyz):
        lat, lon = _latlon(xyz)
        x = np.sin(lat)
        s = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
        out = np.zeros_like(x)
        pmm = np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))
        for m in range(0, self.lmax + 1):
            if m > 0:
                pmm = -math.sqrt((2 * m + 1) / (2.0 * m)) * s * pmm
            ca = np.zeros_like(x)
            cb = np.zeros_like(x)
            p_prev, p = None, pmm
            for l in range(m, self.lmax + 1):
                if l == m + 1:
                    p_prev, p = p, math.sqrt(2 * m + 3) * x * pmm
                elif l > m + 1:
                    a_ = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                    b_ = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                    p_prev, p = p, a_ * (x * p - b_ * p_prev)
                if l >= 1:
                    if self.a[l, m] != 0.0:
                        ca += self.a[l, m] * p
                    if m > 0 and self.b[l, m] != 0.0:
                        cb += self.b[l, m] * p
            if m == 0:
                out += ca
            else:
                out += math.sqrt(2.0) * (ca * np.cos(m * lon) + cb * np.sin(m * lon))
        return out


def _rotate(xyz, axis, ang):
    """Rotate unit vectors xyz about unit vectors axis by angle ang (Rodrigues)."""
    c, s = math.cos(ang), math.sin(ang)
    return xyz * c + np.cross(axis, xyz) * s + axis * np.sum(axis * xyz, axis=-1, keepdims=True) * (1 - c)


def _normal_derivative(fun, mid, tangent, radius, delta=1e-5):
    """d fun / d n_left at mid, n_left = mid x tangent (left of the tangent), in 1/m."""
    # moving along n_left = rotating about the tangent axis
    p = _rotate(mid, tangent, -delta)
    m = _rotate(mid, tangent, delta)
    return (fun(p) - fun(m)) / (2.0 * delta * radius)


def _zonal_balance(ufun, radius, omega, g, mean_depth, nq=200001, anchor="mean"):
    """Depth profile h(lat) from g dh/dlat = -R u (2 Omega sin(lat) + u tan(lat)/R),
    integrated by the trapezoid rule on a fine latitude grid and shifted to the
    requested area-weighted mean (``anchor="mean"``) or equatorial value
    (``anchor="equator"``).  Returns a callable h(lat)."""
    lat = np.linspace(-math.pi / 2, math.pi / 2, nq)
    u = ufun(lat)
    with np.errstate(invalid="ignore", divide="ignore"):
        tan = np.where(np.abs(np.cos(lat)) > 1e-14, np.tan(lat), 0.0)
    rhs = -radius * u * (2.0 * omega * np.sin(lat) + u * tan / radius) / g
    h = np.concatenate([[0.0], np.cumsum(0.5 * (rhs[1:] + rhs[:-1]) * np.diff(lat))])
    w = np.cos(lat)
    mean = np.sum(0.5 * (h[1:] * w[1:] + h[:-1] * w[:-1]) * np.diff(lat)) / 2.0
    ref = mean if anchor == "mean" else np.interp(0.0, lat, h)
    h = h - ref + mean_depth
    return lambda la: np.interp(la, lat, h)


class Sampling:
    """The per-point quantities every workload evaluates on one grid (node
    latitudes, edge latitudes and the eastward component of each edge tangent),
    computed once for many seeded members on the same grid."""

    def __init__(self, node_xyz, edge_mid, edge_tan):
        self.node_xyz = np.asarray(node_xyz, dtype=np.float64)
        self.edge_mid = np.asarray(edge_mid, dtype=np.float64)
        self.edge_tan = np.asarray(edge_tan, dtype=np.float64)
        self.node_lat, _ = _latlon(self.node_xyz)
        east, _ = _east_north(self.edge_mid)
        self.edge_lat, _ = _latlon(self.edge_mid)
        self.east_tan = np.sum(east * self.edge_tan, axis=-1)


class Workload:
    """A seeded initial condition: call ``fields(node_xyz, edge_mid, edge_tan)``.

    Positions are unit vectors; ``edge_tan`` is the unit tangent of each edge
    (direction of positive normal velocity).  Returns (dh [m], u [m/s]) where
    dh is the depth perturbation about ``mean_depth``.
    """

    def __init__(self, kind, seed=0, radius=6.371e6, omega=7.292e-5, g=9.80616, mean_depth=1.0e4, alpha=0.0):
        self.kind, self.seed = kind, seed
        self.radius, self.omega, self.g, self.mean_depth = radius, omega, g, mean_depth
        rng = np.random.Generator(np.random.PCG64(seed))
        if kind == "harmonic":
            self._harm = _Harmonic(seed)
            # scale so that max |dh| over a dense sampling is 100 m
            t = np.linspace(-1, 1, 181)
            ll = np.linspace(-math.pi, math.pi, 361)
            T, L = np.meshgrid(np.arcsin(t), ll, indexing="ij")
            pts = np.stack([np.cos(T) * np.cos(L), np.cos(T) * np.sin(L), np.sin(T)], axis=-1)
            self._scale = 100.0 / np.max(np.abs(self._harm(pts)))
            self.f0 = 2.0 * omega * math.sin(math.pi / 4)
        elif kind == "jet":
            self.lat0 = math.radians(rng.uniform(20.0, 60.0))
            self.width = math.radians(7.0)
            self.u0 = 80.0
            lon = rng.uniform(-math.pi, math.pi, 3)
            lat = np.radians(rng.uniform(-70.0, 70.0, 3))
            self.bumps = np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], axis=-1)
            self.bump_amp, self.bump_radius = 120.0, 5.0e5
            self._h = _zonal_balance(self._ujet, radius, omega, g, mean_depth)
        elif kind == "turbulence":
            # random-phase vorticity with energy spectrum E(l) ~ (l/32)^2 below
            # degree 32 and (l/32)^-3 above, rms velocity 20 m/s, the stream
            # function psi_lm = -R^2 zeta_lm / (l (l + 1)) and geostrophic depth
            # g dh = f0 psi (f0 = 2 Omega sin 45 deg), mean depth 10 km
            lmax = 96
            ls = np.arange(lmax + 1, dtype=np.float64)
            E = np.where(ls < 32, (ls / 32.0) ** 2, (np.maximum(ls, 1.0) / 32.0) ** -3.0)
            E[0] = 0.0
            a = np.zeros((lmax + 1, lmax + 1))
            b = np.zeros((lmax + 1, lmax + 1))
            for l in range(1, lmax + 1):
                ca = rng.standard_normal(l + 1)
                cb = rng.standard_normal(l + 1)
                cb[0] = 0.0
                norm = math.sqrt(np.sum(ca ** 2) + np.sum(cb ** 2))
                # sum_m |psi_lm|^2 l (l + 1) is the degree's share of the kinetic energy
                amp = math.sqrt(E[l] / (l * (l + 1))) / norm
                a[l, : l + 1] = amp * ca
                b[l, : l + 1] = amp * cb
            ke = sum(l * (l + 1) * (np.sum(a[l] ** 2) + np.sum(b[l, 1:] ** 2)) for l in range(1, lmax + 1))
            # mean |u|^2 = sum l (l + 1) psi_lm^2 / (4 pi R^2) for orthonormal harmonics
            scale = 20.0 / math.sqrt(ke / (4.0 * math.pi * radius ** 2))
            self._psi = _Spectral(lmax, scale * a, scale * b)
            self.f0 = 2.0 * omega * math.sin(math.pi / 4)
        elif kind in ("tc1_cosine", "tc1_smooth"):
            self.mean_depth = 0.0
            self.u0 = 2.0 * math.pi * radius / (12.0 * DAY)
            self.bell_h, self.bell_L = 1000.0, radius / 3.0
            self.alpha = alpha
            # v = U a x r^ with the unit axis a: east component U (cos(lat) cos(alpha)
            # + sin(lat) cos(lon) sin(alpha)), north component -U sin(lon) sin(alpha)
            self.axis = np.array([-math.sin(alpha), 0.0, math.cos(alpha)])
        elif kind == "tc2":
            self.u0 = 2.0 * math.pi * radius / (12.0 * DAY)
            gH = 2.94e4
            self._h = _zonal_balance(lambda la: self.u0 * np.cos(la), radius, omega, g, gH / g, anchor="equator")
        else:
            raise ValueError(kind)

    def _ujet(self, lat):
        return self.u0 * np.exp(-(((lat - self.lat0) / self.width) ** 2))

    def _bell(self, xyz):
        xyz = np.asarray(xyz, dtype=np.float64)
        xyz = xyz / np.linalg.norm(xyz, axis=-1, keepdims=True)
        r = self.radius * np.arccos(np.clip(xyz[..., 0], -1.0, 1.0))   # distance to lat 0, lon 0
        H, L = self.bell_h, self.bell_L
        if self.kind == "tc1_cosine":
            return np.where(r < L, 0.5 * H * (1.0 + np.cos(math.pi * np.minimum(r, L) / L)), 0.0)
        inside = r < math.sqrt(2.0) * L
        rr = np.where(inside, r, 0.0)
        return np.where(inside, H * np.exp(rr * rr / (rr * rr - 2.0 * L * L)), 0.0)

    def exact(self, xyz, t):
        """Depth at time t of the advection test: the initial bell rotated by U t / R."""
        back = _rotate(np.asarray(xyz, dtype=np.float64), self.axis, -self.u0 * t / self.radius)
        return self._bell(back)

    def depth(self, xyz, lat=None):
        """Total depth h at unit-sphere points (lat: their latitudes, if known)."""
        xyz = np.asarray(xyz, dtype=np.float64)
        if self.kind.startswith("tc1"):
            return self._bell(xyz)
        if self.kind == "harmonic":
            return self.mean_depth + self._scale * self._harm(xyz)
        if self.kind == "turbulence":
            return self.mean_depth + self.f0 * self._psi(xyz) / self.g
        if lat is None:
            lat, _ = _latlon(xyz)
        h = self._h(lat)
        if self.kind == "jet":
            for b in self.bumps:
                ang = np.arctan2(np.linalg.norm(np.cross(xyz, b), axis=-1), xyz @ b)
                h = h + self.bump_amp * np.exp(-((ang * self.radius / self.bump_radius) ** 2))
        return h

    def velocity(self, mid, tan):
        """Normal velocity component along ``tan`` at edge midpoints."""
        mid = np.asarray(mid, dtype=np.float64)
        tan = np.asarray(tan, dtype=np.float64)
        if self.kind == "harmonic":
            psi = lambda p: self.g * self._scale * self._harm(p) / self.f0
            # u = k x grad(psi);  u . t = -d psi / d n_left
            return -_normal_derivative(psi, mid, tan, self.radius)
        if self.kind == "turbulence":
            return -_normal_derivative(self._psi, mid, tan, self.radius)
        if self.kind.startswith("tc1"):
            m = mid / np.linalg.norm(mid, axis=-1, keepdims=True)
            return self.u0 * np.sum(np.cross(self.axis, m) * tan, axis=-1)
        east, _ = _east_north(mid)
        lat, _ = _latlon(mid)
        uz = self._ujet(lat) if self.kind == "jet" else self.u0 * np.cos(lat)
        return uz * np.sum(east * tan, axis=-1)

    def fields(self, node_xyz, edge_mid, edge_tan):
        dh = self.depth(node_xyz) - self.mean_depth
        return dh, self.velocity(edge_mid, edge_tan)

    def fields_on(self, S):
        """fields() on a precomputed Sampling (the same values)."""
        if self.kind not in ("jet", "tc2"):
            return self.fields(S.node_xyz, S.edge_mid, S.edge_tan)
        dh = self.depth(S.node_xyz, S.node_lat) - self.mean_depth
        uz = self._ujet(S.edge_lat) if self.kind == "jet" else self.u0 * np.cos(S.edge_lat)
        return dh, uz * S.east_tan
