"""Mutation check of the oracle's pins: one plausible mistake at a time (a dropped
term, a wrong sign, index or operand) is planted in a copy of ``oracle/`` and the
oracle's CPU tests are run on the copy.  Every mistake that can change a result
must make a test fail; the few that cannot are listed with the reason.

    python tests/oracle_mutations.py            # all, six at a time
    python tests/oracle_mutations.py 3 17       # some of them

Exit status 1 when a mistake that can change a result survives.  Takes a few
minutes on eight cores; not part of the test suite.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [  # (oracle file, text, replacement, label[, why it cannot change a result])
 ("trisk.py", "return 0.5 * (h[L.edges[:, 0]] + h[L.edges[:, 1]]) * u", "return h[L.edges[:, 0]] * u", "F upwind depth"),
 ("trisk.py", "out += np.where(ok, L.nbr_sign[:, k] * F[ee] * L.l_e[ee], 0.0)", "out += np.where(ok, L.nbr_sign[:, k] * F[ee] * L.d_e[ee], 0.0)", "div uses d_e"),
 ("trisk.py", "return (B[L.edges[:, 1]] - B[L.edges[:, 0]]) / L.d_e", "return (B[L.edges[:, 0]] - B[L.edges[:, 1]]) / L.d_e", "grad sign"),
 ("trisk.py", "return (B[L.edges[:, 1]] - B[L.edges[:, 0]]) / L.d_e", "return (B[L.edges[:, 1]] - B[L.edges[:, 0]]) / L.l_e", "grad over l_e"),
 ("trisk.py", "0.25 * L.l_e[ee] * L.d_e[ee] * u[ee] ** 2", "0.5 * L.l_e[ee] * L.d_e[ee] * u[ee] ** 2", "K factor"),
 ("trisk.py", "return np.sum(L.tri_esign * u[e] * L.d_e[e], axis=1) / L.A_v", "return np.sum(L.tri_esign * u[e] * L.l_e[e], axis=1) / L.A_v", "curl uses l_e"),
 ("trisk.py", "return np.sum(L.kite * h[L.tri], axis=1) / L.A_v", "return np.mean(h[L.tri], axis=1)", "h_v equal thirds"),
 ("trisk.py", "return (vorticity(L, u) + L.f_v) / depth_at_triangles(L, dh, H)", "return vorticity(L, u) / depth_at_triangles(L, dh, H)", "q without f"),
 ("trisk.py", "kp = (k + o - 1) % deg", "kp = (k + o) % deg", "Coriolis kite index"),
 ("trisk.py", "w = 0.5 - csum", "w = 0.5 + csum", "Coriolis weight sign"),
 ("trisk.py", "psi += np.where(ok, w * phi * 0.5 * (qe[ekk] + qe[e2]), 0.0)", "psi += np.where(ok, w * phi * qe[ekk], 0.0)", "Coriolis q not averaged"),
 ("trisk.py", "qe = 0.5 * (q[L.left] + q[L.right])", "qe = q[L.left]", "q_e one triangle"),
 ("trisk.py", "return g * dh + kinetic_energy(L, u)", "return g * dh", "B without K"),
 ("trisk.py", "b = coriolis_tendency(L, F, q) - gradient(L, B)", "b = coriolis_tendency(L, F, q) + gradient(L, B)", "trend grad sign"),
 ("trisk.py", "return gradient(L, divergence(L, u)) - perp_gradient(L, vorticity(L, u))", "return gradient(L, divergence(L, u)) + perp_gradient(L, vorticity(L, u))", "vector Laplacian sign"),
 ("transform.py", "return hf[odd] - np.sum(st * hf[K], axis=1)", "return hf[odd] + np.sum(st * hf[K], axis=1)", "predict sign"),
 ("transform.py", "    s = Hy.Akm[j] / C.A_i[Hy.K[j]]\n    np.add.at", "    s = Hy.Akm[j] / Hy.Am[j][:, None]\n    np.add.at", "update weight area"),
 ("transform.py", "return 0.5 * (s[:, 0] * uf[h[:, 0]] + s[:, 1] * uf[h[:, 1]])", "return 0.5 * (s[:, 0] * uf[h[:, 0]] + uf[h[:, 1]])", "R_u sign dropped"),
 ("transform.py", "b[:, 1] = np.sum(tf * e2, axis=1)", "b[:, 1] = np.sum(tf * e1, axis=1)", "P_u rhs component"),
 ("transform.py", "M = np.stack([t1, t2, xi * t1, eta * t1, xi * t2, eta * t2], axis=1)", "M = np.stack([t1, t2, xi * t1, eta * t1, xi * t2, 0.5 * eta * t2], axis=1)", "P_u condition scaled",
  "equivalent: a constraint with zero right-hand side scaled; the minimum-norm weights are the same"),
 ("transform.py", "return 0.5 * (a - b), uf[VS.int_edge] - pi", "return 0.5 * (a + b), uf[VS.int_edge] - pi", "velocity detail sign"),
 ("transform.py", "delta = 0.5 * (2.0 * uc - ph[:, 0] - ph[:, 1])\n    uf = np.full", "delta = 0.0 * uc\n    uf = np.full", "inverse velocity mean"),
 ("transform.py", "F1 = 0.5 * (F_in_k - F_in_l) + 0.5 * (A(k, m) - A(l, m)) * c[m]", "F1 = 0.5 * (F_in_k - F_in_l)", "R_F0 centre term"),
 ("transform.py", "+ 0.5 * kml(k, FS.m_lp, FS.pp1)", "+ kml(k, FS.m_lp, FS.pp1)", "R'_F half weight"),
 ("transform.py", "return A(a, x) * A(b, x) / FS.Am[x] * (c[a] - c[b])", "return A(a, x) * A(b, x) / FS.Am[x] * (c[b] - c[a])", "kml sign"),
 ("transform.py", "return g1 * self.seg1 + g2 * self.seg2", "return g1 * self.seg1 - g2 * self.seg2", "x_T component sign"),
 ("adapt.py", "        S[Hy.mid[j - 1][se]] = True\n", "", "significance midpoint"),
 ("adapt.py", "            t |= dilate(F, ch)", "            t |= ch", "children not dilated"),
 ("adapt.py", "            T[j - 1] |= T[j][: Hy.levels[j - 1].N]", "            pass", "closure to coarse"),
 ("adapt.py", "        T[j][Hy.K[j][oddlive].ravel()] = True", "        pass", "closure prediction parents"),
 ("adapt.py", "GHOST_HOPS = 5", "GHOST_HOPS = 4", "ghost hops",
  "equivalent on these grids: four hops already hold every stencil of a live point; five is the reading"),
 ("adapt.py", "        live_e[j] = edges_touching(L, live_n[j])", "        live_e[j] = edges_within(L, live_n[j])", "edge liveness"),
 ("adapt.py", "vals = np.where(live_n[K], hf[K], hc[K])", "vals = hc[K]", "prolong ignores live fine"),
 ("adapt.py", "uf[h0[a]] = s0[a] * (2.0 * uc[a] - s1[a] * uf[h1[a]])", "uf[h0[a]] = s0[a] * (ph[a, 0] + delta[a])", "prolong half ignores sibling"),
 ("model.py", "mh = max(float(np.nanmax(np.abs(self.dh[j][self.live_n[j]]), initial=0.0)) for j in self.levels)", "mh = max(float(np.nanmax(np.abs(self.dh[j]), initial=0.0)) for j in self.levels)", "threshold over ghosts"),
 ("model.py", "e = self.eps * math.sqrt(self.eps) if self.regime == 1 else self.eps", "e = self.eps * self.eps if self.regime == 1 else self.eps", "regime exponent"),
 ("model.py", "(k1[0][j] + 2.0 * k2[0][j] + 2.0 * k3[0][j] + k4[0][j])", "(k1[0][j] + k2[0][j] + 2.0 * k3[0][j] + 2.0 * k4[0][j])", "RK4 weights h"),
 ("model.py", "h3 = {j: 2.0 / 3.0 * h0[j] + 1.0 / 3.0 * h2[j] + dt / 6.0 * k[0][j] for j in self.levels}", "h3 = {j: 1.0 / 3.0 * h0[j] + 2.0 / 3.0 * h2[j] + dt / 6.0 * k[0][j] for j in self.levels}", "SSP weights"),
 ("model.py", "            cov = self.covered(j - 1)\n            hf", "            cov = self.live_n[j][: C.N].copy()\n            hf", "partial transform all even"),
 ("model.py", "w = np.sqrt(f[ln] ** 2 + self.g * h[ln] * (math.pi / dx) ** 2)", "w = np.sqrt(f[ln] ** 2 + self.g * h[ln] * (math.pi / dx))", "omega as printed"),
 ("model.py", "        bad[Hy.K[j + 1][dead].ravel()] = True\n", "", "covered ignores odd"),
 ("model.py", "                    B[j][cov_n] = B[j + 1][: C.N][cov_n]\n", "", "B not restricted"),
 ("model.py", "Q[j][cov_e] = 0.5 * (s0[cov_e] * Q[j + 1][h0[cov_e]] + s1[cov_e] * Q[j + 1][h1[cov_e]])", "Q[j][cov_e] = s0[cov_e] * Q[j + 1][h0[cov_e]]", "Q restriction one half"),
 ("model.py", "                F[j][rf] = Fint[rf] / C.l_e[rf]\n", "", "flux not restricted"),
 ("model.py", "return math.fsum((L.A_i * (self.H + self.dh[self.jmin])).tolist())", "return math.fsum((L.A_i * self.dh[self.jmin]).tolist())", "mass without H"),
 ("model.py", "- 0.5 * c2 * c2 * AS", "- 0.0 * c2 * c2 * AS", "energy offset"),
 ("model.py", "        self.partial_transform()\n        self.fill_ghosts()\n", "        self.partial_transform()\n", "ghosts after partial transform",
  "equivalent: the adaptation that follows reads no ghost the partial transform changes, then refills them"),
 ("model.py", "f = 2.0 * self.Hy.omega * L.xyz[:, 2]", "f = 2.0 * self.Hy.omega * L.xyz[:, 2] / L.radius", "dt f scale"),
 ("grid.py", "self.f_v = 2.0 * omega * self.cc[:, 2]", "self.f_v = omega * self.cc[:, 2]", "f_v factor 2"),
 ("grid.py", " + triangle_area(p, self.cc, normalize(prv + p))", "", "kite half dropped"),
 ("grid.py", "self.l_e = arc_length(self.cc[self.left], self.cc[self.right]) * R", "self.l_e = self.d_e / math.sqrt(3.0)", "l_e of an equilateral grid"),
 ("grid.py", "new_xyz = normalize(xyz[parents[:, 0]] + xyz[parents[:, 1]])", "new_xyz = 0.5 * (xyz[parents[:, 0]] + xyz[parents[:, 1]])", "midpoint not projected"),
 ("grid.py", "return math.sqrt(2.0 * 4.0 * math.pi * radius * radius / (math.sqrt(3.0) * N))", "return math.sqrt(4.0 * math.pi * radius * radius / N)", "Table 1 spacing"),
 ("mlp.py", "r = ((b + 0x7FFF + lsb) >> 16) << 16", "r = ((b + 0x8000) >> 16) << 16", "BF16 ties away from zero"),
 ("mlp.py", "r = ((b + 0x7FFF + lsb) >> 16) << 16", "r = (b >> 16) << 16", "BF16 truncation"),
 ("mlp.py", "g = (pos_w * y * (p - 1.0) + (1.0 - y) * p) / n", "g = (y * (p - 1.0) + (1.0 - y) * p) / n", "gradient without pos_w"),
 ("mlp.py", "return L, X.T @ dz, dz.sum(axis=0), a.T @ g, float(g.sum())", "return L, X.T @ dz, dz.sum(axis=0), z.T @ g, float(g.sum())", "w2 gradient pre-activation"),
 ("mlp.py", "mh = m / (1 - b1 ** t)", "mh = m", "Adam bias correction"),
 ("transform.py", "np.subtract.at(even, Hy.K[j].ravel(), (s * hdet[:, None]).ravel())", "np.add.at(even, Hy.K[j].ravel(), (s * hdet[:, None]).ravel())", "inverse update sign"),
 ("transform.py", "hf[Hy.odd[j]] = hdet + np.sum(st * even[Hy.K[j]], axis=1)", "hf[Hy.odd[j]] = hdet + np.sum(st * hc[Hy.K[j]], axis=1)", "inverse predicts from coarse"),
 ("model.py", "        return self.live_n[j + 1][: C.N] & ~bad", "        return ~bad", "covered without the even node",
  "equivalent under the closure: a live odd node of M_k makes k's even node live (k is one of its parents)"),
 ("model.py", "                F[j][rf] = Fint[rf] / C.l_e[rf]", "                F[j][rf] = Fint[rf] / C.d_e[rf]", "restricted flux over d_e"),
 ("model.py", "dx = grid.nominal_spacing(j, L.radius)", "dx = grid.nominal_spacing(self.jmax, L.radius)", "dt spacing of Jmax"),
 ("trisk.py", "out += np.where(ok, L.nbr_sign[:, k] * F[ee] * L.l_e[ee], 0.0)", "out += np.where(ok, F[ee] * L.l_e[ee], 0.0)", "div without orientation"),
 ("adapt.py", "        out[nb[ok & S]] = True", "        out[nb[ok]] = True", "dilate everything"),
]


def run(i, tmp):
    f, old, new, label = MUTATIONS[i][:4]
    d = os.path.join(tmp, f"m{i:02d}")
    for sub in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("__pycache__", "_build"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    p = os.path.join(d, "oracle", f)
    s = open(p).read()
    if s.count(old) != 1:
        return i, label, "NOT APPLIED (text not found once)"
    open(p, "w").write(s.replace(old, new))
    tests = sorted(t for t in os.listdir(os.path.join(d, "tests")) if t.startswith("test_oracle_"))
    r = subprocess.run([sys.executable, "-m", "pytest", *[f"tests/{t}" for t in tests], "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=d, capture_output=True, text=True,
                       timeout=1800, env=dict(os.environ, OMP_NUM_THREADS="1"))
    failed = [ln[7:] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return i, label, ("caught by " + failed[0].split(" - ")[0]) if r.returncode else "SURVIVED"


def main():
    sel = range(len(MUTATIONS)) if len(sys.argv) < 2 else [int(x) for x in sys.argv[1:]]
    bad = 0
    with tempfile.TemporaryDirectory() as tmp, ThreadPoolExecutor(6) as ex:
        for i, label, res in ex.map(lambda k: run(k, tmp), sel):
            why = MUTATIONS[i][4] if len(MUTATIONS[i]) > 4 else None
            if res == "SURVIVED" and why:
                res = "survives, " + why
            elif res == "SURVIVED" or res.startswith("NOT"):
                bad += 1
            print(f"{i:2d} {label:32s} {res}", flush=True)
    sys.exit(1 if bad else 0)


if __name__ == "__main__":
    main()
