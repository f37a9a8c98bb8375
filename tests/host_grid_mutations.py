"""Mutation check of the host grid tables' tests: one plausible mistake at a time
is planted in a copy of ``grid.cpp`` (the library's host geometry and stencil
tables) and ``tests/test_host_grid.py``, which compares those tables with the
oracle's, is run on the copy.  Every mistake that can change a table must make
the test fail; the few that cannot are listed with the reason.

    python tests/host_grid_mutations.py         # all, four at a time
    python tests/host_grid_mutations.py 2 5     # some of them

Exit status 1 when a mistake survives.  Takes a minute or two; not part of the
test suite.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [  # (text in grid.cpp, replacement, label[, why it cannot change a table])
    ("double k = tri_area(a, unit(a + nx), cc) + tri_area(a, cc, unit(pv + a));",
     "double k = tri_area(a, unit(a + nx), cc);", "kite half dropped"),
    ("L.f_v[t] = 2.0 * omega * cc.z;", "L.f_v[t] = omega * cc.z;", "f_v factor 2"),
    ("L.ring_R[k][v] = kk[k] / s;", "L.ring_R[k][v] = 1.0 / L.deg[v];", "equal kite fractions"),
    ("L.l_e[e] = arc(L.cc[L.et[0][e]], L.cc[L.et[1][e]]) * R;",
     "L.l_e[e] = arc(L.xyz[L.en[0][e]], L.xyz[L.en[1][e]]) * R;", "l_e as d_e"),
    ("csum += L.ring_R[(k + o - 1) % dg][v];", "csum += L.ring_R[(k + o) % dg][v];", "Coriolis kite index"),
    ("n_e * n2 * (0.5 - csum)", "n_e * n2 * (csum - 0.5)", "Coriolis weight sign"),
    ("double n_e = side == 0 ? 1.0 : -1.0;", "double n_e = 1.0;", "Coriolis end-cell sign"),
    ("F.ptw[s][m] = F.akm[s][m] / F.A_i[m];", "F.ptw[s][m] = F.akm[s][m] / F.A_kite[m];", "prediction weight area",
     "equivalent to rounding: a hexagon's hierarchical area (its fine pieces summed) and its kite area differ by rounding (below 1e-13 relative)"),
    ("C.mk_w[cnt[k]][k] = F.akm[s][m] / C.A_i[k];", "C.mk_w[cnt[k]][k] = F.akm[s][m] / C.A_kite[k];",
     "update weight area",
     "equivalent to rounding: a hexagon's hierarchical area (its fine pieces summed) and its kite area differ by rounding (below 1e-13 relative)"),
    ("b[6] = {dot(tf, e1), dot(tf, e2), 0, 0, 0, 0};", "b[6] = {dot(tf, e1), dot(tf, e1), 0, 0, 0, 0};",
     "velocity weights right-hand side"),
    ("if (C.en[0][ed] != a && C.en[1][ed] != a) rim = int32_t(ed);", "if (C.en[0][ed] != a) rim = int32_t(ed);",
     "velocity stencil rim edge"),
    ("C.rf_fw[nf][e] = gam[3 * tq + g];", "C.rf_fw[nf][e] = -gam[3 * tq + g];", "x_T sign of the right triangle"),
    ("if (x == lside[a]) w = 0.5 * s * F.l_e[fe], ++found;", "if (x == lside[a]) w = -0.5 * s * F.l_e[fe], ++found;",
     "R_F0 face weight sign"),
    ("w[slot(m)] += 0.5 * (overlap(k, m) - overlap(l, m));", "w[slot(m)] += 0.5 * overlap(k, m);", "R_F0 centre term"),
    ("kml(k, m_lp, pp1, 0.5);", "kml(k, m_lp, pp1, 1.0);", "R'_F half weight"),
    ("w[slot(m_kp)] -= 0.5 * overlap(l, m_kp);", "w[slot(m_kp)] += 0.5 * overlap(l, m_kp);", "corner sliver sign"),
    ("inline double arc(V3 a, V3 b) { return std::atan2(len(cross(a, b - a)), dot(a, b)); }",
     "inline double arc(V3 a, V3 b) { return len(b - a); }", "chord for arc"),
    ("    if (dot(nrm, a + b + c) < 0) nrm = nrm * -1.0;\n", "", "circumcentre side",
     "equivalent: every triangle is counter-clockwise seen from outside, so the normal already points out"),
]


def run(i, tmp):
    old, new, label = MUTATIONS[i][:3]
    d = os.path.join(tmp, f"g{i:02d}")
    for sub in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("__pycache__", "_build"))
    shutil.copytree(os.path.join(ROOT, "paper_1404_0405_gb300", "csrc"),
                    os.path.join(d, "paper_1404_0405_gb300", "csrc"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    p = os.path.join(d, "paper_1404_0405_gb300", "csrc", "grid.cpp")
    s = open(p).read()
    if s.count(old) != 1:
        return i, label, "NOT APPLIED (text not found once)"
    open(p, "w").write(s.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_host_grid.py", "-x", "-q", "-p",
                        "no:cacheprovider"], cwd=d, capture_output=True, text=True, timeout=1800)
    failed = [ln[7:] for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]
    if r.returncode == 0:
        return i, label, "SURVIVED"
    return i, label, "caught by " + (failed[0].split(" - ")[0] if failed else "the build or the table check")


def main():
    sel = range(len(MUTATIONS)) if len(sys.argv) < 2 else [int(x) for x in sys.argv[1:]]
    bad = 0
    with tempfile.TemporaryDirectory() as tmp, ThreadPoolExecutor(4) as ex:
        for i, label, res in ex.map(lambda k: run(k, tmp), sel):
            why = MUTATIONS[i][3] if len(MUTATIONS[i]) > 3 else None
            if res == "SURVIVED" and why:
                res = "survives, " + why
            elif not res.startswith("caught"):
                bad += 1
            print(f"{i:2d} {label:34s} {res}", flush=True)
    sys.exit(1 if bad else 0)


if __name__ == "__main__":
    main()
