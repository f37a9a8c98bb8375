"""The library's host-built grid tables (grid.cpp, compiled here with g++, no GPU)
against the oracle: positions, topology, geometry, TRiSK reconstruction, overlap
areas, velocity prediction and restricted-flux coefficients.  These tables are
the library's fixed inputs; the kernels only combine them."""
import os
import subprocess

import numpy as np
import pytest

from lib_mapping import LevelMap
from oracle import grid, transform, trisk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1404_0405_gb300", "csrc")
JMIN, JMAX, PATCH = 2, 5, 4


def geo_tol(j):
    """Two FP64 constructions agree to ~ulp/dx: node positions are rounded off the
    sphere by an ulp, which moves circumcentres by ~ulp/dx (dx ~ 2^-j radians)."""
    return 2e-14 * 4.0 ** j


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    out = tmp_path_factory.mktemp("host_grid")
    exe = str(out / "host_grid_dump")
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-I", CSRC, os.path.join(CSRC, "grid.cpp"),
           os.path.join(ROOT, "tests", "host_grid_dump.cpp"), "-o", exe]
    subprocess.run(cmd, check=True)
    subprocess.run([exe, str(JMIN), str(JMAX), str(PATCH), str(out)], check=True)

    def rd(name, dtype, shape=None):
        a = np.fromfile(out / name, dtype=dtype)
        return a.reshape(shape) if shape else a

    rd.exe = exe
    return rd


@pytest.mark.parametrize("patch", [1, 4, 8, 16])
def test_index_tables_in_bounds(dump, patch):
    """Every id the device gathers through lies in its array (the validator the
    library runs on each grid it builds), for every patch side; a planted
    out-of-range id is found and named."""
    ok = subprocess.run([dump.exe, "2", "6", str(patch), "--check"], capture_output=True, text=True)
    assert ok.returncode == 0 and ok.stdout.strip() == "tables ok", ok.stdout
    bad = subprocess.run([dump.exe, "2", "6", str(patch), "--check-corrupt"], capture_output=True, text=True)
    assert bad.returncode == 3 and bad.stdout.startswith("cor_i of level 6"), bad.stdout


@pytest.fixture(scope="module")
def ora():
    return grid.Hierarchy(JMIN, JMAX)


@pytest.fixture(scope="module")
def maps(dump, ora):
    m = {}
    for j in range(JMIN, JMAX + 1):
        xyz = dump(f"L{j}_xyz", np.float64, (-1, 3))
        en = dump(f"L{j}_en", np.int32, (2, -1)).T
        tn = dump(f"L{j}_tn", np.int32, (3, -1)).T
        m[j] = LevelMap(xyz, en, ora.levels[j], lib_tris=tn)
    return m


def test_topology_and_geometry(dump, ora, maps):
    for j in range(JMIN, JMAX + 1):
        L, M = ora.levels[j], maps[j]
        assert L.N == M.node.size and L.E == M.edge.size
        A = dump(f"L{j}_A_i", np.float64)
        assert np.abs(A / L.A_i[M.node] - 1).max() < geo_tol(j)
        for name, ref in (("d_e", L.d_e), ("l_e", L.l_e)):
            v = dump(f"L{j}_{name}", np.float64)
            assert np.abs(v / ref[M.edge] - 1).max() < geo_tol(j)
        Av = dump(f"L{j}_A_v", np.float64)
        assert np.abs(Av / L.A_v[M.tri] - 1).max() < geo_tol(j)
        # left triangle of each library edge is the oracle's left (same orientation) or right
        et = dump(f"L{j}_et", np.int32, (2, -1))
        left_ora = np.where(M.sign > 0, L.left[M.edge], L.right[M.edge])
        assert np.array_equal(M.tri[et[0]], left_ora)


def test_coriolis_parameters(dump, ora, maps):
    """f = 2 Omega sin(latitude) at the triangles' circumcentres (the hexagon
    vertices) and at the nodes."""
    two_omega = 2.0 * ora.omega
    for j in range(JMIN, JMAX + 1):
        L, M = ora.levels[j], maps[j]
        fv = dump(f"L{j}_f_v", np.float64)
        assert np.abs(fv - L.f_v[M.tri]).max() < geo_tol(j) * two_omega
        fn = dump(f"L{j}_f_n", np.float64)
        assert np.abs(fn - two_omega * L.xyz[M.node, 2]).max() < 1e-12 * two_omega


def test_lifting_weights(dump, ora, maps):
    """Predict weights s~_km = A_km / A_m of every odd fine node (Eq. 1) and update
    weights s_km = A_km / A_k of every coarse node over M_k (Eq. 2)."""
    for j in range(JMIN + 1, JMAX + 1):
        C, Mc, Mf = ora.levels[j - 1], maps[j - 1], maps[j]
        par = dump(f"L{j}_par", np.int32, (4, -1))
        ptw = dump(f"L{j}_ptw", np.float64, (4, -1))
        odd_lib = np.nonzero(par[0] >= 0)[0]
        r = Mf.node[odd_lib] - C.N
        K, st = ora.K[j][r], ora.Akm[j][r] / ora.Am[j][r][:, None]
        lib_par = Mf.node[par[:, odd_lib].T]
        o1, o2 = np.argsort(lib_par, axis=1), np.argsort(K, axis=1)
        rows = np.arange(r.size)[:, None]
        assert np.array_equal(lib_par[rows, o1], K[rows, o2])
        assert np.abs(ptw[:, odd_lib].T[rows, o1] - st[rows, o2]).max() < geo_tol(j)
        # update weights, coarse node by coarse node
        want = {}
        for rr in range(ora.K[j].shape[0]):
            for col in range(ora.K[j].shape[1]):
                k = int(ora.K[j][rr, col])
                want.setdefault(k, {})[C.N + rr] = ora.Akm[j][rr, col] / C.A_i[k]
        mk_i = dump(f"L{j - 1}_mk_i", np.int32, (12, -1))
        mk_w = dump(f"L{j - 1}_mk_w", np.float64, (12, -1))
        for kl in range(C.N):
            got = {int(Mf.node[m]): w for m, w in zip(mk_i[:, kl], mk_w[:, kl]) if m >= 0}
            ref = want[int(Mc.node[kl])]
            assert got.keys() == ref.keys()
            assert max(abs(got[m] - ref[m]) for m in ref) < geo_tol(j)


def test_coriolis_weights(dump, ora, maps):
    rng = np.random.default_rng(0)
    for j in range(JMIN, JMAX + 1):
        L, M = ora.levels[j], maps[j]
        F = rng.standard_normal(L.E)
        q = rng.standard_normal(L.T)
        ref = trisk.coriolis_tendency(L, F, q)
        ci = dump(f"L{j}_cor_i", np.int32, (10, -1))
        cw = dump(f"L{j}_cor_w", np.float64, (10, -1))
        et = dump(f"L{j}_et", np.int32, (2, -1))
        Fl = M.edges_to_lib(F)
        ql = q[M.tri]
        qe = 0.5 * (ql[et[0]] + ql[et[1]])
        lib = np.sum(cw * Fl[ci] * 0.5 * (qe[None, :] + qe[ci]), axis=0)
        assert np.abs(M.edges_to_ora(lib) - ref).max() < geo_tol(j) * np.abs(ref).max()


def test_overlaps_and_parents(dump, ora, maps):
    for j in range(JMIN + 1, JMAX + 1):
        L, M = ora.levels[j], maps[j]
        par = dump(f"L{j}_par", np.int32, (4, -1))
        akm = dump(f"L{j}_akm", np.float64, (4, -1))
        odd_lib = np.nonzero(par[0] >= 0)[0]
        odd_ora = M.node[odd_lib]
        assert np.all(odd_ora >= ora.levels[j - 1].N)
        r = odd_ora - ora.levels[j - 1].N
        K = ora.K[j][r]
        Ak = ora.Akm[j][r]
        lib_par = M.node[par[:, odd_lib].T]
        lib_a = akm[:, odd_lib].T
        o1, o2 = np.argsort(lib_par, axis=1), np.argsort(K, axis=1)
        rows = np.arange(r.size)[:, None]
        assert np.array_equal(lib_par[rows, o1], K[rows, o2])
        scale = ora.Am[j][r][:, None]
        assert np.abs(lib_a[rows, o1] - Ak[rows, o2]).max() / scale.max() < geo_tol(j)


def test_velocity_prediction(dump, ora, maps):
    rng = np.random.default_rng(1)
    for j in range(JMIN + 1, JMAX + 1):
        C, F = ora.levels[j - 1], ora.levels[j]
        Mc, Mf = maps[j - 1], maps[j]
        VS = transform.VelocityStencils(ora, j)
        uc = rng.standard_normal(C.E)
        ph, pi = transform.velocity_predict(VS, uc)
        vst = dump(f"L{j}_vst", np.int32, (12, -1))
        vw = dump(f"L{j}_vw", np.float64, (12, -1))
        pred = np.sum(vw * Mc.edges_to_lib(uc)[vst], axis=0)          # per library fine edge
        # interior fine edges: compare along the oracle's fine edge orientation
        fe_lib = Mf.inv_edge[VS.int_edge.ravel()]
        got = pred[fe_lib] * Mf.sign[fe_lib]
        assert np.abs(got - pi.ravel()).max() < geo_tol(j) * np.abs(pi).max()
        # halves: library half h of library coarse edge E, along the library coarse direction
        half = dump(f"L{j - 1}_half", np.int32, (2, -1))
        for h in range(2):
            Eo = Mc.edge
            sgn = Mc.sign
            ho = np.where(sgn > 0, h, 1 - h)
            ref = ph[Eo, ho] * sgn
            assert np.abs(pred[half[h]] - ref).max() < geo_tol(j) * np.abs(ph).max()


def test_restricted_flux(dump, ora, maps):
    rng = np.random.default_rng(2)
    for j in range(JMIN + 1, JMAX + 1):
        C, F = ora.levels[j - 1], ora.levels[j]
        Mc, Mf = maps[j - 1], maps[j]
        Ff = rng.standard_normal(F.E)
        c = trisk.divergence(F, Ff)
        ref = transform.restrict_flux(transform.FluxStencils(ora, j), Ff, F.l_e, c)
        fi = dump(f"L{j - 1}_rf_fi", np.int32, (12, -1))
        fw = dump(f"L{j - 1}_rf_fw", np.float64, (12, -1))
        ci = dump(f"L{j - 1}_rf_ci", np.int32, (11, -1))
        cw = dump(f"L{j - 1}_rf_cw", np.float64, (11, -1))
        lib = np.sum(fw * Mf.edges_to_lib(Ff)[fi], axis=0) + np.sum(cw * Mf.nodes_to_lib(c)[ci], axis=0)
        assert np.abs(Mc.edges_to_ora(lib) - ref).max() < geo_tol(j) * np.abs(ref).max()


def _halo_positions(p):
    """The halo slots of a tile of side p, in table order, as (kind, a, b, o): nodes
    (a, b in -1..p+1), edges o = 0, 1, 2 from (a, b) along +a, +a+b, +b (a in -1..p
    or -1..p+1, b likewise, so that both ends are in the node range), triangles t0
    (a,b),(a+1,b),(a+1,b+1) and t1 (a,b),(a+1,b+1),(a,b+1) (a, b in -1..p); each
    block row-major without the patch's own positions 0..p-1."""
    def block(A, B):
        return [(a, b) for a in range(-1, A + 1) for b in range(-1, B + 1) if not (0 <= a < p and 0 <= b < p)]
    out = [("n", a, b, 0) for a, b in block(p + 1, p + 1)]
    for o, (A, B) in enumerate([(p, p + 1), (p, p), (p + 1, p)]):
        out += [("e", a, b, o) for a, b in block(A, B)]
    for t in range(2):
        out += [("t", a, b, t) for a, b in block(p, p)]
    return out


def test_tiles_are_lattice_neighbourhoods(dump):
    """Every regular tile's halo table lays out a triangular lattice around its
    patch (Sec. 5.2): each listed edge joins the nodes at its two lattice
    positions in its stated direction, each listed triangle holds its three
    lattice nodes counter-clockwise with the stated vertex first, every node is a
    hexagon (degree 6), and the tiles near the twelve pentagons -- 40 patches per
    level once a lozenge side holds more than one patch -- are the irregular ones."""
    lay = _halo_positions(PATCH)
    p = PATCH
    for j in range(JMIN, JMAX + 1):
        xyz = dump(f"L{j}_xyz", np.float64, (-1, 3))
        en = dump(f"L{j}_en", np.int32, (2, -1)).T
        tn = dump(f"L{j}_tn", np.int32, (3, -1)).T
        irr = dump(f"L{j}_tile_irr", np.uint8)
        halo = dump(f"L{j}_tile_halo", np.int32)
        n = 2 ** j
        np_ = n // p if n >= p else 1
        npatch = 10 * np_ * np_
        assert irr.size == npatch + 1 and irr[-1] == 1
        if n <= p:   # one patch per lozenge: every tile holds pentagons
            assert irr.all()
            continue
        assert halo.size == npatch * len(lay)
        assert int(irr[:-1].sum()) == (npatch if np_ <= 2 else 40), (j, int(irr[:-1].sum()))
        halo = halo.reshape(npatch, len(lay))
        nelem = 10 * n * n
        deg = np.bincount(en.ravel(), minlength=xyz.shape[0])
        for P in np.flatnonzero(irr[:-1] == 0)[:25]:
            node = {}
            for a in range(p):
                for b in range(p):
                    node[(a, b)] = P * p * p + a * p + b
            for (kind, a, b, o), v in zip(lay, halo[P]):
                if kind == "n":
                    node[(a, b)] = int(v)
            assert all(deg[v] == 6 for v in node.values())
            step = [(1, 0), (1, 1), (0, 1)]
            for (kind, a, b, o), v in zip(lay, halo[P]):
                if kind == "e":
                    e, rev = int(v) >> 1, int(v) & 1
                    ends = (node[(a, b)], node[(a + step[o][0], b + step[o][1])])
                    assert tuple(en[e]) == (ends[::-1] if rev else ends)
                elif kind == "t":
                    t, sft = int(v) >> 2, int(v) & 3
                    loc = [(a, b), (a + 1, b), (a + 1, b + 1)] if o == 0 else [(a, b), (a + 1, b + 1), (a, b + 1)]
                    ids = [node[q] for q in loc]
                    assert [int(tn[t][(c + sft) % 3]) for c in range(3)] == ids
                    x0, x1, x2 = xyz[ids]
                    assert np.dot(np.cross(x1 - x0, x2 - x0), x0 + x1 + x2) > 0   # counter-clockwise
            # the own edges and triangles follow the element layout
            for a in range(p):
                for b in range(p):
                    el = P * p * p + a * p + b
                    for o in range(3):
                        assert tuple(en[o * nelem + el]) == (node[(a, b)], node[(a + step[o][0], b + step[o][1])])
