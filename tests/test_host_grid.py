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
