"""Maps between the library's grid order and the oracle's (tests only).

The two sides build the same nested grid independently and number it
differently; nodes are matched by position, edges and triangles by their nodes,
and an edge's velocity sign by its orientation."""
import numpy as np
from scipy.spatial import cKDTree


class LevelMap:
    """lib -> oracle maps of one level.

    node[i_lib] = i_ora;  edge[e_lib] = e_ora with sign[e_lib] = +1 when both
    sides orient the edge the same way;  tri[t_lib] = t_ora (when given)."""

    def __init__(self, lib_xyz, lib_edges, ora_level, lib_tris=None):
        L = ora_level
        d, idx = cKDTree(L.xyz).query(lib_xyz)
        assert d.max() < 1e-12, f"node positions differ by {d.max()}"
        assert np.unique(idx).size == idx.size
        self.node = idx
        self.inv_node = np.empty_like(idx)
        self.inv_node[idx] = np.arange(idx.size)
        a, b = idx[lib_edges[:, 0]], idx[lib_edges[:, 1]]
        key = np.minimum(a, b) * L.N + np.maximum(a, b)
        okey = L.edges[:, 0] * L.N + L.edges[:, 1]
        order = np.argsort(okey)
        pos = np.searchsorted(okey[order], key)
        e = order[np.clip(pos, 0, okey.size - 1)]
        assert np.array_equal(okey[e], key), "edge sets differ"
        self.edge = e
        self.sign = np.where(L.edges[e, 0] == a, 1.0, -1.0)
        self.inv_edge = np.empty_like(e)
        self.inv_edge[e] = np.arange(e.size)
        self.inv_sign = np.empty_like(self.sign)
        self.inv_sign[e] = self.sign
        if lib_tris is not None:
            s = np.sort(idx[lib_tris], axis=1)
            ks = (s[:, 0] * L.N + s[:, 1]) * L.N + s[:, 2]
            so = np.sort(L.tri, axis=1)
            ko = (so[:, 0] * L.N + so[:, 1]) * L.N + so[:, 2]
            oo = np.argsort(ko)
            t = oo[np.searchsorted(ko[oo], ks)]
            assert np.array_equal(ko[t], ks), "triangle sets differ"
            self.tri = t

    # oracle-ordered arrays -> library order
    def nodes_to_lib(self, x_ora):
        return x_ora[self.node]

    def edges_to_lib(self, u_ora):
        return u_ora[self.edge] * self.sign

    # library-ordered arrays -> oracle order
    def nodes_to_ora(self, x_lib):
        return x_lib[self.inv_node]

    def edges_to_ora(self, u_lib):
        return u_lib[self.inv_edge] * self.inv_sign


def lib_edge_geometry(xyz, edges):
    """Midpoints and unit tangents (origin -> end) of the library's edges."""
    a, b = xyz[edges[:, 0]], xyz[edges[:, 1]]
    m = a + b
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    t = b - a
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return m, t
