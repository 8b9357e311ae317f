"""Mesh, DoF numbering and affine geometry, FP64 (oracle; test infrastructure only).

  * Each element maps the reference simplex affinely: x = x0 + J xhat, with the columns of
    J the edge vectors x_i - x0. Elements with det J <= 0 are rejected.
  * Global DoFs are the distinct physical node positions: a node of element e sits at
    sum_v lam_v x_v (its barycentric coordinates times the element's vertices); nodes that
    coincide (shared vertices, edges, faces) are one DoF. The KMV node sets are symmetric
    on every edge and face, so the positions of a shared node agree between neighbours up
    to rounding. This is checked against the topological count
    V + E_edges*(edge nodes) + F*(face nodes) + T*(interior nodes).
  * Point location (Section 4.2): the containing element is the lowest-numbered element
    whose barycentric coordinates at the point are all >= -1e-12.
"""
import numpy as np
from scipy.spatial import cKDTree


class Mesh:
    def __init__(self, verts, cells, elem):
        verts = np.asarray(verts, dtype=np.float64)
        cells = np.asarray(cells, dtype=np.int64)
        d = verts.shape[1]
        if cells.shape[1] != d + 1 or elem.dim != d:
            raise ValueError("cells must be simplices matching the element dimension")
        self.dim, self.elem = d, elem
        self.verts, self.cells = verts, cells
        self.E = len(cells)
        x0 = verts[cells[:, 0]]
        self.J = np.stack([verts[cells[:, j + 1]] - x0 for j in range(d)], axis=2)  # (E,d,d)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0):
            raise ValueError("element with det J <= 0 (inverted or degenerate)")
        self.Jinv = np.linalg.inv(self.J)
        # physical coordinates of every element node
        self.X = np.einsum("qv,evd->eqd", elem.bary, verts[cells])  # (E, n, d)
        scale = np.max(verts.max(0) - verts.min(0))
        key = np.round(self.X.reshape(-1, d) / (1e-9 * scale)).astype(np.int64)
        uniq, inv = np.unique(key, axis=0, return_inverse=True)
        self.dof = inv.reshape(self.E, elem.n)
        self.N = len(uniq)
        self.coords = np.zeros((self.N, d))
        self.coords[self.dof.ravel()] = self.X.reshape(-1, d)
        self._check_count()
        self._boundary_facets()

    def _check_count(self):
        d, el = self.dim, self.elem
        c = self.cells
        edges = set()
        faces = set()
        for a in range(d + 1):
            for b in range(a + 1, d + 1):
                edges.update(map(tuple, np.sort(c[:, [a, b]], axis=1)))
        nv = len(np.unique(c))
        if d == 2:
            ne_nodes = el.counts[1] // 3
            expect = nv + len(edges) * ne_nodes + self.E * el.counts[2]
        else:
            for f in ([0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]):
                faces.update(map(tuple, np.sort(c[:, f], axis=1)))
            expect = (nv + len(edges) * (el.counts[1] // 6) + len(faces) * (el.counts[2] // 4)
                      + self.E * el.counts[3])
        if expect != self.N:
            raise RuntimeError(f"DoF count {self.N} != topological count {expect}")

    def _boundary_facets(self):
        """Facets that belong to exactly one element, as (element, i) with i the local
        vertex opposite the facet."""
        d = self.dim
        F = np.concatenate([np.sort(self.cells[:, [j for j in range(d + 1) if j != i]], axis=1)
                            for i in range(d + 1)])
        owner_e = np.tile(np.arange(self.E), d + 1)
        owner_i = np.repeat(np.arange(d + 1), self.E)
        _, inv, cnt = np.unique(F, axis=0, return_inverse=True, return_counts=True)
        once = cnt[inv] == 1
        self.bfacets = list(zip(owner_e[once].tolist(), owner_i[once].tolist()))

    def facet_measure(self, e, i):
        others = [j for j in range(self.dim + 1) if j != i]
        P = self.verts[self.cells[e, others]]
        if self.dim == 2:
            return float(np.linalg.norm(P[1] - P[0]))
        return float(0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0])))

    def locate(self, points, tol=1e-12):
        """(element index, reference coordinates) of each point; raises if outside.
        Candidates are the 64 elements with the nearest centroids (every element that
        touches the point is among them on any mesh graded by at most a few times per
        element); the whole mesh is searched if none of them contains the point."""
        points = np.atleast_2d(np.asarray(points, dtype=np.float64))
        tree = cKDTree(self.verts[self.cells].mean(axis=1))
        out_e = np.empty(len(points), dtype=np.int64)
        out_x = np.empty((len(points), self.dim))
        for p_i, p in enumerate(points):
            _, cand = tree.query(p, k=min(64, self.E))
            for cands in (np.sort(np.atleast_1d(cand)), np.arange(self.E)):
                xh = np.einsum("eab,eb->ea", self.Jinv[cands], p - self.verts[self.cells[cands, 0]])
                lam = np.concatenate([1.0 - xh.sum(1, keepdims=True), xh], axis=1)
                ok = np.where(np.all(lam >= -tol, axis=1))[0]
                if len(ok):
                    out_e[p_i], out_x[p_i] = cands[ok[0]], xh[ok[0]]
                    break
            else:
                raise ValueError(f"point {p} is outside the mesh")
        return out_e, out_x
