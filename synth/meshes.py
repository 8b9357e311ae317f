"""Seeded simplex meshes (inputs only).

  structured_tri   squares split into two right triangles (the 1 km x 1 km homogeneous
                   forward case: 64 x 64 squares, 8192 triangles)
  adapted_tri      waveform-adapted triangular mesh: edge length l_e(x) = c(x) / (C f)
                   (Eq. gpwl), gradation limited to 15 % (Section 3.3), points placed by a
                   DistMesh-style force balance (Persson & Strang) on scipy's Delaunay
  kuhn_tets        a depth-graded structured hexahedral grid, each box split into 6 Kuhn
                   tetrahedra (stand-in for a 3D waveform-adapted mesher)

Coordinates are in km; 2D points are (x, z) with z the depth (positive downward).
All cells are returned with positive orientation.
"""
import numpy as np
from scipy.spatial import Delaunay


def structured_tri(nx, ny, Lx=1.0, Ly=1.0, x0=0.0, y0=0.0):
    xs = np.linspace(x0, x0 + Lx, nx + 1)
    ys = np.linspace(y0, y0 + Ly, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = np.arange((nx + 1) * (ny + 1)).reshape(nx + 1, ny + 1)
    a = vid[:-1, :-1].ravel()
    b = vid[1:, :-1].ravel()
    c = vid[1:, 1:].ravel()
    d = vid[:-1, 1:].ravel()
    cells = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])
    return verts, cells


def orient(verts, cells):
    """Flip cells with negative signed volume."""
    cells = cells.copy()
    P = verts[cells]
    if verts.shape[1] == 2:
        det = ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
               - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    else:
        det = np.linalg.det(np.stack([P[:, i] - P[:, 0] for i in (1, 2, 3)], axis=2))
    neg = det < 0
    cells[neg, 1], cells[neg, 2] = cells[neg, 2].copy(), cells[neg, 1].copy()
    return cells


def limit_gradation(h, dx, g=0.15, iters=10000):
    """Smallest size field below h with |grad h| <= g on a regular grid (8-neighbour
    propagation h_i <- min(h_i, h_j + g |x_i - x_j|) until nothing changes)."""
    h = h.copy()
    shifts = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)]
    for _ in range(iters):
        old = h.copy()
        for sx, sy in shifts:
            dist = dx * np.hypot(sx, sy)
            nb = np.full_like(h, np.inf)
            src = h[max(0, -sx):h.shape[0] - max(0, sx), max(0, -sy):h.shape[1] - max(0, sy)]
            nb[max(0, sx):h.shape[0] - max(0, -sx), max(0, sy):h.shape[1] - max(0, -sy)] = src
            h = np.minimum(h, nb + g * dist)
        if np.array_equal(h, old):
            break
    return h


def adapted_tri(cfun, f_peak, C, box, seed=0, grid_dx=None, gradation=0.15, iters=12):
    """Waveform-adapted mesh of the rectangle box = (x0, x1, z0, z1).

    cfun(points) -> velocity (km/s); l_e = c / (C f_peak) limited to the given gradation.
    """
    rng = np.random.default_rng(seed)
    x0, x1, z0, z1 = box
    Lx, Lz = x1 - x0, z1 - z0
    # size field on a grid
    cmin_guess = float(np.min(cfun(np.stack(np.meshgrid(np.linspace(x0, x1, 64),
                                                        np.linspace(z0, z1, 64)), -1).reshape(-1, 2))))
    hmin_est = cmin_guess / (C * f_peak)
    gdx = grid_dx or hmin_est / 2
    gx = np.arange(x0, x1 + gdx, gdx)
    gz = np.arange(z0, z1 + gdx, gdx)
    GX, GZ = np.meshgrid(gx, gz, indexing="ij")
    hgrid = cfun(np.stack([GX.ravel(), GZ.ravel()], 1)).reshape(GX.shape) / (C * f_peak)
    hgrid = limit_gradation(hgrid, gdx, gradation)

    def hfun(p):
        ix = np.clip(((p[:, 0] - x0) / gdx), 0, len(gx) - 1.001)
        iz = np.clip(((p[:, 1] - z0) / gdx), 0, len(gz) - 1.001)
        i0 = ix.astype(int)
        j0 = iz.astype(int)
        fx = ix - i0
        fz = iz - j0
        return ((1 - fx) * (1 - fz) * hgrid[i0, j0] + fx * (1 - fz) * hgrid[i0 + 1, j0]
                + (1 - fx) * fz * hgrid[i0, j0 + 1] + fx * fz * hgrid[i0 + 1, j0 + 1])

    h0 = float(hgrid.min())
    # boundary points: spacing from h along each side
    def side(pa, pb):
        L = np.linalg.norm(np.subtract(pb, pa))
        ts = np.linspace(0, 1, max(2, int(L / (h0 / 4)) + 1))
        pts = np.outer(1 - ts, pa) + np.outer(ts, pb)
        inv_h = 1.0 / hfun(pts)
        s = np.concatenate([[0], np.cumsum(0.5 * (inv_h[1:] + inv_h[:-1]) * np.diff(ts) * L)])
        m = max(1, int(round(s[-1])))
        tt = np.interp(np.linspace(0, s[-1], m + 1), s, ts)
        return np.outer(1 - tt, pa) + np.outer(tt, pb)

    corners = [(x0, z0), (x1, z0), (x1, z1), (x0, z1)]
    bpts = np.vstack([side(corners[i], corners[(i + 1) % 4])[:-1] for i in range(4)])
    nb = len(bpts)
    # interior points: hexagonal lattice at spacing h0 thinned with probability (h0/h)^2
    dy = h0 * np.sqrt(3) / 2
    ys = np.arange(z0 + dy / 2, z1, dy)
    rows = []
    for j, y in enumerate(ys):
        xs = np.arange(x0 + (h0 / 2 if j % 2 else h0 / 4), x1, h0)
        rows.append(np.stack([xs, np.full_like(xs, y)], 1))
    P = np.vstack(rows)
    keep = rng.random(len(P)) < (h0 / hfun(P)) ** 2
    P = P[keep]
    margin = 0.3 * hfun(P)
    P = P[(P[:, 0] > x0 + margin) & (P[:, 0] < x1 - margin) & (P[:, 1] > z0 + margin)
          & (P[:, 1] < z1 - margin)]
    pts = np.vstack([bpts, P])
    for it in range(iters):
        tri = Delaunay(pts)
        T = tri.simplices
        bars = np.unique(np.sort(np.vstack([T[:, [0, 1]], T[:, [1, 2]], T[:, [0, 2]]]), 1), axis=0)
        vec = pts[bars[:, 0]] - pts[bars[:, 1]]
        L = np.hypot(vec[:, 0], vec[:, 1])
        hb = hfun(0.5 * (pts[bars[:, 0]] + pts[bars[:, 1]]))
        L0 = hb * 1.2 * np.sqrt(np.sum(L**2) / np.sum(hb**2))
        F = np.maximum(L0 - L, 0.0)
        Fv = (F / L)[:, None] * vec
        move = np.zeros_like(pts)
        np.add.at(move, bars[:, 0], Fv)
        np.add.at(move, bars[:, 1], -Fv)
        move[:nb] = 0.0
        pts = pts + 0.2 * move
        pts[:, 0] = np.clip(pts[:, 0], x0, x1)
        pts[:, 1] = np.clip(pts[:, 1], z0, z1)
    tri = Delaunay(pts)
    T = tri.simplices
    V = pts[T]
    area = 0.5 * np.abs((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1])
                        - (V[:, 1, 1] - V[:, 0, 1]) * (V[:, 2, 0] - V[:, 0, 0]))
    T = T[area > 1e-6 * h0 * h0]
    used = np.unique(T)
    remap = -np.ones(len(pts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    verts = pts[used]
    cells = orient(verts, remap[T])
    return verts, cells


def kuhn_tets(xs, ys, zs):
    """Boxes of the tensor grid xs x ys x zs, each split into the 6 Kuhn tetrahedra
    (all sharing the main diagonal), so that neighbouring boxes match face to face."""
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    vid = np.arange(verts.shape[0]).reshape(nx + 1, ny + 1, nz + 1)
    c = {}
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                c[(dx, dy, dz)] = vid[dx:nx + dx, dy:ny + dy, dz:nz + dz].ravel()
    tets = []
    import itertools
    for perm in itertools.permutations(range(3)):
        path = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in perm:
            cur[ax] = 1
            path.append(tuple(cur))
        tets.append(np.stack([c[p] for p in path], 1))
    cells = np.concatenate(tets)
    return verts, orient(verts, cells)
