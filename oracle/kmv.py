"""KMV mass-lumped reference elements, FP64 (oracle; test infrastructure only).

What this computes (Section 3.2, "Higher-order mass lumping", and Section 4.1): for a
degree-k Kong-Mulder-Veldhuizen (KMV) element the finite element space is P_k enriched by
bubble functions, the nodes of the nodal basis are also the points of a quadrature rule,
and integrating the mass matrix with that rule makes it diagonal.

  * Node positions: KMV2tri and KMV3tri from Fig. 2dels, KMV2tet and KMV3tet from
    Fig. 3dels. The paper does not print KMV4tri / KMV5tri nodes; here they are solved
    from the symmetric moment equations (Newton from a coarse start, then checked for
    positivity, inclusion and unisolvence) at the degree k + k' - 2 of the classical
    mass-lumping condition (7 and 10). Their node positions are not compared with the
    paper's own tables; their accuracy is pinned instead by the convergence order k + 1
    of a manufactured solution (tests/test_oracle_wave.py).
  * Weights: one weight per symmetry orbit, solved from the moment equations (exact
    integration of monomials up to the highest degree the nodes admit).
  * Space: P_k plus bubbles (b = product of barycentrics):
      tri k=2: P2 + b            (7)      tri k=3: P3 + b*P1   (12)
      tri k=4: P4 + b*P2         (18)     tri k=5: P5 + b*P4   (30)
      tet k=2: P2 + face bubbles + interior bubble                         (15)
      tet k=3: P3 + face bubbles * P1(face) + interior bubble * P1         (32)
    The node counts are those implied by the grid-density coefficients of Table gwpl and
    by the Overthrust line (G/C = 6.97/3.0) of Section 5.5; the text's "50 nodes" for
    KMV3tet conflicts with Fig. 3dels, which lists 32.
  * Nodal basis by Vandermonde inversion; derivative matrices Dhat[d][q][j] =
    d(phi_j)/d(xhat_d) at node q.
"""
import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------------------
# Polynomials in reference coordinates: dict {exponent tuple: coefficient}
# ----------------------------------------------------------------------------------------


def _pmul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(a + b for a, b in zip(ea, eb))
            out[e] = out.get(e, 0.0) + ca * cb
    return {e: c for e, c in out.items() if c != 0.0}


def _mono(e):
    return {tuple(e): 1.0}


def _bary(dim):
    """Barycentric coordinates as polynomials: lam0 = 1 - sum x, lam_i = x_i."""
    one = tuple([0] * dim)
    lam0 = {one: 1.0}
    for d in range(dim):
        e = [0] * dim
        e[d] = 1
        lam0[tuple(e)] = -1.0
    lams = [lam0]
    for d in range(dim):
        e = [0] * dim
        e[d] = 1
        lams.append(_mono(e))
    return lams


def _monomials(dim, deg, exact_degree=None):
    """All exponent tuples of total degree <= deg (or == exact_degree if given)."""
    out = []
    for e in itertools.product(range(deg + 1), repeat=dim):
        s = sum(e)
        if (exact_degree is None and s <= deg) or (exact_degree is not None and s == exact_degree):
            out.append(e)
    out.sort(key=lambda e: (sum(e), tuple(-x for x in e)))
    return out


def peval(p, X):
    """Evaluate polynomial p at points X (m, dim)."""
    X = np.asarray(X, dtype=np.float64)
    v = np.zeros(X.shape[0])
    for e, c in p.items():
        t = np.full(X.shape[0], c)
        for d, a in enumerate(e):
            if a:
                t = t * X[:, d] ** a
        v += t
    return v


def pgrad(p, X):
    """Gradient of p at points X: (m, dim)."""
    X = np.asarray(X, dtype=np.float64)
    dim = X.shape[1]
    g = np.zeros((X.shape[0], dim))
    for e, c in p.items():
        for d in range(dim):
            if e[d] == 0:
                continue
            t = np.full(X.shape[0], c * e[d])
            for dd, a in enumerate(e):
                aa = a - 1 if dd == d else a
                if aa:
                    t = t * X[:, dd] ** aa
            g[:, d] += t
    return g


def simplex_monomial_integral(e):
    """Exact integral of x^e over the reference simplex {x_i >= 0, sum x_i <= 1}:
    prod(e_i!) / (|e| + dim)!  (Dirichlet integral)."""
    dim = len(e)
    return math.prod(math.factorial(a) for a in e) / math.factorial(sum(e) + dim)


# ----------------------------------------------------------------------------------------
# Symmetry orbits of barycentric points
# ----------------------------------------------------------------------------------------


def orbit(bary):
    """All distinct permutations of a barycentric tuple, as barycentric rows."""
    seen = []
    for perm in itertools.permutations(bary):
        if not any(np.allclose(perm, s, atol=1e-14, rtol=0) for s in seen):
            seen.append(perm)
    return np.array(seen, dtype=np.float64)


def bary_to_ref(B):
    """Barycentric rows (lam0, lam1, ...) -> reference coordinates (lam1, lam2, ...)."""
    return np.asarray(B)[:, 1:].copy()


def _orbit_spec_points(spec):
    """spec: list of barycentric generator tuples -> (points, orbit index per point)."""
    pts, lab = [], []
    for i, g in enumerate(spec):
        o = orbit(g)
        pts.append(o)
        lab += [i] * len(o)
    return np.vstack(pts), np.array(lab)


def poly_integral(p):
    """Exact integral of polynomial p over the reference simplex."""
    return sum(c * simplex_monomial_integral(e) for e, c in p.items())


def solve_orbit_weights(points_ref, labels, dim, max_degree=12, tol=1e-13, space=()):
    """One weight per orbit from the moment equations sum_q w_q m(x_q) = int m, for all
    monomials m of degree <= D, together with every function of the element space
    ``space`` (the lumped mass must reproduce the integral of every basis function).
    Returns (weights per point, highest exact degree D). The weights are taken at the
    highest D whose least-squares residual is below tol.

    For all elements here but KMV2tet the space lies inside P_D and the extra rows are
    redundant; for KMV2tet the degree-3 equations leave a one-parameter family and the
    interior-bubble row fixes it (vertex 17/840, edge 32/840, face 81/840, interior
    256/840 of the volume)."""
    norbit = labels.max() + 1
    best = None
    for D in range(0, max_degree + 1):
        polys = [_mono(e) for e in _monomials(dim, D)] + list(space)
        A = np.zeros((len(polys), norbit))
        rhs = np.zeros(len(polys))
        for r, p in enumerate(polys):
            val = peval(p, points_ref)
            for o in range(norbit):
                A[r, o] = val[labels == o].sum()
            rhs[r] = poly_integral(p)
        if np.linalg.matrix_rank(A) < norbit:
            continue  # underdetermined at this degree: go higher
        w, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        res = np.max(np.abs(A @ w - rhs))
        if res < tol:
            best = (w[labels], D)
        elif best is not None:
            break
    if best is None:
        raise ValueError("no moment-exact weights for these nodes")
    return best


# ----------------------------------------------------------------------------------------
# KMV4tri / KMV5tri: Newton on the symmetric moment equations
# ----------------------------------------------------------------------------------------

# Orbit kinds for the triangle: 'v' vertex, 'm' edge midpoint, 'e' edge pair (t, 1-t, 0),
# '3' interior (a, a, 1-2a), '6' interior (a, b, 1-a-b).
_NPAR = {"v": 0, "m": 0, "e": 1, "3": 1, "6": 2}


def _gen(kind, p):
    if kind == "v":
        return (1.0, 0.0, 0.0)
    if kind == "m":
        return (0.5, 0.5, 0.0)
    if kind == "e":
        return (p[0], 1.0 - p[0], 0.0)
    if kind == "3":
        return (p[0], p[0], 1.0 - 2.0 * p[0])
    if kind == "6":
        return (p[0], p[1], 1.0 - p[0] - p[1])
    raise ValueError(kind)


def _orbit_fixed_perms(kind):
    """Permutation list giving a fixed point order for each orbit kind, so that the
    Jacobian of the moment map is smooth in the parameters."""
    if kind == "v":
        return [(0, 1, 2), (1, 0, 2), (1, 2, 0)]
    if kind == "m":
        return [(0, 1, 2), (0, 2, 1), (2, 0, 1)]
    if kind == "3":
        return [(0, 1, 2), (0, 2, 1), (2, 0, 1)]
    return list(itertools.permutations(range(3)))  # 'e', '6': 6 points


def _orbit_points_param(kind, p):
    g = np.array(_gen(kind, p))
    return np.array([g[list(pp)] for pp in _orbit_fixed_perms(kind)])


def _split_kind(kind):
    """'e' -> ('e', None) free edge pair; ('e', t) -> edge pair held fixed at t."""
    if isinstance(kind, tuple):
        return kind[0], np.array(kind[1:], dtype=np.float64)
    return kind, None


def _moment_residual_jac(kinds, x, D):
    monos = _monomials(2, D)
    exact = np.array([simplex_monomial_integral(e) for e in monos])
    r = -exact.copy()
    J = np.zeros((len(monos), len(x)))
    k = 0
    for kind in kinds:
        kind, fixed = _split_kind(kind)
        npar = 0 if fixed is not None else _NPAR[kind]
        p = fixed if fixed is not None else x[k:k + npar]
        w = x[k + npar]
        X = bary_to_ref(_orbit_points_param(kind, p))
        for r_i, e in enumerate(monos):
            m = _mono(e)
            vals = peval(m, X)
            r[r_i] += w * vals.sum()
            J[r_i, k + npar] = vals.sum()
            if npar:
                g = pgrad(m, X)  # (npts, 2)
                for j in range(npar):
                    dp = np.zeros(npar)
                    dp[j] = 1.0
                    # the orbit points are affine in the parameters: exact difference
                    dX = bary_to_ref(_orbit_points_param(kind, p + dp)) - X
                    J[r_i, k + j] = w * np.sum(g * dX)
        k += npar + 1
    return r, J


def newton_orbit_rule(kinds, params0, D, iters=60):
    """Gauss-Newton on the moment equations over the free orbit parameters and all
    weights. A kind given as a tuple (kind, value) is an orbit held at a fixed position.
    Initial weights come from a linear least-squares solve at the starting positions."""
    pts, lab = [], []
    k = 0
    for i, kind in enumerate(kinds):
        kd, fixed = _split_kind(kind)
        npar = 0 if fixed is not None else _NPAR[kd]
        p = fixed if fixed is not None else np.array(params0[k:k + npar])
        B = _orbit_points_param(kd, p)
        pts.append(bary_to_ref(B))
        lab += [i] * len(B)
        k += npar
    pts = np.vstack(pts)
    lab = np.array(lab)
    monos = _monomials(2, D)
    A = np.zeros((len(monos), len(kinds)))
    for r_i, e in enumerate(monos):
        vals = peval(_mono(e), pts)
        for o in range(len(kinds)):
            A[r_i, o] = vals[lab == o].sum()
    w0, *_ = np.linalg.lstsq(A, np.array([simplex_monomial_integral(e) for e in monos]),
                             rcond=None)
    x = []
    k = 0
    for i, kind in enumerate(kinds):
        kd, fixed = _split_kind(kind)
        npar = 0 if fixed is not None else _NPAR[kd]
        x += list(params0[k:k + npar]) + [w0[i]]
        k += npar
    x = np.array(x, dtype=np.float64)
    for _ in range(iters):
        r, J = _moment_residual_jac(kinds, x, D)
        step, *_ = np.linalg.lstsq(J, r, rcond=None)
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    r, _ = _moment_residual_jac(kinds, x, D)
    return x, float(np.max(np.abs(r)))


# Coarse starting points (two significant digits) for the Newton solves; orbit structures
# are readings (the paper does not list these elements' nodes):
#   KMV4tri: vertices, edge midpoints, one edge pair, two interior 3-orbits; the degree-7
#     equations have a unique solution.
#   KMV5tri: vertices, two edge pairs, three interior 3-orbits and one interior 6-orbit
#     (3 + 12 + 15 = 30 nodes), every position free; the moment equations up to degree
#     10 = k + k' - 2 (k' = 7, the degree of b*P4) are 14 S3-invariant conditions on 14
#     unknowns. Multistart Gauss-Newton finds one positive, unisolvent solution (the
#     same one from every start that converges); the starts below lie near it.
_KMV4_KINDS = ["v", "m", "e", "3", "3"]
_KMV4_START = [0.21, 0.42, 0.13]
_KMV4_DEGREE = 7
_KMV5_KINDS = ["v", "e", "e", "3", "3", "3", "6"]
_KMV5_START = [0.36, 0.13, 0.058, 0.46, 0.26, 0.22, 0.70]
_KMV5_DEGREE = 10


def _solved_tri_nodes(k):
    if k == 4:
        kinds, start, D = _KMV4_KINDS, _KMV4_START, _KMV4_DEGREE
    elif k == 5:
        kinds, start, D = _KMV5_KINDS, _KMV5_START, _KMV5_DEGREE
    else:
        raise ValueError(k)
    x, res = newton_orbit_rule(kinds, start, D)
    if res > 1e-13:
        raise RuntimeError(f"KMV{k}tri moment solve did not converge (residual {res:g})")
    gens = []
    kk = 0
    for kind in kinds:
        kd, fixed = _split_kind(kind)
        npar = 0 if fixed is not None else _NPAR[kd]
        gens.append(_gen(kd, fixed if fixed is not None else x[kk:kk + npar]))
        kk += npar + 1
    return gens


# ----------------------------------------------------------------------------------------
# The element
# ----------------------------------------------------------------------------------------


class KMVElement:
    """A KMV reference element.

    Attributes
      dim, k, n                dimension, degree, number of nodes
      bary (n, dim+1)          barycentric coordinates of the nodes
      nodes (n, dim)           reference coordinates
      weights (n,)             lumping weights (sum = reference volume 1/dim!)
      exact_degree             highest degree integrated exactly by (nodes, weights)
      Dhat (dim, n, n)         Dhat[d, q, j] = d phi_j / d xhat_d at node q
      facet_nodes[i]           local nodes on the facet opposite vertex i
      facet_weights[i]         lumped facet-rule weights for those nodes (sum = facet
                               reference measure: 1 in 2D, 1/2 in 3D)
      counts                   (vertex, edge, face, interior) node counts
    """

    def __init__(self, dim, k, gens, space):
        self.dim, self.k = dim, k
        B, lab = _orbit_spec_points(gens)
        order = np.argsort((B > 1e-14).sum(axis=1), kind="stable")  # vertices first
        self.bary = B[order]
        lab = lab[order]
        self.nodes = bary_to_ref(self.bary)
        self.n = len(self.nodes)
        self.weights, self.exact_degree = solve_orbit_weights(self.nodes, lab, dim, space=space)
        self.space = space
        V = np.stack([peval(p, self.nodes) for p in space], axis=1)  # V[i, m] = p_m(x_i)
        if V.shape != (self.n, self.n):
            raise ValueError(f"space dimension {V.shape[1]} != node count {self.n}")
        self.vandermonde_cond = np.linalg.cond(V)
        self.C = np.linalg.inv(V)  # phi_j = sum_m p_m C[m, j]
        G = np.stack([pgrad(p, self.nodes) for p in space], axis=2)  # (q, d, m)
        self.Dhat = np.einsum("qdm,mj->dqj", G, self.C)
        nz = (self.bary > 1e-14).sum(axis=1)
        self.counts = tuple(int((nz == c).sum()) for c in range(1, dim + 2))
        self._facets()

    def basis(self, X):
        """phi_j(X) for reference points X (m, dim) -> (m, n)."""
        P = np.stack([peval(p, X) for p in self.space], axis=1)
        return P @ self.C

    def basis_grad(self, X):
        """grad phi_j(X) -> (m, dim, n)."""
        G = np.stack([pgrad(p, X) for p in self.space], axis=2)
        return np.einsum("xdm,mj->xdj", G, self.C)

    def _facets(self):
        self.facet_nodes, self.facet_weights = [], []
        for i in range(self.dim + 1):
            on = np.where(np.abs(self.bary[:, i]) < 1e-14)[0]
            others = [j for j in range(self.dim + 1) if j != i]
            Bf = self.bary[on][:, others]  # barycentric on the facet
            # orbit labels on the facet: sorted barycentric tuple
            keys = [tuple(np.round(np.sort(b), 12)) for b in Bf]
            uniq = sorted(set(keys))
            lab = np.array([uniq.index(kk) for kk in keys])
            w, _ = solve_orbit_weights(bary_to_ref(Bf), lab, self.dim - 1)
            self.facet_nodes.append(on)
            self.facet_weights.append(w)


def _tri_space(k):
    lam = _bary(2)
    b = _pmul(_pmul(lam[0], lam[1]), lam[2])
    space = [_mono(e) for e in _monomials(2, k)]
    extra = {2: [0], 3: [1], 4: [2], 5: [3, 4]}[k]
    for deg in extra:
        for e in _monomials(2, deg, exact_degree=deg):
            space.append(_pmul(b, _mono(e)))
    return space


def _tet_space(k):
    lam = _bary(3)
    bT = _pmul(_pmul(lam[0], lam[1]), _pmul(lam[2], lam[3]))
    space = [_mono(e) for e in _monomials(3, k)]
    for i in range(4):
        f = [j for j in range(4) if j != i]
        bF = _pmul(_pmul(lam[f[0]], lam[f[1]]), lam[f[2]])
        if k == 2:
            space.append(bF)
        else:
            space.append(_pmul(bF, lam[f[0]]))
            space.append(_pmul(bF, lam[f[1]]))
    if k == 2:
        space.append(bT)
    else:
        for j in range(4):
            space.append(_pmul(bT, lam[j]))
    return space


def kmv_tri(k):
    """KMVktri for k = 2..5."""
    if k == 2:  # Fig. 2dels, KMV2tri: vertices, edge midpoints, centroid
        gens = [(1.0, 0.0, 0.0), (0.5, 0.5, 0.0), (1 / 3, 1 / 3, 1 / 3)]
    elif k == 3:  # Fig. 2dels, KMV3tri node coordinates
        t = 0.2934695559090401
        a = 0.2073451756635909
        gens = [(1.0, 0.0, 0.0), (t, 1.0 - t, 0.0), (a, a, 1.0 - 2.0 * a)]
    elif k in (4, 5):
        gens = [(1.0, 0.0, 0.0)] + _solved_tri_nodes(k)[1:]
    else:
        raise ValueError("KMV triangles are supported for k = 2..5")
    return KMVElement(2, k, gens, _tri_space(k))


def kmv_tet(k):
    """KMVktet for k = 2, 3 (Fig. 3dels)."""
    if k == 2:
        gens = [(1.0, 0, 0, 0), (0.5, 0.5, 0, 0), (1 / 3, 1 / 3, 1 / 3, 0), (0.25, 0.25, 0.25, 0.25)]
    elif k == 3:
        t = 0.314210342418033
        a = 0.21548220313557542
        gens = [(1.0, 0, 0, 0), (t, 1.0 - t, 0, 0), (a, a, 1.0 - 2.0 * a, 0),
                (1 / 6, 1 / 6, 1 / 6, 0.5)]
    else:
        raise ValueError("KMV tetrahedra are supported for k = 2, 3")
    return KMVElement(3, k, gens, _tet_space(k))


def kmv(dim, k):
    return kmv_tri(k) if dim == 2 else kmv_tet(k)
