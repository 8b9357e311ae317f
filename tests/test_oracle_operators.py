"""Pins for the oracle's global operators (Appendix A) against closed forms and
invariants: the lumped mass sums to the domain measure, stiffness rows sum to zero, K is
symmetric positive semi-definite, and the discrete operators reproduce the PDE exactly on
the polynomials the KMV rule integrates exactly (patch tests)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble, kmv, wave
from oracle import mesh as om
from synth import meshes


def _mesh2(k, n=6, perturb=0.15, seed=0):
    V, C = meshes.structured_tri(n, n, 1.0, 1.0)
    rng = np.random.default_rng(seed)
    inner = (V[:, 0] > 1e-9) & (V[:, 0] < 1 - 1e-9) & (V[:, 1] > 1e-9) & (V[:, 1] < 1 - 1e-9)
    V = V.copy()
    V[inner] += perturb / n * rng.uniform(-1, 1, (inner.sum(), 2))
    return om.Mesh(V, C, kmv.kmv_tri(k))


def _mesh3(k, n=3):
    g = np.linspace(0, 1, n + 1)
    V, C = meshes.kuhn_tets(g, g, g)
    return om.Mesh(V, C, kmv.kmv_tet(k))


CASES = [("tri", k) for k in (2, 3, 4, 5)] + [("tet", k) for k in (2, 3)]


def _mesh(kind, k):
    return _mesh2(k) if kind == "tri" else _mesh3(k)


@pytest.mark.parametrize("kind,k", CASES)
def test_mass_sums_to_measure_and_boundary_to_perimeter(kind, k):
    m = _mesh(kind, k)
    M = assemble.lumped_mass(m)
    assert abs(M.sum() - 1.0) < 1e-13
    assert np.all(M > 0)
    Mb = assemble.boundary_mass(m)
    perim = 4.0 if kind == "tri" else 6.0
    assert abs(Mb.sum() - perim) < 1e-12


@pytest.mark.parametrize("kind,k", CASES)
def test_stiffness_rowsum_symmetry_psd(kind, k):
    m = _mesh(kind, k)
    rng = np.random.default_rng(3)
    c = rng.uniform(1.5, 4.5, m.N)
    K = assemble.stiffness(m, c * c)
    scale = abs(K).max()
    assert np.abs(K @ np.ones(m.N)).max() < 1e-12 * scale * 10
    u, v = rng.standard_normal((2, m.N))
    assert abs(u @ (K @ v) - v @ (K @ u)) < 1e-12 * scale * m.N
    if m.N < 3000:
        ev = np.linalg.eigvalsh(K.toarray())
        assert ev.min() > -1e-10 * ev.max()
        assert np.sum(ev < 1e-9 * ev.max()) == 1  # constants only


def _patch_degree(kind, k):
    """Degree m of the polynomials on which M^{-1} K u = -Lap u holds at interior nodes:
    grad phi_i . grad u and phi_i Lap u must be integrated exactly, i.e.
    k' + m - 2 <= D with k' the top degree of the space and D the rule's exactness."""
    kp = {("tri", 2): 3, ("tri", 3): 4, ("tri", 4): 5, ("tri", 5): 7, ("tet", 2): 4, ("tet", 3): 5}
    D = {("tri", 2): 3, ("tri", 3): 5, ("tri", 4): 7, ("tri", 5): 10, ("tet", 2): 3, ("tet", 3): 5}
    return D[(kind, k)] - kp[(kind, k)] + 2


@pytest.mark.parametrize("kind,k", CASES)
def test_patch_test_discrete_laplacian(kind, k):
    """For u a polynomial of degree <= m (c = 1): (K u)_i = -int phi_i Lap u = -M_i Lap u
    at every interior node, because the KMV rule integrates both integrands exactly."""
    m = _mesh(kind, k)
    deg = max(1, min(_patch_degree(kind, k), k))
    rng = np.random.default_rng(4)
    monos = kmv._monomials(m.dim, deg)
    p = {e: c for e, c in zip(monos, rng.standard_normal(len(monos)))}
    u = kmv.peval(p, m.coords)
    lap = np.zeros(m.N)
    for e, cf in p.items():
        for d in range(m.dim):
            if e[d] >= 2:
                ee = list(e)
                ee[d] -= 2
                lap += cf * e[d] * (e[d] - 1) * kmv.peval({tuple(ee): 1.0}, m.coords)
    K = assemble.stiffness(m, np.ones(m.N))
    M = assemble.lumped_mass(m)
    Mb = assemble.boundary_mass(m)
    interior = Mb == 0
    lhs = (K @ u)[interior] / M[interior]
    assert np.max(np.abs(lhs + lap[interior])) < 1e-8 * max(1.0, np.abs(lap).max())


@pytest.mark.parametrize("kind,k", CASES)
def test_divergence_and_gradient_operators(kind, k):
    """(D p)_i = int p . grad phi_i = -M_i div p at interior nodes for a linear field p;
    M^{-1} G_k u = d_k u exactly for u in P_k; D_k = G_k^T."""
    m = _mesh(kind, k)
    D, G = assemble.div_and_grad(m)
    M = assemble.lumped_mass(m)
    interior = assemble.boundary_mass(m) == 0
    rng = np.random.default_rng(5)
    A = rng.standard_normal((m.dim, m.dim))
    b = rng.standard_normal(m.dim)
    P = m.coords @ A.T + b  # p(x) = A x + b, div p = trace(A)
    DP = sum(D[kk] @ P[:, kk] for kk in range(m.dim))
    assert np.max(np.abs(DP[interior] / M[interior] + np.trace(A))) < 1e-9
    monos = kmv._monomials(m.dim, k)
    p = {e: c for e, c in zip(monos, rng.standard_normal(len(monos)))}
    u = kmv.peval(p, m.coords)
    gu = kmv.pgrad(p, m.coords)
    for kk in range(m.dim):
        assert np.max(np.abs(G[kk] @ u / M - gu[:, kk])) < 1e-8
        assert abs(D[kk] - G[kk].T).max() < 1e-15


def test_gershgorin_bounds_true_spectral_radius():
    m = _mesh2(3, n=8)
    ops = wave.Operators(m, np.full(m.N, 2.0), 1.0)
    Minv = 1.0 / ops.M
    L = spla.LinearOperator((m.N, m.N), matvec=lambda x: Minv * (ops.K @ x))
    rho_true = abs(spla.eigs(L, k=1, which="LM", return_eigenvectors=False)[0])
    rho_g = (2.0 / ops.cfl_dt()) ** 2
    assert rho_g >= rho_true * (1 - 1e-10)
    assert rho_g < 4 * rho_true


def test_point_matrix_reproduces_polynomials():
    m = _mesh2(4)
    rng = np.random.default_rng(6)
    pts = rng.uniform(0.02, 0.98, (20, 2))
    H = assemble.point_matrix(m, pts)
    assert np.allclose(np.asarray(H.sum(axis=1)).ravel(), 1.0, atol=1e-12)
    monos = kmv._monomials(2, 4)
    p = {e: c for e, c in zip(monos, rng.standard_normal(len(monos)))}
    assert np.allclose(H @ kmv.peval(p, m.coords), kmv.peval(p, pts), atol=1e-10)


def test_point_location_ties_go_to_lowest_element():
    m = _mesh2(2, perturb=0.0)
    v = m.verts[m.cells[5, 0]]  # a shared vertex
    e, xh = m.locate([v])
    owners = np.where((m.cells == m.cells[5, 0]).any(axis=1))[0]
    assert e[0] == owners.min()


def test_rejects_inverted_elements():
    V, C = meshes.structured_tri(2, 2)
    C = C.copy()
    C[0, [1, 2]] = C[0, [2, 1]]
    with pytest.raises(ValueError):
        om.Mesh(V, C, kmv.kmv_tri(2))
