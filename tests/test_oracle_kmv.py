"""Pins for the oracle's KMV reference elements (Section 3.2, Figs. 2dels and 3dels,
Table gwpl). Every check compares with something the paper or the mathematics fixes,
not with the oracle itself."""
import math
import os

import numpy as np
import pytest

from oracle import kmv
from synth import meshes
from oracle import mesh as om

GOLD = os.path.join(os.path.dirname(__file__), "golden")

TRI = [2, 3, 4, 5]
TET = [2, 3]


def _elements():
    return [kmv.kmv_tri(k) for k in TRI] + [kmv.kmv_tet(k) for k in TET]


@pytest.fixture(scope="module")
def elements():
    return _elements()


def test_node_counts():
    assert [kmv.kmv_tri(k).n for k in TRI] == [7, 12, 18, 30][:len(TRI)]
    assert [kmv.kmv_tet(k).n for k in TET] == [15, 32]


def test_kmv2tri_is_the_textbook_seven_point_rule():
    """Vertex 1/20, edge-midpoint 2/15, centroid 9/20 of the area (the classical
    degree-3 seven-point rule; the KMV2tri nodes of Fig. 2dels)."""
    e = kmv.kmv_tri(2)
    area = 0.5
    w = dict()
    for b, wt in zip(e.bary, e.weights):
        w.setdefault(int((b > 1e-14).sum()), set()).add(round(wt / area, 14))
    assert w == {1: {round(1 / 20, 14)}, 2: {round(2 / 15, 14)}, 3: {round(9 / 20, 14)}}


def test_newton_reproduces_paper_kmv3tri_nodes():
    """The moment-equation solver used for KMV4tri/KMV5tri, started away from the answer,
    lands on the KMV3tri nodes printed in Fig. 2dels."""
    gold = {}
    for line in open(os.path.join(GOLD, "kmv_nodes_paper.txt")):
        if line.startswith("KMV3tri"):
            _, kind, v = line.split()
            gold[kind] = float(v)
    x, res = kmv.newton_orbit_rule(["v", "e", "3"], [0.25, 0.25], 5)
    assert res < 1e-14
    t = min(x[1], 1 - x[1])
    assert abs(t - gold["edge"]) < 1e-13
    assert abs(x[3] - gold["interior"]) < 1e-13


def test_paper_tet_nodes_are_used():
    gold = {}
    for line in open(os.path.join(GOLD, "kmv_nodes_paper.txt")):
        if line.startswith("KMV3tet"):
            _, kind, v = line.split()
            gold[kind] = float(v)
    e = kmv.kmv_tet(3)
    params = set(np.round(e.bary.ravel(), 12))
    for v in gold.values():
        assert round(v, 12) in params


@pytest.mark.parametrize("dim,k,degree", [(2, 2, 3), (2, 3, 5), (2, 4, 7), (2, 5, 10),
                                          (3, 2, 3), (3, 3, 5)])
def test_exactness_degree_and_positivity(dim, k, degree):
    """Brute force: integrate every monomial up to the degree with the rule and compare
    with the Dirichlet integral; the next degree must fail for at least one monomial."""
    e = kmv.kmv(dim, k)
    assert e.exact_degree == degree
    assert np.all(e.weights > 0)
    assert np.all(e.bary > -1e-14)
    for D in range(degree + 1):
        for ex in kmv._monomials(dim, D, exact_degree=D):
            approx = np.sum(e.weights * np.prod(e.nodes ** np.array(ex), axis=1))
            exact = math.prod(math.factorial(a) for a in ex) / math.factorial(sum(ex) + dim)
            assert abs(approx - exact) < 1e-13
    worst = 0.0
    for ex in kmv._monomials(dim, degree + 1, exact_degree=degree + 1):
        approx = np.sum(e.weights * np.prod(e.nodes ** np.array(ex), axis=1))
        exact = math.prod(math.factorial(a) for a in ex) / math.factorial(sum(ex) + dim)
        worst = max(worst, abs(approx - exact))
    assert worst > 1e-8


def test_kmv2tet_integrates_its_interior_bubble():
    """KMV2tet: the degree-3 equations leave one free weight; the rule must integrate the
    element's interior bubble lam0 lam1 lam2 lam3 exactly (1/7! on the reference tet)."""
    e = kmv.kmv_tet(2)
    lam = np.concatenate([1 - e.nodes.sum(1, keepdims=True), e.nodes], axis=1)
    assert abs(np.sum(e.weights * lam.prod(1)) - 1 / math.factorial(7)) < 1e-15


def test_nodal_basis_is_kronecker_and_partition_of_unity(elements):
    for e in elements:
        assert np.allclose(e.basis(e.nodes), np.eye(e.n), atol=1e-10)
        X = np.random.default_rng(1).dirichlet(np.ones(e.dim + 1), 50)[:, 1:]
        assert np.allclose(e.basis(X).sum(1), 1.0, atol=1e-11)
        assert np.allclose(e.Dhat.sum(axis=2), 0.0, atol=1e-9)


def test_polynomial_reproduction_and_exact_gradients(elements):
    """Interpolating a degree-k polynomial at the nodes reproduces it everywhere and
    Dhat gives its exact gradient at the nodes (P_k is inside every KMV space)."""
    rng = np.random.default_rng(2)
    for e in elements:
        monos = kmv._monomials(e.dim, e.k)
        coef = rng.standard_normal(len(monos))
        p = {m: c for m, c in zip(monos, coef)}
        X = rng.dirichlet(np.ones(e.dim + 1), 40)[:, 1:]
        vals = kmv.peval(p, e.nodes)
        assert np.allclose(e.basis(X) @ vals, kmv.peval(p, X), atol=1e-10)
        grad = np.einsum("dqj,j->qd", e.Dhat, vals)
        assert np.allclose(grad, kmv.pgrad(p, e.nodes), atol=1e-9)


def test_dhat_against_central_differences(elements):
    """Brute force: d phi_j / d x_d at the nodes by central differences of the basis."""
    h = 1e-6
    for e in elements:
        fd = np.zeros_like(e.Dhat)
        for d in range(e.dim):
            dx = np.zeros(e.dim)
            dx[d] = h
            fd[d] = (e.basis(e.nodes + dx) - e.basis(e.nodes - dx)) / (2 * h)
        assert np.max(np.abs(fd - e.Dhat)) < 1e-6 * max(1.0, np.max(np.abs(e.Dhat)))


def test_facet_rules(elements):
    """Lumped boundary rule on each facet: positive weights, the facet's measure, and at
    least the element's edge Simpson rule for k=2."""
    for e in elements:
        ref = 1.0 if e.dim == 2 else 0.5
        for w in e.facet_weights:
            assert np.all(w > 0)
            assert abs(w.sum() - ref) < 1e-14
    e2 = kmv.kmv_tri(2)
    assert np.allclose(np.sort(e2.facet_weights[0]), [1 / 6, 1 / 6, 4 / 6])


def _ratio(dim, k, n):
    if dim == 2:
        V, C = meshes.structured_tri(n, n)
    else:
        g = np.linspace(0, 1, n + 1)
        V, C = meshes.kuhn_tets(g, g, g)
    m = om.Mesh(V, C, kmv.kmv(dim, k))
    return m.N / m.E


def _ratio_limit(dim, k):
    """N/E on an unbounded mesh: the boundary adds O(1/n), removed by Richardson
    extrapolation from meshes of n and 2n cells per side."""
    n = 16 if dim == 2 else 3
    return 2 * _ratio(dim, k, 2 * n) - _ratio(dim, k, n)


def test_dof_per_element_matches_grid_density_table():
    """(G/C)^dim from Table gwpl and the Overthrust line equals N/E of the element on a
    large mesh (2 % allowance for the rounding of the table's three-digit G and C)."""
    for line in open(os.path.join(GOLD, "table_gwpl.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, dim, G, C = line.split()
        dim = int(dim)
        k = int(name[3])
        if dim == 2 and k not in TRI:
            continue
        expect = (float(G) / float(C)) ** dim
        got = _ratio_limit(dim, k)
        assert abs(got - expect) / expect < 0.02, (name, got, expect)
