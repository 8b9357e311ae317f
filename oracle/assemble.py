"""Global operators of Appendix A, assembled as FP64 sparse matrices (oracle; test
infrastructure only).

All integrals use the element's own KMV rule (nodes = quadrature points, Section 3.2), so
the mass-like matrices are diagonal and a nodal coefficient (c^2, sigma) is sampled at the
node. Notation: w_q the reference weights, |J_e| = det J_e, grad phi_j(x_q) =
J_e^{-T} Dhat[:, q, j].

  M        (M_u = M_omega = M_p^{x_k})_ii  = sum_e sum_{q -> i} w_q |J_e|
  K        K_ij = sum_e sum_q w_q |J_e| c^2(x_q) grad phi_i(x_q) . grad phi_j(x_q)
  Mb       lumped boundary mass of the Clayton-Engquist term  int_{dOmega} phi_i phi_j ds,
           with the element's facet nodes as the facet rule's points
  Dk       (D^{x_k})_ij = sum_e w_j |J_e| d_k phi_i(x_j): (D P)_i = int p . grad phi_i.
           This is the integrated-by-parts form of -int (div p) v with n . p = 0 on the
           boundary (Section 2.2 states that boundary condition for the forward problem);
           Appendix A prints the same matrix with the roles of i and j swapped.
  Gk       (G_k)_ij = sum_{e ∋ i} w_i |J_e| d_k phi_j(x_i): the lumped, mass-weighted
           gradient tested against phi_i. D_{u,2} = diag(Psi2_kk c^2) G_k and
           D_{omega,3} = diag(Psi3_kk c^2) G_k (Eq. acoustic_pml_II carries the c^2 that
           Appendix A omits). G_k = D_k^T exactly.
  H        H_rj = phi_j(x_r) in the element containing x_r (Section 4.2); the source
           vector of a point source is the same row (its transpose).
"""
import numpy as np
import scipy.sparse as sp


def lumped_mass(mesh):
    w = mesh.elem.weights[None, :] * mesh.detJ[:, None]
    return np.bincount(mesh.dof.ravel(), weights=w.ravel(), minlength=mesh.N)


def physical_dhat(mesh, e_slice):
    """grad phi_j(x_q) for elements e_slice: (E, q, d, j)."""
    return np.einsum("eab,bqj->eqaj", np.transpose(mesh.Jinv[e_slice], (0, 2, 1)),
                     mesh.elem.Dhat)


def stiffness(mesh, c2, chunk=20000):
    n = mesh.elem.n
    w = mesh.elem.weights
    rows, cols, vals = [], [], []
    for s in range(0, mesh.E, chunk):
        sl = slice(s, min(s + chunk, mesh.E))
        B = physical_dhat(mesh, sl)                      # (e, q, d, j)
        dof = mesh.dof[sl]
        coef = w[None, :] * mesh.detJ[sl, None] * c2[dof]  # (e, q)
        Ke = np.einsum("eq,eqai,eqaj->eij", coef, B, B)
        rows.append(np.repeat(dof, n, axis=1).ravel())
        cols.append(np.tile(dof, (1, n)).ravel())
        vals.append(Ke.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.N, mesh.N))


def boundary_mass(mesh):
    """Lumped int_{dOmega} phi_i phi_i ds per node (zero off the boundary)."""
    el = mesh.elem
    ref_measure = 1.0 if mesh.dim == 2 else 0.5
    Mb = np.zeros(mesh.N)
    for e, i in mesh.bfacets:
        scale = mesh.facet_measure(e, i) / ref_measure
        np.add.at(Mb, mesh.dof[e, el.facet_nodes[i]], el.facet_weights[i] * scale)
    return Mb


def div_and_grad(mesh, chunk=20000):
    """Lists D[k], G[k] (k = 0..dim-1) of sparse N x N matrices (see module docstring)."""
    n, d = mesh.elem.n, mesh.dim
    w = mesh.elem.weights
    rows, cols, vals = [], [], [[] for _ in range(d)]
    for s in range(0, mesh.E, chunk):
        sl = slice(s, min(s + chunk, mesh.E))
        B = physical_dhat(mesh, sl)                  # (e, q, a, j)
        dof = mesh.dof[sl]
        wq = w[None, :] * mesh.detJ[sl, None]        # (e, q)
        # G_k[i = node q, j] = w_q |J| d_k phi_j(x_q)
        rows.append(np.repeat(dof, n, axis=1).ravel())
        cols.append(np.tile(dof, (1, n)).ravel())
        for k in range(d):
            vals[k].append((wq[:, :, None] * B[:, :, k, :]).ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    G = [sp.csr_matrix((np.concatenate(vals[k]), (r, c)), shape=(mesh.N, mesh.N)) for k in range(d)]
    D = [g.T.tocsr() for g in G]
    return D, G


def point_matrix(mesh, points):
    """Rows phi_j(x_r) for each point (Section 4.2), as a sparse (npoints, N) matrix."""
    e, xh = mesh.locate(points)
    phi = mesh.elem.basis(xh)  # (m, n)
    n = mesh.elem.n
    rows = np.repeat(np.arange(len(points)), n)
    return sp.csr_matrix((phi.ravel(), (rows, mesh.dof[e].ravel())),
                         shape=(len(points), mesh.N))
