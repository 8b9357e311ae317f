"""Leapfrog forward solve, discrete adjoint and gradient, FP64 (oracle; test
infrastructure only).

State Q^n = [U^n, P^n, Y^n] (Section 3.4): U the pressure, P the auxiliary vector (one
block per direction) and Y = omega (3D only); P and Y exist only when a damping layer is
present. The recurrence is Eq. (forward3):

    A_{n+1} Q^{n+1} + A_n Q^n + A_{n-1} Q^{n-1} = F^n,     F^n = [b^n, 0, 0]

with b^n_i = w(t_n) phi_i(x_s) for a point source (Section 4.2), Q^0 = Q^{-1} = 0, and
records d^n = H U^n for n = 0..Nt.

Readings of the printed block matrices (garbled in the paper: Delta^{-2} and
(2 Delta t^{-1}) typos, M_{u,2} written for M_{u,3}, the row-2 entry of A_{n-1} in column
3, omega-row signs; a literal reading makes the P update leapfrog on a decay term, which is
unstable):

  u rows    A_{n+1} = M/dt^2 + M1/(2dt)          (central differences, Eq. Leapfrog)
            A_n     = -2M/dt^2 + M3 + K | D | M_{omega,1}
            A_{n-1} = M/dt^2 - M1/(2dt)
  P rows    A_{n+1} = M (1/dt + Psi1/2)           (damping term Crank-Nicolson,
            A_n     = D_{u,2} | M(-1/dt + Psi1/2) | -D_{omega,3}   coupling explicit)
  Y row     A_{n+1} = M/dt, A_n = -M | 0 | -M/dt  (Y^{n+1} = Y^n + dt U^n)

  M1 = M tr(Psi1) + c Mb (the Clayton-Engquist term of Appendix A), M3 = M tr(Psi3) in 3D
  and M sigma_x sigma_z in 2D (the paper's "tr Psi2" in Eq. forward2d_I vanishes for the
  traceless Psi2 and is read as det Psi1), M_{omega,1} = M det(Psi1).
  Psi1 = diag(sigma_k); Psi2_kk = sigma_k - sum_{l != k} sigma_l; Psi3_kk = prod_{l != k}
  sigma_l (from the complex coordinate stretch that yields Eqs. acoustic_pml-III with the
  paper's signs).

Adjoint (Section 3.5): with the Lagrangian L = J + sum_n Lam^n . R^n the multipliers obey
the transposed recurrence run backwards,

    A_{n+1}^T Lam^{m-1} = -dJ/dQ^m - A_n^T Lam^m - A_{n-1}^T Lam^{m+1},   Lam^{Nt} = 0,

with dJ/dU^m = H^T (d^m - dtilde^m). The u-block of Lam is the adjoint field u^dagger in
the sign convention of Eq. (acoustic_pml_adj) (source -(u - utilde)); Eq.
(acoustic_pml_FEM_adj) prints the opposite source sign, and the finite-difference check
decides for this one.

Gradient, Eq. (gradient3): M G = sum_n int 2 c grad u^dagger(t_n) . grad u(t_n) delta c,
evaluated with the KMV rule (c and the integrand sampled at the nodes), no dt factor
(Section 3.5). Away from the boundary and the damping layer this is the exact derivative of
the discrete J; the layer and boundary terms are masked (Section 5.1).
"""
import numpy as np
import scipy.sparse as sp

from . import assemble


class Operators:
    """Assembled blocks for one mesh, velocity, time step and damping configuration.

    sigma: None (no layer) or (N, dim) nodal damping per direction.
    absorbing: include the lumped Clayton-Engquist boundary term.
    """

    def __init__(self, mesh, c, dt, sigma=None, absorbing=False):
        self.mesh, self.dt = mesh, dt
        N, d = mesh.N, mesh.dim
        c = np.asarray(c, dtype=np.float64)
        self.c = c
        self.M = assemble.lumped_mass(mesh)
        self.K = assemble.stiffness(mesh, c * c)
        self.Mb = assemble.boundary_mass(mesh) if absorbing else np.zeros(N)
        M = self.M
        layer = sigma is not None
        s = np.zeros((N, d)) if sigma is None else np.asarray(sigma, dtype=np.float64)
        self.sigma = s
        trPsi1 = s.sum(1)
        if d == 2:
            m3 = s[:, 0] * s[:, 1]
            detPsi1 = None
        else:
            m3 = s[:, 0] * s[:, 1] + s[:, 0] * s[:, 2] + s[:, 1] * s[:, 2]
            detPsi1 = s[:, 0] * s[:, 1] * s[:, 2]
        M1 = M * trPsi1 + c * self.Mb
        M3 = M * m3
        Au_p = M / dt**2 + M1 / (2 * dt)
        Au_m = M / dt**2 - M1 / (2 * dt)
        Auu = sp.diags(-2 * M / dt**2 + M3) + self.K
        self.nblk = 1
        if not layer:
            self.A_plus = Au_p
            self.A_minus = Au_m
            self.A0 = Auu.tocsr()
        else:
            D, G = assemble.div_and_grad(mesh)
            self.D, self.G = D, G
            psi2 = np.stack([s[:, k] - (trPsi1 - s[:, k]) for k in range(d)], axis=1)
            blocks = [[Auu] + [D[k] for k in range(d)]]
            Ap = [Au_p]
            Am = [Au_m]
            if d == 3:
                psi3 = np.stack([np.prod(np.delete(s, k, axis=1), axis=1) for k in range(d)], axis=1)
                blocks[0].append(sp.diags(M * detPsi1))
            for k in range(d):
                row = [sp.diags(psi2[:, k] * c * c) @ G[k]]
                for l in range(d):
                    row.append(sp.diags(M * (-1.0 / dt + s[:, k] / 2)) if l == k else None)
                if d == 3:
                    row.append(-(sp.diags(psi3[:, k] * c * c) @ G[k]))
                blocks.append(row)
                Ap.append(M * (1.0 / dt + s[:, k] / 2))
                Am.append(np.zeros(N))
            if d == 3:
                blocks.append([sp.diags(-M)] + [None] * d + [sp.diags(-M / dt)])
                Ap.append(M / dt)
                Am.append(np.zeros(N))
            self.A0 = sp.bmat(blocks, format="csr")
            self.A_plus = np.concatenate(Ap)
            self.A_minus = np.concatenate(Am)
            self.nblk = len(Ap)

    # -- time stepping ------------------------------------------------------------------
    def forward(self, rhs, nt, H, store=False):
        """rhs(n) -> u-block right-hand side b^n (N,). Returns records (nt+1, R) and, if
        store, the pressure history U (nt+1, N)."""
        N = self.mesh.N
        Q_old = np.zeros(self.nblk * N)
        Q = np.zeros(self.nblk * N)
        rec = np.zeros((nt + 1, H.shape[0]))
        hist = np.zeros((nt + 1, N)) if store else None
        F = np.zeros(self.nblk * N)
        for n in range(nt):
            F[:N] = rhs(n)
            Q_new = (F - self.A0 @ Q - self.A_minus * Q_old) / self.A_plus
            Q_old, Q = Q, Q_new
            rec[n + 1] = H @ Q[:N]
            if store:
                hist[n + 1] = Q[:N]
        return rec, hist

    def adjoint(self, H, residual, U_hist=None, r=1, offset=0):
        """Backward transposed recurrence. residual = d - dtilde, (nt+1, R).
        Returns (Lam_u history (nt+1, N), gradient sum g (N,) or None). g_i is
        sum_n 2 c_i sum_{e ∋ i} w_i |J_e| grad u^dagger^n(x_i) . grad U^n(x_i).

        Subsampling (Section 3.6): with r > 1 only the time levels n = offset (mod r) enter
        the sum, each with weight r (the rectangle rule on a time grid r times coarser), so
        that only every r-th forward wavefield is needed."""
        N = self.mesh.N
        nt = residual.shape[0] - 1
        L_next = np.zeros(self.nblk * N)   # Lam^{m+1}
        L = np.zeros(self.nblk * N)        # Lam^m (Lam^{nt} = 0)
        A0T = self.A0.T.tocsr()
        hist = np.zeros((nt + 1, N))
        g = np.zeros(N) if U_hist is not None else None
        GR = self._node_gradients() if U_hist is not None else None
        rhs = np.zeros(self.nblk * N)
        for m in range(nt, 0, -1):
            rhs[:] = 0.0
            rhs[:N] = -(H.T @ residual[m])
            L_prev = (rhs - A0T @ L - self.A_minus * L_next) / self.A_plus
            L_next, L = L, L_prev
            hist[m - 1] = L[:N]
            if g is not None and (m - 1 - offset) % r == 0:
                g += r * self._integrand(GR, L[:N], U_hist[m - 1])
        return hist, g

    # -- gradient (Eq. gradient3) -------------------------------------------------------
    def _node_gradients(self):
        """Sparse maps U -> d_k U at every (element, node) pair, plus the weights
        2 c_q w_q |J_e| and the DoF of each pair."""
        mesh = self.mesh
        n, d = mesh.elem.n, mesh.dim
        B = assemble.physical_dhat(mesh, slice(0, mesh.E))  # (e, q, a, j)
        rows = np.arange(mesh.E * n).repeat(n)
        cols = np.repeat(mesh.dof[:, None, :], n, axis=1).ravel()  # (e, q, j) -> dof[e, j]
        maps = [sp.csr_matrix((B[:, :, k, :].ravel(), (rows, cols)), shape=(mesh.E * n, mesh.N))
                for k in range(d)]
        wt = (2.0 * self.c[mesh.dof] * mesh.elem.weights[None, :] * mesh.detJ[:, None]).ravel()
        return maps, wt, mesh.dof.ravel()

    def _integrand(self, GR, Ladj, U):
        maps, wt, dofs = GR
        acc = np.zeros(len(wt))
        for Gk in maps:
            acc += (Gk @ Ladj) * (Gk @ U)
        return np.bincount(dofs, weights=wt * acc, minlength=self.mesh.N)

    def gradient(self, g, mask=None):
        """G = M^{-1} g (Eq. gradient3), zeroed where mask is False."""
        G = g / self.M
        if mask is not None:
            G = np.where(mask, G, 0.0)
        return G

    # -- CFL and energy -----------------------------------------------------------------
    def cfl_dt(self):
        """dt_CFL = 2 / sqrt(rho(M^{-1}K)), rho bounded by Gershgorin (Eq. spectral)."""
        rowsum = np.asarray(abs(self.K).sum(axis=1)).ravel()
        return 2.0 / np.sqrt(np.max(rowsum / self.M))

    def energy(self, U_new, U_old):
        """Discrete energy at n+1/2 of the undamped leapfrog scheme."""
        dU = U_new - U_old
        return 0.5 * dU @ (self.M * dU) / self.dt**2 + 0.5 * U_new @ (self.K @ U_old)


def misfit(rec, rec_obs):
    """J = 1/2 sum_n sum_r (d - dtilde)^2, plain sums with no dt (Eq. l2error read as in
    Section 3.5)."""
    r = rec - rec_obs
    return 0.5 * float(np.sum(r * r))


def point_source_rhs(mesh, x_s, wavelet):
    """b^n = w(t_n) phi(x_s) (Section 4.2)."""
    b = np.asarray(assemble.point_matrix(mesh, np.atleast_2d(x_s)).todense()).ravel()
    wav = np.asarray(wavelet, dtype=np.float64)
    return lambda n: wav[n] * b
