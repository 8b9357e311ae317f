"""Minimal full-waveform-inversion outer loop (Algorithm 1, Section 4.3): L-BFGS with bound
constraints on the wavespeed and a line search that enforces the strong Wolfe conditions
(SciPy's L-BFGS-B, the bound-constrained form of the L-BFGS method the paper runs through
ROL), over the misfit J(c) = 1/2 sum over shots, steps and receivers of (d - dtilde)^2 (Eq.
l2error) and its discrete gradient dJ/dc (Eq. gradient3 before the mass solve).

Every forward, adjoint and gradient computation runs in the CUDA library (fwi_forward_shot,
fwi_adjoint_misfit, fwi_gradient_raw); this module only sums the shot batches' J and dJ/dc on
the host and hands them to the optimizer. The velocity lives at the mesh's DoFs (library
order, Mesh.dof_coords) and the mesh must have a fixed time step, so that c changes the
operator and not the time grid.
"""
import numpy as np

from . import lib


class ShotSet:
    """The shots of an inversion as batches on one resident mesh: batches[i] a lib.Batch,
    wavelets[i] [S_i][Nt] and observed[i] [S_i][Nt+1][R] float32 arrays or tensors (host or
    device), in the layouts fwi_forward_shot and fwi_adjoint_misfit take."""

    def __init__(self, mesh, batches, wavelets, observed):
        if mesh.params.dt <= 0:
            raise ValueError("the inversion needs a mesh with a fixed time step (dt > 0)")
        if not (len(batches) == len(wavelets) == len(observed)):
            raise ValueError("one wavelet and one observed record array per batch")
        self.mesh, self.batches, self.wavelets, self.observed = mesh, batches, wavelets, observed
        self._rec = [None] * len(batches)
        self.evaluations = 0

    def misfit_and_gradient(self, c):
        """(J, dJ/dc) at velocity c [N] (host float64): every batch's forward solve, adjoint
        solve against its observed records and masked raw gradient, summed."""
        self.mesh.set_velocity(np.ascontiguousarray(c, dtype=np.float64))
        J = 0.0
        g = np.zeros(self.mesh.N)
        gi = np.zeros(self.mesh.N)
        for i, b in enumerate(self.batches):
            if self._rec[i] is None:
                self._rec[i] = np.zeros((b.S, self.mesh.nsteps + 1, b.R), dtype=np.float32)
            b.forward(self.wavelets[i], self._rec[i])
            b.adjoint_misfit(self.observed[i])
            J += b.gradient_raw(gi)
            g += gi
        self.evaluations += 1
        return J, g


def invert(shots, c0, bounds=(1.0, 5.0), maxiter=10, history_size=10, gtol=1e-12):
    """Runs L-BFGS-B from c0 within bounds (km/s; the paper bounds the wavespeed to [1, 5]
    km/s in its Marmousi2 inversions, Section 5.4). Returns (c, history) with history a list of dicts (iteration, J,
    evaluations) for c0 and every accepted iterate."""
    from scipy.optimize import minimize

    last = {}

    def fun(c):
        J, g = shots.misfit_and_gradient(c)
        last["x"], last["J"] = np.array(c, copy=True), J
        return J, g

    history = []
    J0, _ = fun(np.asarray(c0, dtype=np.float64))
    history.append({"iteration": 0, "J": J0, "evaluations": shots.evaluations})

    def cb(c):
        # the line search evaluated the accepted iterate last; evaluate only if it did not
        J = last["J"] if np.array_equal(c, last.get("x")) else fun(c)[0]
        history.append({"iteration": len(history), "J": J, "evaluations": shots.evaluations})

    res = minimize(fun, np.asarray(c0, dtype=np.float64), jac=True, method="L-BFGS-B",
                   bounds=[bounds] * len(c0), callback=cb,
                   options={"maxiter": maxiter, "maxcor": history_size, "gtol": gtol,
                            "ftol": 1e-15})
    return res.x, history


__all__ = ["ShotSet", "invert", "lib"]
