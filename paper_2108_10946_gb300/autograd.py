"""torch.autograd.Function over the misfit J(c) of a batch of shots.

forward(c) runs the forward solve (fwi_forward_shot, checkpoints every ``ckpt_stride``
steps), then the discrete adjoint against the observed records with the forward wavefield
recomputed segment by segment from the checkpoints (fwi_adjoint_misfit), which yields both
J = 1/2 sum (d - dtilde)^2 (Eq. l2error) and dJ/dc (the right-hand side of Eq. gradient3,
masked in the damping layer and the water). backward returns the saved dJ/dc scaled by the
incoming gradient. The velocity lives at the mesh's DoFs (library order, see
Mesh.dof_coords); the mesh must have been created with a fixed time step (dt > 0), so that
c changes the operator and not the time grid.

All numerical work runs in the CUDA library; this module passes pointers.
"""
import torch

from . import lib


class FWIMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, mesh, batch, wavelet, observed):
        if mesh.params.dt <= 0:
            raise ValueError("FWIMisfit needs a mesh with a fixed time step (dt > 0)")
        mesh.set_velocity(c.detach().to("cpu", torch.float64).numpy())
        rec = torch.empty((batch.S, mesh.nsteps + 1, batch.R), device="cuda", dtype=torch.float32)
        batch.forward(wavelet, rec)
        batch.adjoint_misfit(observed)
        g = torch.empty(mesh.N, device="cuda", dtype=torch.float64)
        J = batch.gradient_raw(g)
        ctx.save_for_backward(g)
        ctx.c_meta = (c.device, c.dtype)
        return torch.tensor(J, dtype=torch.float64, device=c.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        dev, dt = ctx.c_meta
        return (gJ.to(g.device) * g).to(dev, dt), None, None, None, None


def misfit(c, mesh, batch, wavelet, observed):
    """J(c) with autograd support (see FWIMisfit)."""
    return FWIMisfit.apply(c, mesh, batch, wavelet, observed)


__all__ = ["FWIMisfit", "misfit", "lib"]
