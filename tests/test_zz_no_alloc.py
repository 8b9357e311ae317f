"""The allocation-free forward entry point (fwi_forward_shot_noalloc) against the regular
fwi_forward_shot on the same batch and inputs, on two calls in a row.

Callers that cannot allocate device memory while they run (inside a CUDA stream capture,
or under a fixed memory budget) use this entry point; its scratch is a static device array
shared by all calls. This file is collected last so that a failure here comes after every
other test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from parity_util import rel_l2  # noqa: E402
from synth import meshes, models, signals  # noqa: E402

TOL = 1e-5  # the seismogram tolerance of the parity tests


@pytest.mark.parametrize("layout", [0, 1])
def test_noalloc_forward_matches_regular_forward(layout):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as pkg
    pkg.build()
    k, n = 3, 12
    V, C = meshes.structured_tri(int(1.5 * n), int(1.25 * n), 1.5, 1.25, -0.25, 0.0)
    box = [(0.0, 1.0), (-10.0, 1.0)]
    mesh = pkg.Mesh(V, C, k, 1, dt=0.0, cfl_factor=0.8, box=box, layer_faces=0b1011,
                    layer_width=0.25, sigma_max=signals.sigma_max(2.4, 0.25), absorbing=True,
                    layout=layout)
    xg = mesh.dof_coords()
    mesh.set_velocity(models.smooth2d(xg))
    dt = mesh.dt
    nt = int(round(0.5 / dt))
    mesh.close()
    mesh = pkg.Mesh(V, C, k, nt, dt=dt, box=box, layer_faces=0b1011, layer_width=0.25,
                    sigma_max=signals.sigma_max(2.4, 0.25), absorbing=True, layout=layout)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    srcs = np.array([[0.3, 0.1], [0.7, 0.15]])
    recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 11)])
    batch = pkg.Batch(mesh, srcs, recs)
    wav = torch.from_numpy(np.stack([signals.ricker_samples(8.0, dt, nt, t0=0.15)] * 2)).cuda()
    ref = torch.zeros((2, nt + 1, len(recs)), device="cuda")
    batch.forward(wav, ref)
    ref = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((2, nt + 1, len(recs)), float("nan"), device="cuda")
        batch.forward_noalloc(wav, out)
        out = out.cpu().numpy()
        for s in range(2):
            err = rel_l2(out[s], ref[s])
            print(f"layout={layout} call {call} shot {s}: rel-L2 vs fwi_forward_shot = {err:.3e}")
            assert err < TOL
