"""The allocation-free forward entry point (fwi_forward_shot_noalloc) against the regular
fwi_forward_shot on the same batch and inputs, on two calls in a row.

Callers that cannot allocate device memory while they run (a service that reserves its
device memory budget at start-up, or a process whose device memory comes from an allocator
the library cannot call) use this entry point; its scratch is a static device array shared
by all calls. This file is collected last so that a failure here comes after every other
test has run."""
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
    outs = [torch.full((2, nt + 1, len(recs)), float("nan"), device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        free_before, _ = torch.cuda.mem_get_info()
        batch.forward_noalloc(wav, outs[call])
        free_after, _ = torch.cuda.mem_get_info()
        if call == 1:  # the first call on the device may load modules; the second allocates nothing
            assert free_after == free_before
        out = outs[call].cpu().numpy()
        for s in range(2):
            err = rel_l2(out[s], ref[s])
            print(f"layout={layout} call {call} shot {s}: rel-L2 vs fwi_forward_shot = {err:.3e}")
            assert err < TOL


def test_noalloc_refuses_a_batch_beyond_its_static_scratch():
    """The static scratch holds 4 Mi floats: a plain-layout batch with 32 shots over ~144k
    shared DoFs needs more, and the call returns FWI_EINVAL before launching anything; the
    regular forward still runs on that batch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as pkg
    from paper_2108_10946_gb300.lib import FWI_EINVAL, FwiError
    pkg.build()
    n, nt = 190, 4
    V, C = meshes.structured_tri(n, n)
    mesh = pkg.Mesh(V, C, 2, nt, dt=1e-4, layout=1, ckpt_stride=4)
    mesh.set_velocity(np.full(mesh.N, 1.5))
    shared = mesh.N - C.shape[0]  # KMV2tri: one interior DoF per element
    assert shared * 32 > 4 << 20
    srcs = np.column_stack([np.linspace(0.1, 0.9, 32), np.full(32, 0.3)])
    batch = pkg.Batch(mesh, srcs, np.array([[0.5, 0.8]]))
    wav = torch.zeros((32, nt), device="cuda")
    out = torch.zeros((32, nt + 1, 1), device="cuda")
    with pytest.raises(FwiError, match="static scratch") as ei:
        batch.forward_noalloc(wav, out)
    assert ei.value.code == FWI_EINVAL
    batch.forward(wav, out)
    batch.close()
    mesh.close()
