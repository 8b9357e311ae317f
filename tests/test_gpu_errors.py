"""Error paths of the library on the GPU, through the C ABI. None of them faults the GPU:
a time step above the stability limit only grows the wavefield to Inf (the kernels flag
the non-finite value and the call returns FWI_ERANGE); an oversized batch only fails a
cudaMalloc (FWI_ENOMEM). After each, the same process runs a normal solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import meshes, models, signals  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as p
    p.build()
    p.load()
    return p


def _healthy_forward(pkg, V, C, k, dt, nt=60):
    mesh = pkg.Mesh(V, C, k, nt, dt=dt, ckpt_stride=20)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    b = pkg.Batch(mesh, np.array([[0.5, 0.3]]), np.array([[0.4, 0.8], [0.6, 0.8]]))
    rec = torch.zeros((1, nt + 1, 2), device="cuda")
    b.forward(torch.from_numpy(signals.ricker_samples(8.0, dt, nt)[None]).float().cuda(), rec)
    assert torch.isfinite(rec).all() and rec.abs().max() > 0
    b.close()
    mesh.close()


@pytest.mark.parametrize("layout", [0, 1])
def test_unstable_time_step_returns_erange(pkg, layout):
    """dt at twice the Gershgorin bound of Eq. spectral: the leapfrog recurrence is unstable
    (its amplification factor exceeds 1 for the highest modes) and the wavefield overflows."""
    from paper_2108_10946_gb300.lib import FWI_ERANGE, FwiError
    V, C = meshes.structured_tri(10, 10)
    probe = pkg.Mesh(V, C, 2, 1, dt=0.0, cfl_factor=1.0)
    probe.set_velocity(models.smooth2d(probe.dof_coords()))
    dt_cfl = probe.dt
    probe.close()
    nt = 3000
    mesh = pkg.Mesh(V, C, 2, nt, dt=2.0 * dt_cfl, ckpt_stride=100, layout=layout)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    b = pkg.Batch(mesh, np.array([[0.5, 0.3], [0.3, 0.6]]), np.array([[0.4, 0.8]]))
    wav = torch.from_numpy(np.stack([signals.ricker_samples(8.0, 2 * dt_cfl, nt)] * 2)).float().cuda()
    rec = torch.zeros((2, nt + 1, 1), device="cuda")
    with pytest.raises(FwiError, match="non-finite") as ei:
        b.forward(wav, rec)
    assert ei.value.code == FWI_ERANGE
    b.close()
    mesh.close()
    _healthy_forward(pkg, V, C, 2, 0.8 * dt_cfl)


def test_batch_beyond_device_memory_returns_enomem(pkg):
    """A batch whose checkpoints alone exceed the GPU's memory (32 shots, a checkpoint
    every step of a 2e6-step record): fwi_batch_create returns FWI_ENOMEM, frees what it had
    allocated, and the next batch is created and runs."""
    from paper_2108_10946_gb300.lib import FWI_ENOMEM, FwiError
    V, C = meshes.structured_tri(10, 10)
    nt = 2_000_000
    mesh = pkg.Mesh(V, C, 2, nt, dt=1e-4, ckpt_stride=1)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    free0, total = torch.cuda.mem_get_info()
    need = mesh.batch_bytes(32, 1)
    assert need > 1.1 * total  # the checkpoint array alone is about 328 GB
    srcs = np.column_stack([np.linspace(0.1, 0.9, 32), np.full(32, 0.3)])
    with pytest.raises(FwiError) as ei:
        pkg.Batch(mesh, srcs, np.array([[0.4, 0.8]]))
    assert ei.value.code == FWI_ENOMEM
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20  # the partial allocations were released
    mesh.close()
    probe = pkg.Mesh(V, C, 2, 1, dt=0.0, cfl_factor=0.8)
    probe.set_velocity(models.smooth2d(probe.dof_coords()))
    dt = probe.dt
    probe.close()
    _healthy_forward(pkg, V, C, 2, dt)


def test_tensor_core_wait_that_gives_up_returns_etimedout(pkg):
    """The tensor-core adjoint kernel's mbarrier waits are bounded. With the batch's limit set
    to 0 polls every first wait gives up at once: the kernel stops early (after a wait with
    the full limit for its MMAs in flight and freeing its tensor memory), the call returns
    FWI_ETIMEDOUT, and with the default limit restored the same batch gives the gradient of a
    healthy run."""
    from paper_2108_10946_gb300.lib import FWI_ETIMEDOUT, FwiError
    V, C = meshes.structured_tri(12, 12)
    probe = pkg.Mesh(V, C, 4, 1, dt=0.0, cfl_factor=0.8)
    probe.set_velocity(models.smooth2d(probe.dof_coords()))
    dt = probe.dt
    probe.close()
    nt = 120
    mesh = pkg.Mesh(V, C, 4, nt, dt=dt, ckpt_stride=20, tensor_cores=1)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    b = pkg.Batch(mesh, np.array([[0.5, 0.3], [0.3, 0.6], [0.6, 0.4], [0.4, 0.2]]),
                  np.array([[0.4, 0.8], [0.6, 0.8]]))
    wav = torch.from_numpy(np.stack([signals.ricker_samples(8.0, dt, nt)] * 4)).float().cuda()
    rec = torch.zeros((4, nt + 1, 2), device="cuda")
    G0 = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    b.forward(wav, rec)
    res = (0.1 * rec).contiguous()
    b.adjoint(res)
    b.gradient(G0)
    b.forward(wav, rec)
    b.set_wait_limit(0)
    with pytest.raises(FwiError, match="gave up") as ei:
        b.adjoint(res)
    assert ei.value.code == FWI_ETIMEDOUT
    b.set_wait_limit(-1)
    G1 = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    b.gradient(G1)  # clears what the failed call accumulated
    b.forward(wav, rec)
    b.adjoint(res)
    b.gradient(G1)
    rel = float(torch.linalg.norm(G1 - G0) / torch.linalg.norm(G0))
    print(f"gradient after the timed-out call against before: rel-L2 {rel:.2e}")
    assert rel < 1e-5  # the same computation; only the order of the atomic sums differs
    b.close()
    mesh.close()


def test_invalid_arguments_of_the_batch_calls_return_einval(pkg):
    """Host-side argument checks of the serving and gradient calls: a segment of 0 steps or
    longer than the mesh's record, a reset mask naming a lane beyond the batch, an adjoint
    before any forward solve, per-shot gradients after a summed adjoint, a gradient-mode
    change while the accumulators hold sums of the other kind. Each returns FWI_EINVAL
    before any launch, and the batch keeps working."""
    from paper_2108_10946_gb300.lib import FWI_EINVAL, FwiError
    V, C = meshes.structured_tri(8, 8)
    probe = pkg.Mesh(V, C, 2, 1, dt=0.0, cfl_factor=0.8)
    probe.set_velocity(models.smooth2d(probe.dof_coords()))
    dt = probe.dt
    probe.close()
    nt = 40
    mesh = pkg.Mesh(V, C, 2, nt, dt=dt, ckpt_stride=10)
    mesh.set_velocity(models.smooth2d(mesh.dof_coords()))
    b = pkg.Batch(mesh, np.array([[0.5, 0.3], [0.3, 0.4]]), np.array([[0.4, 0.8], [0.6, 0.8]]))
    wav = np.stack([signals.ricker_samples(8.0, dt, nt)] * 2).astype(np.float32)
    rec = np.zeros((2, nt + 1, 2), np.float32)

    def einval(call):
        with pytest.raises(FwiError) as ei:
            call()
        assert ei.value.code == FWI_EINVAL

    einval(lambda: b.adjoint(np.zeros((2, nt + 1, 2), np.float32)))  # no forward yet
    einval(lambda: b.forward_segment(0, 0, np.ascontiguousarray(wav[:, :1]), None))
    einval(lambda: b.forward_segment(nt + 1, 0, np.zeros((2, nt + 1), np.float32), None))
    einval(lambda: b.forward_segment(5, 0b100, np.ascontiguousarray(wav[:, :5]), None))  # lane 2 of 2
    b.forward(wav, rec)
    b.adjoint(0.1 * rec)
    einval(lambda: b.gradient_lanes(np.zeros((2, mesh.N))))  # the adjoint summed the shots
    b.set_gradient_lanes(True)
    b.forward(wav, rec)
    einval(lambda: b.adjoint(0.1 * rec))  # accumulators still hold the summed form
    G = np.zeros(mesh.N)
    b.gradient(G)  # clears them
    b.forward(wav, rec)
    b.adjoint(0.1 * rec)
    Gl = np.zeros((2, mesh.N))
    J = b.gradient_lanes(Gl)
    assert np.all(np.isfinite(Gl)) and np.all(J > 0)
    b.close()
    mesh.close()
