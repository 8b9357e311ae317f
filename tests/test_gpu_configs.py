"""GPU runs of two of the workload configurations the method is measured on:

config 1 (Section 5.2.1, Eq. receiver_error_calc): the 1 km square at c = 1.5 km/s, 64 x 64
  squares split into 8192 right triangles, KMV2tri, a 5 Hz Ricker at the centre, 100
  receivers on the line 100 m below the top, 1.0 s at 0.9 of the Gershgorin step, no damping
  layer (natural walls). The FP32 records must match the FP64 oracle to 1e-5, and both must
  match the method-of-images Green's function within the paper's 5 % threshold.
config 3 (Section 5.1, Table gradient_verification): FWI gradient at 3 Hz with KMV3tri on
  the marine window, a start model smoothed with a 500 m Gaussian (water kept), observed
  records from the true model, checkpoints every 50 steps; the adjoint gradient through the
  torch.autograd.Function against central finite differences of J along 5 seeded directions
  at h = 1e-2 and 1e-3 of max |c|."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import analytic  # noqa: E402
from parity_util import OracleCase, rel_l2  # noqa: E402
from synth import meshes, models, signals  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as p
    p.build()
    p.load()
    return p


def test_config1_square_kmv2_records_and_green_function(pkg):
    V, C = meshes.structured_tri(64, 64)
    assert C.shape[0] == 8192
    c0, f = 1.5, 5.0
    cfun = lambda X: np.full(len(X), c0)
    probe = OracleCase(V, C, 2, cfun, 1.0, 1)
    dt = 0.9 * probe.ops.cfl_dt()
    nt = int(round(1.0 / dt))
    orc = OracleCase(V, C, 2, cfun, dt, nt)
    assert orc.mesh.N == 24833
    recs = np.stack([np.linspace(0.005, 0.995, 100), np.full(100, 0.9)], 1)
    src = np.array([0.5, 0.5])
    wav = signals.ricker_samples(f, dt, nt).astype(np.float32)
    rec_o, _ = orc.forward(src, recs, wav.astype(np.float64))
    mesh = pkg.Mesh(V, C, 2, nt, dt=dt)
    mesh.set_velocity(np.full(mesh.N, c0))
    b = pkg.Batch(mesh, src[None], recs)
    rec = torch.zeros((1, nt + 1, 100), device="cuda")
    b.forward(torch.from_numpy(wav[None]).cuda(), rec)
    rec = rec.cpu().numpy()[0]
    err = rel_l2(rec, rec_o)
    # Eq. receiver_error_calc against the image sum (trapezoid in time over 101 samples)
    step = max(1, nt // 100)
    idx = np.arange(0, nt + 1, step)
    times = idx * dt
    ex = np.stack([analytic.box_image_sum(r, src, times, c0, f, 1.0, 1.0) for r in recs], axis=1)

    def E(d):
        num = np.trapezoid(np.sum((d[idx] - ex) ** 2, axis=1), times)
        return np.sqrt(num / np.trapezoid(np.sum(ex ** 2, axis=1), times))

    print(f"config 1: N={mesh.N}, {nt} steps of {dt:.3e} s; GPU vs oracle rel-L2 {err:.3e}; "
          f"E(GPU) {E(rec):.4%}, E(oracle) {E(rec_o):.4%}")
    assert err < 1e-5
    assert E(rec) < 0.05 and abs(E(rec) - E(rec_o)) < 1e-4
    b.close()
    mesh.close()


def test_config3_gradient_against_finite_differences(pkg):
    from paper_2108_10946_gb300.autograd import misfit
    true = models.marine2d(0)
    start = models.smoothed(true, 0.5)
    f, k = 3.0, 3
    box = (6.0, 8.0, 0.0, 1.5)
    V, cells = meshes.adapted_tri(true, f, 15.0, box, seed=0, iters=10)
    lay = dict(box=[(6.2, 7.8), (-10.0, 1.3)], faces=0b1011, width=0.2,
               smax=signals.sigma_max(4.7, 0.2))
    kw = dict(box=lay["box"], layer_faces=lay["faces"], layer_width=lay["width"],
              sigma_max=lay["smax"], absorbing=True, water_speed=1.51)
    probe = pkg.Mesh(V, cells, k, 1, dt=0.0, cfl_factor=0.9, **kw)
    xg = probe.dof_coords()
    probe.set_velocity(true(xg))
    dt = probe.dt  # the true model's step, kept fixed for every c below
    probe.close()
    nt = int(round(1.5 / dt))
    m = pkg.Mesh(V, cells, k, nt, dt=dt, ckpt_stride=50, **kw)
    xg = m.dof_coords()
    m.set_velocity(true(xg))
    srcs = np.stack([np.linspace(6.4, 7.6, 4), np.full(4, 0.05)], 1)
    recs = np.stack([np.linspace(6.1, 7.9, 20), np.full(20, 0.1)], 1)
    b = pkg.Batch(m, srcs, recs)
    wav = torch.from_numpy(np.stack([signals.ricker_samples(f, dt, nt)] * 4)).float().cuda()
    obs = torch.zeros((4, nt + 1, len(recs)), device="cuda")
    b.forward(wav, obs)
    c0 = torch.tensor(start(xg), dtype=torch.float64, requires_grad=True)
    J = misfit(c0, m, b, wav, obs)
    J.backward()
    g = c0.grad.numpy()
    # seeded smooth directions supported where the gradient is not masked (below the water,
    # inside the physical domain), tapered to zero at that support's edge
    inside = (xg[:, 0] > 6.35) & (xg[:, 0] < 7.65) & (xg[:, 1] > 0.55) & (xg[:, 1] < 1.15)
    taper = np.where(inside, np.sin(np.pi * (xg[:, 0] - 6.35) / 1.3) *
                     np.sin(np.pi * (xg[:, 1] - 0.55) / 0.6), 0.0)
    rng = np.random.default_rng(3)
    cmax = float(np.max(start(xg)))
    rows = []
    for trial in range(5):
        kx, kz, ph = rng.uniform(2, 8), rng.uniform(2, 8), rng.uniform(0, 2 * np.pi)
        delta = taper * np.sin(kx * xg[:, 0] + ph) * np.cos(kz * xg[:, 1])
        an = float(delta @ g)
        for hrel in (1e-2, 1e-3):
            h = hrel * cmax
            with torch.no_grad():
                Jp = misfit(c0 + h * torch.from_numpy(delta), m, b, wav, obs).item()
                Jm = misfit(c0 - h * torch.from_numpy(delta), m, b, wav, obs).item()
            fd = (Jp - Jm) / (2 * h)
            rows.append((trial, hrel, fd, an, abs(fd - an) / abs(an)))
    print(f"config 3: N={m.N}, {nt} steps, J(start) = {J.item():.6e}")
    for trial, hrel, fd, an, rel in rows:
        print(f"  direction {trial} h = {hrel:.0e} max|c|: FD {fd:+.6e}  adjoint {an:+.6e}  rel {rel:.2e}")
    assert all(r[4] < 1e-2 for r in rows)
    b.close()
    m.close()


def test_fwi_loop_reduces_misfit_and_model_error(pkg):
    """Algorithm 1 end to end on the config-3 window: L-BFGS-B within [1, 5] km/s over the
    library's misfit and gradient (two batches of four shots) from the 500 m-smoothed start
    model. J must fall at every accepted iterate and the model error outside the masked
    water and layer must shrink."""
    from paper_2108_10946_gb300 import fwi
    true = models.marine2d(0)
    start = models.smoothed(true, 0.5)
    f, k = 3.0, 3
    box = (6.0, 8.0, 0.0, 1.5)
    V, cells = meshes.adapted_tri(true, f, 15.0, box, seed=0, iters=10)
    lay = dict(box=[(6.2, 7.8), (-10.0, 1.3)], faces=0b1011, width=0.2,
               smax=signals.sigma_max(4.7, 0.2))
    kw = dict(box=lay["box"], layer_faces=lay["faces"], layer_width=lay["width"],
              sigma_max=lay["smax"], absorbing=True, water_speed=1.51)
    probe = pkg.Mesh(V, cells, k, 1, dt=0.0, cfl_factor=0.8, **kw)
    probe.set_velocity(true(probe.dof_coords()))
    dt = probe.dt
    probe.close()
    nt = int(round(1.5 / dt))
    m = pkg.Mesh(V, cells, k, nt, dt=dt, ckpt_stride=50, **kw)
    xg = m.dof_coords()
    ct, c0 = true(xg), start(xg)
    m.set_velocity(ct)
    recs = np.stack([np.linspace(6.1, 7.9, 40), np.full(40, 0.1)], 1)
    batches, wavs, obs = [], [], []
    for xs in (np.linspace(6.3, 7.7, 4), np.linspace(6.5, 7.5, 4)):
        b = pkg.Batch(m, np.stack([xs, np.full(4, 0.05)], 1), recs)
        w = torch.from_numpy(np.stack([signals.ricker_samples(f, dt, nt)] * 4)).float().cuda()
        o = torch.zeros((4, nt + 1, len(recs)), device="cuda")
        b.forward(w, o)
        batches.append(b), wavs.append(w), obs.append(o)
    shots = fwi.ShotSet(m, batches, wavs, obs)
    c, hist = fwi.invert(shots, c0, bounds=(1.0, 5.0), maxiter=6)
    free = (ct >= 1.51) & (xg[:, 0] > 6.2) & (xg[:, 0] < 7.8) & (xg[:, 1] < 1.3)
    e0 = np.linalg.norm((c0 - ct)[free]) / np.linalg.norm(ct[free])
    e1 = np.linalg.norm((c - ct)[free]) / np.linalg.norm(ct[free])
    Js = [h["J"] for h in hist]
    print(f"FWI: J {' -> '.join(f'{j:.4e}' for j in Js)} in {shots.evaluations} evaluations; "
          f"model error {e0:.4%} -> {e1:.4%}")
    assert all(b_ <= a_ for a_, b_ in zip(Js, Js[1:]))
    assert Js[-1] < 0.7 * Js[0]
    assert e1 < e0
    assert np.all(c >= 1.0) and np.all(c <= 5.0)
    for b in batches:
        b.close()
    m.close()
