"""GPU tests of the systems around the hot path: the continuous-batching shot server (same
result alone and in the mix, latency bookkeeping, HBM admission) and the autograd wrapper
(gradient against central finite differences of the same misfit and against the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from parity_util import OracleCase, match_dofs, rel_l2  # noqa: E402
from synth import meshes, models, signals  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as p
    p.build()
    return p


def _mesh(pkg, k, n, T=0.5, layout=0, dt=None):
    V, C = meshes.structured_tri(n, n, 1.0, 1.0)
    if dt is None:
        m = pkg.Mesh(V, C, k, 1, dt=0.0, cfl_factor=0.8)
        m.set_velocity(models.smooth2d(m.dof_coords()))
        dt = m.dt
        m.close()
    nt = int(round(T / dt))
    m = pkg.Mesh(V, C, k, nt, dt=dt, layout=layout, ckpt_stride=20)
    m.set_velocity(models.smooth2d(m.dof_coords()))
    return m, V, C, dt, nt


def test_server_result_same_alone_and_in_the_mix(pkg):
    from paper_2108_10946_gb300.serving import Request, ShotServer
    recs = np.array([[x, 0.85] for x in np.linspace(0.1, 0.9, 9)])
    m2, *_ = _mesh(pkg, 2, 12)
    m3, *_ = _mesh(pkg, 3, 10)
    meshes_ = {"a": (m2, recs), "b": (m3, recs)}
    rng = np.random.default_rng(0)

    def wavelet(mesh, f):
        return signals.ricker_samples(f, mesh.dt, mesh.nsteps, t0=1.2 / f)

    # alone: one request, one-shot batch
    srv = ShotServer(meshes_, hbm_budget_bytes=8 << 30, max_batch=1, workers=1)
    alone = srv.submit(Request(0, "a", [0.5, 0.3], wavelet(m2, 8.0)))
    alone.event.wait(120)
    srv.close()
    assert alone.error is None
    # in the mix: the same request among others on two meshes, several workers and batches
    srv = ShotServer(meshes_, hbm_budget_bytes=8 << 30, max_batch=4, workers=2)
    reqs = []
    for i in range(10):
        name = "a" if i % 3 else "b"
        mesh = m2 if name == "a" else m3
        src = [rng.uniform(0.2, 0.8), rng.uniform(0.1, 0.4)]
        reqs.append(srv.submit(Request(i + 1, name, src, wavelet(mesh, rng.uniform(6, 9)))))
        if i == 4:
            target = srv.submit(Request(99, "a", [0.5, 0.3], wavelet(m2, 8.0)))
    for r in reqs + [target]:
        assert r.event.wait(300)
        assert r.error is None, r.error
    st = srv.stats()
    srv.close()
    err = rel_l2(target.records, alone.records)
    print(f"alone vs in the mix: rel-L2 {err:.3e}; stats {st}")
    assert err < 1e-5
    assert st["shots"] == 11 and st["p99_s"] >= st["p50_s"] > 0


def test_server_admission_respects_budget(pkg):
    from paper_2108_10946_gb300.serving import Request, ShotServer
    recs = np.array([[0.5, 0.85]])
    m2, *_ = _mesh(pkg, 2, 10)
    need1 = m2.batch_bytes(1, 1)
    srv = ShotServer({"a": (m2, recs)}, hbm_budget_bytes=int(1.5 * need1), max_batch=4, workers=2)
    rs = [srv.submit(Request(i, "a", [0.5, 0.3], signals.ricker_samples(8.0, m2.dt, m2.nsteps)))
          for i in range(6)]
    for r in rs:
        assert r.event.wait(300) and r.error is None
    assert srv.used <= int(1.5 * need1)  # only one one-shot batch ever fitted
    srv.close()


def test_autograd_gradient_matches_finite_differences_and_oracle(pkg):
    from paper_2108_10946_gb300.autograd import misfit
    k, n, f = 3, 10, 8.0
    m, V, C, dt, nt = _mesh(pkg, k, n, T=0.6)
    xg = m.dof_coords()
    srcs = np.array([[0.5, 0.2], [0.3, 0.25]])
    recs = np.array([[x, 0.85] for x in np.linspace(0.1, 0.9, 9)])
    batch = pkg.Batch(m, srcs, recs)
    wav = torch.from_numpy(np.stack([signals.ricker_samples(f, dt, nt)] * 2)).cuda()
    ctrue = models.smooth2d(xg) * (1 + 0.05 * np.exp(-np.sum((xg - [0.5, 0.55]) ** 2, 1) / 0.02))
    m.set_velocity(ctrue)
    obs = torch.zeros((2, nt + 1, len(recs)), device="cuda")
    batch.forward(wav, obs)
    c0 = torch.tensor(models.smooth2d(xg), dtype=torch.float64, requires_grad=True)
    J = misfit(c0, m, batch, wav, obs)
    J.backward()
    g = c0.grad.numpy()
    inside = (xg[:, 0] > 0.2) & (xg[:, 0] < 0.8) & (xg[:, 1] > 0.2) & (xg[:, 1] < 0.8)
    delta = np.where(inside, np.sin(3 * xg[:, 0]) * np.cos(2 * xg[:, 1]), 0.0)
    h = 2e-3
    with torch.no_grad():
        Jp = misfit(c0 + h * torch.from_numpy(delta), m, batch, wav, obs).item()
        Jm = misfit(c0 - h * torch.from_numpy(delta), m, batch, wav, obs).item()
    fd = (Jp - Jm) / (2 * h)
    an = float(delta @ g)
    print(f"autograd: FD {fd:.6e} vs adjoint {an:.6e} (rel {abs(fd - an) / abs(an):.2e})")
    assert abs(fd - an) < 2e-3 * abs(an)
    # against the oracle's M G (Eq. control_deriv) on the same inputs
    orc = OracleCase(V, C, k, models.smooth2d, dt, nt)
    obs_np = obs.cpu().numpy().astype(np.float64)
    res = [orc.forward(srcs[s], recs, wav[s].cpu().numpy().astype(np.float64))[0] - obs_np[s]
           for s in range(2)]
    Go = orc.gradient(list(srcs), recs, [w.astype(np.float64) for w in wav.cpu().numpy()], res)
    perm = match_dofs(orc.mesh.coords, xg, 1.0)
    err = rel_l2(g[perm], orc.ops.M * Go)
    print(f"autograd dJ/dc vs oracle M G: rel-L2 {err:.3e}")
    assert err < 1e-4
