"""GPU tests of the systems around the hot path: the continuous-batching shot server (same
result alone and in the mix, latency bookkeeping, HBM admission) and the autograd wrapper
(gradient against central finite differences of the same misfit and against the oracle)."""
import time

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


def test_forward_segment_lanes_match_whole_records(pkg):
    """fwi_forward_segment with lanes that start their shots at different segment boundaries
    (reset bits) gives each lane the records fwi_forward_shot gives the same shot from t = 0:
    lanes are independent, and a reset lane starts from the zero state."""
    m, V, C, dt, nt = _mesh(pkg, 3, 10, T=0.4)
    # sources close enough to the receivers that every lane's record carries the direct
    # wave well above the FP32 noise of a run-to-run repeat
    srcs = np.array([[0.5, 0.6], [0.3, 0.55], [0.7, 0.65], [0.4, 0.6]])
    recs = np.array([[x, 0.85] for x in np.linspace(0.1, 0.9, 9)])
    wav = np.stack([signals.ricker_samples(f, dt, nt, t0=0.15) for f in (6.0, 7.0, 8.0, 9.0)])
    wav = wav.astype(np.float32)
    ref = np.zeros((4, nt + 1, len(recs)), np.float32)
    b = pkg.Batch(m, srcs, recs)
    b.forward(wav, ref)
    nseg = 17
    start = [0, 1, 3, 4]  # segment index at which each lane starts its shot
    out = np.zeros_like(ref)
    w = np.zeros((4, nseg), np.float32)
    rec = np.zeros((4, nseg + 1, len(recs)), np.float32)
    c = 0
    while True:
        w[:] = 0.0
        reset, live = 0, False
        for s in range(4):
            t = (c - start[s]) * nseg
            if c == start[s]:
                reset |= 1 << s
            if 0 <= t < nt:
                live = True
                seg = wav[s, t:t + nseg]
                w[s, :len(seg)] = seg
        if not live:
            break
        b.forward_segment(nseg, reset, w, rec)
        for s in range(4):
            t = (c - start[s]) * nseg
            if 0 <= t < nt:
                n = min(nseg, nt - t)
                out[s, t:t + n + 1] = rec[s, :n + 1]
        c += 1
    for s in range(4):
        err = rel_l2(out[s], ref[s])
        print(f"lane {s} (starts at step {start[s] * nseg}): segments vs whole record rel-L2 {err:.3e}")
        assert err < 1e-6
    b.close()
    m.close()


def test_server_result_same_alone_and_in_the_mix(pkg):
    """A forward request and a gradient request give the same records, gradient and misfit
    alone (one-shot batches through the library) and inside a mixed stream served by the
    continuous-batching server (rolling forward batches with admission every 20 steps,
    gradient batches with per-shot gradients, two meshes, two workers)."""
    from paper_2108_10946_gb300.serving import Request, ShotServer
    recs = np.array([[x, 0.85] for x in np.linspace(0.1, 0.9, 9)])
    m2, *_ = _mesh(pkg, 2, 12, T=3.0)  # a long record: later requests arrive during it
    m3, *_ = _mesh(pkg, 3, 10)
    meshes_ = {"a": (m2, recs), "b": (m3, recs)}
    rng = np.random.default_rng(0)

    def wavelet(mesh, f):
        return signals.ricker_samples(f, mesh.dt, mesh.nsteps, t0=1.2 / f).astype(np.float32)

    src_f, src_g = np.array([0.5, 0.3]), np.array([0.4, 0.2])
    wav_f, wav_g = wavelet(m2, 8.0), wavelet(m2, 7.0)
    obs_g = (0.5 * rng.standard_normal((m2.nsteps + 1, len(recs))) * 1e-3).astype(np.float32)
    # alone: one-shot batches straight through the library
    b = pkg.Batch(m2, src_f[None], recs)
    rec_alone = np.zeros((1, m2.nsteps + 1, len(recs)), np.float32)
    b.forward(wav_f[None], rec_alone)
    b.close()
    b = pkg.Batch(m2, src_g[None], recs)
    b.set_gradient_lanes(True)
    rec_g = np.zeros((1, m2.nsteps + 1, len(recs)), np.float32)
    b.forward(wav_g[None], rec_g)
    b.adjoint_misfit(obs_g[None])
    G_alone = np.zeros((1, m2.N))
    J_alone = b.gradient_lanes(G_alone)[0]
    b.close()
    # in the mix: three forward requests on mesh a, submitted together, start a rolling batch
    # of four lanes; the forward target arrives while they are part way through their record
    # and joins the free lane
    srv = ShotServer(meshes_, hbm_budget_bytes=8 << 30, max_batch=4, workers=2, segment=20)
    reqs = []

    def request(i, name, obs=False):
        mesh = m2 if name == "a" else m3
        src = [rng.uniform(0.2, 0.8), rng.uniform(0.1, 0.4)]
        o = np.zeros((mesh.nsteps + 1, len(recs)), np.float32) if obs else None
        return Request(i, name, src, wavelet(mesh, rng.uniform(6, 9)), observed=o)

    def submit(i, name, obs=False):
        reqs.append(srv.submit(request(i, name, obs)))

    reqs.extend(srv.submit_many([request(i, "a") for i in (1, 2, 3)]))
    t0 = time.perf_counter()
    while reqs[0].start is None and time.perf_counter() - t0 < 60:
        time.sleep(0.001)
    time.sleep(0.003)
    tf = srv.submit(Request(98, "a", src_f, wav_f))
    for i in range(4, 15):
        submit(i, "a" if i % 3 else "b", obs=i % 4 == 1)
        if i == 8:
            tg = srv.submit(Request(99, "a", src_g, wav_g, observed=obs_g))
    for r in reqs + [tf, tg]:
        assert r.event.wait(300)
        assert r.error is None, r.error
    st = srv.stats()
    srv.close()
    err_f = rel_l2(tf.records, rec_alone[0])
    err_g = rel_l2(tg.gradient, G_alone[0])
    err_r = rel_l2(tg.records, rec_g[0])
    print(f"alone vs in the mix: forward records rel-L2 {err_f:.3e} (admitted mid-record: "
          f"{tf.mid_record}); gradient rel-L2 {err_g:.3e}, records {err_r:.3e}, J {tg.misfit:.9e} "
          f"vs {J_alone:.9e}; stats {st}")
    assert err_f < 1e-5 and err_r < 1e-5
    assert err_g < 1e-5 and abs(tg.misfit - J_alone) <= 1e-6 * J_alone
    assert st["shots"] == 16 and st["p99_s"] >= st["p50_s"] > 0
    assert tf.mid_record and st["admitted_mid_record"] > 0


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
