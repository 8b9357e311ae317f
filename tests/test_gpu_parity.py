"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same
seeded inputs. Seismograms must agree to 1e-5 relative L2 per shot and gradients to 1e-4
(FP32 GPU vs FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from parity_util import OracleCase, match_dofs, rel_l2  # noqa: E402
from synth import meshes, models, signals  # noqa: E402

REC_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10946_gb300 as pkg
    pkg.build()
    pkg.load()
    return pkg


def _case2d(k, n=12, layer=False):
    """Unit square (plus a 0.25 km layer on the sides and bottom when layer=True)."""
    if layer:
        V, C = meshes.structured_tri(int(1.5 * n), int(1.25 * n), 1.5, 1.25, -0.25, 0.0)
        lay = dict(box=[(0.0, 1.0), (-10.0, 1.0)], faces=0b1011, width=0.25,
                   smax=signals.sigma_max(2.4, 0.25))
    else:
        V, C = meshes.structured_tri(n, n)
        lay = None
    rng = np.random.default_rng(k)
    inner = (V[:, 0] > V[:, 0].min() + 1e-9) & (V[:, 0] < V[:, 0].max() - 1e-9) & \
            (V[:, 1] > 1e-9) & (V[:, 1] < V[:, 1].max() - 1e-9)
    V = V.copy()
    V[inner] += 0.2 / n * rng.uniform(-1, 1, (inner.sum(), 2))
    return V, C, lay


# GPU forms of the time step: (layout, tensor_cores)
SIMT, TC, PLAIN = (0, -1), (0, 1), (1, 0)


def _run_both(lib, V, C, k, lay, T, srcs, recs, absorbing, grad=False, cfun=models.smooth2d,
              f=8.0, layout=0, tensor_cores=0):
    # dt from the oracle's Gershgorin estimate, passed to both sides; T long enough for the
    # direct and reflected arrivals to cross the receivers
    probe = OracleCase(V, C, k, cfun, 1.0, 1, layer=lay, absorbing=absorbing)
    dt = 0.8 * probe.ops.cfl_dt()
    nt = int(round(T / dt))
    orc = OracleCase(V, C, k, cfun, dt, nt, layer=lay, absorbing=absorbing)
    kw = {}
    if lay is not None:
        box = [tuple(b) for b in lay["box"]]
        kw = dict(box=box, layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"])
    mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=absorbing, ckpt_stride=17, layout=layout,
                    tensor_cores=tensor_cores, **kw)
    xg = mesh.dof_coords()
    perm = match_dofs(orc.mesh.coords, xg, 1.0)  # xg[perm] == oracle coords
    mesh.set_velocity(cfun(xg))
    S = len(srcs)
    wav = np.stack([signals.ricker_samples(f, dt, nt, t0=1.2 / f) for _ in range(S)])
    wav[1::2] *= -0.7
    batch = lib.Batch(mesh, np.array(srcs), np.array(recs))
    rec_gpu = torch.zeros((S, nt + 1, len(recs)), dtype=torch.float32, device="cuda")
    batch.forward(torch.from_numpy(wav).cuda(), rec_gpu)
    rec_gpu = rec_gpu.cpu().numpy()
    rec_orc = [orc.forward(srcs[s], np.array(recs), wav[s].astype(np.float64))[0] for s in range(S)]
    out = dict(rec_gpu=rec_gpu, rec_orc=rec_orc, dt=dt, mesh=mesh, orc=orc, perm=perm)
    if grad:
        ctrue = lambda X: cfun(X) * (1 + 0.05 * np.exp(-np.sum((X - X.mean(0)) ** 2, 1) / 0.02))
        obs_case = OracleCase(V, C, k, ctrue, dt, nt, layer=lay, absorbing=absorbing)
        res = np.stack([rec_orc[s] - obs_case.forward(srcs[s], np.array(recs), wav[s].astype(np.float64))[0]
                        for s in range(S)]).astype(np.float32)
        batch.adjoint(torch.from_numpy(res).cuda())
        G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
        J = batch.gradient(G)
        G = G.cpu().numpy()
        Go = orc.gradient(srcs, np.array(recs), [w.astype(np.float64) for w in wav],
                          [r.astype(np.float64) for r in res])
        out.update(G_gpu=G[perm], G_orc=Go, J=J, J_ref=0.5 * float(np.sum(res.astype(np.float64) ** 2)))
    return out


@pytest.mark.parametrize("form", [SIMT, PLAIN], ids=["chunked", "plain"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_forward_records_2d(lib, k, form):
    """Both data layouts of the forward step: chunked shared-memory assembly and plain
    global atomics."""
    V, C, lay = _case2d(k)
    srcs = [[0.5, 0.3], [0.31, 0.62]]
    recs = [[x, 0.85] for x in np.linspace(0.05, 0.95, 9)]
    o = _run_both(lib, V, C, k, lay, 0.7, srcs, recs, absorbing=False, layout=form[0],
                  tensor_cores=form[1])
    for s in range(2):
        err = rel_l2(o["rec_gpu"][s], o["rec_orc"][s])
        print(f"k={k} form={form} shot {s}: records rel-L2 = {err:.3e}")
        assert err < REC_TOL


@pytest.mark.parametrize("form", [SIMT, TC], ids=["chunked", "chunked-tc"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_forward_and_gradient_2d_layer(lib, k, form):
    V, C, lay = _case2d(k, n=12, layer=True)
    srcs = [[0.5, 0.1], [0.2, 0.15]]
    recs = [[x, 0.9] for x in np.linspace(0.05, 0.95, 11)]
    o = _run_both(lib, V, C, k, lay, 0.7, srcs, recs, absorbing=True, grad=True, layout=form[0],
                  tensor_cores=form[1])
    for s in range(2):
        err = rel_l2(o["rec_gpu"][s], o["rec_orc"][s])
        print(f"k={k} form={form} layer shot {s}: records rel-L2 = {err:.3e}")
        assert err < REC_TOL
    gerr = rel_l2(o["G_gpu"], o["G_orc"])
    print(f"k={k} form={form} layer: gradient rel-L2 = {gerr:.3e}, J {o['J']:.6e} vs {o['J_ref']:.6e}")
    assert gerr < GRAD_TOL
    assert abs(o["J"] - o["J_ref"]) < 1e-10 * abs(o["J_ref"])
    # masked entries are exactly zero on both sides
    assert np.all(o["G_gpu"][~o["orc"].mask] == 0)


@pytest.mark.parametrize("S", [1, 4, 8])
@pytest.mark.parametrize("k", [4, 5])
def test_tensor_core_step_matches_cuda_core_step(lib, k, S):
    """Shot counts the oracle cases above do not reach (one shot per CTA row group, a full
    128-row tile, two shot groups per chunk), with a damping layer, an absorbing boundary and
    chunks that straddle the layer: with tensor_cores = 1 the records are those of the FP32
    CUDA-core forward (the same kernels), and the gradient from the tensor-core adjoint
    matches the CUDA-core one (itself held to the oracle above) within the gradient bound."""
    V, C, lay = _case2d(k, n=14, layer=True)
    dt = 0.8 * OracleCase(V, C, k, models.smooth2d, 1.0, 1, layer=lay, absorbing=True).ops.cfl_dt()
    nt = int(round(0.6 / dt))
    rng = np.random.default_rng(S)
    srcs = np.column_stack([rng.uniform(0.1, 0.9, S), rng.uniform(0.05, 0.3, S)])
    recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 13)])
    wav = np.stack([signals.ricker_samples(rng.uniform(6, 9), dt, nt, t0=0.15) for _ in range(S)])
    box = [tuple(b) for b in lay["box"]]
    out = {}
    for name, tcf in (("cuda", -1), ("tc", 1)):
        mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=True, ckpt_stride=17, box=box,
                        layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"],
                        tensor_cores=tcf)
        xg = mesh.dof_coords()
        mesh.set_velocity(models.smooth2d(xg))
        batch = lib.Batch(mesh, srcs, recs)
        rec = torch.zeros((S, nt + 1, len(recs)), device="cuda")
        batch.forward(torch.from_numpy(wav).float().cuda(), rec)
        res = (0.1 * rec).contiguous()
        batch.adjoint(res)
        G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
        batch.gradient(G)
        out[name] = (rec.cpu().numpy(), G.cpu().numpy(), xg)
        batch.close()
        mesh.close()
    (rc, Gc, xc), (rt, Gt, xt) = out["cuda"], out["tc"]
    assert np.array_equal(xc, xt)
    for s in range(S):  # same kernels; only the order of shared-memory atomics differs
        err = rel_l2(rt[s], rc[s])
        print(f"k={k} S={S} shot {s}: records rel-L2 = {err:.3e}")
        assert err < 1e-6
    gerr = rel_l2(Gt, Gc)
    print(f"k={k} S={S}: tensor-core vs CUDA-core gradient rel-L2 = {gerr:.3e}")
    assert gerr < GRAD_TOL


def test_gershgorin_dt_matches_oracle(lib):
    V, C, _ = _case2d(3)
    mesh = lib.Mesh(V, C, 3, 10, dt=0.0, cfl_factor=0.8)
    xg = mesh.dof_coords()
    mesh.set_velocity(models.smooth2d(xg))
    orc = OracleCase(V, C, 3, models.smooth2d, 1.0, 1)
    assert abs(mesh.dt - 0.8 * orc.ops.cfl_dt()) < 1e-12 * mesh.dt


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("k", [2, 3])
def test_forward_and_gradient_3d_layer(lib, k, layout):
    """KMV2tet / KMV3tet with the 3D damping layer (u, p in R^3, omega) and the absorbing
    boundary: records and gradient against the oracle."""
    g = np.linspace(0.0, 1.0, 6)
    gz = np.linspace(0.0, 0.8, 5)
    V, C = meshes.kuhn_tets(g, g, gz)
    lay = dict(box=[(0.2, 0.8), (0.2, 0.8), (-10.0, 0.6)], faces=0b101111, width=0.2,
               smax=signals.sigma_max(2.2, 0.2))
    srcs = [[0.5, 0.5, 0.1], [0.4, 0.55, 0.15]]
    recs = [[x, y, 0.5] for x in (0.3, 0.5, 0.7) for y in (0.35, 0.65)]
    o = _run_both(lib, V, C, k, lay, 0.5, srcs, recs, absorbing=True, grad=True,
                  cfun=models.smooth3d, f=6.0, layout=layout)
    for s in range(2):
        err = rel_l2(o["rec_gpu"][s], o["rec_orc"][s])
        print(f"3D k={k} layout={layout} shot {s}: records rel-L2 = {err:.3e}")
        assert err < REC_TOL
    gerr = rel_l2(o["G_gpu"], o["G_orc"])
    print(f"3D k={k} layout={layout}: gradient rel-L2 = {gerr:.3e}")
    assert gerr < GRAD_TOL


@pytest.mark.parametrize("dim", [2, 3])
def test_shot_batch_of_four_matches_two_batches_of_two(lib, dim):
    """Batches whose shot count is a multiple of 4 finish the halo DoFs with one thread per
    DoF and float4 shot groups; smaller batches with one thread per (DoF, shot). The same
    four shots as one batch of 4 and as two batches of 2 (damping layer, absorbing boundary,
    gradient) must agree to FP32 summation-order noise."""
    if dim == 2:
        V, C, lay = _case2d(3, n=10, layer=True)
        k, cfun = 3, models.smooth2d
        srcs = np.array([[0.5, 0.1], [0.2, 0.15], [0.8, 0.2], [0.35, 0.3]])
        recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 9)])
    else:
        g = np.linspace(0.0, 1.0, 6)
        V, C = meshes.kuhn_tets(g, g, np.linspace(0.0, 0.8, 5))
        lay = dict(box=[(0.2, 0.8), (0.2, 0.8), (-10.0, 0.6)], faces=0b101111, width=0.2,
                   smax=signals.sigma_max(2.2, 0.2))
        k, cfun = 2, models.smooth3d
        srcs = np.array([[0.5, 0.5, 0.1], [0.4, 0.55, 0.15], [0.6, 0.45, 0.2], [0.45, 0.4, 0.12]])
        recs = np.array([[x, y, 0.5] for x in (0.3, 0.5, 0.7) for y in (0.35, 0.65)])
    box = [tuple(b) for b in lay["box"]]
    mesh = lib.Mesh(V, C, k, 1, dt=0.0, cfl_factor=0.8, box=box, layer_faces=lay["faces"],
                    layer_width=lay["width"], sigma_max=lay["smax"], absorbing=True)
    mesh.set_velocity(cfun(mesh.dof_coords()))
    dt = mesh.dt
    mesh.close()
    nt = int(round(0.5 / dt))
    mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=True, ckpt_stride=13, box=box,
                    layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"])
    mesh.set_velocity(cfun(mesh.dof_coords()))
    wav = np.stack([signals.ricker_samples(8.0, dt, nt, t0=0.15) * (1 + 0.1 * i) for i in range(4)])
    wav_d = torch.from_numpy(wav).float().cuda()

    def run(sel):
        b = lib.Batch(mesh, srcs[sel], recs)
        rec = torch.zeros((len(sel), nt + 1, len(recs)), device="cuda")
        b.forward(wav_d[sel].contiguous(), rec)
        b.adjoint((0.1 * rec).contiguous())
        G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
        b.gradient_raw(G)
        b.close()
        return rec.cpu().numpy(), G.cpu().numpy()

    r4, g4 = run([0, 1, 2, 3])
    ra, ga = run([0, 1])
    rb, gb = run([2, 3])
    r2 = np.concatenate([ra, rb])
    for s in range(4):
        err = rel_l2(r4[s], r2[s])
        print(f"dim={dim} shot {s}: batch of 4 vs batches of 2, records rel-L2 = {err:.3e}")
        assert err < 1e-6
    gerr = rel_l2(g4, ga + gb)
    print(f"dim={dim}: gradient rel-L2 = {gerr:.3e}")
    assert gerr < 1e-6


@pytest.mark.parametrize("r", [4, 10])
def test_subsampled_gradient_matches_oracle(lib, r):
    """Gradient subsampling r (Section 3.6): only the time levels n = 0 (mod r) enter Eq.
    gradient3, weight r, and the recompute ring holds ckpt_stride / r wavefields. The GPU
    gradient matches the oracle's subsampled gradient; the printout gives its departure
    from the full (r = 1) gradient and the ring's memory."""
    from oracle import assemble
    k = 3
    V, C, lay = _case2d(k, n=12, layer=True)
    cfun = models.smooth2d
    probe = OracleCase(V, C, k, cfun, 1.0, 1, layer=lay, absorbing=True)
    dt = 0.8 * probe.ops.cfl_dt()
    nt = int(round(0.7 / dt))
    orc = OracleCase(V, C, k, cfun, dt, nt, layer=lay, absorbing=True)
    srcs = np.array([[0.5, 0.1], [0.2, 0.15], [0.7, 0.2], [0.4, 0.12]])
    recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 11)])
    wav = np.stack([signals.ricker_samples(8.0, dt, nt, t0=0.15) * (1 + 0.1 * i) for i in range(4)])
    H = assemble.point_matrix(orc.mesh, recs)
    g_r = np.zeros(orc.mesh.N)
    g_1 = np.zeros(orc.mesh.N)
    recs_o = []
    for s in range(4):
        rec, U = orc.forward(srcs[s], recs, wav[s].astype(np.float64), store=True)
        recs_o.append(rec)
        res = 0.1 * rec.astype(np.float32).astype(np.float64)
        g_r += orc.ops.adjoint(H, res, U_hist=U, r=r)[1]
        g_1 += orc.ops.adjoint(H, res, U_hist=U)[1]
    box = [tuple(b) for b in lay["box"]]
    out = {}
    for stride in (1, r):
        mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=True, ckpt_stride=20, box=box,
                        layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"],
                        grad_stride=stride)
        xg = mesh.dof_coords()
        mesh.set_velocity(cfun(xg))
        perm = match_dofs(orc.mesh.coords, xg, 1.0)
        b = lib.Batch(mesh, srcs, recs)
        rec = torch.zeros((4, nt + 1, len(recs)), device="cuda")
        b.forward(torch.from_numpy(wav).float().cuda(), rec)
        res = torch.from_numpy(np.stack([0.1 * ro for ro in recs_o]).astype(np.float32)).cuda()
        b.adjoint(res)
        G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
        b.gradient(G)
        out[stride] = (G.cpu().numpy()[perm], mesh.batch_bytes(4, len(recs)), mesh.N)
        b.close()
        mesh.close()
    Go_r = orc.ops.gradient(g_r, orc.mask)
    Go_1 = orc.ops.gradient(g_1, orc.mask)
    err = rel_l2(out[r][0], Go_r)
    dep = rel_l2(Go_r, Go_1)
    ring = lambda st: 4 * out[st][2] * 4 * (20 // st)
    print(f"r = {r}: GPU vs oracle (subsampled) rel-L2 {err:.3e}; subsampled vs full gradient "
          f"rel-L2 {dep:.3e}; recompute ring {ring(r) / 1e6:.2f} MB against {ring(1) / 1e6:.2f} MB; "
          f"batch {out[r][1] / 1e6:.2f} MB against {out[1][1] / 1e6:.2f} MB")
    assert err < GRAD_TOL
    assert rel_l2(out[1][0], Go_1) < GRAD_TOL
    assert out[r][1] < out[1][1]


@pytest.mark.parametrize("form", [SIMT, TC, PLAIN], ids=["chunked", "tensor-cores", "plain"])
def test_per_shot_gradients(lib, form):
    """fwi_gradient_lanes returns each shot's own gradient M^-1 g_s and misfit J_s (the
    per-shot terms of Eq. gradient3 that Section 4.5 sums over shots). Every lane matches the
    oracle's gradient of that shot alone, the misfits match 1/2 |residual_s|^2, and the sum
    over lanes equals fwi_gradient (the summed form) on a second identical adjoint solve (to
    the FP32 summation-order noise of the atomics)."""
    layout, tc = form
    k, cfun = (4 if tc == 1 else 3), models.smooth2d  # the tensor-core step serves k = 4, 5
    V, C, lay = _case2d(k, n=10, layer=True)
    srcs = np.array([[0.5, 0.1], [0.2, 0.15], [0.8, 0.2], [0.35, 0.3]])
    recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 9)])
    probe = OracleCase(V, C, k, cfun, 1.0, 1, layer=lay, absorbing=True)
    dt = 0.8 * probe.ops.cfl_dt()
    nt = int(round(0.5 / dt))
    orc = OracleCase(V, C, k, cfun, dt, nt, layer=lay, absorbing=True)
    box = [tuple(b) for b in lay["box"]]
    mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=True, ckpt_stride=13, box=box,
                    layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"],
                    layout=layout, tensor_cores=tc)
    xg = mesh.dof_coords()
    perm = match_dofs(orc.mesh.coords, xg, 1.0)
    mesh.set_velocity(cfun(xg))
    wav = np.stack([signals.ricker_samples(8.0, dt, nt, t0=0.15) * (1 + 0.1 * i) for i in range(4)])
    rng = np.random.default_rng(11)
    res = (0.01 * rng.standard_normal((4, nt + 1, len(recs)))).astype(np.float32)
    b = lib.Batch(mesh, srcs, recs)
    rec = torch.zeros((4, nt + 1, len(recs)), device="cuda")
    wav_d = torch.from_numpy(wav).float().cuda()
    b.set_gradient_lanes(True)
    b.forward(wav_d, rec)
    b.adjoint(torch.from_numpy(res).cuda())
    G = np.zeros((4, mesh.N))
    J = b.gradient_lanes(G)
    # the summed form (the default): its own accumulator, the same sum
    b.set_gradient_lanes(False)
    b.forward(wav_d, rec)
    b.adjoint(torch.from_numpy(res).cuda())
    Gsum = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    Jsum = b.gradient(Gsum)
    Gsum = Gsum.cpu().numpy()
    for s in range(4):
        Go = orc.gradient([srcs[s]], recs, [wav[s].astype(np.float32).astype(np.float64)],
                          [res[s].astype(np.float64)])
        err = rel_l2(G[s][perm], Go)
        Jo = 0.5 * float(np.sum(res[s].astype(np.float64) ** 2))
        print(f"form={form} shot {s}: lane gradient vs oracle rel-L2 {err:.3e}, J {J[s]:.6e} vs {Jo:.6e}")
        assert err < GRAD_TOL
        assert abs(J[s] - Jo) <= 1e-6 * Jo
    serr = rel_l2(G.sum(0), Gsum)
    print(f"form={form}: sum of lanes vs fwi_gradient rel-L2 {serr:.3e}")
    # FP32 summation-order noise; the tensor-core adjoint's own error is larger (3xTF32)
    assert serr < (2e-5 if tc == 1 else 5e-6) and abs(J.sum() - Jsum) <= 1e-12 * Jsum
    # asking for lanes after a summed adjoint is an error, not a silent sum
    b.forward(wav_d, rec)
    b.adjoint(torch.from_numpy(res).cuda())
    with pytest.raises(lib.FwiError):
        b.gradient_lanes(G)
    b.gradient(torch.zeros(mesh.N, dtype=torch.float64, device="cuda"))
    b.close()
    mesh.close()


@pytest.mark.parametrize("k,S,r", [(5, 4, 1), (4, 8, 1), (5, 4, 3)])
def test_gradient_store_matches_recompute(lib, k, S, r):
    """fwi_batch_set_gradient_store: the gradient steps of the persistent kernel read the
    forward field's gradients stored by the recompute instead of contracting the forward
    field again. The gradient equals that of the recompute path (FP32 summation order) and,
    at r = 1, the oracle's, with the damping layer, two shot groups (S = 8) and subsampling
    (r = 3, Section 3.6)."""
    V, C, lay = _case2d(k, n=10, layer=True)
    cfun = models.smooth2d
    rng = np.random.default_rng(k + S + r)
    srcs = np.column_stack([rng.uniform(0.15, 0.85, S), rng.uniform(0.1, 0.35, S)])
    recs = np.array([[x, 0.9] for x in np.linspace(0.05, 0.95, 11)])
    probe = OracleCase(V, C, k, cfun, 1.0, 1, layer=lay, absorbing=True)
    dt = 0.8 * probe.ops.cfl_dt()
    nt = int(round(0.5 / dt))
    box = [tuple(b) for b in lay["box"]]
    mesh = lib.Mesh(V, C, k, nt, dt=dt, absorbing=True, ckpt_stride=12, grad_stride=r, box=box,
                    layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"])
    xg = mesh.dof_coords()
    mesh.set_velocity(cfun(xg))
    wav = np.stack([signals.ricker_samples(rng.uniform(6, 9), dt, nt, t0=0.15) for _ in range(S)])
    wav = wav.astype(np.float32)
    res = (0.01 * rng.standard_normal((S, nt + 1, len(recs)))).astype(np.float32)
    b = lib.Batch(mesh, srcs, recs)
    rec = np.zeros((S, nt + 1, len(recs)), np.float32)
    out = {}
    for store in (False, True):
        b.set_gradient_store(store)
        b.forward(wav, rec)
        b.adjoint(res)
        G = np.zeros(mesh.N)
        out[store] = (G, b.gradient(G))
    err = rel_l2(out[True][0], out[False][0])
    print(f"k={k} S={S} r={r}: stored-gradient vs recompute path rel-L2 {err:.3e}, "
          f"J {out[True][1]:.9e} vs {out[False][1]:.9e}")
    # the two FP32 paths sum the same products in different orders; the time sum of the
    # oscillating integrand cancels, so they part at about 1e-5 (each within the oracle bound)
    assert err < GRAD_TOL and abs(out[True][1] - out[False][1]) <= 1e-12 * out[False][1]
    if r == 1:
        orc = OracleCase(V, C, k, cfun, dt, nt, layer=lay, absorbing=True)
        perm = match_dofs(orc.mesh.coords, xg, 1.0)
        Go = orc.gradient(list(srcs), recs, [w.astype(np.float64) for w in wav],
                          [x.astype(np.float64) for x in res])
        oerr = rel_l2(out[True][0][perm], Go)
        print(f"k={k} S={S}: stored-gradient path vs oracle rel-L2 {oerr:.3e}")
        assert oerr < GRAD_TOL
    b.close()
    mesh.close()
