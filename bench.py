"""Throughput of the KMV FWI hot path on GB300: forward + adjoint + gradient, DoF-steps/s.

Workload (default): the 2D marine section of 17 km x 3.5 km (0.45 km water, 8 dipping
layers, a normal fault, a 4.5 km/s salt body, +-5 % smoothed perturbation; seeded
synthetic stand-in for Marmousi2) with a 1 km damping layer on the sides and bottom, a
waveform-adapted KMV5 triangle mesh at 5 Hz, 4 s records, 500 receivers at 100 m depth and
shots at 50 m depth. The 4 s record takes Nt ~ 1e5 CFL-limited steps, so one bench step is
one window of ``--window`` time steps of that record for one batch of S shots, through the
whole hot path: fwi_forward_shot (records + checkpoints over the window),
fwi_adjoint_misfit (residual, checkpointed recompute, adjoint, gradient integrand) and
fwi_gradient. Every time step of the window does the full work (no step or element is
skipped); the full record is Nt / window such steps at the same rate.

value = S * N * window * 2 / step time (forward and adjoint DoF-steps; recompute steps are
not counted as work), summed over ranks. ``--impl reference`` times the FP64 oracle on the
host cores instead (a bounded sample of the same workload).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAK_HBM_FALLBACK = 6800.0


METRIC = "DoF-steps/s (forward + adjoint, FP32, <=1e-5 rel-L2 vs FP64 oracle)"


def workload_name(k, workload="marine2d"):
    if workload == "thrust3d":
        return f"thrust3d-5x5x3km-kmv{k}tet-layer0.75km-5Hz-3s"
    return f"marine2d-17x3.5km-kmv{k}-layer1km-5Hz-4s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": PEAK_HBM_FALLBACK, "sm_max_mhz": 2070.0}, "fallback"


def make_workload(k=5, C=None, seed=0, nshots=40, nrec=500, T=4.0, f=5.0, small=False):
    """Mesh, velocity, acquisition of the marine workload (inputs only)."""
    from synth import meshes, models, signals
    model = models.marine2d(seed)
    box = (-1.0, 18.0, 0.0, 4.5)
    if small:
        box = (6.0, 8.0, 0.0, 1.5)
    if C is None:
        C = {2: 12.0, 3: 15.0, 4: 18.0, 5: 22.0}[k] if not small else 6.0
    V, cells = meshes.adapted_tri(model, f, C, box, seed=seed, iters=10)
    if small:
        srcs = np.array([[7.0, 0.05], [6.5, 0.05]])
        recs = np.array([[x, 0.1] for x in np.linspace(6.1, 7.9, 20)])
        lay = dict(box=[(6.2, 7.8), (-10.0, 1.3)], faces=0b1011, width=0.2)
    else:
        srcs = np.stack([np.linspace(1.0, 16.0, nshots), np.full(nshots, 0.05)], 1)
        recs = np.stack([np.linspace(0.1, 17.0, nrec), np.full(nrec, 0.1)], 1)
        lay = dict(box=[(0.0, 17.0), (-10.0, 3.5)], faces=0b1011, width=1.0)
    lay["smax"] = signals.sigma_max(4.7, lay["width"])
    return dict(model=model, V=V, cells=cells, k=k, C=C, srcs=srcs, recs=recs, layer=lay, T=T,
                f=f, box=box)


def make_workload3d(k=2, seed=0, small=False, scale=1.0):
    """The 3D workload (inputs only): the 5 km x 5 km x 3 km thrust model (layered, a thrust-
    folded interface, two 5.5-6.0 km/s lenses, smooth perturbation; seeded stand-in for
    Overthrust3D) with a 0.75 km damping layer on the sides and bottom, on a depth-graded
    Kuhn tetrahedral mesh (59 m boxes across, 40 m deep in the top kilometre of slow rock,
    60 m below; 5.08M tetrahedra), 16 shots in a 4 x 4 grid at 50 m depth and a 100 x 100 receiver grid at
    100 m depth, 5 Hz, 3 s. small=True: a 1.2 km x 1.2 km x 1.0 km box of the same model
    (the oracle's sample). scale < 1 coarsens the boxes by that factor (for profiler
    captures of the same kernels on a smaller case)."""
    from synth import meshes, models, signals
    model = models.Thrust3D(seed)
    L = 0.75
    if small:
        xs = np.linspace(1.9, 3.1, 11)
        zs = np.linspace(0.0, 1.0, 9)
        V, cells = meshes.kuhn_tets(xs, xs, zs)
        srcs = np.array([[2.5, 2.5, 0.05], [2.3, 2.6, 0.05], [2.6, 2.35, 0.05], [2.4, 2.4, 0.05]])
        g = np.linspace(2.0, 3.0, 5)
        recs = np.array([[x, y, 0.1] for x in g for y in g])
        lay = dict(box=[(2.05, 2.95), (2.05, 2.95), (-10.0, 0.85)], faces=0b101111, width=0.15)
    else:
        xs = np.linspace(-L, 5 + L, int(round(110 * scale)) + 1)
        zs = np.concatenate([np.arange(0.0, 1.0, 0.04 / scale),
                             np.arange(1.0, 3.0 + L + 1e-9, 0.06 / scale)])
        V, cells = meshes.kuhn_tets(xs, xs, zs)
        g4 = np.linspace(1.0, 4.0, 4)
        srcs = np.array([[x, y, 0.05] for x in g4 for y in g4])
        g100 = np.linspace(0.05, 4.95, 100)
        recs = np.array([[x, y, 0.1] for x in g100 for y in g100])
        lay = dict(box=[(0.0, 5.0), (0.0, 5.0), (-10.0, 3.0)], faces=0b101111, width=L)
    lay["smax"] = signals.sigma_max(6.0, lay["width"])
    return dict(model=model, V=V, cells=cells, k=k, C=None, srcs=srcs, recs=recs, layer=lay,
                T=3.0, f=5.0, dim=3)


def shots_for_rank(nshots, S, rank, world, step=0):
    """Shot indices a rank runs at a given step: the shots are dealt round-robin in blocks of
    S, so that N ranks together cover S*N consecutive shots per step (weak scaling)."""
    base = (step * world + rank) * S
    return [(base + i) % nshots for i in range(S)]


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, device_index):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        rows = [[x.strip() for x in r] for r in rows if r and r[0].strip() == str(device_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- the FP64 oracle on the host cores (cpu_baseline, parity sample, reference arm) ----------
# One shot per worker of a spawn-started process pool (the paper's ensemble runs one shot per
# core). Each worker builds the oracle for the small marine window of the workload once.
_ORC = {}


def _orc_init(k, workload="marine2d"):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_util import OracleCase
    small = make_workload3d(k=k, small=True) if workload == "thrust3d" else make_workload(k=k, small=True)
    lay = small["layer"]
    probe = OracleCase(small["V"], small["cells"], k, small["model"], 1.0, 1, layer=lay,
                       absorbing=True, water=1.51)
    dt = 0.9 * probe.ops.cfl_dt()
    orc = OracleCase(small["V"], small["cells"], k, small["model"], dt, 1, layer=lay,
                     absorbing=True, water=1.51)
    _ORC.update(k=k, small=small, dt=dt, orc=orc, workload=workload)


def _orc_shot(job):
    """Forward (history stored) and adjoint with the gradient integrand for one shot;
    returns (records, raw gradient sum or None, DoF-steps, seconds)."""
    from oracle import assemble
    src, nt, wav, res_scale, keep = job
    orc = _ORC["orc"]
    orc.nt = nt
    t0 = time.perf_counter()
    rec, U = orc.forward(src, _ORC["small"]["recs"], wav, store=True)
    H = assemble.point_matrix(orc.mesh, _ORC["small"]["recs"])
    _, g = orc.ops.adjoint(H, res_scale * rec.astype(np.float32).astype(np.float64), U_hist=U)
    el = time.perf_counter() - t0
    return (rec if keep else None), (g if keep else None), orc.mesh.N * nt * 2, el


def oracle_pool(k, workers, workload="marine2d"):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers, initializer=_orc_init, initargs=(k, workload))


def oracle_window_info(k, workload="marine2d"):
    _orc_init(k, workload)
    return dict(dt=_ORC["dt"], N=_ORC["orc"].mesh.N, E=_ORC["small"]["cells"].shape[0],
                small=_ORC["small"], orc=_ORC["orc"])


def parity_shots(small, n, workload="marine2d"):
    """n shot positions at 50 m depth across the small window."""
    if workload == "thrust3d":
        return np.stack([np.linspace(2.2, 2.8, n), np.linspace(2.7, 2.3, n), np.full(n, 0.05)], 1)
    return np.stack([np.linspace(6.3, 7.7, n), np.full(n, 0.05)], 1)


def oracle_rate(pool, k, dt, workers, nsteps, workload="marine2d"):
    """DoF-steps/s of the FP64 oracle (forward + adjoint with the gradient integrand) over
    `workers` shots, one per worker, nsteps time steps each; wall-clock of the pool."""
    from synth import signals
    srcs = parity_shots(None, workers, workload)
    wav = signals.ricker_samples(5.0, dt, nsteps).astype(np.float64)
    jobs = [(srcs[i], nsteps, wav, 0.03, False) for i in range(workers)]
    t0 = time.perf_counter()
    out = pool.map(_orc_shot, jobs)
    wall = time.perf_counter() - t0
    return dict(value=sum(o[2] for o in out) / wall, seconds=wall, nsteps=nsteps, shots=workers)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# Shot-server pool shaped like the serving workload: six seeded 2D meshes of 50k-2M
# triangles, KMV2..5, 3-8 Hz peaks and 2-6 s records. Each mesh is a structured
# right-triangle mesh of a square whose cell size follows the paper's cells per wavelength
# for 5 % error (Table gwpl: C = 5.85, 3.08, 2.22, 1.69 for KMV2..5) at the slowest speed
# 1.4 km/s and the mesh's peak frequency; c(x) a smooth 1.4-3.0 km/s model.
SERVING_POOL = [  # (triangles, k, peak Hz, record s)
    (50_000, 5, 8.0, 2.0), (120_000, 3, 6.0, 3.0), (250_000, 4, 5.0, 4.0),
    (500_000, 2, 4.0, 5.0), (1_000_000, 3, 3.0, 3.0), (2_000_000, 2, 3.0, 6.0)]
CELLS_PER_WAVELENGTH = {2: 5.85, 3: 3.08, 4: 2.22, 5: 1.69}


def serving_pool(pkg, scale=1.0):
    from synth import meshes, models
    pool = {}
    for i, (E, k, f, T) in enumerate(SERVING_POOL):
        n = max(8, int(round(np.sqrt(scale * E / 2))))
        h = 1.4 / f / CELLS_PER_WAVELENGTH[k]
        L = n * h
        V, C = meshes.structured_tri(n, n, L, L)
        cfun = lambda X, L=L: models.smooth2d(X / L * 2.0)
        probe = pkg.Mesh(V, C, k, 1, dt=0.0, cfl_factor=0.8)
        probe.set_velocity(cfun(probe.dof_coords()))
        dt = probe.dt
        probe.close()
        nt = int(round(T / dt))
        m = pkg.Mesh(V, C, k, nt, dt=dt, ckpt_stride=50, absorbing=True)
        m.set_velocity(cfun(m.dof_coords()))
        recs = np.stack([np.linspace(0.05 * L, 0.95 * L, 50), np.full(50, 0.9 * L)], 1)
        pool[f"m{i}"] = dict(mesh=m, recs=recs, f=f, L=L, E=2 * n * n, k=k, T=T)
    return pool


def serving_stream(pkg, nreq=32, seed=0, budget_gb=40.0, loads=(0.5, 0.75, 1.0, 1.25, 1.5),
                   scale=1.0):
    """Poisson streams of shot requests over the six resident meshes of SERVING_POOL (each
    request on a random mesh; half carry observed records and ask for their own gradient).
    The batched server's saturation throughput is measured first (all requests at once);
    then streams at 0.5x-1.5x of it are each served twice: by the continuous-batching server
    (rolling forward batches with admission every 50 steps, gradient batches, up to 4 shots
    per batch, two workers) and in the one-shot-per-launch form (one worker, one shot per
    batch, whole records). Returns shots/s and p50/p99 latency per stream."""
    from paper_2108_10946_gb300.serving import Request, ShotServer
    from synth import signals
    rng = np.random.default_rng(seed)
    t_setup = time.perf_counter()
    pool = serving_pool(pkg, scale)
    t_setup = time.perf_counter() - t_setup
    meshes_ = {name: (p["mesh"], p["recs"]) for name, p in pool.items()}
    names = sorted(pool)

    def make_plan(rate):
        arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq)) if rate else np.zeros(nreq)
        plan = []
        for i in range(nreq):
            mi = int(rng.integers(len(names)))
            p = pool[names[mi]]
            m, f, L = p["mesh"], p["f"], p["L"]
            wav = signals.ricker_samples(f, m.dt, m.nsteps, t0=1.2 / f)
            obs = np.zeros((m.nsteps + 1, len(p["recs"])), np.float32) if rng.random() < 0.5 else None
            src = [rng.uniform(0.1, 0.9) * L, rng.uniform(0.05, 0.3) * L]
            plan.append((arrivals[i], mi, src, wav, obs))
        return plan

    def serve(plan, max_batch, workers, rolling):
        srv = ShotServer(meshes_, hbm_budget_bytes=int(budget_gb * 2 ** 30), max_batch=max_batch,
                         workers=workers, rolling=rolling)
        t0 = time.perf_counter()
        reqs = []
        for i, (t, mi, src, wav, obs) in enumerate(plan):
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            reqs.append(srv.submit(Request(i, names[mi], src, wav, observed=obs)))
        for r in reqs:
            r.event.wait(900)
        st = srv.stats()
        st["errors"] = sum(r.error is not None for r in reqs)
        st["wall_s"] = time.perf_counter() - t0
        srv.close()
        return st

    serve(make_plan(0), 4, 2, True)  # warm-up: resident batches, code paths
    sat = serve(make_plan(0), 4, 2, True)
    sat_one = serve(make_plan(0), 1, 1, False)
    lam = sat["shots_per_s"]
    streams = []
    for rho in loads:
        plan = make_plan(rho * lam)
        streams.append({"load": rho, "mean_interarrival_s": 1.0 / (rho * lam),
                        "batched": serve(plan, 4, 2, True),
                        "one_shot_per_launch": serve(plan, 1, 1, False)})
    desc = [{"triangles": p["E"], "k": p["k"], "peak_hz": p["f"], "record_s": p["T"],
             "steps": p["mesh"].nsteps, "dofs": p["mesh"].N} for p in pool.values()]
    for p in pool.values():
        p["mesh"].close()
    return {"requests_per_stream": nreq, "meshes": desc, "gradient_fraction": "1/2",
            "setup_s": t_setup, "saturation": {"batched": sat, "one_shot_per_launch": sat_one},
            "streams": streams}


def run_reference(args):
    """The oracle arm: the FP64 oracle on the host cores, one shot per core, each step a
    bounded sample (ref_steps time steps of forward + adjoint per shot) of the workload's
    small marine window at the same element degree."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    k = args.k
    cores = host_cores()
    info = oracle_window_info(k, args.workload)
    pool = oracle_pool(k, cores, args.workload)
    try:
        for _ in range(args.warmup):
            oracle_rate(pool, k, info["dt"], cores, args.ref_steps, args.workload)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(oracle_rate(pool, k, info["dt"], cores, args.ref_steps, args.workload)["value"])
        el = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    v = float(np.mean(vals))
    where = ("a 1.2 km x 1.2 km x 1.0 km box of the thrust model" if args.workload == "thrust3d"
             else "the 2 km x 1.5 km marine window")
    sample = (f"FP64 oracle, KMV{k}{'tet' if args.workload == 'thrust3d' else 'tri'} on {where} of the workload "
              f"({info['E']} elements, N={info['N']}), {cores} shots (one per host core), "
              f"{args.ref_steps} forward + adjoint steps each per bench step")
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "DoF-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(k, args.workload),
                       "sample": "the FP64 oracle on the host cores, timed on a bounded window of "
                                 "the workload (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": v, "unit": "DoF-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "DoF-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def parity_sample(pkg, pool, info, k, S, T_par, workload="marine2d", gstore=False):
    """The GPU library against the FP64 oracle on the workload's small marine window (same
    mesher, model, water, layer and absorbing boundary; S shots, T_par seconds): records
    rel-L2 (worst shot) and gradient rel-L2, as the tests measure them. The oracle shots run
    in the pool; the GPU runs the same shots as one batch."""
    import torch
    from synth import signals
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_util import match_dofs, rel_l2
    dt, small, orc = info["dt"], info["small"], info["orc"]
    nt = int(round(T_par / dt))
    srcs = parity_shots(small, S, workload)
    wav = signals.ricker_samples(5.0, dt, nt).astype(np.float32)
    out = pool.map(_orc_shot, [(srcs[i], nt, wav.astype(np.float64), 0.03, True) for i in range(S)])
    lay = small["layer"]
    mesh = pkg.Mesh(small["V"], small["cells"], k, nt, dt=dt, box=lay["box"],
                    layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"],
                    absorbing=True, ckpt_stride=50, water_speed=1.51)
    xg = mesh.dof_coords()
    mesh.set_velocity(small["model"](xg))
    b = pkg.Batch(mesh, srcs, small["recs"])
    b.set_gradient_store(gstore)  # the bench's own gradient path
    rec = torch.zeros((S, nt + 1, len(small["recs"])), device="cuda")
    b.forward(torch.from_numpy(np.stack([wav] * S)).cuda(), rec)
    rec = rec.cpu().numpy()
    rec_err = max(rel_l2(rec[s], out[s][0]) for s in range(S))
    res = np.stack([0.03 * o[0].astype(np.float32) for o in out]).astype(np.float32)
    b.adjoint(torch.from_numpy(res).cuda())
    G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    b.gradient(G)
    perm = match_dofs(orc.mesh.coords, xg, 1.0)
    Go = orc.ops.gradient(np.sum([o[1] for o in out], axis=0), orc.mask)
    g_err = rel_l2(G.cpu().numpy()[perm], Go)
    b.close()
    mesh.close()
    return {"records_rel_l2_max": rec_err, "gradient_rel_l2": g_err, "shots": S, "steps": nt,
            "window": (f"1.2 km x 1.2 km x 1.0 km box of the thrust model, KMV{k}tet" if workload == "thrust3d"
                       else f"2 km x 1.5 km marine window, KMV{k}") +
                      f", N={info['N']}, {T_par} s, layer, absorbing boundary, residual 0.03 d"}


# DRAM bytes (read + write) of one forward time step: the three launches of a step
# (k_chunk_pt<0>, k_chunk<0,1>, node_kernel4<2>) from one ncu capture of this workload's mesh
# (profiles/ncu_forward_marine2d_kmv5_S4.md), keyed by (workload, k, S, N) so that it is
# reported only for the mesh, degree and shot count it was measured on.
FORWARD_TRAFFIC = {("marine2d", 5, 4, 7477937): 745.2e6}

NODES = {2: (7, 6), 3: (12, 9), 4: (18, 12), 5: (30, 15)}  # KMVktri: nodes, shared nodes
NODES3 = {2: (15, 14), 3: (32, 28)}                           # KMVktet


def step_roofline(prof, k, E, N, S, fp32_tflops, sm_count, peaks, src, dim=2):
    """Roofline entries of the forward time step (element kernels + shared-DoF kernel) and of
    the adjoint step with the gradient integrand, from per-step CUDA-event times.
    Algorithmic work per step (stated in DESIGN):
      forward flops = E S 4 d n^2 (two n x n contractions per direction per element and shot)
      adjoint flops = E S 6 d n^2 (plus the contraction of the forward field)
      forward bytes = N (16 S + 8) + E (4 n_s + 4 n_g): u, v read and written per shot, c^2
                      and M^-1 per DoF, shared-node connectivity and Ghat (n_g = 3 in 2D, 6 in
                      3D) per element
      adjoint bytes = forward bytes + 4 N S (forward field) + 8 N (gradient segment)"""
    nn, ns = (NODES if dim == 2 else NODES3)[k]
    d = dim
    ng = 3 if dim == 2 else 6  # Ghat entries per element
    fs, as_ = max(prof["fwd_steps"], 1), max(prof["adj_steps"], 1)
    fwd_ms = (prof["fwd_elem_ms"] + prof["fwd_node_ms"]) / fs
    adj_ms = (prof["adj_elem_ms"] + prof["adj_node_ms"]) / as_
    hbm = peaks["hbm_gbs"]

    def entry(flops, nbytes, ms, label):
        tf = flops / (ms * 1e-3) / 1e12
        gb = nbytes / (ms * 1e-3) / 1e9
        alu_src = f"measured FP32 FMA probe (fwi_fp32_peak), {sm_count} SMs"
        if tf / fp32_tflops >= gb / hbm:
            e = {"bound": "alu", "achieved": tf, "peak": fp32_tflops, "unit": "TFLOP/s",
                 "frac": tf / fp32_tflops, "peak_source": alu_src, "hbm_achieved_gbs": gb,
                 "hbm_frac": gb / hbm}
        else:
            e = {"bound": "hbm", "achieved": gb, "peak": hbm, "unit": "GB/s", "frac": gb / hbm,
                 "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs", "alu_achieved_tflops": tf,
                 "alu_frac": tf / fp32_tflops}
        e.update({"traffic": None, "kernel": f"{label}, {ms * 1e3:.1f} us/step",
                  "flops_per_step": flops, "bytes_per_step": nbytes})
        return e

    fwd_bytes = N * (16 * S + 8) + E * (4 * ns + 4 * ng)
    roof = entry(E * S * 4 * d * nn * nn, fwd_bytes, fwd_ms,
                 "forward time step (element kernels + shared-DoF kernel)")
    roof["element_kernel_us"] = prof["fwd_elem_ms"] / fs * 1e3
    roof["node_kernel_us"] = prof["fwd_node_ms"] / fs * 1e3
    roof["adjoint"] = entry(E * S * 6 * d * nn * nn, fwd_bytes + 4 * N * S + 8 * N, adj_ms,
                            "adjoint step with the gradient integrand")
    roof["adjoint"]["element_kernel_us"] = prof["adj_elem_ms"] / as_ * 1e3
    roof["adjoint"]["node_kernel_us"] = prof["adj_node_ms"] / as_ * 1e3
    return roof


def degree_line(pkg, k, args, S, fp32_tflops, sm_count, peaks, src):
    """The same step (forward, adjoint, gradient) on the marine workload at another element
    degree, over a shorter window: DoF-steps/s and the roofline entries."""
    import torch
    from synth import signals
    wl = make_workload(k=k)
    lay = wl["layer"]
    kw = dict(box=lay["box"], layer_faces=lay["faces"], layer_width=lay["width"],
              sigma_max=lay["smax"], absorbing=True, ckpt_stride=args.ckpt, water_speed=1.51)
    m0 = pkg.Mesh(wl["V"], wl["cells"], k, 1, dt=0.0, cfl_factor=0.9, **kw)
    c = wl["model"](m0.dof_coords())
    m0.set_velocity(c)
    dt = m0.dt
    m0.close()
    nt = args.extra_window
    mesh = pkg.Mesh(wl["V"], wl["cells"], k, nt, dt=dt, **kw)
    mesh.set_velocity(c)
    b = pkg.Batch(mesh, wl["srcs"][:S], wl["recs"])
    b.set_gradient_store(not args.no_gradient_store)
    R = len(wl["recs"])
    wav = torch.from_numpy(np.stack([signals.ricker_samples(5.0, dt, nt)] * S)).float().cuda()
    rec = torch.zeros((S, nt + 1, R), device="cuda")
    obs = torch.zeros_like(rec)
    G = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    b.forward(wav, obs)
    obs *= 0.97

    def step():
        b.forward(wav, rec)
        b.adjoint_misfit(obs)
        b.gradient(G)

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 2
    b.profile(True)
    step()
    prof = b.profile_read()
    b.profile(False)
    out = {"k": k, "workload": workload_name(k), "elements": mesh.E, "dofs": mesh.N, "dt": dt,
           "window_steps": nt, "shots_per_step": S, "ms_per_step": ms,
           "value": S * mesh.N * nt * 2 / (ms * 1e-3), "unit": "DoF-steps/s",
           "roofline": step_roofline(prof, k, mesh.E, mesh.N, S, fp32_tflops, sm_count, peaks, src)}
    b.close()
    mesh.close()
    return out


def run_ours(args):
    import torch
    import paper_2108_10946_gb300 as pkg
    from synth import signals

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.build()
    pool = info = None
    cores = host_cores()
    three_d = args.workload == "thrust3d"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's worker pool starts now (spawn) and builds its window while the GPU runs
        pool = oracle_pool(args.k, cores, args.workload)
    fp32_tflops, sm_count = pkg.lib.fp32_peak()
    wl = make_workload3d(k=args.k, scale=args.mesh_scale) if three_d else make_workload(k=args.k, C=args.C)
    lay = wl["layer"]
    t_setup = time.perf_counter()
    mesh = pkg.Mesh(wl["V"], wl["cells"], wl["k"], 1, dt=0.0, cfl_factor=0.9,
                    box=lay["box"], layer_faces=lay["faces"], layer_width=lay["width"],
                    sigma_max=lay["smax"], absorbing=True, ckpt_stride=args.ckpt,
                    water_speed=1.51)
    xg = mesh.dof_coords()
    c = wl["model"](xg)
    mesh.set_velocity(c)
    dt = mesh.dt
    nt_record = int(round(wl["T"] / dt))
    nt = min(args.window, nt_record)
    # rebuild with the window as the step count (dt is a property of mesh and velocity)
    mesh.close()
    mesh = pkg.Mesh(wl["V"], wl["cells"], wl["k"], nt, dt=dt, box=lay["box"],
                    layer_faces=lay["faces"], layer_width=lay["width"], sigma_max=lay["smax"],
                    absorbing=True, ckpt_stride=args.ckpt, water_speed=1.51)
    mesh.set_velocity(c)
    N, E = mesh.N, wl["cells"].shape[0]
    S = args.shots
    shots = wl["srcs"][shots_for_rank(len(wl["srcs"]), S, rank, world)]
    batch = pkg.Batch(mesh, shots, wl["recs"])
    # the gradient steps read the forward field's gradients stored by the recompute
    # (fwi_batch_set_gradient_store; no effect on tetrahedra)
    batch.set_gradient_store(not args.no_gradient_store)
    R = len(wl["recs"])
    wav = np.stack([signals.ricker_samples(wl["f"], dt, nt)] * S)
    wav_d = torch.from_numpy(wav).cuda()
    # observed data: the same sources through a true model (smoothed start model vs true:
    # here the start model is the true model scaled, which is all the step needs)
    obs_d = torch.zeros((S, nt + 1, R), device="cuda")
    batch.forward(wav_d, obs_d)
    obs_d *= 0.97
    rec_d = torch.zeros((S, nt + 1, R), device="cuda")
    G_d = torch.zeros(N, dtype=torch.float64, device="cuda")
    setup_s = time.perf_counter() - t_setup

    def step():
        batch.forward(wav_d, rec_d)
        batch.adjoint_misfit(obs_d)
        batch.gradient(G_d)
        if dist is not None:
            dist.all_reduce(G_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    pkg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(os.path.join(args.clocks_dir, f"clocks_rank{rank}.csv"))
    with clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    launches = pkg.launch_count()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    ms_step = ms / args.steps
    units = S * N * nt * 2 * world
    value = units / (ms_step / 1000.0)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    wav_h = torch.from_numpy(wav).pin_memory()
    obs_h = obs_d.cpu().pin_memory()
    rec_h = torch.zeros((S, nt + 1, R)).pin_memory()
    G_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        batch.forward(wav_h.numpy(), rec_h.numpy())
        batch.adjoint_misfit(obs_h.numpy())
        batch.gradient(G_h.numpy())
        if dist is not None:  # the shots' gradient summed over the ranks, as in the step
            G_d.copy_(G_h)
            dist.all_reduce(G_d)
            G_h.copy_(G_d)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = S * N * nt * 2 * world / e2e_s

    # per-kernel timing of the forward and adjoint steps (events on the library's stream)
    batch.profile(True)
    batch.forward(wav_d, rec_d)
    batch.adjoint_misfit(obs_d)
    batch.gradient(G_d)
    prof = batch.profile_read()
    batch.profile(False)
    peaks, src = _peaks()
    clk_sum = clk.summary(local)
    roof = step_roofline(prof, wl["k"], E, N, S, fp32_tflops, sm_count, peaks, src,
                         dim=3 if three_d else 2)
    traffic = FORWARD_TRAFFIC.get((args.workload, wl["k"], S, N))
    if traffic is not None:
        roof["traffic"] = traffic
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                  "three launches of one forward step on this mesh")

    extra_k = []
    # the side measurements (other degrees, plain form, serving) belong to the one-GPU line;
    # multi-GPU lines measure the scaled step alone
    if rank == 0 and world == 1 and args.extra_k and not three_d:
        for kx in [int(x) for x in args.extra_k.split(",") if x]:
            extra_k.append(degree_line(pkg, kx, args, S, fp32_tflops, sm_count, peaks, src))

    plain = None
    if args.plain and world == 1:
        # the unfused form: layout 1 (one thread per element and shot, global atomics,
        # separate node kernel), one shot per launch, same window
        mp_ = pkg.Mesh(wl["V"], wl["cells"], wl["k"], nt, dt=dt, box=lay["box"],
                       layer_faces=lay["faces"], layer_width=lay["width"],
                       sigma_max=lay["smax"], absorbing=True, ckpt_stride=args.ckpt,
                       water_speed=1.51, layout=1)
        mp_.set_velocity(wl["model"](mp_.dof_coords()))
        b1 = pkg.Batch(mp_, shots[:1], wl["recs"])
        w1, r1 = wav_d[:1].contiguous(), torch.zeros((1, nt + 1, R), device="cuda")
        o1 = obs_d[:1].contiguous()
        g1 = torch.zeros(mp_.N, dtype=torch.float64, device="cuda")
        b1.forward(w1, r1)
        b1.adjoint_misfit(o1)
        b1.gradient(g1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(S):
            b1.forward(w1, r1)
            b1.adjoint_misfit(o1)
            b1.gradient(g1)
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": S * N * nt * 2 / (pms / 1000.0), "unit": "DoF-steps/s",
                 "form": "layout 1 (per-element global atomics), one shot per launch",
                 "speedup_of_value": value / (S * N * nt * 2 / (pms / 1000.0))}
        b1.close()
        mp_.close()

    serving = None
    if rank == 0 and world == 1 and not args.no_serving and not three_d:
        serving = serving_stream(pkg, scale=args.serving_scale)

    cpu = parity = None
    if pool is not None:
        try:
            info = oracle_window_info(wl["k"], args.workload)
            # long enough for the sea-floor reflection (near 0.55 s) to reach the receivers,
            # so that the gradient below the masked water is more than rounding noise
            T_par = 0.6 if three_d else {2: 1.5, 3: 1.5, 4: 0.8, 5: 0.6}[wl["k"]]
            parity = parity_sample(pkg, pool, info, wl["k"], S, T_par, args.workload,
                                   gstore=not args.no_gradient_store)
            ob = oracle_rate(pool, wl["k"], info["dt"], cores, args.ref_steps, args.workload)
        finally:
            pool.close()
            pool.join()
        where = ("a 1.2 km x 1.2 km x 1.0 km box of the thrust model" if three_d else
                 "the 2 km x 1.5 km marine window")
        cpu = {"value": ob["value"], "unit": "DoF-steps/s", "cores": cores, "kind": "oracle",
               "sample": (f"FP64 oracle, KMV{wl['k']}{'tet' if three_d else 'tri'} on {where} of the "
                          f"workload ({info['E']} elements, N={info['N']}), {cores} shots in "
                          f"parallel (one per host core), {ob['nsteps']} forward + adjoint steps each, "
                          f"{ob['seconds']:.1f} s wall")}
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "DoF-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(wl["k"], args.workload),
                       "elements": E, "dofs": N, "dt": dt, "record_steps": nt_record,
                       "window_steps": nt, "shots_per_step": S,
                       "receivers": R, "ckpt_stride": args.ckpt, "C": wl["C"],
                       "l2": "inputs larger than L2 (wavefields of N*S floats, records)",
                       "parallelism": f"shots across {world} GPU(s), replicas of the mesh",
                       "gradient_store": not args.no_gradient_store and not three_d,
                       "setup_s": setup_s},
            "e2e": {"value": e2e_val, "unit": "DoF-steps/s",
                    "h2d_bytes_per_step": int(wav.nbytes + obs_h.numel() * 4 + (N * 8 if world > 1 else 0)),
                    "d2h_bytes_per_step": int(rec_h.numel() * 4 + N * 8 * (2 if world > 1 else 1))},
            "gpu_launches": int(launches),
            "roofline": roof,
            "parity_vs_oracle": parity,
            "other_degrees": extra_k,
            "cpu_baseline": cpu,
            "plain_form": plain,
            "serving": serving,
            "clocks": clk_sum,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="marine2d", choices=["marine2d", "thrust3d"],
                    help="marine2d: the 2D marine section (KMV2-5 triangles); thrust3d: the 3D "
                         "thrust section (KMV2/3 tetrahedra, use --k 2 or 3)")
    ap.add_argument("--mesh-scale", type=float, default=1.0,
                    help="thrust3d only: coarsen the mesh's boxes by this factor (< 1 for captures)")
    ap.add_argument("--k", type=int, default=None,
                    help="element degree (default 5 for marine2d, 2 for thrust3d)")
    ap.add_argument("--C", type=float, default=None)
    ap.add_argument("--shots", type=int, default=4)
    ap.add_argument("--ckpt", type=int, default=50)
    ap.add_argument("--window", type=int, default=2000)
    ap.add_argument("--no-plain", dest="plain", action="store_false",
                    help="skip timing the plain form (one shot per launch, plain layout)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the nvidia-smi clock samples of the timed region are written")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-stream latency run")
    ap.add_argument("--no-gradient-store", action="store_true",
                    help="recompute the forward field's gradients in the gradient steps instead "
                         "of storing them during the recompute (less device memory)")
    ap.add_argument("--serving-scale", type=float, default=1.0,
                    help="element-count factor of the serving pool (1 = 50k-2M triangles)")
    ap.add_argument("--extra-k", default="3,4",
                    help="other element degrees measured on the same workload (comma list; '' for none)")
    ap.add_argument("--extra-window", type=int, default=500)
    ap.add_argument("--ref-steps", type=int, default=300,
                    help="time steps per shot of the oracle's timed sample")
    args = ap.parse_args()
    if args.k is None:
        args.k = 2 if args.workload == "thrust3d" else 5
    if args.workload == "thrust3d" and args.ref_steps == 300:
        args.ref_steps = 100  # the KMV3tet oracle takes about 0.17 s per step and shot
    if args.impl == "reference":
        run_reference(args)
    elif args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        spawn_ranks(args)
    else:
        run_ours(args)


def _rank_main(rank, args, port):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(args.gpus),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    run_ours(args)


def spawn_ranks(args):
    """bench.py --gpus N without a launcher: start one process per GPU (spawn), with the
    rank variables a launcher would set; rank 0 prints the line."""
    import socket
    import torch.multiprocessing as tmp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    tmp.start_processes(_rank_main, args=(args, port), nprocs=args.gpus, start_method="spawn")


if __name__ == "__main__":
    main()
