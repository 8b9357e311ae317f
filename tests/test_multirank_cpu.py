"""The multi-GPU path on CPU ranks (gloo, world size 2): shots are dealt to ranks with no
collective on the data path, and the per-rank gradients are summed once by an all-reduce,
which must equal the single-process sum over the same shots (Eq. gradient3 sums over
shots)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_util import OracleCase
    from synth import meshes, models, signals
    V, C = meshes.structured_tri(6, 6)
    probe = OracleCase(V, C, 2, models.smooth2d, 1.0, 1)
    dt = 0.8 * probe.ops.cfl_dt()
    nt = int(0.4 / dt)
    orc = OracleCase(V, C, 2, models.smooth2d, dt, nt)
    srcs = [[0.2, 0.2], [0.4, 0.25], [0.6, 0.2], [0.8, 0.3]]
    recs = np.array([[x, 0.8] for x in np.linspace(0.1, 0.9, 5)])
    w = signals.ricker_samples(8.0, dt, nt).astype(np.float64)
    return orc, srcs, recs, w


def _rank_gradient(orc, srcs, recs, w, shots):
    res = [0.3 * orc.forward(srcs[i], recs, w)[0] for i in shots]
    return orc.gradient([srcs[i] for i in shots], recs, [w] * len(shots), res)


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    orc, srcs, recs, w = _case()
    shots = bench.shots_for_rank(len(srcs), 2, rank, world)
    g = torch.from_numpy(_rank_gradient(orc, srcs, recs, w, shots))
    dist.all_reduce(g)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # max over ranks, as bench.py does for time
    if rank == 0:
        out.put((g.numpy(), float(t.item()), shots))
    dist.destroy_process_group()


def test_shot_dealing_covers_every_shot_once():
    import bench
    for nshots, S, world in ((40, 4, 2), (32, 8, 4), (16, 2, 8)):
        seen = []
        for step in range(nshots // (S * world)):
            for rank in range(world):
                seen += bench.shots_for_rank(nshots, S, rank, world, step)
        assert sorted(seen) == list(range(nshots))


def test_two_rank_gradient_allreduce_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    g2, tmax, _ = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    orc, srcs, recs, w = _case()
    g1 = _rank_gradient(orc, srcs, recs, w, [0, 1, 2, 3])
    assert tmax == 2.0
    assert np.allclose(g2, g1, rtol=1e-12, atol=1e-14 * np.abs(g1).max())
