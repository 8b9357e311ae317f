"""Shared helpers for the GPU-vs-oracle parity tests: run the same seeded case through the
CUDA library (C ABI via the ctypes binding) and through the FP64 oracle, and compare."""
import numpy as np

from oracle import assemble, kmv, wave
from oracle import mesh as om


def layer_sigma(coords, box, faces, width, smax):
    """sigma_d = smax (distance into the layer / width)^2 on the faces listed in the bit mask
    (bit 2d: below box[d][0], bit 2d+1: above box[d][1]) - the oracle-side evaluation of the
    quadratic profile of Section 2.1."""
    N, d = coords.shape
    s = np.zeros((N, d))
    for a in range(d):
        lo, hi = box[a]
        if faces & (1 << (2 * a)):
            dist = lo - coords[:, a]
            s[:, a] += np.where(dist > 0, (dist / width) ** 2, 0.0)
        if faces & (1 << (2 * a + 1)):
            dist = coords[:, a] - hi
            s[:, a] += np.where(dist > 0, (dist / width) ** 2, 0.0)
    return smax * s


def match_dofs(xa, xb, scale):
    """Permutation p with xb[p] == xa (DoFs matched by position)."""
    ka = {tuple(np.round(x / (1e-8 * scale)).astype(np.int64)): i for i, x in enumerate(xa)}
    p = np.empty(len(xb), dtype=np.int64)
    for j, x in enumerate(xb):
        p[ka[tuple(np.round(x / (1e-8 * scale)).astype(np.int64))]] = j
    return p


class OracleCase:
    """FP64 oracle for one mesh/velocity/layer configuration."""

    def __init__(self, verts, cells, k, cfun, dt, nt, layer=None, absorbing=False, water=0.0):
        dim = verts.shape[1]
        self.mesh = om.Mesh(verts, cells, kmv.kmv(dim, k))
        self.c = cfun(self.mesh.coords)
        self.sigma = None
        if layer is not None:
            self.sigma = layer_sigma(self.mesh.coords, layer["box"], layer["faces"], layer["width"],
                                     layer["smax"])
        self.ops = wave.Operators(self.mesh, self.c, dt, sigma=self.sigma, absorbing=absorbing)
        self.nt = nt
        self.mask = np.ones(self.mesh.N, dtype=bool)
        if self.sigma is not None:
            self.mask &= ~np.any(self.sigma > 0, axis=1)
        if water > 0:
            self.mask &= ~(self.c < water)

    def forward(self, src, recs, wavelet, store=False):
        H = assemble.point_matrix(self.mesh, recs)
        return self.ops.forward(wave.point_source_rhs(self.mesh, src, wavelet), self.nt, H, store=store)

    def gradient(self, src_list, recs, wavelets, residuals):
        H = assemble.point_matrix(self.mesh, recs)
        g = np.zeros(self.mesh.N)
        for src, w, res in zip(src_list, wavelets, residuals):
            _, U = self.forward(src, recs, w, store=True)
            _, gi = self.ops.adjoint(H, res, U_hist=U)
            g += gi
        return self.ops.gradient(g, self.mask)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


# ---- oracle shots in a process pool (spawn start: safe next to a CUDA context) ------------

def _oracle_shot(args):
    spec, src, recs, wavelet, res_scale = args
    from synth import models
    model = models.marine2d(spec.get("model_seed", 0))
    orc = OracleCase(spec["V"], spec["cells"], spec["k"], model, spec["dt"], spec["nt"],
                     layer=spec["layer"], absorbing=spec["absorbing"], water=spec["water"])
    need_grad = res_scale is not None
    rec, U = orc.forward(src, recs, wavelet, store=need_grad)
    g = None
    if need_grad:
        H = assemble.point_matrix(orc.mesh, recs)
        _, g = orc.ops.adjoint(H, res_scale * rec.astype(np.float32).astype(np.float64), U_hist=U)
    return rec, g


def oracle_shots(spec, srcs, recs, wavelets, res_scale=None, workers=4):
    """FP64 oracle records (and, if res_scale is given, the raw gradient sums g of Eq.
    gradient3 for the residual res_scale * float32(records)) of every shot on the marine
    model, one shot per worker of a spawn-started process pool. spec: V, cells, k, dt, nt,
    layer (dict or None), absorbing, water."""
    import multiprocessing as mp
    jobs = [(spec, np.asarray(s, np.float64), np.asarray(recs, np.float64),
             np.asarray(w, np.float64), res_scale) for s, w in zip(srcs, wavelets)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, len(jobs))) as pool:
        out = pool.map(_oracle_shot, jobs)
    return [o[0] for o in out], [o[1] for o in out]
