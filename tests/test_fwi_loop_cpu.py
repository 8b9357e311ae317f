"""Host logic of the FWI outer loop (Algorithm 1) without a GPU: ShotSet sums the misfit and
the raw gradient over its shot batches, and invert() drives L-BFGS-B within the bounds. Fake
batches stand in for the library (a quadratic misfit per batch with a known minimiser)."""
import numpy as np

from paper_2108_10946_gb300 import fwi


class FakeMesh:
    def __init__(self, N):
        self.N = N
        self.nsteps = 3
        self.c = None

        class P:
            dt = 1e-3
        self.params = P()

    def set_velocity(self, c):
        self.c = np.array(c)


class FakeBatch:
    """J_b(c) = 1/2 sum w_b (c - t_b)^2: its forward/adjoint/gradient_raw calls mimic the
    library's sequence and return J_b and dJ_b/dc."""
    S, R = 1, 2

    def __init__(self, mesh, weight, target):
        self.mesh, self.w, self.t = mesh, weight, target
        self.calls = []

    def forward(self, wavelet, rec):
        self.calls.append("forward")

    def adjoint_misfit(self, observed):
        self.calls.append("adjoint_misfit")

    def gradient_raw(self, out):
        self.calls.append("gradient_raw")
        r = self.mesh.c - self.t
        out[:] = self.w * r
        return 0.5 * float(np.sum(self.w * r * r))


def test_shot_set_sums_batches_and_invert_reaches_the_bounded_minimum():
    N = 50
    rng = np.random.default_rng(0)
    m = FakeMesh(N)
    t1, t2 = rng.uniform(1.5, 4.5, N), rng.uniform(1.5, 4.5, N)
    t2[:5] = 6.0  # the combined minimiser lies outside the bounds there
    w1, w2 = rng.uniform(0.5, 2, N), rng.uniform(0.5, 2, N)
    bs = [FakeBatch(m, w1, t1), FakeBatch(m, w2, t2)]
    shots = fwi.ShotSet(m, bs, [None, None], [None, None])
    c0 = np.full(N, 2.5)
    J, g = shots.misfit_and_gradient(c0)
    assert np.isclose(J, 0.5 * np.sum(w1 * (c0 - t1) ** 2 + w2 * (c0 - t2) ** 2))
    assert np.allclose(g, w1 * (c0 - t1) + w2 * (c0 - t2))
    assert bs[0].calls == ["forward", "adjoint_misfit", "gradient_raw"]
    c, hist = fwi.invert(shots, c0, bounds=(1.0, 5.0), maxiter=50)
    exact = np.clip((w1 * t1 + w2 * t2) / (w1 + w2), 1.0, 5.0)
    assert np.allclose(c, exact, atol=1e-6)
    assert np.all(c <= 5.0) and np.all(c >= 1.0)
    Js = [h["J"] for h in hist]
    assert all(b <= a + 1e-12 for a, b in zip(Js, Js[1:]))
