"""Closed forms used to pin the oracle (test infrastructure only).

  * Ricker wavelet (the paper names it, Section 2.1, but prints no formula). Reading:
    w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0, t0 = 1/f.
  * 2D free-space Green's function of u_tt - c^2 Lap u = delta(x) delta(t):
    G(r, t) = H(ct - r) / (2 pi c sqrt(c^2 t^2 - r^2)); the response to w(t) delta(x_s)
    is G convolved in time with w. The substitution tau = r/c + s^2 removes the
    inverse square-root singularity; the remaining smooth integral is done by adaptive
    Gauss-Kronrod quadrature.
  * In the box [0, Lx] x [0, Ly] with natural (Neumann) boundaries the exact solution is
    the sum over the images at (+-x_s + 2 m Lx, +-y_s + 2 n Ly), all with sign +.
"""
import numpy as np
from scipy.integrate import quad


def ricker(t, f, t0=None):
    t0 = 1.0 / f if t0 is None else t0
    a = (np.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def green2d_ricker(r, t, c, f):
    """u(r, t) = int_{r/c}^{t} w(t - tau) / (2 pi c sqrt(c^2 tau^2 - r^2)) dtau."""
    if t <= r / c:
        return 0.0
    smax = np.sqrt(t - r / c)

    def integrand(s):
        tau = r / c + s * s
        return ricker(t - tau, f) / (np.pi * c * np.sqrt(c * (c * tau + r)))

    val, _ = quad(integrand, 0.0, smax, limit=400, epsabs=1e-13, epsrel=1e-11)
    return val


def box_image_sum(x_rec, x_src, times, c, f, Lx, Ly):
    """Exact pressure at x_rec for a Ricker point source at x_src in the Neumann box."""
    T = float(np.max(times))
    reach = c * T
    out = np.zeros(len(times))
    mx = int(np.ceil(reach / (2 * Lx))) + 1
    my = int(np.ceil(reach / (2 * Ly))) + 1
    for m in range(-mx, mx + 1):
        for sx in (x_src[0], -x_src[0]):
            for n in range(-my, my + 1):
                for sy in (x_src[1], -x_src[1]):
                    ix, iy = sx + 2 * m * Lx, sy + 2 * n * Ly
                    r = np.hypot(x_rec[0] - ix, x_rec[1] - iy)
                    if r > reach:
                        continue
                    for k, t in enumerate(times):
                        out[k] += green2d_ricker(r, t, c, f)
    return out
