"""Source signals fed to the solvers (inputs only)."""
import numpy as np


def ricker_samples(f, dt, nt, t0=None, dtype=np.float32):
    """Ricker wavelet w(t_n), t_n = n dt, n = 0..nt-1, centred at t0 = 1/f (unit peak).
    The paper forces every source with a Ricker wavelet of a given peak frequency
    (Section 2.1); it prints no formula, so the common form is used."""
    t0 = 1.0 / f if t0 is None else t0
    a = (np.pi * f * (np.arange(nt) * dt - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(dtype)


def sigma_max(c_max, width, R=1e-3):
    """Peak damping of the quadratic layer profile for a target reflection R:
    (3 c_max / (2 L)) ln(1/R) (a standard choice; the paper does not give the amplitude)."""
    return 1.5 * c_max / width * np.log(1.0 / R)
