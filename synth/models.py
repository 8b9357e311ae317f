"""Seeded synthetic P-wavespeed models (km/s), evaluated at arbitrary points (inputs only).

  smooth2d / smooth3d   small analytic models for parity tests
  MarineModel2D         17 x 3.5 km marine section standing in for Marmousi2/BP2004: 0.45 km
                        water at 1.5 km/s, 8 layers with seeded dipping interfaces (<= 10 deg),
                        a 60-degree normal fault with 200 m throw below 1 km, a 4.5 km/s salt
                        body, +-5 % Gaussian-smoothed perturbation (200 m correlation) below the
                        water, clipped to [1.5, 4.7]; gridded at 10 m and sampled bilinearly
                        (Section 4.6); outside the section the edge values extend into the
                        damping layer
  ThrustModel3D         5 x 5 x 3 km section standing in for Overthrust3D: layers with a
                        thrust-folded interface, two 5.5-6.0 km/s lenses, smooth perturbation,
                        c in [1.5, 6.0]
"""
import numpy as np
from scipy.ndimage import gaussian_filter


def smooth2d(X):
    return 1.6 + 0.6 * X[:, 1] + 0.2 * np.sin(2.0 * X[:, 0]) * np.cos(1.5 * X[:, 1])


def smooth3d(X):
    return 1.6 + 0.5 * X[:, 2] + 0.15 * np.sin(2.0 * X[:, 0]) * np.cos(1.5 * X[:, 1])


class Grid2D:
    """Bilinear sampling of a regular grid, clamped at the edges."""

    def __init__(self, x0, z0, dx, values):
        self.x0, self.z0, self.dx, self.v = x0, z0, dx, values

    def __call__(self, P):
        nx, nz = self.v.shape
        fx = np.clip((P[:, 0] - self.x0) / self.dx, 0, nx - 1 - 1e-9)
        fz = np.clip((P[:, 1] - self.z0) / self.dx, 0, nz - 1 - 1e-9)
        i = fx.astype(int)
        j = fz.astype(int)
        ax, az = fx - i, fz - j
        v = self.v
        return ((1 - ax) * (1 - az) * v[i, j] + ax * (1 - az) * v[i + 1, j]
                + (1 - ax) * az * v[i, j + 1] + ax * az * v[i + 1, j + 1])


def marine2d(seed=0, Lx=17.0, Lz=3.5, water=0.45, dx=0.01):
    rng = np.random.default_rng(seed)
    xs = np.arange(0, Lx + dx / 2, dx)
    zs = np.arange(0, Lz + dx / 2, dx)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    # 8 layers with dipping planar interfaces
    base = np.linspace(water + 0.25, Lz - 0.3, 8)
    dips = np.deg2rad(rng.uniform(-10, 10, 8))
    vel = np.linspace(1.7, 4.2, 9)
    # normal fault at x_f, 60 degrees, 200 m throw for depths below 1 km
    xf = rng.uniform(6.0, 11.0)
    hanging = (X - xf) > (Z - 1.0) / np.tan(np.deg2rad(60.0))
    Zs = np.where(hanging & (Z > 1.0), Z - 0.2, Z)
    c = np.full(X.shape, vel[0])
    for i in range(8):
        iface = base[i] + np.tan(dips[i]) * (X - Lx / 2)
        c = np.where(Zs > iface, vel[i + 1], c)
    # salt body (smooth super-ellipse blob ~3 x 1 km)
    sx, sz = rng.uniform(4.0, 13.0), rng.uniform(1.8, 2.6)
    r = ((X - sx) / 1.5) ** 4 + ((Z - sz) / 0.5) ** 4
    c = np.where(r < 1.0, 4.5, c)
    # +-5 % smoothed perturbation below the water
    pert = gaussian_filter(rng.standard_normal(X.shape), sigma=0.2 / dx)
    pert *= 0.05 / max(np.abs(pert).max(), 1e-12)
    c = c * (1 + pert)
    c = np.where(Z < water, 1.5, c)
    c = np.clip(c, 1.5, 4.7)
    return Grid2D(0.0, 0.0, dx, c)


def smoothed(model, sigma_km):
    """Gaussian-smoothed copy (FWI start model), water kept exact (c < 1.51 km/s)."""
    v = gaussian_filter(model.v, sigma=sigma_km / model.dx)
    v = np.where(model.v < 1.51, model.v, v)
    return Grid2D(model.x0, model.z0, model.dx, v)


class Thrust3D:
    def __init__(self, seed=0, Lx=5.0, Ly=5.0, Lz=3.0):
        rng = np.random.default_rng(seed)
        self.L = (Lx, Ly, Lz)
        self.base = np.linspace(0.3, Lz - 0.3, 6)
        self.vel = np.linspace(1.8, 4.8, 7)
        self.fold = rng.uniform(0.1, 0.3, 2)
        self.lens = [(rng.uniform(1, 4), rng.uniform(1, 4), rng.uniform(1.2, 2.4), rng.uniform(5.5, 6.0))
                     for _ in range(2)]
        self.ph = rng.uniform(0, 2 * np.pi, 3)

    def __call__(self, P):
        x, y, z = P[:, 0], P[:, 1], P[:, 2]
        c = np.full(len(P), self.vel[0])
        for i, b in enumerate(self.base):
            iface = b + (self.fold[0] * np.sin(1.2 * x + self.ph[0]) + 0.05 * x) * (i % 2)
            c = np.where(z > iface, self.vel[i + 1], c)
        for (lx, ly, lz, lv) in self.lens:
            r = ((x - lx) / 0.8) ** 2 + ((y - ly) / 0.8) ** 2 + ((z - lz) / 0.3) ** 2
            c = np.where(r < 1, lv, c)
        c = c * (1 + 0.03 * np.sin(3 * x + self.ph[1]) * np.cos(2 * y + self.ph[2]))
        c = np.where(z < 0.1, 1.5, c)
        return np.clip(c, 1.5, 6.0)
