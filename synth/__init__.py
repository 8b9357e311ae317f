"""Seeded synthetic workload generators (meshes, velocity models, acquisition geometry,
source signals).

This package holds no arithmetic of the method: it builds the inputs that both the CUDA
path and the FP64 oracle consume. The paper's datasets (Marmousi2, BP2004, Overthrust3D)
are not available; these generators stand in for them with the paper's shapes (17 km x
3.5 km marine section with a 0.45 km water layer, 1.5-4.7 km/s, 40 shots, 500 receivers,
5 Hz Ricker; a 5 x 5 x 3 km 3D section).
"""
