"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: only parameter sets (the
workload shapes) and seeded random arrays fed to both sides.
"""
import math

import numpy as np

# 2D 256^2, isotropic band at 0.25 k_Nyq (p = 2, axes 1:1, s = 2, w = 0.05)
C0 = dict(shape=(256, 256), p=2.0, axes=(1.0, 1.0), rot=0.0, k0=0.25, width=0.05, supp=2.0,
          levels=(0.0,), nr=128, ntheta=1)
# 2D 4096^2 ensemble: p = 4, 2:1 semi-axes rotated 30 degrees, band 0.15, width 0.03, s = 4
C1 = dict(shape=(4096, 4096), p=4.0, axes=(1.0, 0.5), rot=math.radians(30.0), k0=0.15, width=0.03,
          supp=4.0, levels=(0.0, 0.5, -0.5), nr=64, ntheta=36, nfields=64)
# 3D 512^3 / 1024^3: p = 6, semi-axes 1:1:0.5, band 0.2, width 0.04, s = 2
C2 = dict(shape=(512, 512, 512), p=6.0, axes=(1.0, 1.0, 0.5), rot=0.0, k0=0.2, width=0.04, supp=2.0,
          levels=(0.0,), nr=256, ntheta=1)


def filter_kwargs(cfg):
    return {k: cfg[k] for k in ("p", "axes", "rot", "k0", "width", "supp")}


def random_field(shape, seed, dtype=np.float64):
    """Seeded standard-normal field (for the standalone threshold/spectrum calls)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def random_filter(ndim, seed):
    """Seeded filter parameters drawn over the ranges of the ragged workload."""
    r = np.random.default_rng(seed)
    axes = (1.0,) + tuple(r.uniform(0.5, 2.0, size=ndim - 1))
    return dict(p=float(r.uniform(1.0, 8.0)), axes=axes, rot=float(r.uniform(0.0, math.pi)),
                k0=float(r.uniform(0.05, 0.4)), width=float(r.uniform(0.01, 0.1)),
                supp=float(r.choice([2.0, 4.0, 6.0])))
