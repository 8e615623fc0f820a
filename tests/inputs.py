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


def mlp_params(seed, widths=(8, 256, 256, 256, 128), in_pad=32):
    """Seeded parameters of the surrogate network (flat, layer by layer W then b):
    W uniform within +-1.5/sqrt(fan_in) (padding columns 0), b uniform within +-0.2."""
    r = np.random.default_rng(seed)
    out = []
    for l in range(len(widths) - 1):
        n_out, fan = widths[l + 1], widths[l]
        n_in = max(in_pad, fan) if l == 0 else fan
        W = np.zeros((n_out, n_in))
        W[:, :fan] = r.uniform(-1.5, 1.5, (n_out, fan)) / math.sqrt(fan)
        out += [W.reshape(-1), r.uniform(-0.2, 0.2, n_out)]
    return np.concatenate(out).astype(np.float32)


def mlp_rows(rows, seed, width=8):
    """Seeded network inputs on [-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (rows, width)).astype(np.float32)


def surrogate_thetas(rows, seed):
    """Seeded raw parameters over the surrogate's ranges: p in [1, 8], semi-axis ratios in
    [0.5, 2], rotation in [0, pi), k0 in [0.05, 0.4], width in [0.01, 0.1], s in {2, 4, 6},
    level in [-1, 1] (the ragged workload's draws)."""
    r = np.random.default_rng(seed)
    t = np.empty((rows, 8))
    t[:, 0] = r.uniform(1.0, 8.0, rows)
    t[:, 1] = r.uniform(0.5, 2.0, rows)
    t[:, 2] = r.uniform(0.5, 2.0, rows)
    t[:, 3] = r.uniform(0.0, math.pi, rows)
    t[:, 4] = r.uniform(0.05, 0.4, rows)
    t[:, 5] = r.uniform(0.01, 0.1, rows)
    t[:, 6] = r.choice([2.0, 4.0, 6.0], rows)
    t[:, 7] = r.uniform(-1.0, 1.0, rows)
    return t.astype(np.float32)
