"""Helpers of the GPU parity tests (comparisons only; no arithmetic of the method)."""
import math

import numpy as np
import torch

import oracle

FIELD_REL_L2 = 2e-6      # relative L2 of the FP32 field against the FP64 oracle
FIELD_MAX_ABS = 1e-4     # max |error| in units of the field rms
MAP_BAND = 1e-4          # sites with |f_oracle - t| below this (x rms) may differ
BIN_REL = 1e-4           # relative error of a bin sum
BIN_FLOOR = 1e-9         # bins below this fraction of the peak bin are compared absolutely


def f32(v):
    return float(np.float32(v))


def filters(hf_mod, **kw):
    """The same parameters, rounded to FP32 once, for the GPU and the oracle."""
    kw = dict(kw)
    axes = tuple(f32(a) for a in kw.pop("axes", (1.0, 1.0, 1.0)))
    vals = {k: f32(v) for k, v in kw.items() if k in ("p", "rot", "k0", "width", "supp")}
    form = int(kw.get("form", 0))
    g = hf_mod.Filter(axes=axes, form=form, **vals)
    o = oracle.Filter(axes=axes, form=form, **vals)
    return g, o


def np_(t):
    return t.detach().cpu().numpy()


def rel_l2(got, want):
    return float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def check_field(got, want, rel=FIELD_REL_L2):
    got = np.asarray(got, dtype=np.float64)
    rms = math.sqrt(float(np.mean(want * want)))
    r = rel_l2(got, want)
    m = float(np.abs(got - want).max()) / rms
    assert r <= rel, f"field relative L2 {r:.3e} > {rel:.1e}"
    assert m <= FIELD_MAX_ABS, f"field max |err| {m:.3e} rms > {FIELD_MAX_ABS:.1e}"
    return r, m


def check_maps(got, want, f_oracle, levels):
    """Bit-exact except where |f - t| < MAP_BAND rms; returns mismatches per level."""
    rms = math.sqrt(float(np.mean(f_oracle * f_oracle)))
    bad = []
    for i, t in enumerate(levels):
        diff = got[i] != want[i]
        near = np.abs(f_oracle - t) < MAP_BAND * rms
        assert not np.any(diff & ~near), f"level {t}: {int((diff & ~near).sum())} sign errors away from the level"
        bad.append(int(diff.sum()))
    return bad


def check_bins(got_sums, want_sums, got_counts=None, want_counts=None, flips=0, N=None):
    """Relative BIN_REL per bin (absolute below BIN_FLOOR of the peak bin mean),
    plus the exact effect bound of `flips` differing +-1 sites:
    |d sum_b| <= 4 D sqrt(c sum_b / N) + 4 D^2 c / N."""
    got_sums = np.asarray(got_sums, np.float64)
    want_sums = np.asarray(want_sums, np.float64)
    if got_counts is not None:
        np.testing.assert_array_equal(np.asarray(got_counts), np.asarray(want_counts))
    c = np.asarray(want_counts if want_counts is not None else np.ones_like(want_sums), np.float64)
    mean = np.where(c > 0, want_sums / np.maximum(c, 1), 0.0)
    floor = BIN_FLOOR * mean.max() * c
    tol = BIN_REL * np.abs(want_sums) + floor
    if flips:
        tol = tol + 4 * flips * np.sqrt(c * np.abs(want_sums) / N) + 4 * flips * flips * c / N
    err = np.abs(got_sums - want_sums)
    worst = int(np.argmax(err - tol))
    assert np.all(err <= tol), (f"bin {worst}: got {got_sums[worst]!r} want {want_sums[worst]!r} "
                                f"(count {c[worst]:.0f}, tol {tol[worst]:.3e})")
    nz = want_sums > floor
    return float(np.max(err[nz] / np.abs(want_sums[nz]))) if nz.any() else 0.0


def dev_zeros(n, dtype):
    return torch.zeros(n, dtype=dtype, device="cuda")
