"""Pins of the oracle's window variance sigma_F^2(R) (Eq. (1), Sec. II.A)."""
import math

import numpy as np
import pytest

import oracle
from oracle import Filter


def band_limited_field(shape, seed):
    # a generated field: A = 0 on every Nyquist plane, so its trigonometric interpolant is unambiguous
    return oracle.generate(shape, Filter(p=2.0, axes=(1.0,) * len(shape), k0=0.3, width=0.2, supp=2.0), seed)


def interpolant(y):
    """Signed modes k and coefficients c of g(x) = sum c e^{i k.x} interpolating y."""
    Y = np.fft.fftn(y) / y.size
    grids = np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in y.shape], indexing="ij")
    k = np.stack([2 * np.pi * g / n for g, n in zip(grids, y.shape)], axis=-1).reshape(-1, y.ndim)
    return k, Y.reshape(-1)


def ball_average_by_quadrature(y, R, nr=24, nang=48):
    """Average of the interpolant over a ball of radius R at every lattice point, by
    Gauss-Legendre in the radius and product rules over the angles (no Bessel functions)."""
    k, c = interpolant(y)
    xr, wr = np.polynomial.legendre.leggauss(nr)
    rho = 0.5 * R * (xr + 1.0)
    if y.ndim == 2:
        th = 2 * np.pi * np.arange(nang) / nang
        pts = np.stack([np.outer(rho, np.cos(th)), np.outer(rho, np.sin(th))], axis=-1).reshape(-1, 2)
        w = np.outer(0.5 * R * wr * rho, np.full(nang, 2 * np.pi / nang)).reshape(-1) / (np.pi * R * R)
    else:
        xt, wt = np.polynomial.legendre.leggauss(nang // 2)
        ph = 2 * np.pi * np.arange(nang) / nang
        st = np.sqrt(1 - xt * xt)
        dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(xt, np.ones_like(ph))], -1)
        pts = (rho[:, None, None, None] * dirs[None]).reshape(-1, 3)
        w = (0.5 * R * wr * rho * rho)[:, None, None] * wt[None, :, None] * np.full(nang, 2 * np.pi / nang)[None, None]
        w = w.reshape(-1) / (4.0 / 3.0 * np.pi * R ** 3)
    # the average at x0 is sum_k c_k e^{i k.x0} sum_q w_q e^{i k.p_q}
    kernel = np.exp(1j * pts @ k.T).T @ w
    X0 = np.stack(np.meshgrid(*[np.arange(n) for n in y.shape], indexing="ij"), -1).reshape(-1, y.ndim)
    return (np.exp(1j * X0 @ k.T) @ (c * kernel)).real


@pytest.mark.parametrize("shape,radii", [((8, 8), (0.7, 1.5, 3.2)), ((4, 4, 4), (0.6, 1.3))])
def test_window_variance_matches_quadrature(shape, radii):
    y = band_limited_field(shape, 3)
    got = oracle.window_variance(y, radii)
    for R, g in zip(radii, got):
        avg = ball_average_by_quadrature(y, R)
        want = float(np.mean((avg - avg.mean()) ** 2))
        assert abs(g - want) <= 1e-9 * max(want, 1e-12) + 1e-12, (R, g, want)


def test_window_variance_small_window_is_the_variance():
    for shape in ((32, 16), (8, 16, 8)):
        y = oracle.noise(shape, 5)
        got = oracle.window_variance(y, [1e-9])[0]
        assert abs(got - y.var()) < 1e-12 * y.var()


def test_white_noise_is_standard_nonhyperuniform():
    # unit white noise: sigma^2(R) v1(R) -> 1 (the spectrum is flat), less the part of the
    # ball's transform beyond the Brillouin zone, about 4 / (pi^2 R) in 2D
    R = np.array([6.0, 8.0, 12.0])
    acc = np.zeros_like(R)
    M = 24
    for e in range(M):
        acc += oracle.window_variance(oracle.noise((128, 128), 2, e), R)
    ratio = acc / M * np.pi * R ** 2
    assert np.all(np.abs(ratio - (1.0 - 4.0 / (np.pi ** 2 * R))) < 0.08), ratio


def test_filter_expectation_matches_realisations():
    shape = (64, 64)
    filt = Filter(p=3.0, axes=(1.0, 0.6), rot=0.4, k0=0.25, width=0.08, supp=2.0)
    R = [1.0, 3.0, 6.0]
    acc = np.zeros(3)
    M = 48
    for e in range(M):
        acc += oracle.window_variance(oracle.generate(shape, filt, 1, e), R)
    want = oracle.window_variance_filter(shape, filt, R)
    assert np.all(np.abs(acc / M / want - 1.0) < 0.15), (acc / M, want)
    np.testing.assert_allclose(oracle.window_variance_filter(shape, filt, R, sigma_f=2.0), 4.0 * want, rtol=1e-13)


@pytest.mark.parametrize("s,slope", [(2.0, -3.0), (4.0, -3.0), (0.5, -2.5), (0.0, -2.0)])
def test_class_scaling_2d(s, slope):
    # Sec. II.A: spectra ~ |k|^s at small k give sigma^2 ~ R^-(d+1) for s > 1 (class I),
    # R^-(d+s) for 0 < s < 1 (class III) and R^-d for a spectrum that does not vanish
    # at k = 0 (standard nonhyperuniform); the paper-form filter (k0 = 0) has
    # chi ~ K^s near K = 0
    shape = (1024, 1024)
    filt = Filter(p=2.0, axes=(1.0, 1.0), width=0.08, supp=s, form=1)
    R = np.array([48.0, 64.0, 96.0, 128.0])
    v = oracle.window_variance_filter(shape, filt, R)
    fit = np.polyfit(np.log(R), np.log(v), 1)[0]
    assert abs(fit - slope) < 0.15, fit


def test_class_scaling_3d():
    shape = (64, 64, 64)
    filt = Filter(p=2.0, axes=(1.0, 1.0, 1.0), width=0.25, supp=2.0, form=1)
    R = np.array([6.0, 8.0, 12.0])
    v = oracle.window_variance_filter(shape, filt, R)
    fit = np.polyfit(np.log(R), np.log(v), 1)[0]
    assert abs(fit + 4.0) < 0.25, fit
