"""Pins of the oracle's generator, sign maps and binned spectra (CPU only)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import Filter
from tests import inputs

F2 = Filter(p=3.0, axes=(1.0, 0.5), rot=0.5, k0=0.3, width=0.08, supp=2.0)
F3 = Filter(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.3, width=0.1, supp=2.0)


def brute_dft(a, sign):
    shape = a.shape
    out = np.zeros(shape, np.complex128)
    X = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for k in itertools.product(*[range(n) for n in shape]):
        ph = sum(k[d] * X[d] / shape[d] for d in range(len(shape)))
        out[k] = (a * np.exp(sign * 2j * np.pi * ph)).sum()
    return out


def signed(i, n):
    return i if i < n // 2 else i - n


@pytest.mark.parametrize("shape,filt", [((8, 8), F2), ((8, 16), F2), ((4, 8, 8), F3)])
def test_generate_brute_force(shape, filt):
    # every step from its definition: DFT sums, A from the pinned filter, inverse sums, Eq. (15)
    z = oracle.noise(shape, seed=3, field_idx=2)
    X = brute_dft(z, -1)
    H = np.zeros(shape)
    for k in itertools.product(*[range(n) for n in shape]):
        H[k] = oracle.filter_value(shape, [signed(k[d], shape[d]) for d in range(len(shape))], filt)
    g = brute_dft(H * X, +1).real / z.size
    f = (g - g.mean()) / g.std()
    got = oracle.generate(shape, filt, seed=3, field_idx=2)
    np.testing.assert_allclose(got, f, atol=1e-11)


@pytest.mark.parametrize("shape,filt", [((128, 64), F2), ((16, 32, 8), F3)])
def test_generate_with_library_fft(shape, filt):
    z = oracle.noise(shape, seed=1)
    G = np.fft.fftn(z) * oracle.filter_grid(shape, filt)
    g = np.fft.ifftn(G).real
    f = (g - g.mean()) / g.std()
    got, spec = oracle.generate(shape, filt, seed=1, return_spectrum=True)
    np.testing.assert_allclose(got, f, atol=1e-11)
    assert np.abs(spec - G).max() < 1e-11 * np.abs(G).max()


def test_generate_real_zero_mean_unit_variance():
    f = oracle.generate((64, 128), F2, seed=4)
    assert abs(f.mean()) < 1e-13 and abs(f.var() - 1.0) < 1e-12
    mi, rms = oracle.inverse_realness((64, 128), F2, seed=4)
    assert mi <= 1e-12 * rms
    f2 = oracle.generate((64, 128), F2, seed=4, sigma_f=2.5)
    np.testing.assert_allclose(f2, 2.5 * f, rtol=1e-13, atol=1e-13)


def test_wiener_khinchin_ensemble():
    # E |G(n)|^2 / N = A(n)^2 for unit white noise: check the ensemble ratio is 1
    shape = (32, 32)
    H2 = oracle.filter_grid(shape, F2) ** 2
    acc = np.zeros(shape)
    M = 64
    for e in range(M):
        _, G = oracle.generate(shape, F2, seed=9, field_idx=e, return_spectrum=True)
        acc += np.abs(G) ** 2 / G.size
    sel = H2 > 1e-3
    ratio = (acc[sel] / H2[sel]) / M
    # each mode's mean of M exponential(1) draws (Hermitian pairs are not independent)
    assert abs(ratio.mean() - 1.0) < 4.0 / math.sqrt(M * sel.sum() / 2)
    assert np.all(ratio < 3.0)


def test_sign_map_convention():
    f = np.array([-1.0, -0.0, 0.0, 1e-300, 0.5, 0.49999])
    assert list(oracle.threshold(f, 0.0)) == [-1, 1, 1, 1, 1, 1]
    assert list(oracle.threshold(f, 0.5)) == [-1, -1, -1, -1, 1, -1]


def test_map_spectrum_parseval_and_dc():
    f = oracle.generate((64, 64), F2, seed=2)
    m = oracle.threshold(f, 0.0).astype(np.float64)
    S = oracle.spectrum_modes(m)
    assert S.sum() == pytest.approx(m.size, rel=1e-12)
    assert S[0, 0] == pytest.approx(m.sum() ** 2 / m.size, rel=1e-12, abs=1e-12)
    Sf = oracle.spectrum_modes(f)
    assert Sf[0, 0] < 1e-20 and Sf.sum() == pytest.approx(f.size, rel=1e-12)


def test_spectrum_of_a_cosine():
    # y = cos(2 pi (3 x0 / 32 + 5 x1 / 64)): S = N/4 at the two modes +-(3, 5), zero elsewhere
    x0, x1 = np.meshgrid(np.arange(32), np.arange(64), indexing="ij")
    y = np.cos(2 * np.pi * (3 * x0 / 32 + 5 * x1 / 64))
    S = oracle.spectrum_modes(y)
    assert S[3, 5] == pytest.approx(y.size / 4, rel=1e-12)
    assert S[-3, -5] == pytest.approx(y.size / 4, rel=1e-12)
    S[3, 5] = S[-3, -5] = 0
    assert np.abs(S).max() < 1e-18 * y.size
    sums, counts = oracle.spectrum_bins(y, nr=32, ntheta=1)
    kap = math.hypot(2 * 3 / 32, 2 * 5 / 64)
    b = int(math.floor(32 * kap))
    assert sums[b] == pytest.approx(y.size / 2, rel=1e-12)
    assert abs(sums.sum() - y.size / 2) < 1e-9


def _float_bin(shape, idx, nr, ntheta):
    kap = [2.0 * idx[d] / shape[d] for d in range(len(shape))]
    r = math.sqrt(sum(k * k for k in kap))
    if r >= 1.0:
        return None, r * nr
    th = 0.0
    if ntheta > 1 and (kap[0] != 0 or kap[1] != 0):
        th = math.atan2(kap[1], kap[0]) % math.pi
    return int(r * nr) * ntheta + int(th / (math.pi / ntheta)), r * nr


@pytest.mark.parametrize("shape,nr,ntheta", [((32, 32), 16, 1), ((32, 64), 24, 1), ((64, 64), 32, 12),
                                             ((16, 16, 32), 8, 1)])
def test_bin_membership_matches_float_geometry(shape, nr, ntheta):
    # away from the boundaries the exact integer rule agrees with plain floating geometry
    checked = 0
    for k in itertools.product(*[range(n) for n in shape]):
        idx = [signed(k[d], shape[d]) for d in range(len(shape))]
        want, rr = _float_bin(shape, idx, nr, ntheta)
        if abs(rr - round(rr)) < 1e-9:
            continue
        if ntheta > 1 and (idx[0] or idx[1]):
            th = math.atan2(2.0 * idx[1] / shape[1], 2.0 * idx[0] / shape[0]) % math.pi
            t = th / (math.pi / ntheta)
            if abs(t - round(t)) < 1e-9:
                continue
        got = oracle.bin_of(shape, idx, nr, ntheta)
        assert got == (-1 if want is None else want), (idx, got, want)
        checked += 1
    assert checked > 0.8 * np.prod(shape)


def test_bin_boundaries_half_open():
    # radial: |kappa| = 0.5 exactly falls in bin nr/2; angular: 45 degrees opens sector j = ntheta/4
    assert oracle.bin_of((32, 32), (8, 0), 16, 1) == 8
    assert oracle.bin_of((32, 32), (4, 4), 16, 4) == int(16 * math.hypot(0.25, 0.25)) * 4 + 1
    assert oracle.bin_of((32, 32), (0, 5), 16, 4) == int(16 * 5 / 16) * 4 + 2
    assert oracle.bin_of((32, 32), (-3, 0), 16, 4) == int(16 * 3 / 16) * 4 + 0
    assert oracle.bin_of((32, 32), (0, -16), 16, 4) == -1


def test_bin_counts_and_sums_consistent():
    shape, nr, nt = (32, 64), 16, 6
    y = inputs.random_field(shape, 3)
    sums, counts = oracle.spectrum_bins(y, nr, nt)
    S = oracle.spectrum_modes(y)
    want_s = np.zeros(nr * nt)
    want_c = np.zeros(nr * nt, np.int64)
    inside = 0
    for k in itertools.product(range(shape[0]), range(shape[1])):
        idx = [signed(k[0], shape[0]), signed(k[1], shape[1])]
        b = oracle.bin_of(shape, idx, nr, nt)
        if b >= 0:
            want_s[b] += S[k]
            want_c[b] += 1
        kap2 = (2.0 * idx[0] / shape[0]) ** 2 + (2.0 * idx[1] / shape[1]) ** 2
        inside += kap2 < 1.0
    np.testing.assert_array_equal(counts, want_c)
    np.testing.assert_allclose(sums, want_s, rtol=1e-12, atol=1e-12)
    assert counts.sum() == inside


def test_arcsine_law_for_zero_threshold():
    # E[m(x) m(x+r)] = (2/pi) arcsin rho(r) for the sign of a Gaussian field (t = 0)
    shape = (32, 32)
    H2 = oracle.filter_grid(shape, F2) ** 2
    rho = np.fft.ifftn(H2).real
    rho /= rho.flat[0]
    want = np.fft.fftn(2.0 / np.pi * np.arcsin(np.clip(rho, -1, 1))).real / 1.0
    acc = np.zeros(shape)
    M = 96
    for e in range(M):
        f = oracle.generate(shape, F2, seed=21, field_idx=e)
        acc += oracle.spectrum_modes(oracle.threshold(f, 0.0).astype(np.float64))
    acc /= M
    # compare the ensemble power in a few radial shells (sample-variance bound)
    sel = want > 0.05 * want.max()
    assert abs(acc[sel].sum() / want[sel].sum() - 1.0) < 0.08


def _phi2_equal(t, rho):
    """P(X < t, Y < t) for standard normals with correlation rho: Phi(t)^2 plus the
    integral over r from 0 to rho of the bivariate density at (t, t), which with
    r = sin(u) is exp(-t^2 / (1 + sin u)) / (2 pi) du (Gauss-Legendre in u)."""
    from scipy.stats import norm

    x, w = np.polynomial.legendre.leggauss(48)
    top = np.arcsin(np.clip(np.asarray(rho, np.float64), -1.0, 1.0))
    u = 0.5 * top[..., None] * (x + 1.0)
    integral = 0.5 * top * np.sum(w * np.exp(-t * t / (1.0 + np.sin(u))), axis=-1) / (2.0 * np.pi)
    return norm.cdf(t) ** 2 + integral


def test_bivariate_normal_quadrature_against_scipy():
    # the quadrature used by the t != 0 pin below, against scipy's own bivariate normal CDF
    from scipy.stats import multivariate_normal

    for t in (-0.5, 0.0, 0.5, 1.2):
        for rho in (-0.9, -0.3, 0.0, 0.4, 0.95):
            want = multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]]).cdf([t, t])
            assert abs(_phi2_equal(t, rho) - want) < 1e-6, (t, rho)


@pytest.mark.parametrize("level", [0.5, -0.5])
def test_map_spectrum_for_nonzero_threshold(level):
    # m = sgn(f - t) of a unit-variance Gaussian field with correlation rho(r):
    # E[m(x) m(x+r)] = 1 - 4 Phi(t) + 4 Phi_2(t, t; rho(r)), so away from DC the
    # ensemble spectrum of the map is the DFT of that covariance (t = 0 is the
    # arcsine law above); rho = IDFT(A^2) / sum A^2 (Wiener-Khinchin, Sec. II.B)
    from scipy.stats import norm

    shape = (32, 32)
    H2 = oracle.filter_grid(shape, F2) ** 2
    rho = np.fft.ifftn(H2).real
    rho /= rho.flat[0]
    mean = 1.0 - 2.0 * norm.cdf(level)
    cov = 1.0 - 4.0 * norm.cdf(level) + 4.0 * _phi2_equal(level, rho) - mean * mean
    want = np.fft.fftn(cov).real
    acc = np.zeros(shape)
    M = 128
    for e in range(M):
        f = oracle.generate(shape, F2, seed=23, field_idx=e)
        acc += oracle.spectrum_modes(oracle.threshold(f, level).astype(np.float64))
    acc /= M
    # the sum of the covariance spectrum over all modes is N C(0) = N (1 - mean^2)
    assert abs(want.sum() / (want.size * (1.0 - mean * mean)) - 1.0) < 1e-9
    sel = want > 0.05 * want.max()
    sel[0, 0] = False  # DC carries the squared mean, checked below
    # (128 fields put the sample error near 1%; a level off by 0.2 sigma moves these by 10-15%)
    assert abs(acc[sel].sum() / want[sel].sum() - 1.0) < 0.03
    # and the broadband part a threshold adds (modes far from the band) within its sample band
    far = (want < 0.05 * want.max()) & (want > 0)
    far[0, 0] = False
    assert abs(acc[far].sum() / want[far].sum() - 1.0) < 0.04
    # DC holds the squared mean: E S(0) = N E[mbar^2] = N mean^2 + (the covariance's DC term)
    N = acc.size
    assert abs(acc[0, 0] / (N * mean * mean + want[0, 0]) - 1.0) < 0.06


def test_noise_dft_at_matches_fft():
    shape = (8, 16, 4)
    z = oracle.noise(shape, seed=5, field_idx=1)
    X = np.fft.fftn(z)
    modes = [(0, 0, 0), (1, 2, 1), (-3, 7, -2), (-4, -8, 0), (2, -5, 1)]
    got = oracle.noise_dft_at(shape, 5, 1, modes)
    for q, m in enumerate(modes):
        assert abs(got[q] - X[tuple(i % n for i, n in zip(m, shape))]) < 1e-10


def test_pipeline_consistency():
    cfg = dict(inputs.C0)
    shape = (64, 64)
    filt = Filter(**inputs.filter_kwargs(cfg))
    out = oracle.pipeline(shape, filt, seed=0, levels=(0.0, 0.5), nr=32, ntheta=1)
    f = oracle.generate(shape, filt, seed=0)
    np.testing.assert_array_equal(out["f"], f)
    np.testing.assert_array_equal(out["maps"][1], oracle.threshold(f, 0.5))
    s, c = oracle.spectrum_bins(oracle.threshold(f, 0.5).astype(float), 32, 1)
    np.testing.assert_array_equal(out["sums_m"][1], s)
    np.testing.assert_array_equal(out["counts_m"][1], c)
    np.testing.assert_array_equal(out["counts_f"], c)


def test_filter_without_power_gives_a_zero_field():
    # a band far outside the lattice (k0 = 3 k_Nyq, w = 0.01): A underflows to 0 at every
    # mode, Var g = 0 and Eq. (15) is read as f = 0; the maps are all +1 at t <= 0
    filt = Filter(p=2.0, axes=(1.0, 1.0), k0=3.0, width=0.01, supp=2.0)
    assert oracle.filter_grid((32, 32), filt).max() == 0.0
    r = oracle.pipeline((32, 32), filt, 1, levels=(0.0, 0.5), nr=16)
    assert np.all(r["f"] == 0.0)
    assert np.all(r["maps"][0] == 1) and np.all(r["maps"][1] == -1)
    assert np.all(r["sums_f"] == 0.0)


@pytest.mark.parametrize("shape,nr,nt", [((8, 16), 4, 3), ((16, 8), 8, 1), ((4, 8, 8), 4, 1)])
def test_half_bins_are_bin_of_each_stored_mode(shape, nr, nt):
    # the stored half spectrum [..][n_last/2], axes before the last in FFT order
    got = oracle.half_bins(shape, nr, nt).reshape(shape[:-1] + (shape[-1] // 2,))
    for pos in itertools.product(*[range(n) for n in shape[:-1]], range(shape[-1] // 2)):
        idx = [signed(pos[d], shape[d]) for d in range(len(shape) - 1)] + [pos[-1]]
        assert got[pos] == oracle.bin_of(shape, idx, nr, nt)
