"""Pins of the oracle's filter A = sqrt(chi), Eqs. (8), (12), (13) (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from oracle import Filter


def test_superellipse_p2_is_euclidean():
    f = Filter(p=2.0, axes=(1.0, 1.0))
    rng = np.random.default_rng(0)
    for k in rng.uniform(-1, 1, size=(50, 2)):
        assert oracle.superellipse(k, f) == pytest.approx(math.hypot(*k), rel=1e-14)
    f3 = Filter(p=2.0, axes=(1.0, 1.0, 1.0))
    for k in rng.uniform(-1, 1, size=(20, 3)):
        assert oracle.superellipse(k, f3) == pytest.approx(np.linalg.norm(k), rel=1e-14)


def test_superellipse_p1_is_diamond_and_large_p_is_square():
    f1 = Filter(p=1.0, axes=(1.0, 0.5))
    fbig = Filter(p=400.0, axes=(1.0, 0.5))
    for k in [(0.3, 0.1), (-0.2, 0.4), (0.05, -0.33)]:
        assert oracle.superellipse(k, f1) == pytest.approx(abs(k[0]) / 1.0 + abs(k[1]) / 0.5, rel=1e-14)
        assert oracle.superellipse(k, fbig) == pytest.approx(max(abs(k[0]), abs(k[1]) / 0.5), rel=5e-3)


def test_superellipse_homogeneous_degree_one():
    f = Filter(p=3.3, axes=(1.0, 0.7, 1.6))
    k = np.array([0.1, -0.25, 0.3])
    assert oracle.superellipse(2.5 * k, f) == pytest.approx(2.5 * oracle.superellipse(k, f), rel=1e-13)


def test_rotation_pi_is_identity_and_half_pi_swaps_axes():
    base = dict(p=3.0, k0=0.2, width=0.05, supp=2.0)
    f0 = Filter(axes=(1.0, 0.5), rot=0.0, **base)
    fpi = Filter(axes=(1.0, 0.5), rot=math.pi, **base)
    fh = Filter(axes=(1.0, 0.5), rot=math.pi / 2, **base)
    fswap = Filter(axes=(0.5, 1.0), rot=0.0, **base)
    for k in [(0.3, 0.1), (-0.2, 0.4), (0.05, -0.33), (0.7, 0.0)]:
        assert oracle.superellipse(k, fpi) == pytest.approx(oracle.superellipse(k, f0), rel=1e-12)
        assert oracle.superellipse(k, fh) == pytest.approx(oracle.superellipse(k, fswap), rel=1e-12)


def test_rotation_direction():
    # the semi-axis a points at angle rot: a wavevector along that angle has K = |k| / a
    f = Filter(p=2.0, axes=(2.0, 0.5), rot=math.radians(30))
    k = 0.4 * np.array([math.cos(math.radians(30)), math.sin(math.radians(30))])
    assert oracle.superellipse(k, f) == pytest.approx(0.4 / 2.0, rel=1e-12)


def test_kstar_closed_forms():
    # paper form (k0 = 0): the maximum of K^alpha exp(-K^2 / (2 sigma^2)) is at sigma sqrt(alpha)
    f = Filter(form=1, k0=0.3, width=0.07, supp=20.0)
    assert oracle.kstar(f) == pytest.approx(0.07 * math.sqrt(20.0), rel=1e-14)
    # no suppression: the maximum is the band centre
    assert oracle.kstar(Filter(k0=0.3, width=0.05, supp=0.0)) == pytest.approx(0.3, rel=1e-14)


def test_filter_is_one_at_the_maximum_lattice_point():
    # k0 = 0.25, w = 0.25, s = 2 puts K* at 0.5 = kappa of n = 4 on a 16-point axis
    f = Filter(p=2.0, axes=(1.0, 1.0), k0=0.25, width=0.25, supp=2.0)
    assert oracle.kstar(f) == pytest.approx(0.5, rel=1e-15)
    assert oracle.filter_value((16, 16), (4, 0), f) == pytest.approx(1.0, abs=1e-15)
    assert oracle.filter_value((16, 16), (0, -4), f) == pytest.approx(1.0, abs=1e-15)
    H = oracle.filter_grid((64, 64), f)
    assert H.max() <= 1.0 + 1e-15


def test_filter_gaussian_special_case_is_amplitude():
    # s = 0: chi = exp(-(K-k0)^2 / (2 w^2)) and A = sqrt(chi) = exp(-(K-k0)^2 / (4 w^2))
    f = Filter(p=2.0, axes=(1.0, 1.0), k0=0.25, width=0.125, supp=0.0)
    # kappa = 2 n / 32: n = 6 -> 0.375 = k0 + w
    assert oracle.filter_value((32, 32), (6, 0), f) == pytest.approx(math.exp(-0.25), rel=1e-14)
    assert oracle.filter_value((32, 32), (4, 0), f) == pytest.approx(1.0, rel=1e-14)


def test_filter_zero_at_dc_and_nyquist_planes():
    f = Filter(p=4.0, axes=(1.0, 0.5), rot=0.4, k0=0.2, width=0.2, supp=2.0)
    H = oracle.filter_grid((16, 32), f)
    assert H[0, 0] == 0.0
    assert np.all(H[8, :] == 0.0) and np.all(H[:, 16] == 0.0)
    f3 = Filter(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.2, supp=2.0)
    H3 = oracle.filter_grid((8, 16, 8), f3)
    assert H3[0, 0, 0] == 0.0
    assert np.all(H3[4] == 0) and np.all(H3[:, 8] == 0) and np.all(H3[:, :, 4] == 0)
    assert (H3 > 0).sum() > 100


def test_filter_even():
    f = Filter(p=3.0, axes=(1.0, 0.6), rot=0.7, k0=0.2, width=0.1, supp=4.0)
    H = oracle.filter_grid((32, 64), f)
    Hm = H[(-np.arange(32)) % 32][:, (-np.arange(64)) % 64]
    np.testing.assert_allclose(H, Hm, rtol=1e-13, atol=0)


@pytest.mark.parametrize("s", [1.0, 2.0, 4.0])
def test_small_k_power_law(s):
    # chi ~ K^s as K -> 0 (the small-k expansion of the paper's form, k0 = 0): A ~ K^(s/2)
    f = Filter(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.05, supp=s, form=1)
    n = 1 << 14
    a1 = oracle.filter_value((n, 4), (1, 0), f)
    a2 = oracle.filter_value((n, 4), (2, 0), f)
    slope = math.log(a2 ** 2 / a1 ** 2) / math.log(2.0)
    assert slope == pytest.approx(s, abs=2e-3)


def test_no_suppression_is_a_plain_gaussian_band():
    # Eq. (13) with alpha = 0: chi = C exp(-K^2 / (2 sigma^2)), maximal (1) at K -> 0
    f = Filter(p=2.0, axes=(1.0, 1.0), width=0.1, supp=0.0, form=1)
    for idx in ([1, 0], [3, 4], [10, 0]):
        K = oracle.superellipse([2 * i / 64 for i in idx], f)
        assert abs(oracle.filter_value((64, 64), idx, f) - math.exp(-K * K / (4 * 0.01))) < 1e-14
