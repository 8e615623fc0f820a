"""Pins of the oracle's noise-shaped binarisation (first-order sigma-delta
along axis 0, in strips).  Sec. II.B observes that the plain sign map loses
the field's hyperuniform scaling, and Sec. IV leaves binarisations that keep
it to future work; this is the strategy built here.  With
u = clamp(g (f - t), -1, 1), each column of each strip runs v = u + e,
m = sgn(v) (+1 at v = 0), e <- v - m from e = 0.

The pins do not re-run that recurrence: they check worked examples done by
hand, closed forms (zero input, saturated input), the invariants the
recurrence implies (|e| <= 1, the prefix sums of m - u are -e, exact for
dyadic inputs), the first-difference form of the quantisation error in
Fourier space (against numpy's FFT), strip independence, the automatic gain
against numpy, and the purpose of the method: near k = 0 the map's spectrum
is far below the plain sign map's.
"""
import numpy as np
import pytest

import oracle
from tests import inputs


def test_worked_example_by_hand():
    # u = (0.5, 0.5, -0.25, 0.75), gain 1, one strip of 4 rows:
    #   v = 0.5  -> m = +1, e = -0.5
    #   v = 0    -> m = +1 (v >= 0), e = -1
    #   v = -1.25 -> m = -1, e = -0.25
    #   v = 0.5  -> m = +1, e = -0.5
    f = np.array([0.5, 0.5, -0.25, 0.75], np.float32).reshape(4, 1)
    m, e = oracle.sigma_delta(f, gain=1.0, strip=4, return_error=True)
    assert m.ravel().tolist() == [1, 1, -1, 1]
    assert e.ravel().tolist() == [-0.5, -1.0, -0.25, -0.5]
    # two strips of 2 rows: the second strip restarts from e = 0
    #   strip 0: v = 0.5 -> +1, e = -0.5; v = 0 -> +1, e = -1
    #   strip 1: v = -0.25 -> -1, e = 0.75; v = 1.5 -> +1, e = 0.5
    m, e = oracle.sigma_delta(f, gain=1.0, strip=2, return_error=True)
    assert m.ravel().tolist() == [1, 1, -1, 1]
    assert e.ravel().tolist() == [-0.5, -1.0, 0.75, 0.5]
    # level and gain: f = 3, t = 1, g = 0.25 gives u = 0.5 at every row
    #   e: 0 -> -0.5 -> 0 -> -0.5 ..., m alternates +1, +1?  v = 0.5 -> +1 (e -0.5),
    #   v = 0 -> +1 (e -1), v = -0.5 -> -1 (e 0.5), v = 1 -> +1 (e 0): period 4, mean 1/2
    m = oracle.sigma_delta(np.full((8, 1), 3.0, np.float32), t=1.0, gain=0.25, strip=8)
    assert m.ravel().tolist() == [1, 1, -1, 1, 1, 1, -1, 1]


def test_columns_and_axis():
    # every column runs on its own along axis 0: a 4 x 3 lattice whose columns
    # are three different worked sequences
    cols = [[0.5, 0.5, -0.25, 0.75], [0.0, 0.0, 0.0, 0.0], [-1.0, -1.0, 1.0, 1.0]]
    f = np.array(cols, np.float32).T.copy()
    m = oracle.sigma_delta(f, gain=1.0, strip=4)
    assert m[:, 0].tolist() == [1, 1, -1, 1]
    assert m[:, 1].tolist() == [1, -1, 1, -1]
    assert m[:, 2].tolist() == [-1, -1, 1, 1]
    # 3D: the recurrence runs along axis 0 only, each (i1, i2) its own column
    g = inputs.random_field((16, 4, 8), 3, np.float32)
    m3 = oracle.sigma_delta(g, gain=0.4, strip=16)
    for i1 in range(4):
        for i2 in range(8):
            col = np.ascontiguousarray(g[:, i1, i2]).reshape(16, 1)
            assert (oracle.sigma_delta(col, gain=0.4, strip=16).ravel() == m3[:, i1, i2]).all()


def test_zero_and_saturated_inputs():
    # u = 0: e alternates 0, -1, so the map alternates +1, -1 down every column
    # of every strip (a checkerboard along axis 0 at the Nyquist wavenumber)
    m, e = oracle.sigma_delta(np.zeros((32, 16), np.float32), gain=1.0, strip=8, return_error=True)
    want = np.where(np.arange(32) % 2 == 0, 1, -1)[:, None] * np.ones((1, 16), np.int64)
    assert (m == want).all()
    assert (e == np.where(np.arange(32) % 2 == 0, -1.0, 0.0)[:, None]).all()
    # f == t everywhere: max |f - t| = 0, the automatic gain is 0 and u = 0
    assert oracle.sd_gain(np.full((8, 8), 2.5, np.float32), 2.5) == 0.0
    assert (oracle.sigma_delta(np.full((8, 8), 2.5, np.float32), t=2.5) == want[:8, :8]).all()
    # |u| = 1 (saturated by the clamp): e stays 0 and m = sgn(f - t)
    f = inputs.random_field((64, 32), 5, np.float32)
    f = np.where(np.abs(f) < 0.1, 0.5, f).astype(np.float32)
    m, e = oracle.sigma_delta(f, gain=1e6, strip=64, return_error=True)
    assert (m == np.where(f >= 0, 1, -1)).all() and (e == 0).all()


@pytest.mark.parametrize("gain", [0.0, 0.375, 2.0])
def test_error_bound_and_prefix_sums(gain):
    # |e| <= 1, and within every strip the prefix sums of m - u equal -e (the
    # quantisation error is a first difference): exact in FP32 for dyadic data
    rng = np.random.default_rng(11)
    f = (rng.integers(-1024, 1025, size=(64, 48)) / 1024.0).astype(np.float32)
    g = 1.0 if gain == 0.0 else gain
    u = np.clip(f * np.float32(g), -1, 1).astype(np.float64)
    for h in (64, 16, 1):
        m, e = oracle.sigma_delta(f, gain=g, strip=h, return_error=True)
        assert np.abs(e).max() <= 1.0
        d = (m - u).reshape(64 // h, h, 48)
        assert np.array_equal(np.cumsum(d, axis=1), -e.reshape(64 // h, h, 48).astype(np.float64))
    # random FP32 data: the same identity up to the rounding of 64 additions
    f = inputs.random_field((64, 48), 12, np.float32)
    m, e = oracle.sigma_delta(f, gain=gain, strip=32, return_error=True)
    g = oracle.sd_gain(f) if gain == 0.0 else gain
    u = np.clip(f.astype(np.float64) * g, -1, 1)
    assert np.abs(e).max() <= 1.0
    d = (m - u).reshape(2, 32, 48)
    assert np.abs(np.cumsum(d, axis=1) + e.reshape(2, 32, 48)).max() < 64 * 2.0 ** -22


def test_quantisation_error_is_a_first_difference_in_fourier_space():
    # one strip over the whole axis: q = m - u = e_prev - e with e_prev = 0 at
    # row 0, so along axis 0 Q(n0) = (w - 1) E(n0) - e_last with w = exp(-2 pi i n0 / N0)
    f = inputs.random_field((128, 64), 21, np.float32)
    m, e = oracle.sigma_delta(f, strip=128, return_error=True)
    g = oracle.sd_gain(f)
    u = np.clip((f * np.float32(g)).astype(np.float32), -1, 1).astype(np.float64)
    Q = np.fft.fft(m - u, axis=0)
    E = np.fft.fft(e.astype(np.float64), axis=0)
    w = np.exp(-2j * np.pi * np.arange(128) / 128)[:, None]
    want = (w - 1) * E - e[-1].astype(np.float64)[None, :]
    assert np.abs(Q - want).max() < 1e-9 * np.abs(Q).max() + 1e-5


def test_strips_are_independent():
    f = inputs.random_field((64, 32), 31, np.float32)
    g = oracle.sd_gain(f)
    m = oracle.sigma_delta(f, gain=g, strip=16)
    for s in range(4):
        part = np.ascontiguousarray(f[16 * s:16 * (s + 1)])
        assert (oracle.sigma_delta(part, gain=g, strip=16) == m[16 * s:16 * (s + 1)]).all()
    # the automatic gain of the whole field is used in every strip
    assert (oracle.sigma_delta(f, strip=16) == m).all()
    # strip 0 is min(n0, 256)
    assert (oracle.sigma_delta(f) == oracle.sigma_delta(f, strip=64)).all()
    with pytest.raises(ValueError):
        oracle.sigma_delta(f, strip=48)


def test_automatic_gain_against_numpy():
    for seed, t in ((1, 0.0), (2, 0.5), (3, -1.25)):
        f = inputs.random_field((32, 32), seed, np.float32)
        want = np.float32(1.0) / np.abs(f - np.float32(t)).max()
        assert oracle.sd_gain(f, t) == want


def test_level_sets_the_volume_fraction_of_u():
    # each column's mean of m tracks that of u = g (f - t) within 1 / h
    f = inputs.random_field((256, 64), 41, np.float32)
    for t in (-0.5, 0.0, 0.7):
        g = oracle.sd_gain(f, t)
        m = oracle.sigma_delta(f, t=t, gain=g, strip=256)
        u = np.clip((f.astype(np.float64) - t) * g, -1, 1)
        assert np.abs(m.mean(axis=0) - u.mean(axis=0)).max() <= 1.0 / 256 + 1e-6


def test_keeps_the_small_k_suppression_the_sign_map_loses():
    # Sec. II.B: the sign map refills the spectrum near k = 0.  Over eight
    # hyperuniform fields (s = 2, band at k0 = 0.25), the sigma-delta map's
    # lowest radial bins stay 30 to 200 times below the sign map's,
    # and they rise with k (no plateau at k -> 0)
    shape, nr = (128, 128), 32
    filt = oracle.Filter(p=2, axes=(1, 1), k0=0.25, width=0.05, supp=2)
    acc = {"sign": 0.0, "sd": 0.0}
    for seed in range(8):
        f = oracle.generate(shape, filt, seed).astype(np.float32)
        for name, y in (("sign", oracle.threshold(f, 0.0)), ("sd", oracle.sigma_delta(f))):
            s, c = oracle.spectrum_bins(y, nr)
            acc[name] = acc[name] + s / c
    sign, sd = acc["sign"] / 8, acc["sd"] / 8
    assert sign[1:4].min() > 0.3
    assert (sd[1:4] < 0.03 * sign[1:4]).all()
    assert sd[1] < sd[3] < sd[6]


def test_keeps_the_small_k_suppression_in_3d():
    # the same in 3D: eight 64^3 fields (s = 2, band at k0 = 0.4), strips of the whole
    # axis; the lowest bins stay below 4% of the sign map's.  Their floor (about
    # E[e^2] / h, h = 64 here) is the strip starts' term
    shape, nr = (64, 64, 64), 32
    filt = oracle.Filter(p=2, axes=(1, 1, 1), k0=0.4, width=0.08, supp=2)
    acc = {"sign": 0.0, "sd": 0.0}
    for seed in range(8):
        f = oracle.generate(shape, filt, seed).astype(np.float32)
        for name, y in (("sign", oracle.threshold(f, 0.0)), ("sd", oracle.sigma_delta(f))):
            s, c = oracle.spectrum_bins(y, nr)
            acc[name] = acc[name] + s / c
    sign, sd = acc["sign"] / 8, acc["sd"] / 8
    assert sign[1:5].min() > 0.3
    assert (sd[1:5] < 0.04 * sign[1:5]).all()
    assert sd[1:5].max() < 0.05
    assert sd[2] < sd[6] < sd[10]


def test_window_variance_keeps_the_fields_class():
    # Sec. II.A defines hyperuniformity by the window variance of Eq. (1):
    # sigma^2(R) falls faster than R^-d.  Eight 256^2 fields with s = 2 fall as
    # R^-(d+1) = R^-3; the sign map's local slope drifts back toward -d = -2, the
    # noise-shaped map's stays with the field's
    shape = (256, 256)
    filt = oracle.Filter(p=2, axes=(1, 1), k0=0.25, width=0.05, supp=2)
    radii = np.array([8.0, 11.3, 16.0, 22.6, 32.0])
    acc = {"f": 0.0, "sign": 0.0, "sd": 0.0}
    for seed in range(8):
        f = oracle.generate(shape, filt, seed).astype(np.float32)
        for name, y in (("f", f), ("sign", oracle.threshold(f, 0.0)), ("sd", oracle.sigma_delta(f))):
            acc[name] = acc[name] + oracle.window_variance(y.astype(np.float64), radii)
    slope = {k: np.polyfit(np.log(radii), np.log(v), 1)[0] for k, v in acc.items()}
    local = {k: np.diff(np.log(v)) / np.diff(np.log(radii)) for k, v in acc.items()}
    assert slope["f"] == pytest.approx(-3.0, abs=0.1)
    assert slope["sd"] == pytest.approx(slope["f"], abs=0.15)
    assert local["sd"].max() < -2.8
    assert local["sign"][-1] > -2.4 and local["sign"][-1] > local["sign"][0]
