"""Pins of the oracle's k-space noise (Sec. II.B, i.i.d. Gaussian coefficients
drawn directly on the lattice with the Hermitian pairing of a real field)."""
import math

import numpy as np
import pytest

import oracle
from oracle import Filter

scipy_stats = pytest.importorskip("scipy.stats")

F2 = Filter(p=3.0, axes=(1.0, 0.5), rot=0.5, k0=0.3, width=0.08, supp=2.0)
F3 = Filter(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.3, width=0.1, supp=2.0)


def mirror(X):
    idx = tuple((-np.arange(n)) % n for n in X.shape)
    return X[np.ix_(*idx)]


@pytest.mark.parametrize("shape", [(8, 16), (16, 8), (4, 4), (8, 8, 8), (4, 16, 8), (16, 4, 32)])
def test_hermitian_pairing_gives_a_real_field(shape):
    X = oracle.kspace_noise(shape, seed=5, field_idx=1)
    assert np.array_equal(X, np.conj(mirror(X)))
    # self-conjugate modes (every index 0 or N/2) are real
    for corner in np.ndindex(*([2] * len(shape))):
        k = tuple(c * n // 2 for c, n in zip(corner, shape))
        assert X[k].imag == 0.0
    x = oracle.fftn(X, inverse=True) / X.size
    assert np.abs(x.imag).max() <= 1e-12 * np.sqrt((x.real ** 2).mean())


def test_half_spectrum_draw_closed_form():
    # interior modes of the half: |X|^2 / (N/2) = -2 ln u_a and arg X = 2 pi u_b, with
    # (u_a, u_b) the first pair of Philox block J = row (N_last/4 + 1) + k_last // 2
    # (counter word 3 = 1) for even k_last, the second for odd k_last
    seed = 0x1234_5678_9ABC
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for shape in ((8, 16), (4, 8, 32)):
        N, nlast = int(np.prod(shape)), shape[-1]
        X = oracle.kspace_noise(shape, seed=seed, field_idx=3)
        for idx in np.ndindex(*shape[:-1]):
            row = int(np.ravel_multi_index(idx, shape[:-1]))
            for kl in range(1, nlast // 2):
                J = row * (nlast // 4 + 1) + kl // 2
                x = oracle.philox4x32_10([J, 0, 3, 1], key).astype(np.float64)
                u = (x + 0.5) / 2.0 ** 32
                ua, ub = (u[0], u[1]) if kl % 2 == 0 else (u[2], u[3])
                z = X[idx + (kl,)]
                assert abs(abs(z) ** 2 / (N / 2) - (-2.0 * math.log(ua))) < 1e-12 * max(1.0, abs(z) ** 2)
                assert abs(np.angle(z * np.exp(-2j * np.pi * ub))) < 1e-12


def test_hermitian_plane_takes_the_smaller_row():
    # on k_last = 0 the mode with the smaller row index is the drawn one
    shape = (8, 16)
    X = oracle.kspace_noise(shape, seed=2)
    key = [2, 0]
    for n0 in (1, 2, 3):
        J = n0 * 5
        x = oracle.philox4x32_10([J, 0, 0, 1], key).astype(np.float64)
        u = (x + 0.5) / 2.0 ** 32
        r = math.sqrt(64.0) * math.sqrt(-2.0 * math.log(u[0]))
        want = r * np.exp(2j * np.pi * u[1])
        assert abs(X[n0, 0] - want) < 1e-12 * r
        assert abs(X[8 - n0, 0] - np.conj(want)) < 1e-12 * r
    # self-conjugate (4, 0): sqrt(N) Re Z of its own draw
    x = oracle.philox4x32_10([4 * 5, 0, 0, 1], key).astype(np.float64)
    u = (x + 0.5) / 2.0 ** 32
    want = math.sqrt(128.0) * math.sqrt(-2.0 * math.log(u[0])) * math.cos(2 * math.pi * u[1])
    assert abs(X[4, 0] - want) < 1e-12 * max(1.0, abs(want))


def test_moments_of_the_coefficients():
    shape = (256, 256)
    N = 256 * 256
    X = oracle.kspace_noise(shape, seed=7)
    half = X[:, 1:128].reshape(-1) / math.sqrt(N)  # independent interior modes
    m = half.size
    assert abs((np.abs(half) ** 2).mean() - 1.0) < 5.0 / math.sqrt(m)
    assert abs((half.real ** 2).mean() - 0.5) < 5.0 * math.sqrt(0.5 / m)
    assert abs((half.imag ** 2).mean() - 0.5) < 5.0 * math.sqrt(0.5 / m)
    assert abs((half.real * half.imag).mean()) < 5.0 * math.sqrt(0.25 / m)
    # neighbours in k_last share a Philox block but not a pair: uncorrelated
    a = X[:, 1:127:2].reshape(-1)
    b = X[:, 2:128:2].reshape(-1)
    assert abs((a * np.conj(b)).mean() / N) < 5.0 / math.sqrt(a.size)
    assert abs((np.abs(a) ** 2 * np.abs(b) ** 2).mean() / N ** 2 - 1.0) < 10.0 / math.sqrt(a.size)
    # other field indices and seeds give other numbers
    Y = oracle.kspace_noise(shape, seed=7, field_idx=1)
    assert abs((X[:, 1:128] * np.conj(Y[:, 1:128])).mean() / N) < 5.0 / math.sqrt(m)


def test_inverse_is_unit_white_noise():
    shape = (256, 256)
    x = (oracle.fftn(oracle.kspace_noise(shape, seed=3), inverse=True) / (256 * 256)).real
    # Var x = sum E|X|^2 / N^2 = 1, Gaussian, uncorrelated neighbours
    n = x.size
    assert abs(x.mean()) < 5.0 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 6.0 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(x.reshape(-1)[::3], "norm").pvalue > 1e-4
    for ax in (0, 1):
        r = (x * np.roll(x, 1, axis=ax)).mean() / x.var()
        assert abs(r) < 5.0 / math.sqrt(n)


@pytest.mark.parametrize("shape,filt", [((32, 64), F2), ((8, 16, 16), F3)])
def test_generate_kspace_steps(shape, filt):
    # the same filter, inverse and normalisation as the real-space path, on the k-space coefficients
    X = oracle.kspace_noise(shape, seed=4, field_idx=2)
    G = X * oracle.filter_grid(shape, filt)
    g = np.fft.ifftn(G).real
    f = (g - g.mean()) / g.std()
    got, spec = oracle.generate(shape, filt, seed=4, field_idx=2, return_spectrum=True, noise="kspace")
    np.testing.assert_allclose(got, f, atol=1e-11)
    assert np.abs(spec - G).max() < 1e-11 * np.abs(G).max()
    assert abs(got.mean()) < 1e-13 and abs(got.var() - 1.0) < 1e-12


def test_wiener_khinchin_kspace_ensemble():
    shape = (32, 32)
    H2 = oracle.filter_grid(shape, F2) ** 2
    acc = np.zeros(shape)
    M = 64
    for e in range(M):
        _, G = oracle.generate(shape, F2, seed=9, field_idx=e, return_spectrum=True, noise="kspace")
        acc += np.abs(G) ** 2 / G.size
    sel = H2 > 1e-3
    ratio = (acc[sel] / H2[sel]) / M
    assert abs(ratio.mean() - 1.0) < 4.0 / math.sqrt(M * sel.sum() / 2)
    assert np.all(ratio < 3.0)


def test_kspace_and_real_space_agree_in_distribution():
    # binned map spectra of the two noise modes agree within their sampling error
    shape = (64, 64)
    M = 24
    acc = {}
    for mode in ("real", "kspace"):
        s = np.zeros(32)
        s2 = np.zeros(32)
        for e in range(M):
            r = oracle.pipeline(shape, F2, seed=1, field_idx=e, levels=(0.0,), nr=32, noise=mode)
            v = r["sums_m"][0] / np.maximum(r["counts_m"][0], 1)
            s += v
            s2 += v * v
        acc[mode] = (s / M, np.sqrt(np.maximum(s2 / M - (s / M) ** 2, 0.0) / M))
    (a, ea), (b, eb) = acc["real"], acc["kspace"]
    z = np.abs(a - b) / np.sqrt(ea ** 2 + eb ** 2 + 1e-30)
    sel = (ea > 0) & (eb > 0)
    assert np.median(z[sel]) < 1.5 and z[sel].max() < 6.0


def test_pipeline_kspace_consistency():
    shape = (32, 32)
    r = oracle.pipeline(shape, F2, seed=3, levels=(0.0, 0.5), nr=16, noise="kspace")
    f = oracle.generate(shape, F2, seed=3, noise="kspace")
    np.testing.assert_array_equal(r["f"], f)
    np.testing.assert_array_equal(r["maps"][1], oracle.threshold(f, 0.5))
    with pytest.raises(ValueError):
        oracle.generate(shape, F2, seed=3, noise="fourier")
