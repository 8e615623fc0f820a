"""Pins of the oracle's own radix-2 DFT (CPU only)."""
import itertools

import numpy as np
import pytest

import oracle


def brute_dft(a, sign=-1):
    """O(N^2) DFT from the definition, one output at a time."""
    shape = a.shape
    out = np.zeros(shape, np.complex128)
    grids = [np.arange(n) for n in shape]
    X = np.meshgrid(*grids, indexing="ij")
    for k in itertools.product(*[range(n) for n in shape]):
        ph = sum(k[d] * X[d] / shape[d] for d in range(len(shape)))
        out[k] = (a * np.exp(sign * 2j * np.pi * ph)).sum()
    return out


@pytest.mark.parametrize("shape", [(8,), (16,), (8, 8), (8, 16), (16, 4), (4, 4, 4), (2, 4, 8)])
def test_fft_matches_definition(shape):
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    np.testing.assert_allclose(oracle.fftn(a), brute_dft(a, -1), atol=1e-11)
    np.testing.assert_allclose(oracle.fftn(a, inverse=True), brute_dft(a, +1), atol=1e-11)


@pytest.mark.parametrize("shape", [(256, 256), (64, 32), (32, 16, 64)])
def test_fft_matches_library(shape):
    rng = np.random.default_rng(5)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = np.fft.fftn(a)
    got = oracle.fftn(a)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_fft_roundtrip_and_parseval():
    rng = np.random.default_rng(9)
    a = rng.standard_normal((64, 128))
    X = oracle.fftn(a)
    back = oracle.fftn(X, inverse=True) / a.size
    assert np.abs(back - a).max() < 1e-13
    np.testing.assert_allclose((np.abs(X) ** 2).sum() / a.size, (a * a).sum(), rtol=1e-13)


def test_real_input_hermitian():
    a = np.random.default_rng(1).standard_normal((16, 32))
    X = oracle.fftn(a)
    Xm = np.conj(X[(-np.arange(16)) % 16][:, (-np.arange(32)) % 32])
    assert np.abs(X - Xm).max() < 1e-12
