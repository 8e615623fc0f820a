"""Pins of the oracle's noise: Philox4x32-10 and Box-Muller (CPU only)."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    # published known-answer vectors of Salmon et al. (SC'11)
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_noise_bits_layout():
    # word i is component i & 3 of the block with counter (i >> 2, 0, field, 0)
    bits = oracle.noise_bits((4, 6), seed=0x1234_0000_0007, field_idx=5).reshape(-1)
    for j in range(6):
        blk = oracle.philox4x32_10([j, 0, 5, 0], [0x0000_0007, 0x1234])
        assert list(bits[4 * j: 4 * j + 4]) == list(blk)


def test_noise_bits_uniform_chi2():
    bits = oracle.noise_bits((1 << 18,), seed=3).astype(np.uint64)
    top = (bits >> np.uint64(24)).astype(np.int64)  # 256 cells
    counts = np.bincount(top, minlength=256)
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4


def test_noise_fields_and_seeds_differ():
    a = oracle.noise_bits((1024,), seed=1, field_idx=0)
    b = oracle.noise_bits((1024,), seed=1, field_idx=1)
    c = oracle.noise_bits((1024,), seed=2, field_idx=0)
    assert (a != b).mean() > 0.99 and (a != c).mean() > 0.99


def test_box_muller_radius_and_angle():
    # Box-Muller closed form: z0^2 + z1^2 = -2 ln u0 and atan2(z1, z0) = 2 pi u1 (mod 2 pi)
    shape = (4096,)
    bits = oracle.noise_bits(shape, seed=11).astype(np.float64)
    z = oracle.noise(shape, seed=11)
    u = (bits + 0.5) / 2.0 ** 32
    for pair in (0, 2):
        z0, z1 = z[pair::4], z[pair + 1::4]
        u0, u1 = u[pair::4], u[pair + 1::4]
        np.testing.assert_allclose(z0 * z0 + z1 * z1, -2.0 * np.log(u0), rtol=1e-12)
        ang = np.mod(np.arctan2(z1, z0), 2 * np.pi)
        d = np.abs(np.angle(np.exp(1j * (ang - 2 * np.pi * u1))))
        assert d.max() < 1e-9


def test_noise_is_standard_normal():
    z = oracle.noise((1 << 20,), seed=7)
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 6.0 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z[:200_000], "norm").pvalue > 1e-4
    # neighbours (same block, different block) are uncorrelated
    for lag in (1, 2, 3, 4, 5):
        r = np.corrcoef(z[:-lag], z[lag:])[0, 1]
        assert abs(r) < 5.0 / np.sqrt(z.size)
