"""Host-side logic of the binding and the drivers, on the CPU: the paper's unit
conversion (Sec. III: physical sigma on a box of side L), the k-plane
reconstruction from the stored half spectrum used by the sweeps' log S(k)
images, the image writer, and the seeded parameter draws of the ragged and
surrogate workloads.  No kernel runs here."""
import math
import os

import numpy as np
import pytest

from paper_2509_08675_gb300 import builder

builder.build()  # the binding loads the library at import

from paper_2509_08675_gb300 import hufield as hf  # noqa: E402
from paper_2509_08675_gb300 import sweeps  # noqa: E402


def test_paper_filter_units():
    # Sec. III.A: 1024^2 on a box of side 100 with sigma = 2: k_Nyq = pi n / L,
    # so the width in Nyquist units is 2 / (pi 10.24); the paper's form has k0 = 0, s = alpha
    f = hf.paper_filter(alpha=20.0, sigma=2.0, p=1.5, axes=(1.0, 0.5), n=1024, L=100.0)
    assert f.form == 1 and f.k0 == 0.0 and f.supp == 20.0 and f.p == 1.5
    assert f.width == pytest.approx(2.0 / (math.pi * 1024 / 100.0), rel=1e-15)
    assert tuple(f.axes) == (1.0, 0.5)
    # 3D: 256^3 on a box of side 25
    g = hf.paper_filter(alpha=20.0, sigma=2.0, p=2.0, axes=(1.0, 1.0, 1.0), n=256, L=25.0)
    assert g.width == pytest.approx(2.0 * 25.0 / (math.pi * 256), rel=1e-15)


@pytest.mark.parametrize("shape", [(8, 8), (16, 32), (64, 16)])
def test_full_plane_mirrors_the_half_spectrum(shape):
    # the full S(n) of a real field against its stored half [n0][k1 < n1/2]
    y = np.random.default_rng(3).standard_normal(shape)
    S = np.abs(np.fft.fft2(y)) ** 2 / y.size
    half = S[:, : shape[1] // 2]
    got = sweeps.full_plane(half)
    want = np.fft.fftshift(S)
    nyq = np.fft.fftshift(np.arange(shape[1]) == shape[1] // 2)  # the unstored k1 = -n1/2 column
    assert np.isnan(got[:, nyq]).all()
    np.testing.assert_allclose(got[:, ~nyq], want[:, ~nyq], rtol=1e-12)


def test_log10_safe_floors_relative_to_the_peak():
    a = np.array([0.0, 1e-20, 1.0, 100.0])
    out = sweeps.log10_safe(a, floor=1e-6)
    np.testing.assert_allclose(out, [-4.0, -4.0, 0.0, 2.0])


def test_write_pgm_scales_to_bytes(tmp_path):
    img = np.array([[0.0, 0.5], [1.0, np.nan]])
    path = os.path.join(tmp_path, "a.pgm")
    sweeps.write_pgm(path, img)
    raw = open(path, "rb").read()
    header = b"P5 2 2 255\n"
    assert raw.startswith(header)
    assert list(raw[len(header):]) == [0, 128, 255, 0]  # NaN written as the low end


def test_surrogate_parameter_draws():
    from paper_2509_08675_gb300 import surrogate

    t = surrogate.draw_thetas(4000, 11)
    assert t.dtype == np.float32 and t.shape == (4000, 8)
    lo = [1.0, 0.5, 0.5, 0.0, 0.05, 0.01, 2.0, -1.0]
    hi = [8.0, 2.0, 2.0, math.pi, 0.4, 0.1, 6.0, 1.0]
    for j in range(8):
        assert t[:, j].min() >= np.float32(lo[j]) and t[:, j].max() <= np.float32(hi[j])
    assert set(np.unique(t[:, 6]).tolist()) == {2.0, 4.0, 6.0}
    np.testing.assert_array_equal(t, surrogate.draw_thetas(4000, 11))
    assert not np.array_equal(t, surrogate.draw_thetas(4000, 12))
    f = surrogate.theta_filter(t[0])
    assert f.p == float(t[0, 0]) and tuple(f.axes) == (float(t[0, 1]), float(t[0, 2]))
    assert (f.rot, f.k0, f.width, f.supp) == tuple(float(v) for v in t[0, 3:7])


def test_levels_and_radii_marshalling():
    # FP32 arrays for the C ABI (range checks are the library's: HUFIELD_ERR_INVALID_ARG)
    lv, n = hf._levels((0.0, 0.5, -0.5))
    assert n == 3 and [lv[i] for i in range(3)] == [0.0, 0.5, -0.5]
    lv, n = hf._levels(())
    assert n == 0 and len(lv) == 1  # never a zero-length array
    r, n = hf._radii(np.array([1.0, 2.5, 1e-3]))
    assert n == 3 and [r[i] for i in range(3)] == [1.0, 2.5, float(np.float32(1e-3))]
