"""Window variance sigma_F^2(R) (Eq. (1)) through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import filters, np_

pytestmark = pytest.mark.gpu

RADII = [0.0, 0.5, 1.0, 2.5, 4.0, 8.0, 16.0]
WINDOW_REL = 2e-5  # FP32 spectrum, FP64 window terms and sums


def gpu_window(hf, plan, y, radii):
    out = torch.empty(len(radii), dtype=torch.float64, device="cuda")
    ws = plan.workspace(3, 0)
    hf.hufield_window_variance(plan, y, radii, out, ws)
    torch.cuda.synchronize()
    return np_(out)


CASES = [((256, 256), inputs.filter_kwargs(inputs.C0)), ((64, 128), dict(p=3.0, axes=(1.0, 0.5), rot=0.6,
         k0=0.3, width=0.1, supp=4.0)), ((32, 16, 64), inputs.filter_kwargs(inputs.C2)),
         ((64, 64, 64), inputs.filter_kwargs(inputs.C2))]


@pytest.mark.parametrize("shape,fk", CASES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else None)
def test_window_variance_of_fields_and_maps(hf, shape, fk):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    f = torch.empty(shape, dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, gf, 2, 1, f, ws)
    m = torch.empty((1,) + tuple(shape), dtype=torch.int8, device="cuda")
    hf.hufield_threshold(plan, f, [0.0], m)
    torch.cuda.synchronize()
    for y, yo in ((f, np_(f).astype(np.float64)), (m[0], np_(m[0]).astype(np.float64)),
                  (f.to(torch.bfloat16), np_(f.to(torch.bfloat16).float()).astype(np.float64))):
        got = gpu_window(hf, plan, y, RADII)
        want = oracle.window_variance(yo, RADII)
        np.testing.assert_allclose(got, want, rtol=WINDOW_REL, atol=1e-12 * want[0])


def test_window_variance_white_noise_and_nyquist(hf):
    # white noise has all of its Nyquist plane: the plane's plain DFT must be right
    for shape in ((128, 64), (16, 32, 32)):
        plan = hf.Plan(shape)
        y = torch.from_numpy(oracle.noise(shape, 9).astype(np.float32)).cuda()
        got = gpu_window(hf, plan, y, RADII)
        want = oracle.window_variance(np_(y).astype(np.float64), RADII)
        np.testing.assert_allclose(got, want, rtol=WINDOW_REL)


FILTERS = [((1024, 1024), dict(p=2.0, axes=(1.0, 1.0), width=0.08, supp=2.0, form=1)),
           ((512, 512), inputs.filter_kwargs(inputs.C1)),
           ((256, 256), dict(p=2.0, axes=(1.0, 1.0), width=0.1, supp=0.0, form=1)),
           ((64, 64, 64), inputs.filter_kwargs(inputs.C2)),
           ((32, 64, 16), dict(p=2.5, axes=(1.0, 0.7, 1.3), rot=1.1, k0=0.25, width=0.08, supp=6.0))]


@pytest.mark.parametrize("shape,fk", FILTERS, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else None)
def test_window_variance_filter(hf, shape, fk):
    gf, of = filters(hf, **fk)
    gf.sigma_f = 1.5
    plan = hf.Plan(shape)
    radii = [0.0, 1.0, 3.0, 8.0, 24.0, 64.0]
    out = torch.empty(len(radii), dtype=torch.float64, device="cuda")
    hf.hufield_window_variance_filter(plan, gf, radii, out, plan.workspace(0, 0))
    torch.cuda.synchronize()
    want = oracle.window_variance_filter(shape, of, radii, sigma_f=1.5)
    # FP32 filter amplitudes (relative ~1e-6 each)
    np.testing.assert_allclose(np_(out), want, rtol=1e-4)


def test_window_variance_class_scaling(hf):
    # Sec. II.A: sigma^2 ~ R^-(d+1) for s > 1 (class I), R^-d without suppression
    shape = (1024, 1024)
    R = [48.0, 64.0, 96.0, 128.0]
    plan = hf.Plan(shape)
    out = torch.empty(len(R), dtype=torch.float64, device="cuda")
    for s, slope in ((2.0, -3.0), (0.0, -2.0)):
        gf, _ = filters(hf, p=2.0, axes=(1.0, 1.0), width=0.08, supp=s, form=1)
        hf.hufield_window_variance_filter(plan, gf, R, out, plan.workspace(0, 0))
        torch.cuda.synchronize()
        fit = np.polyfit(np.log(R), np.log(np_(out)), 1)[0]
        assert abs(fit - slope) < 0.15, (s, fit)


def test_window_variance_rejects_bad_radii(hf):
    plan = hf.Plan((32, 32))
    y = torch.zeros((32, 32), device="cuda")
    out = torch.empty(65, dtype=torch.float64, device="cuda")
    ws = plan.workspace(3, 0)
    for radii in ([], [-1.0], [float("nan")], [1.0] * 65):
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_window_variance(plan, y, radii, out, ws)
        assert e.value.status == hf.ERR_INVALID_ARG
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_window_variance(plan, y, [1.0], out, plan.workspace(2, 0))
    assert e.value.status == hf.ERR_WS_TOO_SMALL
