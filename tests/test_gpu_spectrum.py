"""Standalone sign maps and spectrum calls on seeded fields against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_bins, dev_zeros, np_

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(8, 8), (256, 256), (16, 8, 32)])
def test_threshold_exact(hf, shape):
    plan = hf.Plan(shape)
    y = inputs.random_field(shape, 1, np.float32)
    levels = (0.0, 0.5, -0.5, 1.25)
    maps = torch.empty((len(levels),) + shape, dtype=torch.int8, device="cuda")
    hf.hufield_threshold(plan, torch.from_numpy(y).cuda(), levels, maps)
    yb = torch.from_numpy(y).to(torch.bfloat16)
    maps_b = torch.empty_like(maps)
    hf.hufield_threshold(plan, yb.cuda(), levels, maps_b)
    torch.cuda.synchronize()
    for i, t in enumerate(levels):
        np.testing.assert_array_equal(np_(maps[i]), oracle.threshold(y.astype(np.float64), np.float32(t)))
        np.testing.assert_array_equal(np_(maps_b[i]), oracle.threshold(yb.float().numpy().astype(np.float64),
                                                                        np.float32(t)))


SPEC_CASES = [((256, 256), 128, 1), ((64, 128), 32, 12), ((512, 512), 64, 36), ((16, 8, 32), 8, 1),
              ((32, 32, 32), 16, 1), ((8, 8), 4, 1), ((8, 4096), 64, 1), ((4096, 8), 64, 2)]


@pytest.mark.parametrize("shape,nr,nt", SPEC_CASES)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "i8"])
def test_spectrum_parity(hf, shape, nr, nt, dtype):
    plan = hf.Plan(shape)
    y = inputs.random_field(shape, 2, np.float32)
    if dtype == "f32":
        t = torch.from_numpy(y)
    elif dtype == "bf16":
        t = torch.from_numpy(y).to(torch.bfloat16)
    else:
        t = torch.from_numpy(np.where(y >= 0, 1, -1).astype(np.int8))
    yo = t.float().numpy().astype(np.float64)
    s, c = dev_zeros(nr * nt, torch.float64), dev_zeros(nr * nt, torch.int64)
    ws = plan.workspace(1, nr * nt)
    hf.hufield_spectrum(plan, t.cuda(), nr, nt, False, s, c, ws)
    hf.hufield_spectrum(plan, t.cuda(), nr, nt, True, s, c, ws)  # accumulate doubles both
    torch.cuda.synchronize()
    ws_, wc = oracle.spectrum_bins(yo, nr, nt)
    check_bins(np_(s) / 2, ws_, np_(c) // 2, wc)
    mean = torch.empty(nr * nt, dtype=torch.float64, device="cuda")
    hf.hufield_bins_mean(s, c, mean)
    torch.cuda.synchronize()
    np.testing.assert_allclose(np_(mean), np.where(wc > 0, ws_ / np.maximum(wc, 1), 0), rtol=2e-4, atol=1e-12)
