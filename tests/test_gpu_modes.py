"""Per-mode spectra (hufield_spectrum_modes, hufield_filter_modes) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import filters, np_

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256), (64, 128), (16, 32, 64), (64, 64, 64)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_spectrum_modes(hf, shape):
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C2 if len(shape) == 3 else inputs.C1))
    plan = hf.Plan(shape)
    f = torch.empty(shape, dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, gf, 1, 0, f, plan.workspace(0, 0))
    m = torch.empty((1,) + tuple(shape), dtype=torch.int8, device="cuda")
    hf.hufield_threshold(plan, f, [0.0], m)
    M = shape[-1] // 2
    out = torch.empty(int(np.prod(shape)) // 2, dtype=torch.float32, device="cuda")
    for y in (f, m[0]):
        hf.hufield_spectrum_modes(plan, y, out, plan.workspace(1, 0))
        torch.cuda.synchronize()
        want = oracle.spectrum_modes(np_(y).astype(np.float64))[..., :M]
        got = np_(out).reshape(shape[:-1] + (M,)).astype(np.float64)
        scale = want.max()
        assert np.abs(got - want).max() <= 2e-6 * scale
        big = want > 1e-3 * scale
        assert np.abs(got[big] / want[big] - 1.0).max() < 1e-4


@pytest.mark.parametrize("shape,fk", [((256, 256), inputs.filter_kwargs(inputs.C1)),
                                      ((128, 64), dict(p=0.5, axes=(1.0, 0.5), width=0.06, supp=20.0, form=1)),
                                      ((32, 64, 16), inputs.filter_kwargs(inputs.C2)),
                                      ((32, 32, 32), dict(p=100.0, axes=(1.0, 1.0, 1.0), width=0.06, supp=20.0,
                                                          form=1))])
def test_filter_modes(hf, shape, fk):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    out = torch.empty(int(np.prod(shape)) // 2, dtype=torch.float32, device="cuda")
    hf.hufield_filter_modes(plan, gf, out)
    torch.cuda.synchronize()
    M = shape[-1] // 2
    want = (oracle.filter_grid(shape, of) ** 2)[..., :M]
    got = np_(out).reshape(shape[:-1] + (M,)).astype(np.float64)
    assert np.abs(got - want).max() <= 1e-5
    assert got.reshape(-1)[0] == 0.0
