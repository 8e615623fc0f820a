"""Generated field (noise -> r2c -> filter -> c2r -> normalise) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_field, filters, np_, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    ((256, 256), inputs.filter_kwargs(inputs.C0)),
    ((8, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.4, width=0.2, supp=2.0)),
    ((16, 64), dict(p=3.0, axes=(1.0, 0.5), rot=0.7, k0=0.3, width=0.1, supp=4.0)),
    ((64, 32), dict(p=1.0, axes=(1.0, 0.5), width=0.3, supp=2.0, form=1)),
    ((512, 512), inputs.filter_kwargs(inputs.C1)),
    ((4096, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0)),
    ((8, 4096), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0)),
    ((8, 8, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.4, width=0.2, supp=2.0)),
    ((16, 32, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.1, supp=2.0)),
    ((32, 16, 64), dict(p=2.5, axes=(1.0, 0.7, 1.3), rot=1.1, k0=0.25, width=0.08, supp=6.0)),
    ((64, 64, 64), inputs.filter_kwargs(inputs.C2)),
]


@pytest.mark.parametrize("shape,fk", CASES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else None)
def test_generate_parity(hf, shape, fk):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, gf, 0, 3, out, ws)
    torch.cuda.synchronize()
    want = oracle.generate(shape, of, 0, 3)
    check_field(np_(out), want)


# exponents across the paper's range (p from 0.5 to 50) and beyond: the terms
# |kappa_i / a_i|^p of Eq. (12) span hundreds of decades at p = 50 (p = 100
# keeps the FP64 oracle's terms above its underflow on these lattices)
WIDE_P = [
    ((256, 256), dict(p=0.5, axes=(1.0, 0.5), k0=0.2, width=0.05, supp=2.0)),
    ((256, 256), dict(p=20.0, axes=(1.0, 0.5), k0=0.2, width=0.05, supp=2.0)),
    ((256, 256), dict(p=50.0, axes=(1.0, 1.0), k0=0.15, width=0.04, supp=4.0)),
    ((256, 256), dict(p=50.0, axes=(1.0, 0.5), rot=0.4, k0=0.15, width=0.04, supp=4.0)),
    ((128, 128), dict(p=50.0, axes=(1.0, 1.0), width=0.05, supp=20.0, form=1)),
    ((32, 64, 32), dict(p=30.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.05, supp=2.0)),
    ((32, 32, 32), dict(p=100.0, axes=(1.0, 2.0, 0.5), k0=0.3, width=0.08, supp=2.0)),
    # Eq. (13) with alpha = 0 in the paper form: K* = 0, no suppression term
    ((256, 256), dict(p=2.0, axes=(1.0, 1.0), width=0.1, supp=0.0, form=1)),
]


@pytest.mark.parametrize("shape,fk", WIDE_P, ids=lambda v: str(v.get("p")) if isinstance(v, dict) else None)
def test_generate_wide_exponents(hf, shape, fk):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, gf, 4, 1, out, ws)
    torch.cuda.synchronize()
    check_field(np_(out), oracle.generate(shape, of, 4, 1))


@pytest.mark.parametrize("shape", [(256, 256), (32, 16, 64)])
def test_generate_sigma_f_and_seeds(hf, shape):
    gf, of = filters(hf, p=3.0, axes=(1.0, 0.8, 1.2), k0=0.3, width=0.1, supp=2.0)
    gf.sigma_f = 2.5
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    for seed, field in [(1, 0), (2**40 + 3, 9)]:
        hf.hufield_generate(plan, gf, seed, field, out, ws)
        torch.cuda.synchronize()
        check_field(np_(out), oracle.generate(shape, of, seed, field, sigma_f=2.5))


def test_generate_bf16_storage_error(hf):
    # BF16 storage: round to nearest with an 8-bit significand, the error uniform within
    # half an ulp (2^-8 of the binade's base): relative L2 1.6e-3 for a Gaussian field
    shape = (256, 256)
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C0))
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.bfloat16, device="cuda")
    hf.hufield_generate(plan, gf, 0, 0, out, ws)
    torch.cuda.synchronize()
    r = rel_l2(np_(out.float()).astype(np.float64), oracle.generate(shape, of, 0, 0))
    assert 1.3e-3 < r < 2.0e-3


def test_forward_spectrum(hf):
    for shape in [(64, 32), (16, 8, 32), (8, 4096)]:
        plan = hf.Plan(shape)
        ws = plan.workspace(0, 0)
        hf.hufield_forward(plan, 11, 2, ws)
        torch.cuda.synchronize()
        M = shape[-1] // 2
        half = int(np.prod(shape)) // 2
        got = np_(ws[256: 256 + half * 8].view(torch.complex64)).reshape(shape[:-1] + (M,))  # after the header
        X = np.fft.fftn(oracle.noise(shape, 11, 2))[..., :M]
        assert np.abs(got - X).max() < 2e-6 * math.sqrt(np.prod(shape)) * 4
        assert rel_l2(got.astype(np.complex128), X) < 1e-6
