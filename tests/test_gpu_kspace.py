"""k-space noise path (plans with HUFIELD_PLAN_KSPACE_NOISE) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_bins, check_field, filters, np_
from tests.test_gpu_pipeline import compare, run_pipeline

pytestmark = pytest.mark.gpu

CASES = [
    ("C0-256^2", (256, 256), inputs.filter_kwargs(inputs.C0), (0.0,), 128, 1),
    ("2d-8x8", (8, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.4, width=0.3, supp=2.0), (0.0, 0.25), 4, 3),
    ("2d-aniso-16x64", (16, 64), dict(p=3.0, axes=(1.0, 0.5), rot=0.7, k0=0.3, width=0.1, supp=4.0),
     (0.0, 0.5, -0.5), 8, 6),
    ("2d-paper-64x32", (64, 32), dict(p=1.0, axes=(1.0, 0.5), width=0.3, supp=2.0, form=1), (0.0,), 16, 1),
    ("C1-like-512^2", (512, 512), inputs.filter_kwargs(inputs.C1), (0.0, 0.5, -0.5), 64, 36),
    ("2d-4096x8", (4096, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0), (0.0,), 32, 1),
    ("2d-8x4096", (8, 4096), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0), (0.0,), 32, 4),
    ("3d-8^3", (8, 8, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.4, width=0.2, supp=2.0), (0.0,), 4, 1),
    ("3d-16x32x8", (16, 32, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.1, supp=2.0), (0.0, 0.5), 16, 1),
    ("3d-rot-32x16x64", (32, 16, 64), dict(p=2.5, axes=(1.0, 0.7, 1.3), rot=1.1, k0=0.25, width=0.08, supp=6.0),
     (0.0,), 32, 1),
    ("C2-like-64^3", (64, 64, 64), inputs.filter_kwargs(inputs.C2), (0.0,), 32, 1),
]


@pytest.mark.parametrize("name,shape,fk,levels,nr,nt", CASES, ids=[c[0] for c in CASES])
def test_kspace_pipeline_parity(hf, name, shape, fk, levels, nr, nt):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape, kspace=True)
    got = run_pipeline(hf, plan, gf, shape, 5, 2, levels, nr, nt)
    want = oracle.pipeline(shape, of, 5, 2, levels=levels, nr=nr, ntheta=nt, noise="kspace")
    compare(got, want, levels, int(np.prod(shape)))


@pytest.mark.parametrize("shape", [(256, 256), (32, 16, 64)])
def test_kspace_generate_seeds_and_fields(hf, shape):
    gf, of = filters(hf, p=3.0, axes=(1.0, 0.8, 1.2), k0=0.3, width=0.1, supp=2.0)
    plan = hf.Plan(shape, kspace=True)
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    for seed, field in [(1, 0), (2**40 + 3, 9)]:
        hf.hufield_generate(plan, gf, seed, field, out, ws)
        torch.cuda.synchronize()
        check_field(np_(out), oracle.generate(shape, of, seed, field, noise="kspace"))


def test_kspace_differs_from_real_space_noise(hf):
    # the two noise modes give independent fields of the same law
    shape = (256, 256)
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C0))
    outs = []
    for ks in (False, True):
        plan = hf.Plan(shape, kspace=ks)
        ws = plan.workspace(0, 0)
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
        hf.hufield_generate(plan, gf, 0, 0, out, ws)
        torch.cuda.synchronize()
        outs.append(np_(out).astype(np.float64))
    a, b = outs
    assert abs(a.var() - 1.0) < 1e-5 and abs(b.var() - 1.0) < 1e-5
    assert abs(float((a * b).mean())) < 0.1


@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("shape,nf", [((512, 512), 3), ((64, 64, 64), 2)])
def test_kspace_ensemble(hf, shape, nf, lanes):
    fk = inputs.filter_kwargs(inputs.C1 if len(shape) == 2 else inputs.C2)
    gf, of = filters(hf, **fk)
    levels = (0.0, 0.5) if len(shape) == 2 else (0.0,)
    nr, nt = (64, 36) if len(shape) == 2 else (32, 1)
    plan = hf.Plan(shape, kspace=True)
    got = run_pipeline(hf, plan, gf, shape, 7, 4, levels, nr, nt, nfields=nf, lanes=lanes)
    sums_f = np.zeros(nr * nt)
    for e in range(nf):
        want = oracle.pipeline(shape, of, 7, 4 + e, levels=levels, nr=nr, ntheta=nt, noise="kspace")
        check_field(got["f"][e], want["f"])
        sums_f += want["sums_f"]
    check_bins(got["sums_f"], sums_f)
