"""Argument checks of the C ABI: error codes, nothing enqueued."""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_unsupported_dims(hf):
    for shape in [(4, 8), (8, 8192), (12, 16), (8,), (8, 8, 8, 8), (2048, 2048, 1024)]:
        with pytest.raises(hf.HufieldError) as e:
            hf.Plan(shape)
        assert e.value.status in (hf.ERR_UNSUPPORTED_DIMS, hf.ERR_INVALID_ARG)


def test_bad_filters_rejected(hf):
    plan = hf.Plan((32, 32))
    ws = plan.workspace(0, 0)
    out = torch.empty((32, 32), device="cuda")
    bad = [dict(p=0.0), dict(p=float("nan")), dict(width=0.0), dict(supp=-1.0), dict(axes=(1.0, 0.0)),
           dict(sigma_f=0.0), dict(k0=float("inf")), dict(form=2), dict(nyquist=1), dict(rot=float("nan")),
           dict(p=1025.0), dict(axes=(1.0, 2.0 ** 21)), dict(axes=(2.0 ** -21, 1.0))]
    for kw in bad:
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_generate(plan, hf.Filter(**kw), 0, 0, out, ws)
        assert e.value.status == hf.ERR_INVALID_ARG, kw


def test_workspace_checks(hf):
    plan = hf.Plan((64, 64))
    out = torch.empty((64, 64), device="cuda")
    ws = plan.workspace(0, 0)
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_generate(plan, hf.Filter(), 0, 0, out, ws[: ws.numel() - 256])
    assert e.value.status == hf.ERR_WS_TOO_SMALL
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_generate(plan, hf.Filter(), 0, 0, out, ws[8:])
    assert e.value.status == hf.ERR_INVALID_ARG  # misaligned


def test_map_output_alignment(hf):
    # maps are written in units of at most 4 bytes: any 4-byte offset works, others are refused
    plan = hf.Plan((64, 64))
    f = torch.randn((64, 64), device="cuda")
    buf = torch.zeros(64 * 64 + 16, dtype=torch.int8, device="cuda")
    hf.hufield_threshold(plan, f, (0.0,), buf[4:4 + 64 * 64])
    torch.cuda.synchronize()
    want = torch.where(f >= 0, 1, -1).to(torch.int8).flatten()
    assert torch.equal(buf[4:4 + 64 * 64], want)
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_threshold(plan, f, (0.0,), buf[2:2 + 64 * 64])
    assert e.value.status == hf.ERR_INVALID_ARG


def test_bins_and_levels_checks(hf):
    plan = hf.Plan((16, 16, 16))
    ws = plan.workspace(8, 4096)
    f = torch.empty((16, 16, 16), device="cuda")
    maps = torch.empty((9, 16, 16, 16), dtype=torch.int8, device="cuda")
    s = torch.zeros(4096 * 9, dtype=torch.float64, device="cuda")
    c = torch.zeros(4096 * 9, dtype=torch.int64, device="cuda")
    cases = [dict(levels=[0.0] * 9, nr=8, nt=1), dict(levels=[math.nan], nr=8, nt=1), dict(levels=[0.0], nr=0, nt=1),
             dict(levels=[0.0], nr=8, nt=2), dict(levels=[0.0], nr=4097, nt=1)]
    for cs in cases:
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_pipeline(plan, hf.Filter(axes=(1, 1, 1)), 0, 0, f, cs["levels"], maps, cs["nr"], cs["nt"],
                                False, s, c, s, c, ws)
        assert e.value.status == hf.ERR_INVALID_ARG, cs
    with pytest.raises(hf.HufieldError):
        hf.hufield_threshold(plan, f, [], maps)


def test_error_leaves_outputs_untouched(hf):
    plan = hf.Plan((32, 32))
    ws = plan.workspace(0, 0)
    out = torch.full((32, 32), 7.0, device="cuda")
    with pytest.raises(hf.HufieldError):
        hf.hufield_generate(plan, hf.Filter(p=-1.0), 0, 0, out, ws)
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())


def test_largest_lattice_and_empty_ensemble(hf):
    # N = 2^31 voxels is the largest lattice a plan takes; one voxel more of any axis
    # is refused above.  The field there still has mean 0 and variance 1 (Eq. 15).
    shape = (2048, 1024, 1024)
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    f = torch.empty(shape, dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, hf.Filter(p=2.0, axes=(1.0, 1.0, 1.0), k0=0.3, width=0.1, supp=2.0), 5, 0, f, ws)
    torch.cuda.synchronize()
    assert hf.hufield_workspace_status(ws) == hf.OK
    mean = float(f.double().mean())
    var = float(f.double().square().mean())
    assert abs(mean) < 1e-6 and abs(var - 1.0) < 2e-5, (mean, var)
    del f, ws
    torch.cuda.empty_cache()
    # an ensemble of no fields is an argument error and writes nothing
    small = hf.Plan((32, 32))
    wss = small.workspace(1, 8)
    out = torch.full((1, 32, 32), 7.0, device="cuda")
    maps = torch.full((1, 1, 32, 32), 3, dtype=torch.int8, device="cuda")
    s = torch.full((8,), 2.0, dtype=torch.float64, device="cuda")
    c = torch.full((8,), 4, dtype=torch.int64, device="cuda")
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_ensemble(small, hf.Filter(), 0, 0, 0, out, [0.0], maps, 8, 1, False, s, c, s, c, wss)
    assert e.value.status == hf.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((out == 7.0).all()) and bool((maps == 3).all())
    assert bool((s == 2.0).all()) and bool((c == 4).all())
