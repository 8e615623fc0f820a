"""Noise-shaped binarisation (hufield_binarise): the +-1 map of the CUDA path
against the oracle's, site for site, on the same stored field.  Each site is
decided by FP32 operations that both sides take in the same order, so the
maps must be identical.  Covers int8 and one-bit storage, FP32 and BF16
fields, automatic and explicit gains (with the clamp active), levels, every
strip height from one row to the whole axis, 2D and 3D lattices including the
benchmark's full-size fields (4096^2 and 512^3), and argument checks.  The map's
spectrum near k = 0 is checked on the GPU against the sign map's."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_bins, dev_zeros, filters, np_
from tests.test_gpu_maps_bits import unpack

pytestmark = pytest.mark.gpu


def run(hf, plan, f, fmt, level=0.0, gain=0.0, strip=0, ws=None):
    N = f.numel()
    hf.hufield_plan_set_maps_format(plan, fmt)
    if fmt == hf.MAPS_BITS:
        out = torch.full((N // 32,), -1, dtype=torch.int32, device="cuda")  # every bit must be written
    else:
        out = torch.zeros(N, dtype=torch.int8, device="cuda")
    if ws is None and gain == 0.0:
        ws = plan.workspace(0, 0)
    hf.hufield_binarise(plan, f, out, level, gain, strip, ws)
    torch.cuda.synchronize()
    m = np_(out)
    return (unpack(m, N) if fmt == hf.MAPS_BITS else m).reshape(tuple(f.shape))


def host_f32(f: torch.Tensor) -> np.ndarray:
    return np_(f.float())  # BF16 -> FP32 is exact


# (shape, strip, gain, level)
CASES = [
    ((8, 8), 0, 0.0, 0.0),
    ((8, 64), 1, 0.0, 0.0),
    ((64, 128), 16, 0.4, 0.0),
    ((256, 256), 0, 0.0, 0.5),
    ((256, 256), 64, 3.0, -0.25),     # clamp active
    ((1024, 512), 0, 0.0, 0.0),       # strips of 256 rows, four per column
    ((512, 32), 512, 0.0, 1.0),       # one strip over the whole axis
    ((16, 32, 64), 0, 0.0, 0.0),
    ((64, 64, 64), 8, 0.7, 0.3),
    ((256, 8, 16), 256, 0.0, -0.5),
]


@pytest.mark.parametrize("shape,strip,gain,level", CASES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_map_matches_oracle(hf, shape, strip, gain, level, dtype):
    plan = hf.Plan(shape)
    f = torch.from_numpy(inputs.random_field(shape, 7, np.float32)).cuda().to(dtype)
    want = oracle.sigma_delta(host_f32(f), t=level, gain=gain, strip=strip)
    fmts = [hf.MAPS_I8] + ([hf.MAPS_BITS] if int(np.prod(shape)) // shape[0] >= 32 else [])
    for fmt in fmts:
        got = run(hf, plan, f, fmt, level, gain, strip)
        assert np.array_equal(got, want), f"format {fmt}: {(got != want).sum()} sites differ"


def test_generated_fields_twice_in_a_row(hf):
    # a generated hyperuniform field (the 256^2 parity case's filter), the same call
    # twice, then a second field: the automatic gain's reduction word starts from zero
    cfg = inputs.C0
    gf, _ = filters(hf, **inputs.filter_kwargs(cfg))
    plan = hf.Plan(cfg["shape"])
    ws = plan.workspace(0, 0)
    out_f = torch.empty(cfg["shape"], dtype=torch.float32, device="cuda")
    for field in (0, 0, 1):
        hf.hufield_generate(plan, gf, 5, field, out_f, ws)
        got = run(hf, plan, out_f, hf.MAPS_BITS, ws=ws)
        assert np.array_equal(got, oracle.sigma_delta(np_(out_f)))


@pytest.mark.parametrize("name", ["C1", "C2"])
def test_full_size_fields(hf, name):
    # the benchmark's lattices (4096^2 with its filter; 512^3 with its filter), one-bit maps,
    # default strips and the automatic gain, every site against the oracle
    cfg = getattr(inputs, name)
    gf, _ = filters(hf, **inputs.filter_kwargs(cfg))
    plan = hf.Plan(cfg["shape"])
    ws = plan.workspace(0, 0)
    out_f = torch.empty(cfg["shape"], dtype=torch.float32, device="cuda")
    hf.hufield_generate(plan, gf, 0, 0, out_f, ws)
    got = run(hf, plan, out_f, hf.MAPS_BITS, ws=ws)
    f = np_(out_f)
    del out_f
    want = oracle.sigma_delta(f)
    assert np.array_equal(got, want), f"{(got != want).sum()} sites differ"


def test_small_k_spectrum_below_the_sign_maps(hf):
    # Sec. II.B: the sign map refills the spectrum near k = 0; the noise-shaped
    # map keeps it suppressed.  Eight generated 256^2 fields, bins from the GPU.
    cfg = inputs.C0
    gf, _ = filters(hf, **inputs.filter_kwargs(cfg))
    shape, nr = cfg["shape"], 64
    plan = hf.Plan(shape)
    ws = plan.workspace(1, nr)
    out_f = torch.empty(shape, dtype=torch.float32, device="cuda")
    sign = torch.empty(shape, dtype=torch.int8, device="cuda")
    sd = torch.empty(shape, dtype=torch.int8, device="cuda")
    sums = {k: dev_zeros(nr, torch.float64) for k in ("sign", "sd")}
    counts = {k: dev_zeros(nr, torch.int64) for k in ("sign", "sd")}
    for field in range(8):
        hf.hufield_generate(plan, gf, 9, field, out_f, ws)
        hf.hufield_threshold(plan, out_f, (0.0,), sign)
        hf.hufield_binarise(plan, out_f, sd, 0.0, 0.0, 0, ws)
        for k, y in (("sign", sign), ("sd", sd)):
            hf.hufield_spectrum(plan, y, nr, 1, field > 0, sums[k], counts[k], ws)
    torch.cuda.synchronize()
    s_sign = np_(sums["sign"]) / np_(counts["sign"])
    s_sd = np_(sums["sd"]) / np_(counts["sd"])
    assert s_sign[1:5].min() > 0.3
    assert (s_sd[1:5] < 0.03 * s_sign[1:5]).all()
    # the map's spectrum is that of the oracle's map (same sites)
    want_s, want_c = oracle.spectrum_bins(oracle.sigma_delta(np_(out_f)), nr)
    hf.hufield_spectrum(plan, sd, nr, 1, False, sums["sd"], counts["sd"], ws)
    torch.cuda.synchronize()
    check_bins(np_(sums["sd"]), want_s, np_(counts["sd"]), want_c)


def test_rejected_arguments(hf):
    plan = hf.Plan((64, 64))
    f = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros(64 * 64, dtype=torch.int8, device="cuda")
    ws = plan.workspace(0, 0)
    bad = [
        dict(strip=48), dict(strip=128), dict(strip=-1), dict(gain=-1.0), dict(gain=float("inf")),
        dict(gain=float("nan")), dict(level=float("nan")),
    ]
    for kw in bad:
        args = dict(level=0.0, gain=0.5, strip=0, ws=ws) | kw
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_binarise(plan, f, out, **args)
        assert e.value.status == hf.ERR_INVALID_ARG, kw
    with pytest.raises(hf.HufieldError) as e:  # the automatic gain needs the workspace
        hf.hufield_binarise(plan, f, out, 0.0, 0.0, 0, None)
    assert e.value.status == hf.ERR_INVALID_ARG
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_binarise(plan, f, out, 0.0, 0.0, 0, ws[:256])
    assert e.value.status == hf.ERR_WS_TOO_SMALL
    # one-bit maps need 32 columns per row of axis 0
    small = hf.Plan((64, 16))
    hf.hufield_plan_set_maps_format(small, hf.MAPS_BITS)
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_binarise(small, torch.zeros((64, 16), device="cuda"), out, 0.0, 0.5, 0, None)
    assert e.value.status == hf.ERR_INVALID_ARG
    # nothing was written by the refused calls
    assert int(out.abs().sum()) == 0
