"""Whole path (field, sign maps, binned S of field and maps) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_bins, check_field, check_maps, dev_zeros, filters, np_

pytestmark = pytest.mark.gpu


def run_pipeline(hf, plan, gf, shape, seed, field, levels, nr, ntheta, out_dtype=torch.float32, nfields=1, lanes=1):
    N = int(np.prod(shape))
    nb = nr * ntheta
    nlev = len(levels)
    ws = plan.workspace(nlev, nb, lanes=lanes)
    out_f = torch.empty((nfields,) + tuple(shape), dtype=out_dtype, device="cuda")
    maps = torch.empty((nfields, max(nlev, 1)) + tuple(shape), dtype=torch.int8, device="cuda")
    sf, cf = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    sm, cm = dev_zeros(max(nlev, 1) * nb, torch.float64), dev_zeros(max(nlev, 1) * nb, torch.int64)
    if nfields == 1:
        hf.hufield_pipeline(plan, gf, seed, field, out_f, levels, maps, nr, ntheta, False, sf, cf, sm, cm, ws)
    else:
        hf.hufield_ensemble(plan, gf, seed, field, nfields, out_f, levels, maps, nr, ntheta, False, sf, cf, sm, cm,
                            ws)
    torch.cuda.synchronize()
    return {"f": np_(out_f.float()), "maps": np_(maps), "sums_f": np_(sf), "counts_f": np_(cf),
            "sums_m": np_(sm).reshape(-1, nb)[:nlev], "counts_m": np_(cm).reshape(-1, nb)[:nlev]}


def compare(got, want, levels, N, e=0):
    check_field(got["f"][e], want["f"])
    flips = check_maps(got["maps"][e][: len(levels)], want["maps"], want["f"], levels) if levels else []
    check_bins(got["sums_f"], want["sums_f"], got["counts_f"], want["counts_f"])
    for t in range(len(levels)):
        check_bins(got["sums_m"][t], want["sums_m"][t], got["counts_m"][t], want["counts_m"][t], flips=flips[t], N=N)


CASES = [
    ("C0-256^2", (256, 256), inputs.filter_kwargs(inputs.C0), (0.0,), 128, 1),
    ("2d-aniso-16x64", (16, 64), dict(p=3.0, axes=(1.0, 0.5), rot=0.7, k0=0.3, width=0.1, supp=4.0),
     (0.0, 0.5, -0.5), 8, 6),
    ("2d-paper-64x32", (64, 32), dict(p=1.0, axes=(1.0, 0.5), width=0.3, supp=2.0, form=1), (0.0,), 16, 1),
    ("C1-like-512^2", (512, 512), inputs.filter_kwargs(inputs.C1), (0.0, 0.5, -0.5), 64, 36),
    ("2d-8x8", (8, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.4, width=0.3, supp=2.0), (0.0, 0.25), 4, 3),
    ("2d-4096x8", (4096, 8), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0), (0.0,), 32, 1),
    ("2d-8x4096", (8, 4096), dict(p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0), (0.0,), 32, 4),
    ("3d-8^3", (8, 8, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.4, width=0.2, supp=2.0), (0.0,), 4, 1),
    ("3d-16x32x8", (16, 32, 8), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.1, supp=2.0), (0.0, 0.5), 16, 1),
    ("3d-rot-32x16x64", (32, 16, 64), dict(p=2.5, axes=(1.0, 0.7, 1.3), rot=1.1, k0=0.25, width=0.08, supp=6.0),
     (0.0,), 32, 1),
    ("C2-like-64^3", (64, 64, 64), inputs.filter_kwargs(inputs.C2), (0.0,), 32, 1),
]


@pytest.mark.parametrize("name,shape,fk,levels,nr,nt", CASES, ids=[c[0] for c in CASES])
def test_pipeline_parity(hf, name, shape, fk, levels, nr, nt):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 0, 0, levels, nr, nt)
    want = oracle.pipeline(shape, of, 0, 0, levels=levels, nr=nr, ntheta=nt)
    compare(got, want, levels, int(np.prod(shape)))


def wide_tile(L):
    """Columns per tile of the strided pass of length L with enough columns for its
    wide tile: 256 up to L = 16, 4096 / L up to 512, 8192 / L from 1024."""
    return 256 if L <= 16 else (4096 // L if L <= 512 else 8192 // L)


AXIS_LENGTHS = [1 << k for k in range(3, 13)]


@pytest.mark.parametrize("noise", ["real", "kspace"])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("L", AXIS_LENGTHS)
def test_every_axis_length(hf, L, ndim, noise):
    # each strided-pass length in both its tile widths: a few columns (narrow tile) and
    # two wide tiles' worth (n_last / 2 = 2 TB), along axis 0 (2D) and the middle axis (3D)
    w = max(8, 2 * wide_tile(L))
    for shape in ([(L, 8), (L, w)] if ndim == 2 else [(8, L, 8), (8, L, w)]):
        fk = dict(p=2.0, axes=(1.0,) * ndim, k0=0.3, width=0.1, supp=2.0)
        gf, of = filters(hf, **fk)
        plan = hf.Plan(shape, kspace=noise == "kspace")
        nt = 2 if ndim == 2 else 1
        got = run_pipeline(hf, plan, gf, shape, 3, 1, (0.0,), 16, nt)
        want = oracle.pipeline(shape, of, 3, 1, levels=(0.0,), nr=16, ntheta=nt, noise=noise)
        compare(got, want, (0.0,), int(np.prod(shape)))


# Narrow bands (Eqs. 12-13) end well inside the lattice: past the band the
# filtered spectrum is exactly zero in FP32, and the passes after the forward
# transform skip the columns k_last >= kz where every mode is zero.  Cases with
# kz odd, kz inside a tile, rotated 2D and 3D filters, the paper's form and
# small lattices whose tiles span several rows.
BAND_CASES = [
    ("2d-256", (256, 256), dict(p=2.0, axes=(1.0, 1.0), k0=0.2, width=0.02, supp=2.0), 16, 1),
    ("2d-rot-128x512", (128, 512), dict(p=3.0, axes=(1.0, 0.5), rot=0.7, k0=0.15, width=0.02, supp=4.0), 16, 6),
    ("2d-paper-64", (64, 64), dict(p=1.0, axes=(1.0, 0.5), width=0.05, supp=2.0, form=1), 16, 1),
    ("2d-256x16", (256, 16), dict(p=2.0, axes=(1.0, 1.0), k0=0.2, width=0.03, supp=2.0), 16, 1),
    ("3d-32x64x128", (32, 64, 128), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.03, supp=2.0), 16, 1),
    ("3d-rot-64x32x64", (64, 32, 64), dict(p=2.5, axes=(1.0, 0.7, 0.6), rot=1.1, k0=0.15, width=0.03, supp=2.0),
     16, 1),
    ("3d-16x1024x64", (16, 1024, 64), dict(p=2.0, axes=(1.0, 1.0, 1.0), k0=0.1, width=0.02, supp=2.0), 16, 1),
    ("3d-16^3", (16, 16, 16), dict(p=6.0, axes=(1.0, 1.0, 0.5), k0=0.2, width=0.04, supp=2.0), 8, 1),
]


@pytest.mark.parametrize("name,shape,fk,nr,nt", BAND_CASES + [
    ("C1-like-512^2", (512, 512), inputs.filter_kwargs(inputs.C1), 64, 36),
    ("C2-like-64^3", (64, 64, 64), inputs.filter_kwargs(inputs.C2), 32, 1),
    ("C0-256^2", (256, 256), inputs.filter_kwargs(inputs.C0), 128, 1)], ids=lambda v: v if isinstance(v, str) else None)
def test_band_edge_is_exactly_zero(hf, name, shape, fk, nr, nt):
    # the passes skip k_last >= kz: there the FP64 filter (Eqs. 12-13) must be
    # far below the FP32 underflow (2^-126), for k_last and -k_last alike
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    kz = hf.hufield_filter_band_edge(plan, gf)
    M = shape[-1] // 2
    assert 0 < kz <= M
    if name != "C0-256^2":
        assert kz < M  # narrow bands end inside the lattice
    H = oracle.filter_grid(shape, of)
    klast = np.abs(np.fft.fftfreq(shape[-1], 1.0 / shape[-1]))
    if kz < M:
        assert np.abs(H[..., klast >= kz]).max() <= 2.0 ** -139
    with pytest.raises(hf.HufieldError):
        hf.hufield_filter_band_edge(plan, hf.Filter(p=-1.0, axes=(1.0,) * len(shape)))


@pytest.mark.parametrize("noise", ["real", "kspace"])
@pytest.mark.parametrize("name,shape,fk,nr,nt", BAND_CASES, ids=[c[0] for c in BAND_CASES])
def test_narrow_band_parity(hf, name, shape, fk, nr, nt, noise):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape, kspace=noise == "kspace")
    levels = (0.0, 0.4)
    got = run_pipeline(hf, plan, gf, shape, 6, 3, levels, nr, nt, nfields=2)
    sf, cf = 0.0, 0
    sm, cm = 0.0, 0
    for e in range(2):
        want = oracle.pipeline(shape, of, 6, 3 + e, levels=levels, nr=nr, ntheta=nt, noise=noise)
        check_field(got["f"][e], want["f"])
        check_maps(got["maps"][e], want["maps"], want["f"], levels)
        sf, cf = sf + want["sums_f"], cf + want["counts_f"]
        sm, cm = sm + want["sums_m"], cm + want["counts_m"]
    check_bins(got["sums_f"], sf, got["counts_f"], cf)
    for t in range(len(levels)):
        check_bins(got["sums_m"][t], sm[t], got["counts_m"][t], cm[t], flips=2, N=int(np.prod(shape)))
    # generate (no bins) and BF16 output take the same passes
    ws = plan.workspace(0, 0)
    out = torch.empty(shape, dtype=torch.bfloat16, device="cuda")
    hf.hufield_generate(plan, gf, 6, 3, out, ws)
    torch.cuda.synchronize()
    ref = oracle.pipeline(shape, of, 6, 3, levels=(), nr=nr, ntheta=nt, noise=noise)["f"]
    err = np.linalg.norm(np_(out.float()).astype(np.float64) - ref) / np.linalg.norm(ref)
    assert err < 2.5e-3, err


# Corners of the ragged workload's parameter ranges (p in [1, 8], semi-axes in
# [0.5, 2], k0 in [0.05, 0.4], width down to 0.01, s up to 6, levels in [-1, 1]):
# the narrowest bands stretch the filter's rounding the most (a relative error
# of K grows by about 2 |K - k0| K / (w^2 ln 4) in log2 A).
CORNER_CASES = [
    ("2d-1024-p8-far", (1024, 1024), dict(p=8.0, axes=(2.0, 0.5), rot=2.0, k0=0.4, width=0.01, supp=6.0), 0.7, 128),
    ("2d-1024-p1-near", (1024, 1024), dict(p=1.0, axes=(0.5, 2.0), rot=0.3, k0=0.05, width=0.01, supp=2.0), -1.0,
     128),
    ("3d-256-p8-far", (256, 256, 256), dict(p=8.0, axes=(1.0, 2.0, 0.5), rot=1.0, k0=0.4, width=0.01, supp=6.0), 0.0,
     128),
    ("3d-256-p1-near", (256, 256, 256), dict(p=1.0, axes=(1.0, 0.5, 2.0), rot=3.0, k0=0.05, width=0.01, supp=4.0),
     -0.5, 128),
]


@pytest.mark.parametrize("name,shape,fk,level,nr", CORNER_CASES, ids=[c[0] for c in CORNER_CASES])
def test_parameter_range_corners(hf, name, shape, fk, level, nr):
    gf, of = filters(hf, **fk)
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 8, 1, (level,), nr, 1)
    want = oracle.pipeline(shape, of, 8, 1, levels=(level,), nr=nr, ntheta=1)
    compare(got, want, (level,), int(np.prod(shape)))


def test_pipeline_no_levels(hf):
    shape = (64, 64)
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C0))
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 4, 1, (), 16, 1)
    want = oracle.pipeline(shape, of, 4, 1, levels=(), nr=16, ntheta=1)
    check_field(got["f"][0], want["f"])
    check_bins(got["sums_f"], want["sums_f"], got["counts_f"], want["counts_f"])


@pytest.mark.parametrize("lanes,nf", [(1, 3), (2, 3), (2, 6)])
def test_ensemble_accumulates(hf, lanes, nf):
    # lanes = 2: a two-slice workspace runs the odd fields on the plan's second stream
    shape, levels, nr, nt = (64, 128), (0.0, 0.5, -0.5), 16, 6
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C1))
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 0, 5, levels, nr, nt, nfields=nf, lanes=lanes)
    sf = np.zeros(nr * nt)
    cf = np.zeros(nr * nt, np.int64)
    sm = np.zeros((len(levels), nr * nt))
    cm = np.zeros((len(levels), nr * nt), np.int64)
    flips = np.zeros(len(levels), np.int64)
    for e in range(nf):
        w = oracle.pipeline(shape, of, 0, 5 + e, levels=levels, nr=nr, ntheta=nt)
        check_field(got["f"][e], w["f"])
        flips += np.asarray(check_maps(got["maps"][e], w["maps"], w["f"], levels))
        sf += w["sums_f"]
        cf += w["counts_f"]
        sm += w["sums_m"]
        cm += w["counts_m"]
    check_bins(got["sums_f"], sf, got["counts_f"], cf)
    for t in range(len(levels)):
        check_bins(got["sums_m"][t], sm[t], got["counts_m"][t], cm[t], flips=max(2, int(flips[t])),
                   N=int(np.prod(shape)))


def test_two_lane_ensembles_accumulate_across_calls(hf):
    # a second call with accumulate = 1 adds its fields' bins to the first call's,
    # the second lane's field bins included
    shape, levels, nr, nt = (32, 64), (0.0,), 8, 4
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C1))
    plan = hf.Plan(shape)
    nb = nr * nt
    ws = plan.workspace(1, nb, lanes=2)
    out_f = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
    maps = torch.empty((3, 1) + shape, dtype=torch.int8, device="cuda")
    sf, cf = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    sm, cm = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    hf.hufield_ensemble(plan, gf, 4, 0, 3, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, ws)
    hf.hufield_ensemble(plan, gf, 4, 3, 3, out_f, levels, maps, nr, nt, True, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    assert hf.hufield_workspace_status(ws) == hf.OK
    want_s, want_c = 0.0, 0
    for e in range(6):
        w = oracle.pipeline(shape, of, 4, e, levels=levels, nr=nr, ntheta=nt)
        want_s, want_c = want_s + w["sums_f"], want_c + w["counts_f"]
    check_bins(np_(sf), want_s, np_(cf), want_c)
    for e in range(3):  # the second call's fields are the stored ones
        check_field(np_(out_f[e]), oracle.pipeline(shape, of, 4, 3 + e, levels=levels, nr=nr, ntheta=nt)["f"])


def test_pipeline_bf16_maps_from_fp32(hf):
    shape, levels = (128, 128), (0.0, 0.5)
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C0))
    plan = hf.Plan(shape)
    a = run_pipeline(hf, plan, gf, shape, 1, 0, levels, 32, 1)
    b = run_pipeline(hf, plan, gf, shape, 1, 0, levels, 32, 1, out_dtype=torch.bfloat16)
    np.testing.assert_array_equal(a["maps"], b["maps"])
    # same maps; the FP64 bin sums differ only by the order of the atomic adds
    np.testing.assert_allclose(a["sums_m"], b["sums_m"], rtol=1e-6)
    assert 3e-4 < np.linalg.norm(b["f"] - a["f"]) / np.linalg.norm(a["f"]) < 2e-3


def test_field_bins_equal_spectrum_of_stored_field(hf):
    # S_f from the filtered spectrum equals the spectrum call on the stored FP32 field
    shape, nr = (32, 32, 32), 16
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C2))
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 2, 0, (0.0,), nr, 1)
    f = torch.from_numpy(got["f"][0].astype(np.float32)).cuda()
    s, c = dev_zeros(nr, torch.float64), dev_zeros(nr, torch.int64)
    ws = plan.workspace(1, nr)
    hf.hufield_spectrum(plan, f, nr, 1, False, s, c, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np_(c), got["counts_f"])
    np.testing.assert_allclose(np_(s), got["sums_f"], rtol=2e-5, atol=1e-9 * got["sums_f"].max())


@pytest.mark.parametrize("shape,nr,nt", [((128, 64), 16, 6), ((32, 16, 64), 16, 1)])
def test_plan_cached_bins(hf, shape, nr, nt):
    # bins cached at plan time give the same results as bins built per call;
    # a call with other (nr, ntheta) falls back to building them
    levels = (0.0, 0.5)
    gf, of = filters(hf, **inputs.filter_kwargs(inputs.C1 if len(shape) == 2 else inputs.C2))
    plain = hf.Plan(shape)
    cached = hf.Plan(shape)
    hf.hufield_plan_set_bins(cached, nr, nt)
    a = run_pipeline(hf, plain, gf, shape, 3, 1, levels, nr, nt, nfields=2)
    b = run_pipeline(hf, cached, gf, shape, 3, 1, levels, nr, nt, nfields=2)
    np.testing.assert_array_equal(a["counts_f"], b["counts_f"])
    np.testing.assert_array_equal(a["counts_m"], b["counts_m"])
    np.testing.assert_allclose(b["sums_f"], a["sums_f"], rtol=1e-6, atol=1e-9 * a["sums_f"].max())
    np.testing.assert_allclose(b["sums_m"], a["sums_m"], rtol=1e-6)
    want = oracle.pipeline(shape, of, 3, 2, levels=levels, nr=nr, ntheta=nt)
    check_field(b["f"][1], want["f"])
    other = run_pipeline(hf, cached, gf, shape, 3, 1, levels, nr // 2, nt, nfields=1)
    want = oracle.pipeline(shape, of, 3, 1, levels=levels, nr=nr // 2, ntheta=nt)
    check_bins(other["sums_f"], want["sums_f"], other["counts_f"], want["counts_f"])


def test_filter_without_power(hf):
    # a band beyond the Nyquist wavenumber: A = 0 at every mode, Eq. (15) is read as f = 0;
    # the call reports it in the workspace status and adds no field bins
    shape, levels = (64, 32), (0.0, 0.5)
    gf, of = filters(hf, p=2.0, axes=(1.0, 1.0), k0=3.0, width=0.01, supp=2.0)
    plan = hf.Plan(shape)
    got = run_pipeline(hf, plan, gf, shape, 1, 0, levels, 16, 1)
    ws = plan.workspace(len(levels), 16)
    f = torch.empty(shape, device="cuda")
    hf.hufield_generate(plan, gf, 1, 0, f, ws)
    assert hf.hufield_workspace_status(ws) == hf.ERR_NO_POWER
    assert bool((f == 0).all())
    want = oracle.pipeline(shape, of, 1, 0, levels=levels, nr=16)
    assert np.all(got["f"] == 0.0) and np.all(got["sums_f"] == 0.0)
    np.testing.assert_array_equal(got["maps"][0][: len(levels)], want["maps"])
    for t in range(len(levels)):
        check_bins(got["sums_m"][t], want["sums_m"][t], got["counts_m"][t], want["counts_m"][t])
