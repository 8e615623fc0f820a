"""One-bit sign maps (hufield_plan_set_maps_format): the same maps as the int8
ones, bit for bit, through every row-kernel variant (ballot-packed words and
the OR-into-cleared-words path of short rows and one-row tiles), in single
calls, two-lane ensembles and the standalone threshold; the field and every bin
unchanged.  The int8 maps themselves are checked against the FP64 oracle in
test_gpu_pipeline.py."""
import numpy as np
import pytest
import torch

from tests.gpu_common import dev_zeros, filters, np_

pytestmark = pytest.mark.gpu

LEVELS = (0.0, 0.5, -0.5)


def unpack(words: np.ndarray, n: int) -> np.ndarray:
    """+-1 int8 sites of one-bit maps: site i is bit i % 32 of little-endian word i // 32."""
    raw = np.ascontiguousarray(words).view(np.uint8).reshape(*words.shape[:-1], -1)
    bits = np.unpackbits(raw, axis=-1, bitorder="little")[..., :n]
    return bits.astype(np.int8) * 2 - 1


def run(hf, shape, fmt, nfields, levels=LEVELS, nr=16, nt=1, out_dtype=torch.float32):
    gf, _ = filters(hf, p=2.0, axes=(1.0, 0.5, 1.0), rot=0.3, k0=0.25, width=0.08, supp=2.0)
    plan = hf.Plan(shape)
    hf.hufield_plan_set_maps_format(plan, fmt)
    assert hf.hufield_plan_maps_format(plan) == fmt
    N = int(np.prod(shape))
    nlev, nb = len(levels), nr * nt
    ws = plan.workspace(nlev, nb, lanes=2 if nfields > 1 else 1)
    out_f = torch.empty((nfields, N), dtype=out_dtype, device="cuda")
    if fmt == hf.MAPS_BITS:
        # garbage in the words beforehand: every bit must be written
        maps = torch.full((nfields, nlev, N // 32), -1, dtype=torch.int32, device="cuda")
    else:
        maps = torch.empty((nfields, nlev, N), dtype=torch.int8, device="cuda")
    sf, cf = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    sm, cm = dev_zeros(nlev * nb, torch.float64), dev_zeros(nlev * nb, torch.int64)
    if nfields == 1:
        hf.hufield_pipeline(plan, gf, 3, 7, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, ws)
    else:
        hf.hufield_ensemble(plan, gf, 3, 7, nfields, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    m = np_(maps)
    if fmt == hf.MAPS_BITS:
        m = unpack(m, N)
    return {"f": np_(out_f.float()), "maps": m, "bins": [np_(t) for t in (sf, cf, sm, cm)]}


# (shape, what it reaches): row length M = n_last / 2 and rows per tile
SHAPES = [
    ((8, 8), "M = 4, one-row tiles: OR path"),
    ((64, 64), "M = 32: OR path"),
    ((16, 256), "M = 128 in one-row tiles of 8 threads: OR path"),
    ((256, 256), "M = 128, 32-row tiles: ballot, 16 pairs per half-warp"),
    ((64, 512), "M = 256: ballot"),
    ((1024, 1024), "M = 512: ballot"),
    ((256, 4096), "M = 2048: ballot"),
    ((16, 16, 16), "3D, M = 8: OR path"),
    ((8, 16, 256), "3D, M = 128: ballot"),
    ((32, 16, 64), "3D, M = 32: OR path"),
]


def own_threshold(f, levels=LEVELS):
    """The maps of a call's own FP32 field: +1 where f >= t (the kernels compare the stored values)."""
    return np.stack([np.where(f >= t, 1, -1) for t in levels], axis=-2).astype(np.int8)


def same_maps(b, a, levels=LEVELS):
    """Two calls' maps agree except where their fields sit within FP32 rounding of a level:
    the normalisation's sum is added in a run-dependent order, so the two fields may differ
    in the last bit."""
    f = a["f"]
    rms = float(np.sqrt(np.mean(f.astype(np.float64) ** 2)))
    for t, lev in enumerate(levels):
        near = np.abs(f - lev) <= 1e-5 * rms
        np.testing.assert_array_equal(b["maps"][..., t, :][~near], a["maps"][..., t, :][~near])


@pytest.mark.parametrize("shape,what", SHAPES, ids=["x".join(map(str, s[0])) for s in SHAPES])
def test_bit_maps_equal_int8_maps(hf, shape, what):
    a = run(hf, shape, hf.MAPS_I8, 1)
    b = run(hf, shape, hf.MAPS_BITS, 1)
    # exact against the call's own field; across the two calls up to the level band
    np.testing.assert_array_equal(b["maps"], own_threshold(b["f"]))
    np.testing.assert_array_equal(a["maps"], own_threshold(a["f"]))
    np.testing.assert_allclose(b["f"], a["f"], rtol=0, atol=1e-6 * float(np.abs(a["f"]).max()))
    same_maps(b, a)
    # bins: counts exact; sums to the rounding of the shared-memory FP32 run sums and
    # FP64 atomic adds, whose order varies from call to call
    for k, (x, y) in enumerate(zip(b["bins"], a["bins"])):
        if k % 2:
            np.testing.assert_array_equal(x, y)
        else:
            np.testing.assert_allclose(x, y, rtol=1e-6, atol=0)


@pytest.mark.parametrize("shape", [(512, 512), (64, 64), (32, 32, 32)], ids=["512^2", "64^2", "32^3"])
def test_bit_maps_in_two_lane_ensembles(hf, shape):
    # field e's maps at byte (e nlev + t) N / 8: each field's words land in its own block
    a = run(hf, shape, hf.MAPS_I8, 3)
    b = run(hf, shape, hf.MAPS_BITS, 3)
    np.testing.assert_array_equal(b["maps"], own_threshold(b["f"]))
    same_maps(b, a)


def test_bit_maps_with_bf16_fields(hf):
    # the maps threshold the FP32 values before their BF16 rounding: compared across calls
    a = run(hf, (512, 512), hf.MAPS_I8, 1, out_dtype=torch.bfloat16)
    b = run(hf, (512, 512), hf.MAPS_BITS, 1, out_dtype=torch.bfloat16)
    f = a["f"]
    for t, lev in enumerate(LEVELS):
        far = np.abs(f - lev) > 1e-2 * float(np.sqrt(np.mean(f.astype(np.float64) ** 2)))
        np.testing.assert_array_equal(b["maps"][..., t, :][far], a["maps"][..., t, :][far])
        assert (b["maps"][..., t, :] != a["maps"][..., t, :]).sum() <= 8


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_threshold_bits(hf, dtype):
    shape = (128, 256)
    N = int(np.prod(shape))
    g = torch.Generator(device="cpu").manual_seed(5)
    f = torch.randn(N, generator=g).to(dtype).cuda()
    plan = hf.Plan(shape)
    m8 = torch.empty((len(LEVELS), N), dtype=torch.int8, device="cuda")
    hf.hufield_threshold(plan, f, LEVELS, m8)
    hf.hufield_plan_set_maps_format(plan, hf.MAPS_BITS)
    mb = torch.full((len(LEVELS), N // 32), -1, dtype=torch.int32, device="cuda")
    hf.hufield_threshold(plan, f, LEVELS, mb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(unpack(np_(mb), N), np_(m8))


def test_bad_maps_format_refused(hf):
    plan = hf.Plan((64, 64))
    with pytest.raises(hf.HufieldError):
        hf.hufield_plan_set_maps_format(plan, 2)
    assert hf.hufield_plan_maps_format(plan) == hf.MAPS_I8


BATCH_SHAPES = [(8, 8), (16, 16), (32, 32), (64, 128), (8, 8, 8), (16, 16, 16), (32, 32, 32)]


@pytest.mark.parametrize("per_item", [False, True], ids=["batched-chunks", "per-item"])
def test_batch_bit_maps(hf, per_item):
    # rows of 4 and 8 pairs (OR path into words cleared at the graph's start) and of 16
    # or more (per-row words); each item's map from bit f_offset on, exact against the
    # batch's own fields (each site compares its stored FP32 value with the item's level)
    from tests import inputs

    rng = np.random.default_rng(4)
    items = []
    for i in range(21):
        shape = BATCH_SHAPES[i % len(BATCH_SHAPES)]
        gf, _ = filters(hf, **inputs.random_filter(len(shape), 500 + i))
        items.append((shape, gf, 9, i, float(np.float32(rng.uniform(-1, 1))), min(16, min(shape) // 2)))
    batch = hf.Batch(items, per_item=per_item, maps_bits=True)
    total = batch.total_voxels
    out_f = dev_zeros(total, torch.float32)
    words = torch.full((total // 32,), -1, dtype=torch.int32, device="cuda")
    z = [dev_zeros(batch.total_bins, dt) for dt in (torch.float64, torch.int64, torch.float64, torch.int64)]
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    for _ in range(2):  # capture, then replay over the same (dirty) words
        hf.hufield_batch_run(batch, out_f, words, *z, ws)
        torch.cuda.synchronize()
        f_all, m_all = np_(out_f), unpack(np_(words), total)
        for i, (shape, _, _, _, level, _) in enumerate(items):
            N = int(np.prod(shape))
            fo = batch.f_offset[i]
            want = np.where(f_all[fo:fo + N] >= level, 1, -1).astype(np.int8)
            np.testing.assert_array_equal(m_all[fo:fo + N], want)
    batch.close()
