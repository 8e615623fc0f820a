"""Ragged batch (hufield_batch_*): every item of a batch of mixed 2D/3D
lattices and filters matches the oracle, on the first run (graph capture) and
on a replay."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_bins, check_field, check_maps, dev_zeros, filters, np_

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (32, 32), (64, 64), (8, 8, 8), (16, 16, 16), (32, 32, 32)]


def _items(hf, count, seed):
    rng = np.random.default_rng(seed)
    items, oitems = [], []
    for i in range(count):
        shape = SHAPES[int(rng.integers(len(SHAPES)))]
        fk = inputs.random_filter(len(shape), seed * 1000 + i)
        gf, of = filters(hf, **fk)
        level = float(np.float32(rng.uniform(-1, 1)))
        nr = min(128, min(shape) // 2)
        items.append((shape, gf, 7, i, level, nr))
        oitems.append((shape, of, 7, i, level, nr))
    return items, oitems


@pytest.mark.parametrize("lanes", [0, 1, 8])
def test_batch_matches_oracle_and_replays(hf, lanes):
    # lanes 0: the default (two per size class); 8: up to eight side by side
    items, oitems = _items(hf, 14, 1)
    batch = hf.Batch(items, lanes=lanes)
    out_f = dev_zeros(batch.total_voxels, torch.float32)
    maps = dev_zeros(batch.total_voxels, torch.int8)
    sf, cf = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    sm, cm = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    for run in range(2):
        out_f.zero_()
        hf.hufield_batch_run(batch, out_f, maps, sf, cf, sm, cm, ws)
        torch.cuda.synchronize()
        f_all, m_all = np_(out_f), np_(maps)
        for i, (shape, of, seed, field, level, nr) in enumerate(oitems):
            N = int(np.prod(shape))
            fo, bo = batch.f_offset[i], batch.bin_offset[i]
            want = oracle.pipeline(shape, of, seed, field, levels=(level,), nr=nr, ntheta=1)
            check_field(f_all[fo:fo + N].reshape(shape), want["f"])
            flips = check_maps(m_all[fo:fo + N].reshape((1,) + shape), want["maps"], want["f"], (level,))
            check_bins(np_(sf)[bo:bo + nr], want["sums_f"], np_(cf)[bo:bo + nr], want["counts_f"])
            check_bins(np_(sm)[bo:bo + nr], want["sums_m"][0], np_(cm)[bo:bo + nr], want["counts_m"][0],
                       flips=flips[0], N=N)
    batch.close()


def test_batch_outputs_alternating_between_three_sets(hf):
    # sets A, B, A, C, B: the two most recent sets' graphs are kept, the third set's run
    # captures over the least recently used one; every run writes its own buffers
    items, _ = _items(hf, 10, 3)
    batch = hf.Batch(items)
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")

    def buffers():
        return ([dev_zeros(batch.total_voxels, torch.float32), dev_zeros(batch.total_voxels, torch.int8)] +
                [dev_zeros(batch.total_bins, dt) for dt in (torch.float64, torch.int64, torch.float64, torch.int64)])

    sets = {k: buffers() for k in "ABC"}
    got = {}
    for k in "ABACB":
        for t in sets[k]:
            t.zero_()
        hf.hufield_batch_run(batch, *sets[k], ws)
        torch.cuda.synchronize()
        got.setdefault(k, []).append([np_(t) for t in sets[k]])
    # the runs agree to the rounding of their atomically added sums: each field's
    # normalisation (hence a map site within rounding of its level) and the bin sums
    ref = got["A"][0]
    for k, runs in got.items():
        for outs in runs:
            np.testing.assert_allclose(outs[0], ref[0], rtol=0, atol=1e-6 * float(np.abs(ref[0]).max()))
            flips = int((outs[1] != ref[1]).sum())
            assert flips <= 2
            np.testing.assert_array_equal(outs[3], ref[3])
            np.testing.assert_array_equal(outs[5], ref[5])
            np.testing.assert_allclose(outs[2], ref[2], rtol=1e-5)
            if flips == 0:
                np.testing.assert_allclose(outs[4], ref[4], rtol=1e-5)
    batch.close()


@pytest.mark.parametrize("chunk_bytes", [None, 300000])
def test_batched_chunks_equal_per_item_calls(hf, monkeypatch, chunk_bytes):
    # a size class runs its items a chunk at a time through the batched passes; with a
    # small chunk budget (a few fields per chunk: 2D 64^2 spectra are 16 KB, 3D 32^3
    # 128 KB) every lane runs several chunks.  Fields equal the item-by-item path's to
    # FP32 rounding (the row passes may take another tile width, whose code the
    # compiler contracts differently), maps except at sites within that rounding of
    # the level, bins to rounding.
    if chunk_bytes:
        monkeypatch.setenv("HUFIELD_BATCH_CHUNK_BYTES", str(chunk_bytes))
    items, _ = _items(hf, 40, 3)
    outs = []
    for per_item in (False, True):
        batch = hf.Batch(items, per_item=per_item)
        out_f = dev_zeros(batch.total_voxels, torch.float32)
        maps = dev_zeros(batch.total_voxels, torch.int8)
        bins = [dev_zeros(batch.total_bins, dt) for dt in (torch.float64, torch.int64, torch.float64, torch.int64)]
        ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
        hf.hufield_batch_run(batch, out_f, maps, *bins, ws)
        torch.cuda.synchronize()
        assert hf.hufield_workspace_status(ws) == hf.OK
        outs.append((np_(out_f), np_(maps), [np_(b) for b in bins]))
        batch.close()
    (fa, ma, ba), (fb, mb, bb) = outs
    np.testing.assert_allclose(fa, fb, rtol=0, atol=2e-6 * float(np.abs(fb).max()))
    level = np.zeros_like(fa)
    for i, (shape, _, _, _, lv, _) in enumerate(items):
        o = batch.f_offset[i]
        level[o:o + int(np.prod(shape))] = lv
    diff = ma != mb
    assert not np.any(diff & (np.abs(fb - level) > 1e-5)), "sign differs away from the level"
    np.testing.assert_array_equal(ba[1], bb[1])
    np.testing.assert_array_equal(ba[3], bb[3])
    for x, y in zip(ba[::2], bb[::2]):
        np.testing.assert_allclose(x, y, rtol=1e-5, atol=1e-9 * float(np.abs(y).max()) + 8.0 * int(diff.sum()))


def test_batch_rejects_bad_lane_counts(hf):
    items, _ = _items(hf, 3, 2)
    with pytest.raises(hf.HufieldError) as e:
        hf.Batch(items, lanes=9)
    assert e.value.status == hf.ERR_INVALID_ARG


def test_batch_rejects_bad_items(hf):
    gf, _ = filters(hf, p=2.0, axes=(1.0, 1.0), k0=0.3, width=0.1, supp=2.0)
    with pytest.raises(hf.HufieldError):
        hf.Batch([((16, 16), gf, 0, 0, 0.0, 0)])
    with pytest.raises(hf.HufieldError):
        hf.Batch([((12, 16), gf, 0, 0, 0.0, 8)])


def test_batch_one_class_two_lanes_uncached_bins(hf):
    # seven items of one lattice share a plan and run on two lanes in turn; their
    # bin counts differ, so every item builds its bin table in its lane's workspace
    rng = np.random.default_rng(3)
    items, oitems = [], []
    for i in range(7):
        shape = (32, 64)
        gf, of = filters(hf, **inputs.random_filter(2, 500 + i))
        level = float(np.float32(rng.uniform(-1, 1)))
        nr = 8 + 3 * i
        items.append((shape, gf, 11, i, level, nr))
        oitems.append((shape, of, 11, i, level, nr))
    batch = hf.Batch(items)
    out_f = dev_zeros(batch.total_voxels, torch.float32)
    maps = dev_zeros(batch.total_voxels, torch.int8)
    sf, cf = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    sm, cm = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    hf.hufield_batch_run(batch, out_f, maps, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    f_all = np_(out_f)
    for i, (shape, of, seed, field, level, nr) in enumerate(oitems):
        N = int(np.prod(shape))
        fo, bo = batch.f_offset[i], batch.bin_offset[i]
        want = oracle.pipeline(shape, of, seed, field, levels=(level,), nr=nr, ntheta=1)
        check_field(f_all[fo:fo + N].reshape(shape), want["f"])
        check_bins(np_(sf)[bo:bo + nr], want["sums_f"], np_(cf)[bo:bo + nr], want["counts_f"])
    batch.close()


def test_autotuned_batch_matches_oracle(hf):
    items, oitems = _items(hf, 6, 4)
    batch = hf.Batch(items, autotune=True)
    out_f = dev_zeros(batch.total_voxels, torch.float32)
    maps = dev_zeros(batch.total_voxels, torch.int8)
    sf, cf = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    sm, cm = dev_zeros(batch.total_bins, torch.float64), dev_zeros(batch.total_bins, torch.int64)
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    hf.hufield_batch_run(batch, out_f, maps, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    f_all = np_(out_f)
    for i, (shape, of, seed, field, level, nr) in enumerate(oitems):
        N = int(np.prod(shape))
        fo, bo = batch.f_offset[i], batch.bin_offset[i]
        want = oracle.pipeline(shape, of, seed, field, levels=(level,), nr=nr, ntheta=1)
        check_field(f_all[fo:fo + N].reshape(shape), want["f"])
        check_bins(np_(sf)[bo:bo + nr], want["sums_f"], np_(cf)[bo:bo + nr], want["counts_f"])
    batch.close()
