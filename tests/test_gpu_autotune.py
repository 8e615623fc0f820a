"""Plan autotuning (hufield_plan_autotune): the chosen launch choices come
from the candidate sets, the results stay those of the oracle, and a cache
file reproduces a tuning without timing it again."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import filters, np_
from tests.test_gpu_pipeline import compare, run_pipeline

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,cfg,levels,nr,nt", [((64, 64, 64), inputs.C2, (0.0,), 32, 1),
                                                    ((512, 512), inputs.C1, (0.0, 0.5), 64, 36)],
                         ids=["3d-64", "2d-512"])
def test_autotuned_plan_keeps_parity(hf, shape, cfg, levels, nr, nt):
    gf, of = filters(hf, **inputs.filter_kwargs(cfg))
    plan = hf.Plan(shape)
    before = hf.hufield_plan_tuning(plan)
    assert before == {"cta_cap": {"plain": 2, "filter": 2, "bins": 3, "kspace": 2}, "l2_promotion": 0}
    hf.hufield_plan_autotune(plan, gf, len(levels), nr, nt)
    got_t = hf.hufield_plan_tuning(plan)
    assert got_t["cta_cap"]["plain"] in (1, 2, 3) and got_t["cta_cap"]["filter"] in (1, 2, 3)
    assert got_t["cta_cap"]["bins"] in (2, 3, 4) and got_t["l2_promotion"] in (0, 64, 128, 256)
    assert hf.hufield_plan_tile(plan) in (0, 1, 2)
    got = run_pipeline(hf, plan, gf, shape, 2, 0, levels, nr, nt)
    compare(got, oracle.pipeline(shape, of, 2, 0, levels=levels, nr=nr, ntheta=nt), levels, int(np.prod(shape)))


def test_autotune_cache_round_trip(hf, tmp_path, monkeypatch):
    shape = (32, 32, 32)
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C2))
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("HUFIELD_AUTOTUNE_CACHE", str(cache))
    a = hf.Plan(shape)
    hf.hufield_plan_autotune(a, gf, 1, 16, 1)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "32x32x32 nlev=1 nbins=16" in lines[0]
    # a hand-edited entry for the same key wins (the last one for a key is used)
    key = lines[0].split("\t")[0]
    assert len(lines[0].split("\t")[1].split()) == 6  # caps, promotion, tile width
    cache.write_text(cache.read_text() + f"{key}\t1 1 4 1 256\n")  # five fields: an older line, tile 0
    b = hf.Plan(shape)
    hf.hufield_plan_autotune(b, gf, 1, 16, 1)
    assert hf.hufield_plan_tuning(b) == {"cta_cap": {"plain": 1, "filter": 1, "bins": 4, "kspace": 1},
                                         "l2_promotion": 256}
    assert hf.hufield_plan_tile(b) == 0
    assert len(cache.read_text().splitlines()) == 2  # reused, not timed and appended again


def test_autotune_rejects_bad_arguments(hf):
    plan = hf.Plan((32, 32))
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C0))
    for nlev, nr, nt in ((9, 8, 1), (1, 0, 1), (1, 8, 65)):
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_plan_autotune(plan, gf, nlev, nr, nt)
        assert e.value.status == hf.ERR_INVALID_ARG
    assert hf.hufield_plan_tuning(plan)["l2_promotion"] == 0


@pytest.mark.parametrize("shape,cfg,levels,nr,nt", [((1024, 1024), inputs.C1, (0.0, 0.5), 64, 36),
                                                    ((256, 256, 256), inputs.C2, (0.0,), 128, 1)],
                         ids=["2d-1024", "3d-256"])
def test_tile_widths_give_the_same_results(hf, shape, cfg, levels, nr, nt):
    # every strided column is transformed on its own, so the tile width changes
    # only the order of the bin sums: fields and maps are bit-identical, bins agree
    # to rounding and all match the oracle; the cached bin table follows the width
    gf, of = filters(hf, **inputs.filter_kwargs(cfg))
    want = oracle.pipeline(shape, of, 4, 0, levels=levels, nr=nr, ntheta=nt)
    plan = hf.Plan(shape)
    hf.hufield_plan_set_bins(plan, nr, nt)
    ref = None
    for tile in (0, 1, 2, 0):
        hf.hufield_plan_set_tile(plan, tile)
        assert hf.hufield_plan_tile(plan) == tile
        got = run_pipeline(hf, plan, gf, shape, 4, 0, levels, nr, nt)
        compare(got, want, levels, int(np.prod(shape)))
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got["f"], ref["f"]) and np.array_equal(got["maps"], ref["maps"])
            np.testing.assert_allclose(got["sums_m"], ref["sums_m"], rtol=1e-5, atol=1e-9 * ref["sums_m"].max())
            np.testing.assert_array_equal(got["counts_m"], ref["counts_m"])
    with pytest.raises(hf.HufieldError):
        hf.hufield_plan_set_tile(plan, 3)


@pytest.mark.parametrize("shape,cfg,levels,nr,nt,noise", [((1024, 1024), inputs.C1, (0.0, 0.5), 64, 36, "real"),
                                                          ((256, 256, 256), inputs.C2, (0.0,), 128, 1, "real"),
                                                          ((512, 512), inputs.C1, (0.0,), 64, 36, "kspace")],
                         ids=["2d-1024", "3d-256", "2d-512-kspace"])
def test_tile_orders_give_the_same_results(hf, shape, cfg, levels, nr, nt, noise):
    # contiguous chunks and interleaved tiles transform the same columns; only
    # the order of the Parseval and bin sums changes, so every order matches the
    # oracle and the fields agree to an ulp of their normalisation
    gf, of = filters(hf, **inputs.filter_kwargs(cfg))
    plan = hf.Plan(shape, kspace=noise == "kspace")
    hf.hufield_plan_set_bins(plan, nr, nt)
    assert hf.hufield_plan_order(plan) == 0
    want = oracle.pipeline(shape, of, 4, 0, levels=levels, nr=nr, ntheta=nt, noise=noise)
    ref = None
    for tile, order in ((0, 1), (0, 2), (2, 1), (2, 2), (0, 0)):
        hf.hufield_plan_set_tile(plan, tile)
        hf.hufield_plan_set_order(plan, order)
        assert hf.hufield_plan_order(plan) == order
        got = run_pipeline(hf, plan, gf, shape, 4, 0, levels, nr, nt)
        compare(got, want, levels, int(np.prod(shape)))
        if ref is None:
            ref = got
        else:
            np.testing.assert_allclose(got["f"], ref["f"], rtol=3e-7, atol=3e-7 * np.abs(ref["f"]).max())
            np.testing.assert_allclose(got["sums_m"], ref["sums_m"], rtol=1e-5, atol=1e-9 * ref["sums_m"].max())
            np.testing.assert_allclose(got["sums_f"], ref["sums_f"], rtol=1e-5, atol=1e-9 * ref["sums_f"].max())
            np.testing.assert_array_equal(got["counts_m"], ref["counts_m"])
    with pytest.raises(hf.HufieldError):
        hf.hufield_plan_set_order(plan, 3)
