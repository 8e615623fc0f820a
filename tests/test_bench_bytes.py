"""The benchmark's byte model (host logic, no GPU): the pass plan's bytes per
voxel, and how the filter's band edge scales the passes that skip columns."""
import pytest

import bench


def per_voxel(shape, nlev, live, kspace=False):
    n = 1
    for v in shape:
        n *= v
    return bench.field_bytes(shape, nlev, live, kspace=kspace) / n


def test_pass_plan_without_band_edge():
    # 3D, one level: r2c 4, axis-1 forward 8, filter 8, axis-1 inverse 8, c2r 13, map axis-1 8, bins 4
    # (the ~53 B/voxel of the one-axis-per-pass plan)
    assert per_voxel((64, 64, 64), 1, 1.0) == pytest.approx(53.0)
    # 2D, three levels: r2c 4, filter 8, c2r 4 + 4 + 3 + 12, bins 3 x 4
    assert per_voxel((256, 256), 3, 1.0) == pytest.approx(47.0)
    # k-space noise: no r2c or axis-1 forward; the filter pass writes only
    assert per_voxel((64, 64, 64), 1, 1.0, kspace=True) == pytest.approx(53.0 - 4 - 8 - 4)


def test_one_bit_maps_cut_only_the_map_writes():
    # c2r writes each map at 1/8 byte per site instead of 1: 3 levels save 3 x 7/8 B/voxel
    n = 256 * 256
    assert bench.field_bytes((256, 256), 3, 1.0, map_bytes=0.125) / n == pytest.approx(47.0 - 3 * 0.875)
    a = bench.algorithmic_bytes((256, 256), 3, map_bytes=0.125)
    b = bench.algorithmic_bytes((256, 256), 3)
    assert b["c2r"] - a["c2r"] == pytest.approx(3 * 0.875 * n)
    assert all(a[k] == b[k] for k in a if k != "c2r")


def test_band_edge_scales_only_the_pruned_passes():
    # half the columns live: filter 8, axis-1 forward and inverse 8 + 8 and c2r's read 4 halve
    assert per_voxel((64, 64, 64), 1, 0.5) == pytest.approx(53.0 - (8 + 8 + 8 + 4) / 2)
    assert per_voxel((256, 256), 3, 0.5) == pytest.approx(47.0 - (8 + 4) / 2)
    a = bench.algorithmic_bytes((32, 32, 32), 1, live=0.25)
    b = bench.algorithmic_bytes((32, 32, 32), 1, live=1.0)
    for k in ("r2c", "cols_mid_maps", "cols_bins", "counts"):
        assert a[k] == b[k]
    # the bin table is overhead, outside the algorithmic bytes
    assert b["counts"] == 0 and b["cols_bins"] == 4 * 32 ** 3
    o = bench.overhead_bytes((32, 32, 32), 1, live=0.25)
    assert o["cols_bins"] == 32 ** 3 and o["cols_filter"] == pytest.approx(0.25 * 32 ** 3)
    for k in ("cols_mid_fwd", "cols_filter", "cols_mid_inv"):
        assert a[k] == pytest.approx(0.25 * b[k])


def test_ragged_draws_are_seeded_and_in_range():
    # the ragged workload's items: the same for the same seed, sizes from the nine
    # lattices, parameters inside the stated ranges (host logic only)
    from paper_2509_08675_gb300 import hufield as hf

    a = bench.ragged_items(hf, 300, seed=0)
    b = bench.ragged_items(hf, 300, seed=0)
    c = bench.ragged_items(hf, 300, seed=1)
    key = lambda items: [(s, f.p, f.axes, f.rot, f.k0, f.width, f.supp, lvl, nr)  # noqa: E731
                         for s, f, _, _, lvl, nr in items]
    assert key(a) == key(b) and key(a) != key(c)
    sizes = {s for s, *_ in a}
    assert sizes <= set(bench.RAGGED["sizes"]) and len(sizes) == len(bench.RAGGED["sizes"])
    for shape, f, seed, i, level, nr in a:
        assert 1.0 <= f.p <= 8.0 and 0.0 <= f.rot < 3.1416 and 0.05 <= f.k0 <= 0.4 and 0.01 <= f.width <= 0.1
        assert f.supp in (2.0, 4.0, 6.0) and -1.0 <= level <= 1.0 and nr == min(128, shape[0] // 2)
        axes = f.axes[:len(shape)]
        assert all(0.5 <= r <= 2.0 for r in axes[-2:]) and (len(shape) == 2 or axes[0] == 1.0)


def test_binarise_bytes():
    # the field read by the max pass and by the sigma-delta pass, the map written once
    n = 512 ** 3
    assert bench.binarise_bytes((512, 512, 512)) / n == pytest.approx(8.125)
    assert bench.binarise_bytes((4096, 4096), map_bytes=1.0) / 4096 ** 2 == pytest.approx(9.0)
    assert bench.binarise_bytes((256, 256), auto_gain=False) / 256 ** 2 == pytest.approx(4.125)
