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
    # 3D, one level: r2c 4, axis-1 forward 8, filter 9, axis-1 inverse 8, c2r 13, map axis-1 8, bins 5
    assert per_voxel((64, 64, 64), 1, 1.0) == pytest.approx(55.0)
    # 2D, three levels: r2c 4, filter 9, c2r 4 + 4 + 3 + 12, bins 3 x 5
    assert per_voxel((256, 256), 3, 1.0) == pytest.approx(51.0)
    # k-space noise: no r2c or axis-1 forward; the filter pass writes only
    assert per_voxel((64, 64, 64), 1, 1.0, kspace=True) == pytest.approx(55.0 - 4 - 8 - 4)


def test_band_edge_scales_only_the_pruned_passes():
    # half the columns live: filter 9, axis-1 forward and inverse 8 + 8 and c2r's read 4 halve
    assert per_voxel((64, 64, 64), 1, 0.5) == pytest.approx(55.0 - (9 + 8 + 8 + 4) / 2)
    assert per_voxel((256, 256), 3, 0.5) == pytest.approx(51.0 - (9 + 4) / 2)
    a = bench.algorithmic_bytes((32, 32, 32), 1, live=0.25)
    b = bench.algorithmic_bytes((32, 32, 32), 1, live=1.0)
    for k in ("r2c", "cols_mid_maps", "cols_bins", "counts"):
        assert a[k] == b[k]
    for k in ("cols_mid_fwd", "cols_filter", "cols_mid_inv"):
        assert a[k] == pytest.approx(0.25 * b[k])
