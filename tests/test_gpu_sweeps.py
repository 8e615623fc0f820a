"""The paper-native sweep driver (Figs. 1-5 workloads) on reduced grids."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2509_08675_gb300 import sweeps

pytestmark = pytest.mark.gpu


def read_pgm(path):
    with open(path, "rb") as fh:
        data = fh.read()
    head, _, rest = data.partition(b"\n")
    kind, w, h, maxv = head.split()
    assert kind == b"P5" and maxv == b"255"
    img = np.frombuffer(rest, dtype=np.uint8)
    assert img.size == int(w) * int(h)
    return img.reshape(int(h), int(w))


def test_sweep_files_and_parity(hf, tmp_path):
    recs = sweeps.sweep(str(tmp_path), figs=("fig2", "fig5"), seed=3, n_override={2: 64, 3: 16})
    assert len(recs) == len(sweeps.FIGURES["fig2"]["sets"]) + len(sweeps.FIGURES["fig5"]["sets"])
    for r in recs:
        base = os.path.join(str(tmp_path), f"{r['figure']}_{r['tag']}")
        for suffix in ("_field.npy", "_map.npy", "_field.pgm", "_map.pgm", "_logS_field.pgm", ".json"):
            assert os.path.exists(base + suffix), base + suffix
        img = read_pgm(base + "_logS_field.pgm")
        assert img.max() == 255 and img.min() == 0
        rec = json.load(open(base + ".json"))
        assert rec["window_variance_field"][0] < 1.0 and rec["window_variance_field"][-1] < rec["window_variance_field"][0]
    # one set checked against the oracle: paper form, anisotropic, f[y][x] with semi-axes (b, a)
    r = next(r for r in recs if r["figure"] == "fig2" and r["alpha"] == 20.0)
    f = np.load(os.path.join(str(tmp_path), f"fig2_{r['tag']}_field.npy")).astype(np.float64)
    fl = r["filter"]
    of = oracle.Filter(p=float(np.float32(fl["p"])), axes=tuple(float(np.float32(a)) for a in fl["axes"]),
                       width=float(np.float32(fl["width"])), supp=float(np.float32(fl["supp"])), form=1)
    want = oracle.generate((64, 64), of, 3, 0)
    assert np.linalg.norm(f - want) / np.linalg.norm(want) < 2e-6
    assert fl["axes"][:2] == [0.5, 1.0]
    m = np.load(os.path.join(str(tmp_path), f"fig2_{r['tag']}_map.npy"))
    assert set(np.unique(m)) <= {-1, 1}


def test_full_plane_mirror():
    half = np.arange(4 * 3, dtype=np.float64).reshape(4, 3)
    full = np.fft.ifftshift(sweeps.full_plane(half))
    assert np.isnan(full[:, 3]).all()
    for k0 in range(4):
        for k1 in range(1, 3):
            assert full[k0, 6 - k1] == half[(-k0) % 4, k1]
