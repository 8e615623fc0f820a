"""Paper-native workloads (Sec. III): the 2D sweeps of Figs. 1-4 on a 1024^2 grid
of side L = 100 and the 3D exponent sweep of Fig. 5 on a 256^3 grid of side
L = 25, with the paper's form of the filter (Eq. 13 with k0 = 0, sigma = 2 and
the concentration alpha), written to files:

  <fig>_<tag>_field.npy / .pgm        the continuous field (2D: a central
                                       excerpt in the PGM; 3D: three central
                                       orthogonal cuts)
  <fig>_<tag>_map.npy / .pgm          the +-1 sign map (same cuts)
  <fig>_<tag>_logS_field.pgm          log10 S(k) of the field over the k-plane
                                       (3D: the k_x = 0 plane of the filter's
                                       spectrum A(k)^2, as in Fig. 5)
  <fig>_<tag>_logS_map.pgm            log10 S(k) of the sign map (2D)
  <fig>_<tag>.json                     parameters, binned S(k) of field and map,
                                       window variances sigma_F^2(R), timings

Axes: in 2D the field is f[y][x] (axis 0 = y, axis 1 = x) and the paper's
semi-axes (a, b) act on (k_x, k_y), so the filter's per-axis semi-axes are
(b, a).  Volume renderings (Fig. 5, rows 2 and 4) need a graphics stack and are
not made; the orthogonal cuts stand in for them.  Every number comes from the
CUDA library through the C ABI.

    python -m paper_2509_08675_gb300.sweeps --out DIR [--figs fig1 fig3 ...] [--seed S] [--no-arrays]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import hufield as hf

ALPHAS = [0.5, 1.0, 2.0, 20.0, 50.0, 100.0]
P_2D = [0.5, 1.0, 1.5, 2.0, 10.0, 50.0]
P_3D = [0.5, 1.0, 1.5, 2.0, 10.0, 100.0]

FIGURES = {
    # Fig. 1: isotropic (a, b) = (1, 1), p = 1, alpha swept
    "fig1": dict(dim=2, n=1024, L=100.0, ab=(1.0, 1.0), sets=[dict(p=1.0, alpha=a) for a in ALPHAS]),
    # Fig. 2: anisotropic (a, b) = (1, 0.5), p = 1, alpha swept
    "fig2": dict(dim=2, n=1024, L=100.0, ab=(1.0, 0.5), sets=[dict(p=1.0, alpha=a) for a in ALPHAS]),
    # Fig. 3: isotropic, alpha = 20, p swept; 300 x 300 excerpts
    "fig3": dict(dim=2, n=1024, L=100.0, ab=(1.0, 1.0), excerpt=300, sets=[dict(p=p, alpha=20.0) for p in P_2D]),
    # Fig. 4: anisotropic, alpha = 20, p swept
    "fig4": dict(dim=2, n=1024, L=100.0, ab=(1.0, 0.5), excerpt=300, sets=[dict(p=p, alpha=20.0) for p in P_2D]),
    # Fig. 5: 3D, alpha = 20, p swept
    "fig5": dict(dim=3, n=256, L=25.0, ab=(1.0, 1.0), sets=[dict(p=p, alpha=20.0) for p in P_3D]),
}
SIGMA = 2.0
RADII = [1.0, 2.0, 4.0, 8.0, 16.0, 32.0]


def write_pgm(path: str, img: np.ndarray, lo: float | None = None, hi: float | None = None) -> None:
    """8-bit binary PGM of a 2D array, linearly scaled from [lo, hi] (default: its range)."""
    a = np.asarray(img, dtype=np.float64)
    finite = np.isfinite(a)
    lo = float(a[finite].min()) if lo is None else lo
    hi = float(a[finite].max()) if hi is None else hi
    scaled = np.where(finite, (a - lo) / (hi - lo if hi > lo else 1.0), 0.0)
    u8 = np.clip(np.rint(255.0 * scaled), 0, 255).astype(np.uint8)
    with open(path, "wb") as fh:
        fh.write(f"P5 {u8.shape[1]} {u8.shape[0]} 255\n".encode())
        fh.write(u8.tobytes())


def full_plane(half: np.ndarray) -> np.ndarray:
    """The k-plane (2D) from the stored half spectrum [n0][k1], k1 < N/2: the
    mirror S(-n) = S(n) fills k1 < 0; the Nyquist column k1 = -N/2 is not stored
    (NaN).  Returned centred (k = 0 in the middle)."""
    n0, m = half.shape
    full = np.full((n0, 2 * m), np.nan)
    full[:, :m] = half
    neg = half[(-np.arange(n0)) % n0, 1:][:, ::-1]  # S(-k0, -k1) for k1 = m-1 .. 1
    full[:, m + 1:] = neg
    return np.fft.fftshift(full)


def log10_safe(a: np.ndarray, floor: float = 1e-12) -> np.ndarray:
    return np.log10(np.maximum(a, floor * np.nanmax(a)))


def run_set(fig: dict, ps: dict, seed: int, out_dir: str, tag: str, name: str, arrays: bool = True) -> dict:
    dim, n, L = fig["dim"], fig["n"], fig["L"]
    shape = (n,) * dim
    a, b = fig["ab"]
    axes = (b, a) if dim == 2 else (1.0, 1.0, 1.0)
    filt = hf.paper_filter(ps["alpha"], SIGMA, ps["p"], axes, n, L)
    plan = hf.Plan(shape)
    nr = n // 2
    ws = plan.workspace(1, nr)
    f = torch.empty(shape, dtype=torch.float32, device="cuda")
    maps = torch.empty((1,) + shape, dtype=torch.int8, device="cuda")
    sf, cf = torch.zeros(nr, dtype=torch.float64, device="cuda"), torch.zeros(nr, dtype=torch.int64, device="cuda")
    sm, cm = torch.zeros(nr, dtype=torch.float64, device="cuda"), torch.zeros(nr, dtype=torch.int64, device="cuda")
    hf.hufield_pipeline(plan, filt, seed, 0, f, [0.0], maps, nr, 1, False, sf, cf, sm, cm, ws)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hf.hufield_pipeline(plan, filt, seed, 0, f, [0.0], maps, nr, 1, False, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    t_pipe = time.perf_counter() - t0
    t0 = time.perf_counter()
    hf.hufield_generate(plan, filt, seed, 0, f, plan.workspace(0, 0))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0

    half = int(np.prod(shape)) // 2
    spec = torch.empty(half, dtype=torch.float32, device="cuda")
    wsm = plan.workspace(3, 0)
    wv = torch.empty(len(RADII), dtype=torch.float64, device="cuda")
    wvm = torch.empty(len(RADII), dtype=torch.float64, device="cuda")
    hf.hufield_window_variance(plan, f, RADII, wv, wsm)
    hf.hufield_window_variance(plan, maps[0], RADII, wvm, wsm)
    fn = f.cpu().numpy()
    mn = maps[0].cpu().numpy()
    base = os.path.join(out_dir, f"{name}_{tag}")
    if arrays:
        np.save(base + "_field.npy", fn)
        np.save(base + "_map.npy", mn)
    if dim == 2:
        ex = fig.get("excerpt", n)
        c0 = (n - ex) // 2
        write_pgm(base + "_field.pgm", fn[c0:c0 + ex, c0:c0 + ex])
        write_pgm(base + "_map.pgm", mn[c0:c0 + ex, c0:c0 + ex], -1.0, 1.0)
        for y, suffix in ((f, "field"), (maps[0], "map")):
            hf.hufield_spectrum_modes(plan, y, spec, wsm)
            torch.cuda.synchronize()
            img = full_plane(spec.cpu().numpy().astype(np.float64).reshape(n, n // 2))
            write_pgm(base + f"_logS_{suffix}.pgm", log10_safe(img))
    else:
        c = n // 2
        cuts = np.concatenate([fn[c, :, :], fn[:, c, :], fn[:, :, c]], axis=1)
        mcuts = np.concatenate([mn[c, :, :], mn[:, c, :], mn[:, :, c]], axis=1)
        write_pgm(base + "_field.pgm", cuts)
        write_pgm(base + "_map.pgm", mcuts, -1.0, 1.0)
        hf.hufield_filter_modes(plan, filt, spec)
        torch.cuda.synchronize()
        chi = spec.cpu().numpy().astype(np.float64).reshape(n, n, n // 2)
        # the k_x = 0 plane (k_x = last axis): rows k_z (axis 0), columns k_y (axis 1)
        write_pgm(base + "_logS_field.pgm", log10_safe(np.fft.fftshift(chi[:, :, 0])))
    cnt_f, cnt_m = cf.cpu().numpy(), cm.cpu().numpy()
    rec = {"figure": name, "tag": tag, "shape": list(shape), "L": L, "sigma": SIGMA, "alpha": ps["alpha"],
           "p": ps["p"], "ab": [a, b], "seed": seed,
           "filter": {"p": filt.p, "axes": list(filt.axes), "width": filt.width, "supp": filt.supp, "form": 1},
           "S_field_bins": (sf.cpu().numpy() / np.maximum(cnt_f, 1)).tolist(),
           "S_map_bins": (sm.cpu().numpy() / np.maximum(cnt_m, 1)).tolist(),
           "bin_edges_kappa": [i / nr for i in range(nr + 1)],
           "window_radii": RADII, "window_variance_field": wv.cpu().numpy().tolist(),
           "window_variance_map": wvm.cpu().numpy().tolist(),
           "seconds_pipeline": t_pipe, "seconds_generate": t_gen}
    with open(base + ".json", "w") as fh:
        json.dump(rec, fh)
    return rec


def sweep(out_dir: str, figs=("fig1", "fig2", "fig3", "fig4", "fig5"), seed: int = 0, n_override=None,
          arrays: bool = True) -> list:
    """Runs the chosen figures' parameter sets; n_override shrinks the grids (tests);
    arrays=False skips the .npy files (images and JSON only)."""
    os.makedirs(out_dir, exist_ok=True)
    recs = []
    for name in figs:
        fig = dict(FIGURES[name])
        if n_override:
            fig["n"] = n_override[fig["dim"]]
            if "excerpt" in fig:
                fig["excerpt"] = min(fig["excerpt"], fig["n"])
        for ps in fig["sets"]:
            tag = f"p{ps['p']:g}_alpha{ps['alpha']:g}"
            recs.append(run_set(fig, ps, seed, out_dir, tag, name, arrays))
    with open(os.path.join(out_dir, "index.json"), "w") as fh:
        json.dump([{k: r[k] for k in ("figure", "tag", "alpha", "p", "ab", "seconds_generate",
                                      "seconds_pipeline")} for r in recs], fh, indent=1)
    return recs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--figs", nargs="+", default=list(FIGURES), choices=list(FIGURES))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-arrays", action="store_true", help="images and JSON only")
    args = ap.parse_args(argv)
    for r in sweep(args.out, args.figs, args.seed, arrays=not args.no_arrays):
        print(f"{r['figure']} {r['tag']}: generate {1e3 * r['seconds_generate']:.2f} ms, "
              f"pipeline {1e3 * r['seconds_pipeline']:.2f} ms")


if __name__ == "__main__":
    main()
