#!/usr/bin/env python3
"""Throughput of the spectral-filtering generator (generate + threshold + S(k)).

Prints ONE JSON line (rank 0).  Default workload: the 2D 4096^2 ensemble of 64
fields (p = 4, semi-axes 2:1 rotated 30 degrees, band 0.15 k_Nyq, width 0.03,
s = 4, levels 0 and +-0.5 sigma, 64 x 36 radial x angular bins); one step is
the whole ensemble.  Metric: voxels per second of the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun each rank runs its own ensemble (field indices offset by rank,
no data-path collective: weak scaling); timing is max over ranks.  The
reference arm (--impl reference) times the FP64 CPU oracle on a bounded sample
of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # 2D 4096^2 FP32 ensemble of 64 seeds, anisotropic, angularly resolved S(k)
    "ensemble-2d-4096": dict(shape=(4096, 4096), nfields=64, p=4.0, axes=(1.0, 0.5), rot=math.radians(30.0),
                             k0=0.15, width=0.03, supp=4.0, levels=(0.0, 0.5, -0.5), nr=64, ntheta=36),
    # 3D 512^3 single field, superellipsoid p = 6, semi-axes 1:1:0.5
    "3d-512": dict(shape=(512, 512, 512), nfields=1, p=6.0, axes=(1.0, 1.0, 0.5), rot=0.0, k0=0.2, width=0.04,
                   supp=2.0, levels=(0.0,), nr=256, ntheta=1),
    # the same single 512^3 fields, eight per step: two in flight on the ensemble's two lanes
    "3d-512x8": dict(shape=(512, 512, 512), nfields=8, p=6.0, axes=(1.0, 1.0, 0.5), rot=0.0, k0=0.2, width=0.04,
                     supp=2.0, levels=(0.0,), nr=256, ntheta=1),
    "3d-1024": dict(shape=(1024, 1024, 1024), nfields=1, p=6.0, axes=(1.0, 1.0, 0.5), rot=0.0, k0=0.2, width=0.04,
                    supp=2.0, levels=(0.0,), nr=256, ntheta=1),
    # 2D 256^2 isotropic single field (the small oracle case)
    "2d-256": dict(shape=(256, 256), nfields=1, p=2.0, axes=(1.0, 1.0), rot=0.0, k0=0.25, width=0.05, supp=2.0,
                   levels=(0.0,), nr=128, ntheta=1),
}
# ragged batch: 2000 fields, sizes uniform over nine lattices, parameters drawn per field
RAGGED = dict(count=2000, sizes=[(n, n) for n in (64, 128, 256, 512, 1024)] + [(n, n, n) for n in (32, 64, 128, 256)])
METRIC = "voxels/s for gen+threshold+S(k)"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant pass from an ncu capture of the current kernels, keyed by
# (workload, pass); None until captured.
TRAFFIC = {
    ("ensemble-2d-4096", "cols_bins"): 232.5e6,  # k_cols<12, 1, 2, -1, 0, 2>, 3 maps of 4096^2, per launch
    ("3d-512", "c2r"): 1566.0e6,  # k_c2r<8, 4, 0, 1>, 512^3, one-bit map
    ("3d-512x8", "c2r"): 1566.0e6,  # the same kernel on the same lattice
    ("3d-512", "r2c"): 475.7e6,  # k_r2c<8, 4, 0>, 512^3
    ("3d-512x8", "r2c"): 475.7e6,
}
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
E2E_CHUNK = 4  # fields per ensemble call in the end-to-end leg (--e2e-chunk)


def algorithmic_bytes(shape, nlev, field_bytes=4, kspace=False, live=1.0, map_bytes=1.0):
    """Bytes each pass kind must move per launch (one field), by the pass plan:
    r2c writes the half spectrum (4 B/voxel); a strided pass reads and writes it
    (8 B/voxel per spectrum; the filter pass of k-space noise only writes it);
    c2r reads it, writes the field, nlev sign maps (map_bytes per site: 1 for
    int8, 1/8 for one-bit maps) and nlev map spectra; the
    bins pass reads the nlev map spectra.  Only the columns below the filter's
    band edge hold nonzero data after the filter (a fraction `live` = kz /
    (n_last / 2) of the half spectrum): the axis-1 forward, the filter pass and
    the axis-1 inverse move that part, and c2r needs only it.  The bins of each
    mode are a function of its integer indices, so the bin table the binning
    passes read is an implementation choice, counted apart (overhead_bytes)."""
    N = math.prod(shape)
    h = 4 * N  # half spectrum bytes
    return {
        "r2c": h,
        "cols_mid_fwd": 2 * h * live,
        "cols_filter": (1 if kspace else 2) * h * live,
        "cols_mid_inv": 2 * h * live,
        "c2r": h * live + field_bytes * N + nlev * N * map_bytes + nlev * h,
        "cols_mid_maps": 2 * h * nlev,
        "cols_bins": h * nlev,
        "counts": 0,
        "misc": 0,
    }


def overhead_bytes(shape, nlev, live=1.0):
    """Bytes beyond the pass plan that the passes move per launch: the bin table
    (one uint16 per half-spectrum mode, N/2 modes; half of that with the
    paired radial order, counted here at its larger size) read by the filter
    pass over its live columns and by the bins pass once per map, and written
    by the table pass once per plan."""
    N = math.prod(shape)
    tab = N
    return {"cols_filter": tab * live, "cols_bins": tab * nlev, "counts": tab}


def field_bytes(shape, nlev, live, kspace=False, out_bytes=4, map_bytes=1.0):
    """Algorithmic bytes of one field's pipeline (the passes it runs, bin table cached)."""
    algo = algorithmic_bytes(shape, nlev, out_bytes, kspace, live, map_bytes)
    keys = ["cols_filter", "c2r"] + (["cols_bins"] if nlev else [])
    keys += [] if kspace else ["r2c"]
    if len(shape) == 3:
        keys += ["cols_mid_inv"] + ([] if kspace else ["cols_mid_fwd"]) + (["cols_mid_maps"] if nlev else [])
    return sum(algo[k] for k in keys)


def binarise_bytes(shape, map_bytes=0.125, field_bytes=4, auto_gain=True):
    """Bytes one noise-shaped binarisation call must move: the field read by the
    sigma-delta pass (and once more by the max |f - t| pass of the automatic
    gain) and the map written (1/8 byte per site one-bit, 1 int8)."""
    N = math.prod(shape)
    return (2 if auto_gain else 1) * field_bytes * N + map_bytes * N


def band_live(hf, plan, filt, shape):
    """Fraction of the half spectrum below the filter's band edge (hufield_filter_band_edge)."""
    return hf.hufield_filter_band_edge(plan, filt) / (shape[-1] // 2)


def replica_field0(rank: int, nfields: int) -> int:
    """First field index of a rank's ensemble: ranks generate disjoint fields."""
    return rank * nfields


def max_over_ranks(dist, value: float, device) -> float:
    """The slowest rank's time (weak scaling): all-reduce MAX, identity on one rank."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 50 ms during the timed region."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, out_path=None):
        self.proc = None
        self.path = out_path or os.path.join("/tmp", f"hufield_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, bus_id=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if bus_id and parts[1].lower()[-12:] != bus_id.lower()[-12:]:
                continue
            rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(wl, nfields_total, noise="real"):
    """The FP64 oracle on one field of the workload (a bounded sample)."""
    import oracle

    of = oracle.Filter(p=wl["p"], axes=wl["axes"], rot=wl["rot"], k0=wl["k0"], width=wl["width"], supp=wl["supp"])
    t0 = time.perf_counter()
    oracle.pipeline(wl["shape"], of, 0, 0, levels=wl["levels"], nr=wl["nr"], ntheta=wl["ntheta"], noise=noise)
    dt = time.perf_counter() - t0
    N = math.prod(wl["shape"])
    return {"value": N / dt, "unit": "voxels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1 field of {'x'.join(map(str, wl['shape']))} (of {nfields_total} per step), "
                      f"full FP64 pipeline, {dt:.2f} s"}


def run_reference(args, wl, name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    N = math.prod(wl["shape"])
    times = []
    for i in range(args.warmup + args.steps):
        of = oracle.Filter(p=wl["p"], axes=wl["axes"], rot=wl["rot"], k0=wl["k0"], width=wl["width"],
                           supp=wl["supp"])
        t0 = time.perf_counter()
        oracle.pipeline(wl["shape"], of, i, 0, levels=wl["levels"], nr=wl["nr"], ntheta=wl["ntheta"],
                        noise=args.noise)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = N * len(times) / tot
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "shape": list(wl["shape"]), "noise": args.noise,
                       "step_sample": "1 field per step"},
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": f"1 field of {'x'.join(map(str, wl['shape']))} per step"},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ragged_reference(args):
    """The oracle on the ragged workload: each step a bounded sample of the batch's
    items (consecutive items, about 20 s of host time)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle

    items = ragged_items(oracle, RAGGED["count"])
    vox, sec, cnt, nxt = 0, 0.0, 0, 0
    for i in range(args.warmup + args.steps):
        v, s_, c, x = ragged_oracle_sample(items, nxt, 20.0)
        nxt += c
        if i >= args.warmup:
            vox, sec, cnt = vox + x, sec + s_, cnt + c
    value = vox / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ragged-2000", "step_sample": f"about 20 s of consecutive items ({cnt} timed)"},
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": _oracle_threads(), "kind": "oracle",
                             "sample": f"{cnt} consecutive items of the 2000-item batch"},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ragged_items(mod, count, seed=0):
    """The ragged workload, filters as mod.Filter (the binding's or the oracle's):
    a host Philox stream (numpy) draws each field's lattice uniformly from the
    nine sizes and its filter: p in [1, 8], semi-axes (r1, r2) in 2D and
    (1, r1, r2) in 3D with r in [0.5, 2], rotation in [0, pi), k0 in
    [0.05, 0.4], width in [0.01, 0.1], s in {2, 4, 6}; level t in [-1, 1];
    nr = min(128, n / 2) radial bins."""
    import numpy as np

    rng = np.random.Generator(np.random.Philox(seed))
    items = []
    for i in range(count):
        shape = RAGGED["sizes"][int(rng.integers(len(RAGGED["sizes"])))]
        r1, r2 = float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.5, 2.0))
        axes = (r1, r2) if len(shape) == 2 else (1.0, r1, r2)
        filt = mod.Filter(p=float(rng.uniform(1.0, 8.0)), axes=axes, rot=float(rng.uniform(0.0, math.pi)),
                         k0=float(rng.uniform(0.05, 0.4)), width=float(rng.uniform(0.01, 0.1)),
                         supp=float(rng.choice([2.0, 4.0, 6.0])))
        items.append((shape, filt, seed, i, float(rng.uniform(-1.0, 1.0)), min(128, shape[0] // 2)))
    return items


def run_ragged(args):
    """The ragged batch as one CUDA graph launch per step (hufield_batch_run)."""
    import torch

    from paper_2509_08675_gb300 import builder

    builder.build()
    from paper_2509_08675_gb300 import hufield as hf

    torch.cuda.set_device(0)
    print(json.dumps(ragged_line(hf, torch, args)), flush=True)


def ragged_line(hf, torch, args, e2e=True, cpu=True):
    """The ragged workload's bench line (also timed inside the default run)."""
    items = ragged_items(hf, RAGGED["count"])
    bits = args.maps == "bits"
    batch = hf.Batch(items, autotune=True, maps_bits=bits)  # launch choices tuned per size class
    out_f = torch.empty(batch.total_voxels, dtype=torch.float32, device="cuda")
    if bits:  # one bit per site, 32-bit words
        maps = torch.empty(batch.total_voxels // 32, dtype=torch.int32, device="cuda")
    else:
        maps = torch.empty(batch.total_voxels, dtype=torch.int8, device="cuda")
    z = lambda dt: torch.zeros(batch.total_bins, dtype=dt, device="cuda")  # noqa: E731
    sf, cf, sm, cm = z(torch.float64), z(torch.int64), z(torch.float64), z(torch.int64)
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):  # the first run captures the graph
        hf.hufield_batch_run(batch, out_f, maps, sf, cf, sm, cm, ws, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        hf.hufield_batch_run(batch, out_f, maps, sf, cf, sm, cm, ws, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop(None)
    tot_ms = sum(a.elapsed_time(b) for a, b in ev)
    voxels = int(batch.total_voxels)
    value = args.steps * voxels / (tot_ms / 1e3)
    n3 = sum(1 for it in items if len(it[0]) == 3)
    n2 = len(items) - n3
    # pass plan per field with one level (2D 4 + 9 + 13 + 5 = 31 B/voxel, 3D 55 B/voxel
    # without a band edge), each field's filter and band edge
    plans = {tuple(it[0]): hf.Plan(tuple(it[0])) for it in items}
    nbytes = sum(field_bytes(tuple(it[0]), 1, band_live(hf, plans[tuple(it[0])], it[1], it[0]),
                             map_bytes=0.125 if bits else 1.0) for it in items)
    peak, peak_kind = peaks()
    gbs = nbytes / (tot_ms / args.steps / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ragged-2000", "fields_per_step": len(items), "fields_2d": n2, "fields_3d": n3,
                       "voxels_per_step": voxels, "levels": "one per field, t in [-1, 1]", "maps": args.maps,
                       "l2": "flushed between timed steps", "parallelism": "replicas x1",
                       "launch": "one CUDA graph per step (hufield_batch_run)", "autotuned": True},
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "traffic": None, "kernel": "whole batch graph",
                         "peak_source": peak_kind},
            "pipeline": {"bytes_per_voxel": round(nbytes / voxels, 2), "GBps": round(gbs, 1),
                         "frac": round(gbs / peak, 4)},
            "gpu_launches": args.steps * batch.launches(), "clocks": clk, "e2e": None, "cpu_baseline": None}
    if e2e and not args.no_e2e:
        line["e2e"] = ragged_e2e(hf, torch, batch, out_f, maps, (sf, cf, sm, cm), ws, stream, args)
    if cpu and not args.no_cpu_baseline:
        v, sec, cnt, vox = ragged_oracle_sample(items, 0, 15.0)
        line["cpu_baseline"] = {"value": v, "unit": "voxels/s", "cores": _oracle_threads(), "kind": "oracle",
                                "sample": f"the batch's first {cnt} items ({vox} voxels, {sec:.1f} s), full FP64 "
                                          f"pipeline with each item's filter, level and bins"}
    del batch, out_f, maps, ws, flush
    return line


def _oracle_threads():
    import oracle

    return oracle.num_threads()


def ragged_oracle_sample(items, start, seconds):
    """The FP64 oracle on consecutive items of the ragged batch from `start` until
    `seconds` of host time have passed (at least one item): voxels/s, time, items,
    voxels."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    vox, cnt, i = 0, 0, start
    while cnt == 0 or time.perf_counter() - t0 < seconds:
        shape, f, seed, idx, level, nr = items[i % len(items)]
        of = oracle.Filter(p=f.p, axes=f.axes, rot=f.rot, k0=f.k0, width=f.width, supp=f.supp)
        oracle.pipeline(shape, of, seed, idx, levels=(level,), nr=nr, ntheta=1)
        vox += math.prod(shape)
        cnt += 1
        i += 1
    sec = time.perf_counter() - t0
    return vox / sec, sec, cnt, vox


def ragged_e2e(hf, torch, batch, out_f, maps, bins, ws, stream, args):
    """The batch through its public call with every output (fields, maps, bins)
    copied to pinned host memory, steps pipelined: the outputs alternate between
    two device sets, and a second stream copies step i's while step i + 1 runs.
    A step ends when its copies have reached the host; the median of the steps'
    times (CUDA events on the copy stream) is the figure, the wall-clock mean
    beside it."""
    try:
        host_f = torch.empty(out_f.shape, dtype=out_f.dtype, pin_memory=True)
        host_m = torch.empty(maps.shape, dtype=maps.dtype, pin_memory=True)
        host_b = [torch.empty(b.shape, dtype=b.dtype, pin_memory=True) for b in bins]
    except RuntimeError:
        return None
    sets = [(out_f, maps, list(bins)),
            (torch.empty_like(out_f), torch.empty_like(maps), [torch.empty_like(b) for b in bins])]
    copy = torch.cuda.Stream()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]

    def steps(n):
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        ends = []
        for i in range(n):
            f, m, b = sets[i & 1]
            stream.wait_event(copied[i & 1])  # this set's previous copy has left the device
            hf.hufield_batch_run(batch, f, m, *b, ws, stream=stream)
            done[i & 1].record(stream)
            copy.wait_event(done[i & 1])
            with torch.cuda.stream(copy):
                host_f.copy_(f, non_blocking=True)
                host_m.copy_(m, non_blocking=True)
                for h, d in zip(host_b, b):
                    h.copy_(d, non_blocking=True)
            copied[i & 1].record(copy)
            e = torch.cuda.Event(enable_timing=True)
            e.record(copy)
            ends.append(e)
        copy.synchronize()
        stream.synchronize()
        return [start.elapsed_time(ends[0])] + [ends[q - 1].elapsed_time(ends[q]) for q in range(1, n)]

    steps(2)  # warms the pinned pages and the second set's graph
    n = max(3, min(args.steps, 5))
    t0 = time.perf_counter()
    times = steps(n)
    wall = (time.perf_counter() - t0) / n
    dt = sorted(times)[len(times) // 2] / 1e3
    d2h = (out_f.numel() * out_f.element_size() + maps.numel() * maps.element_size()
           + sum(b.numel() * b.element_size() for b in bins))
    del sets
    return {"value": batch.total_voxels / dt, "unit": "voxels/s", "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": int(d2h), "steps": n, "step_ms_median": round(1e3 * dt, 3),
            "step_ms_min": round(min(times), 3), "step_ms_max": round(max(times), 3),
            "wall_ms_mean": round(1e3 * wall, 3),
            "note": "inputs are seeds and filter parameters set at plan time; every output copied to pinned host, "
                    "step i's copies overlapping step i + 1"}


SURROGATE = dict(fields=200000, train_frac=0.9, steps=20000, batch=1024, designs=500, starts=4, iters=300,
                 plain_sample=10, plain_budget=300, plain_seeds=16)


def run_surrogate(args):
    """The surrogate workload (2D 256^2, 128 radial bins of the map's S(k)): data
    from the plain generator, training, 500 inverse designs each confirmed by the
    plain generator (64-field mean within 5% relative L2 of the target), and the
    plain generator's own search (Nelder-Mead, 16 fields per evaluation) on a
    sample of the same targets.  One JSON line: the ratio of GPU-seconds per
    confirmed design, with the surrogate's data and training amortised over the
    designs (value) and without (ratio_marginal).  GPU-seconds are the device
    time of each phase's GPU work (CUDA events around it); host work between
    (planning batches, the search's own logic) is not counted on either side."""
    import numpy as np
    import torch

    from paper_2509_08675_gb300 import builder

    builder.build()
    from paper_2509_08675_gb300 import surrogate as sg

    torch.cuda.set_device(0)
    cfg = dict(SURROGATE)
    if args.fields > 0:
        cfg["fields"] = args.fields
    # smaller runs (profiling): fewer training steps, designs or searched targets
    for key in ("train_steps", "designs", "plain_sample"):
        v = getattr(args, key)
        if v > 0:
            cfg["steps" if key == "train_steps" else key] = v
    n = cfg["fields"]
    ntr = int(cfg["train_frac"] * n)
    clocks = ClockSampler()
    clocks.start()
    th = sg.draw_thetas(n, 100)
    data = sg.generate_dataset(th, seed=7)
    model = sg.Surrogate(seed=3)
    model.fit_stats(data, ntr)
    log = model.train(data, ntr, cfg["steps"], batch=cfg["batch"], log_every=cfg["steps"] // 10)
    # held-out accuracy: predictions against the 64-field means of 200 held-out parameter sets
    hold = th[ntr:ntr + 200]
    Sh = sg.plain_spectra(hold, seed=99, nseeds=64).cpu().numpy()
    ph = model.predict(data.x[ntr:ntr + 200]).cpu().numpy()
    eh = sg.rel_err(ph, Sh)
    # targets: 64-field means at held-out random parameters (cost counted for neither method)
    tt = sg.draw_thetas(cfg["designs"], 555)
    T = sg.plain_spectra(tt, seed=11, nseeds=64)
    Tn = T.cpu().numpy()
    best, L, design_s, allth, order = model.design(T, starts=cfg["starts"], iters=cfg["iters"])
    tv = sg.Timer()  # device time of the verification runs (their batches' planning is host work)
    V = sg.plain_spectra(best, seed=12, nseeds=64, timer=tv).cpu().numpy()
    err = sg.rel_err(V, Tn)
    # a design that fails falls back to the next start by the surrogate's loss (verified the same way)
    retry = np.where(err > sg.CONFIRM)[0]
    if len(retry):
        alt = allth[retry, order[retry, 1]]
        Va = sg.plain_spectra(alt, seed=12, nseeds=64, timer=tv).cpu().numpy()
        ea = sg.rel_err(Va, Tn[retry])
        better = ea < err[retry]
        err[retry[better]] = ea[better]
    verify_s = tv.ms / 1e3
    confirmed = int((err <= sg.CONFIRM).sum())
    # the plain generator's own search on a sample of the targets, its answer
    # confirmed the same way as a design (64 fields)
    ps = []
    ev = sg.Evaluator(13, cfg["plain_seeds"])
    for i in range(cfg["plain_sample"]):
        before = ev.timer.ms
        tc = sg.Timer()
        thp, ep, nev = sg.nelder_mead_search(Tn[i], seed=13, nseeds=cfg["plain_seeds"],
                                             budget=cfg["plain_budget"], rng_seed=i, evaluator=ev)
        Vp = sg.plain_spectra(thp[None, :].astype(np.float32), seed=12, nseeds=64, timer=tc).cpu().numpy()
        ps.append((nev, (ev.timer.ms - before + tc.ms) / 1e3, float(sg.rel_err(Vp, Tn[i:i + 1])[0])))
    ev.close()
    clk = clocks.stop(None)
    plain_s = float(np.mean([p[1] for p in ps]))
    plain_ok = sum(1 for p in ps if p[2] <= sg.CONFIRM)
    plain_per_confirmed = sum(p[1] for p in ps) / max(plain_ok, 1)
    sur_marginal = (design_s + verify_s) / max(confirmed, 1)
    sur_total = (data.gpu_s + log.gpu_s + design_s + verify_s) / max(confirmed, 1)
    line = {"metric": "GPU-seconds per confirmed design: plain-generator search / surrogate (5% rel. L2 of S(k))",
            "value": plain_per_confirmed / sur_total, "unit": "x fewer GPU-seconds (amortised)", "n_gpus": 1,
            "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 weights, f32 accumulation; f32 generator", "data": "synthetic",
            "config": {"workload": "surrogate-256", "shape": [256, 256], "bins": 128, **cfg},
            "surrogate": {
                "designs": cfg["designs"], "confirmed": confirmed, "confirmed_frac": confirmed / cfg["designs"],
                "err_median": float(np.median(err)), "err_p90": float(np.percentile(err, 90)),
                "heldout_pred_err_median": float(np.median(eh)), "heldout_pred_err_p90": float(np.percentile(eh, 90)),
                "gpu_s": {"data": round(data.gpu_s, 3), "train": round(log.gpu_s, 3), "design": round(design_s, 3),
                          "verify": round(verify_s, 3)},
                "train_losses": [round(x, 5) for x in log.losses],
                "gpu_s_per_confirmed_design": {"amortised": sur_total, "marginal": sur_marginal}},
            "plain_search": {"targets": len(ps), "confirmed": plain_ok,
                             "evaluations_mean": float(np.mean([p[0] for p in ps])),
                             "gpu_s_mean": plain_s, "gpu_s_per_confirmed_design": plain_per_confirmed,
                             "errors": [round(p[2], 4) for p in ps]},
            "generator_fields_per_confirmed_design": {
                "plain_search": (sum(p[0] for p in ps) * cfg["plain_seeds"] + 64 * len(ps)) / max(plain_ok, 1),
                "surrogate_marginal": 64 * (cfg["designs"] + len(retry)) / max(confirmed, 1),
                "surrogate_amortised": (64 * (cfg["designs"] + len(retry)) + n) / max(confirmed, 1)},
            "ratio_marginal": plain_per_confirmed / sur_marginal,
            "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="ensemble-2d-4096",
                    choices=sorted(WORKLOADS) + ["ragged-2000", "surrogate-256"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparator (context line)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--train-steps", type=int, default=0, help="surrogate: training steps (default 20000)")
    ap.add_argument("--designs", type=int, default=0, help="surrogate: inverse designs (default 500)")
    ap.add_argument("--plain-sample", type=int, default=0, help="surrogate: targets searched by the plain generator")
    ap.add_argument("--fields", type=int, default=0, help="override fields per step (small profiling cases)")
    ap.add_argument("--also", default="3d-512,3d-512x8,ragged-2000,binarise",
                    help="comma-separated workloads timed in the same run ('' for none)")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="fields per ensemble call in the end-to-end leg (default %d)" % E2E_CHUNK)
    ap.add_argument("--maps", default="bits", choices=["bits", "i8"],
                    help="sign-map storage: one bit per site (default) or one int8 per site")
    ap.add_argument("--order", type=int, default=0, choices=[0, 1, 2],
                    help="strided passes' tile order: 0 default (interleaved), 1 contiguous chunks, 2 interleaved")
    ap.add_argument("--noise", default="real", choices=["real", "kspace"],
                    help="white noise in real space (forward FFT) or drawn as k-space coefficients")
    args = ap.parse_args()
    if args.workload == "surrogate-256":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the surrogate workload compares two GPU "
                              "methods; its plain-search leg is the baseline"}))
            return
        return run_surrogate(args)
    if args.workload == "ragged-2000":
        if args.impl == "reference":
            return run_ragged_reference(args)
        return run_ragged(args)
    wl = dict(WORKLOADS[args.workload])
    if args.fields > 0:
        wl["nfields"] = args.fields
    if args.impl == "reference":
        return run_reference(args, wl, args.workload)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2509_08675_gb300 import builder

    if rank == 0 or world == 1:
        builder.build()
    if dist is not None:
        dist.barrier()
    from paper_2509_08675_gb300 import hufield as hf

    res = measure(hf, torch, wl, args.workload, args, rank, world, dist)
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(hf, torch, res["plan"], res["filt"], wl, args, *res["bufs"], res["field0"], dist, world)
    also = {}
    for name in [n for n in args.also.split(",") if n and n != args.workload] if world == 1 else []:
        if name == "binarise":
            try:  # a context leg: a failure is reported in the line, not in place of it
                also[name] = binarise_line(hf, torch, args)
            except Exception as exc:  # noqa: BLE001
                also[name] = {"error": f"{type(exc).__name__}: {exc}"}
            continue
        if name == "ragged-2000":
            t_r = time.perf_counter()
            r2 = ragged_line(hf, torch, args, cpu=False)
            also[name] = {k: r2[k] for k in ("value", "ms_per_step", "config", "pipeline", "gpu_launches", "clocks",
                                             "e2e")}
            also[name]["wall_s"] = round(time.perf_counter() - t_r, 1)
            continue
        r2 = measure(hf, torch, dict(WORKLOADS[name]), name, args, rank, world, dist)
        also[name] = {k: r2[k] for k in ("value", "ms_per_step", "ms_per_step_one_lane", "lanes", "roofline",
                                         "pipeline", "passes", "clocks")}
        del r2
    comp = {}
    if world == 1 and not args.no_cufft:
        comp[args.workload] = cufft_comparator(hf, torch, wl)
        for name in also:
            if name in WORKLOADS and WORKLOADS[name]["nfields"] == 1:
                comp[name] = cufft_comparator(hf, torch, dict(WORKLOADS[name]))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(wl, wl["nfields"], args.noise)
    if rank == 0:
        shape, nlev = wl["shape"], len(wl["levels"])
        line = {"metric": METRIC, "value": res["value"], "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": args.workload, "shape": list(shape), "fields_per_step": wl["nfields"],
                           "levels": list(wl["levels"]), "bins": [wl["nr"], wl["ntheta"]],
                           "noise": args.noise, "maps": args.maps, "l2": "flushed between timed steps",
                           "parallelism": f"replicas x{world}", "lanes": res["lanes"]},
                "ms_per_step_one_lane": res["ms_per_step_one_lane"],
                "roofline": res["roofline"],
                "pipeline": res["pipeline"],
                "passes": res["passes"],
                "gpu_launches": res["gpu_launches"],
                "clocks": res["clocks"],
                "e2e": e2e,
                "cpu_baseline": cpu}
        if also:
            line["also"] = also
        if comp:
            line["cufft_comparator"] = comp
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measure(hf, torch, wl, name, args, rank, world, dist):
    """Device-timed steps of one workload: per-step CUDA events on the launching
    stream, L2 flushed between steps.  An ensemble runs on two lanes (a
    two-slice workspace: consecutive fields overlap); the per-pass times come
    from the plan's per-launch CUDA events over the same number of steps run
    on one lane, where every launch's events bracket that kernel alone."""
    shape, nf, levels = wl["shape"], wl["nfields"], wl["levels"]
    nlev, nr, nt = len(levels), wl["nr"], wl["ntheta"]
    nb = nr * nt
    N = math.prod(shape)
    fdt = torch.float32 if args.dtype == "f32" else torch.bfloat16
    filt = hf.Filter(p=wl["p"], axes=wl["axes"], rot=wl["rot"], k0=wl["k0"], width=wl["width"], supp=wl["supp"])
    plan = hf.Plan(shape, profile=True, kspace=args.noise == "kspace")
    hf.hufield_plan_set_bins(plan, nr, nt)  # plan-time bin table and counts, as a production caller would
    bits = args.maps == "bits"
    hf.hufield_plan_set_maps_format(plan, hf.MAPS_BITS if bits else hf.MAPS_I8)
    hf.hufield_plan_set_order(plan, args.order)
    ws = plan.workspace(nlev, nb, lanes=2 if nf >= 2 else 1)
    slice_bytes = (hf.hufield_workspace_bytes(plan, nlev, nb) + 255) & ~255
    ws_one = ws[:slice_bytes]  # the first slice alone: one lane
    out_f = torch.empty((nf,) + tuple(shape), dtype=fdt, device="cuda")
    if bits:  # one bit per site, 32-bit words
        maps = torch.empty((nf, nlev, N // 32), dtype=torch.int32, device="cuda")
    else:
        maps = torch.empty((nf, nlev) + tuple(shape), dtype=torch.int8, device="cuda")
    sf = torch.zeros(nb, dtype=torch.float64, device="cuda")
    cf = torch.zeros(nb, dtype=torch.int64, device="cuda")
    sm = torch.zeros(nlev * nb, dtype=torch.float64, device="cuda")
    cm = torch.zeros(nlev * nb, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    field0 = replica_field0(rank, nf)

    def step(i, w=ws):
        hf.hufield_ensemble(plan, filt, 1000 + i, field0, nf, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, w,
                            stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if hf.hufield_workspace_status(ws) != hf.OK:
        raise RuntimeError("device-side timeout during warm-up")
    hf.hufield_profile_read(plan)  # drop warm-up records

    clocks = ClockSampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
        ev[i][0].record(stream)
        step(args.warmup + i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    bus = None
    try:
        pr = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
    except Exception:
        bus = None
    clk = clocks.stop(bus)
    tot_ms = sum(a.elapsed_time(b) for a, b in ev)
    if hf.hufield_workspace_status(ws) != hf.OK:
        raise RuntimeError("device-side timeout during the timed steps")
    tot_ms = max_over_ranks(dist, tot_ms, "cuda")
    value = world * args.steps * nf * N / (tot_ms / 1e3)

    # per-pass times: the same steps on one lane (no overlap between fields)
    hf.hufield_profile_read(plan)  # drop the two-lane records
    one_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step(args.warmup + i, ws_one)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    one_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    prof = hf.hufield_profile_read(plan)
    if hf.hufield_workspace_status(ws_one) != hf.OK:
        raise RuntimeError("device-side timeout during the one-lane steps")

    # roofline of the dominant pass (per-launch CUDA-event times of the one-lane steps)
    live = band_live(hf, plan, filt, shape)
    algo = algorithmic_bytes(shape, nlev, 4 if args.dtype == "f32" else 2, args.noise == "kspace", live,
                             0.125 if bits else 1.0)
    peak, peak_kind = peaks()
    passes = {}
    for k, (ms, cnt) in prof.items():
        if cnt == 0:
            continue
        per = ms / cnt
        gbs = algo.get(k, 0) / (per / 1e3) / 1e9 if algo.get(k, 0) else None
        passes[k] = {"launches": cnt, "ms_total": round(ms, 4), "ms_per_launch": round(per, 5),
                     "GBps": round(gbs, 1) if gbs else None, "frac": round(gbs / peak, 4) if gbs else None}
    dom = max((k for k in passes if algo.get(k, 0)), key=lambda k: passes[k]["ms_total"])
    per_step_bytes = sum(algo[k] * passes[k]["launches"] / args.steps for k in passes if algo.get(k))
    pipe_gbs = per_step_bytes / (tot_ms / args.steps / 1e3) / 1e9
    over = overhead_bytes(shape, nlev, live)
    dom_per = passes[dom]["ms_per_launch"]
    traffic = TRAFFIC.get((name, dom))
    roof = {"bound": "hbm", "achieved": passes[dom]["GBps"], "peak": peak, "unit": "GB/s",
            "frac": passes[dom]["frac"], "traffic": traffic,
            "algorithmic_bytes": algo[dom],
            "traffic_over_algorithmic": round(traffic / algo[dom], 3) if traffic else None,
            "overhead_bytes": over.get(dom, 0),
            "frac_with_overhead": round((algo[dom] + over.get(dom, 0)) / (dom_per / 1e3) / 1e9 / peak, 4),
            "kernel": dom, "peak_source": peak_kind}
    return {"value": value, "ms_per_step": tot_ms / args.steps, "ms_per_step_one_lane": round(one_ms, 4),
            "lanes": 2 if nf >= 2 else 1, "roofline": roof,
            "pipeline": {"bytes_per_voxel": round(per_step_bytes / (nf * N), 2), "GBps": round(pipe_gbs, 1),
                         "frac": round(pipe_gbs / peak, 4), "band_live": round(live, 4)},
            # the one-lane steps launch what the timed steps do, less the one kernel per
            # two-lane ensemble call that joins the second lane's field bins
            "passes": passes,
            "gpu_launches": sum(p["launches"] for p in passes.values()) + (args.steps if nf >= 2 else 0),
            "clocks": clk,
            "plan": plan, "filt": filt, "bufs": (out_f, maps, sf, cf, sm, cm, ws), "field0": field0}


def binarise_line(hf, torch, args, shapes=("ensemble-2d-4096", "3d-512")):
    """Noise-shaped binarisation (hufield_binarise) of one generated field of each
    lattice, maps in the bench's format, automatic gain (the max |f - t| pass, then
    the sigma-delta pass): device time per call by CUDA events on the launching
    stream, L2 flushed between calls.  Bytes per voxel: the field read twice, the
    map written once (4 + 4 + 1/8 with one-bit maps, 4 + 4 + 1 with int8)."""
    peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    bits = args.maps == "bits"
    out = {}
    for name in shapes:
        wl = WORKLOADS[name]
        shape = tuple(wl["shape"])
        N = math.prod(shape)
        filt = hf.Filter(p=wl["p"], axes=wl["axes"], rot=wl["rot"], k0=wl["k0"], width=wl["width"],
                         supp=wl["supp"])
        plan = hf.Plan(shape)
        hf.hufield_plan_set_maps_format(plan, hf.MAPS_BITS if bits else hf.MAPS_I8)
        ws = plan.workspace(0, 0)
        f = torch.empty(shape, dtype=torch.float32, device="cuda")
        hf.hufield_generate(plan, filt, 7, 0, f, ws, stream=stream)
        m = torch.empty(N // 32 if bits else N, dtype=torch.int32 if bits else torch.int8, device="cuda")
        for _ in range(args.warmup):
            hf.hufield_binarise(plan, f, m, 0.0, 0.0, 0, ws, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            hf.hufield_binarise(plan, f, m, 0.0, 0.0, 0, ws, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        bpv = binarise_bytes(shape, 0.125 if bits else 1.0) / N
        gbs = bpv * N / (ms / 1e3) / 1e9
        out[name] = {"shape": list(shape), "ms_per_call": round(ms, 5), "voxels_per_s": N / (ms / 1e3),
                     "bytes_per_voxel": bpv, "GBps": round(gbs, 1), "frac": round(gbs / peak, 4),
                     "peak_source": peak_kind, "strip": min(shape[0], 256), "launches_per_call": 2}
        del f, m, ws, plan
    return out


def cufft_comparator(hf, torch, wl, nfields=4):
    """The same steps with library FFTs (torch.fft = cuFFT) and torch elementwise
    kernels, timed beside ours for context: torch.randn noise, rfftn, multiply by
    the filter (A from hufield_filter_modes), irfftn, normalise, threshold, rfftn of
    each map, |.|^2 and binning by index_add (radial bins, float geometry).  Not a
    product path; no parity claim."""
    shape = tuple(wl["shape"])
    N = math.prod(shape)
    M = shape[-1] // 2
    levels, nr, nt = wl["levels"], wl["nr"], wl["ntheta"]
    filt = hf.Filter(p=wl["p"], axes=wl["axes"], rot=wl["rot"], k0=wl["k0"], width=wl["width"], supp=wl["supp"])
    plan = hf.Plan(shape)
    a2 = torch.empty(N // 2, dtype=torch.float32, device="cuda")
    hf.hufield_filter_modes(plan, filt, a2)
    A = torch.zeros(shape[:-1] + (M + 1,), dtype=torch.float32, device="cuda")
    A[..., :M] = a2.view(shape[:-1] + (M,)).sqrt()
    # radial (and, in 2D, angular) bin of every rfft mode; weight 2 for 0 < k_last < M
    ks = [torch.fft.fftfreq(n, 1.0 / n, device="cuda") * (2.0 / n) for n in shape[:-1]]
    ks.append(torch.arange(M + 1, device="cuda", dtype=torch.float32) * (2.0 / shape[-1]))
    grids = torch.meshgrid(*ks, indexing="ij")
    kap = torch.sqrt(sum(g * g for g in grids))
    rb = torch.floor(kap * nr).long()
    if nt > 1:
        th = torch.atan2(grids[1], grids[0])
        th = torch.where(th < 0, th + math.pi, th)
        sb = torch.clamp(torch.floor(th / math.pi * nt).long(), max=nt - 1)
        idx = rb * nt + sb
    else:
        idx = rb
    keep = (rb < nr).reshape(-1)
    idx = idx.reshape(-1)[keep]
    w = torch.full(shape[:-1] + (M + 1,), 2.0, device="cuda")
    w[..., 0] = 1.0
    w[..., M] = 1.0
    w = w.reshape(-1)[keep]
    nb = nr * nt
    sums = torch.zeros((1 + len(levels)) * nb, dtype=torch.float64, device="cuda")

    def field(i):
        z = torch.randn(shape, device="cuda")
        G = torch.fft.rfftn(z) * A
        P = (G.real ** 2 + G.imag ** 2).reshape(-1)
        tot = (P.reshape(shape[:-1] + (M + 1,)) * torch.where(torch.arange(M + 1, device="cuda") % M == 0, 1.0,
                                                               2.0)).sum()
        f = torch.fft.irfftn(G, s=shape)
        f = f * torch.rsqrt(tot / N / N)
        sums[:nb].index_add_(0, idx, (P[keep] * w * (N / tot)).double())
        for t, lev in enumerate(levels):
            m = torch.where(f >= lev, 1.0, -1.0)
            Y = torch.fft.rfftn(m)
            sums[(1 + t) * nb:(2 + t) * nb].index_add_(0, idx, ((Y.real ** 2 + Y.imag ** 2).reshape(-1)[keep] * w
                                                                / N).double())
        return f

    for i in range(2):
        field(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(nfields):
        field(i)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / nfields
    return {"ms_per_field": round(ms, 4), "value": N / (ms / 1e3), "unit": "voxels/s", "fields_timed": nfields,
            "what": "torch.fft (cuFFT) + torch elementwise, same steps, torch.randn noise; context only"}


def measure_e2e(hf, torch, plan, filt, wl, args, out_f, maps, sf, cf, sm, cm, ws, field0, dist, world):
    """The same steps through the public ensemble call in chunks of E2E_CHUNK
    fields (two lanes each), with every output (fields, sign maps, bins) copied
    to pinned host memory on a second stream: each chunk's copies overlap the
    next chunk's compute, across step boundaries too (a chunk's buffers are
    rewritten only after their copy, the bins only after theirs).  A step ends
    when its bins have reached the host; the median of the steps' times (CUDA
    events on the copy stream) is the figure, the wall-clock mean beside it."""
    shape, nf, levels = wl["shape"], wl["nfields"], wl["levels"]
    nlev, nr, nt = len(levels), wl["nr"], wl["ntheta"]
    N = math.prod(shape)
    try:
        host_f = torch.empty(out_f.shape, dtype=out_f.dtype, pin_memory=True)
        host_m = torch.empty(maps.shape, dtype=maps.dtype, pin_memory=True)
    except RuntimeError:
        return None
    host_bins = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (sf, cf, sm, cm)]
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    step_chunk = args.e2e_chunk if args.e2e_chunk > 0 else E2E_CHUNK
    chunks = [(c, min(nf, c + step_chunk)) for c in range(0, nf, step_chunk)]
    done = [torch.cuda.Event() for _ in chunks]
    copied = [torch.cuda.Event() for _ in chunks]
    bins_copied = torch.cuda.Event()

    def steps(first, n):
        start = torch.cuda.Event(enable_timing=True)
        start.record(comp)
        ends = []
        for i in range(first, first + n):
            for k, (a, b) in enumerate(chunks):
                comp.wait_event(copied[k])  # this chunk's buffers have left the device
                if k == 0:
                    comp.wait_event(bins_copied)  # the previous step's bins too (this call clears them)
                hf.hufield_ensemble(plan, filt, 2000 + i, field0 + a, b - a, out_f[a:b], levels, maps[a:b], nr, nt,
                                    a > 0, sf, cf, sm, cm, ws, stream=comp)
                done[k].record(comp)
                copy.wait_event(done[k])
                with torch.cuda.stream(copy):
                    host_f[a:b].copy_(out_f[a:b], non_blocking=True)
                    host_m[a:b].copy_(maps[a:b], non_blocking=True)
                copied[k].record(copy)
            with torch.cuda.stream(copy):  # the step's result: its bins
                for h, d in zip(host_bins, (sf, cf, sm, cm)):
                    h.copy_(d, non_blocking=True)
            bins_copied.record(copy)
            e = torch.cuda.Event(enable_timing=True)
            e.record(copy)
            ends.append(e)
        copy.synchronize()
        comp.synchronize()
        return [start.elapsed_time(ends[0])] + [ends[q - 1].elapsed_time(ends[q]) for q in range(1, n)]

    nsteps = max(3, min(args.steps, 5))
    steps(0, 1)  # warms the pinned pages
    hf.hufield_profile_read(plan)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    times = steps(1, nsteps)
    wall = (time.perf_counter() - t0) / nsteps
    hf.hufield_profile_read(plan)
    times = [max_over_ranks(dist, t / 1e3, "cuda") for t in times]
    dt = sorted(times)[len(times) // 2]
    d2h = (out_f.numel() * out_f.element_size() + maps.numel() * maps.element_size()
           + sum(t.numel() * t.element_size() for t in (sf, cf, sm, cm)))
    return {"value": world * nf * N / dt, "unit": "voxels/s", "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": int(d2h), "steps": nsteps, "step_ms_median": round(1e3 * dt, 3),
            "step_ms_min": round(1e3 * min(times), 3), "step_ms_max": round(1e3 * max(times), 3),
            "wall_ms_mean": round(1e3 * wall, 3),
            "note": "inputs are seeds and filter parameters passed by value; every output (field, sign maps in "
                    "the plan's format, bins) copied to pinned host, copies overlapping the next chunk's compute"}


if __name__ == "__main__":
    main()
