"""Full-size workloads in the launch configuration the benchmark times (plan-cached
bins, one ensemble call): the 4096^2 ensemble, and 512^3 and 1024^3 fields.
Checked on outputs the oracle computes one by one (noise words, forward
spectrum modes, filter ratios) and on properties that hold at any size."""
import math

import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import dev_zeros, filters, np_

pytestmark = pytest.mark.gpu

CASES = [
    ("C1-4096^2x3", (4096, 4096), inputs.C1, (0.0, 0.5, -0.5), 64, 36, 3, 12),
    ("C2-512^3", (512, 512, 512), inputs.C2, (0.0,), 256, 1, 1, 6),
    ("C2-1024^3", (1024, 1024, 1024), inputs.C2, (0.0,), 256, 1, 1, 2),
]
SEED = 11


def sample_modes(shape, count, rng, of):
    """Signed modes inside the filter's band (A > 0.2), off every Nyquist plane, k_last > 0:
    random directions at the band's radius K* (in units of k_Nyq), rounded to the lattice."""
    ks = oracle.kstar(of)
    out = []
    for _ in range(20000):
        if len(out) == count:
            break
        v = rng.standard_normal(len(shape))
        v[-1] = abs(v[-1])
        v *= ks / np.linalg.norm(v) * rng.uniform(0.8, 1.2)
        m = [int(round(v[d] * shape[d] / 2)) for d in range(len(shape))]
        if m[-1] < 1 or any(abs(m[d]) >= shape[d] // 2 for d in range(len(shape))):
            continue
        if oracle.filter_value(shape, m, of) > 0.2:
            out.append(m)
    assert len(out) == count
    return np.array(out, dtype=np.int64)


def half_index(shape, m):
    """Flat index of signed mode m (k_last >= 0) in the stored half spectrum [..][n_last/2]."""
    M = shape[-1] // 2
    idx = 0
    for d, n in enumerate(shape[:-1]):
        idx = idx * n + (int(m[d]) % n)
    return idx * M + int(m[-1])


@pytest.mark.parametrize("name,shape,cfg,levels,nr,nt,nf,nmodes", CASES, ids=[c[0] for c in CASES])
def test_full_size(hf, name, shape, cfg, levels, nr, nt, nf, nmodes):
    rng = np.random.default_rng(5)
    N = math.prod(shape)
    gf, of = filters(hf, **inputs.filter_kwargs(cfg))
    plan = hf.Plan(shape)
    hf.hufield_plan_set_bins(plan, nr, nt)
    nb = nr * nt
    nlev = len(levels)
    ws = plan.workspace(nlev, nb)
    out_f = torch.empty((nf,) + shape, dtype=torch.float32, device="cuda")
    maps = torch.empty((nf, nlev) + shape, dtype=torch.int8, device="cuda")
    sf, cf = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    sm, cm = dev_zeros(nlev * nb, torch.float64), dev_zeros(nlev * nb, torch.int64)
    hf.hufield_ensemble(plan, gf, SEED, 0, nf, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    assert hf.hufield_workspace_status(ws) == hf.OK

    # 1. noise words of field 0, sampled blocks, against the oracle's Philox
    bits = torch.empty(N, dtype=torch.int32, device="cuda")
    hf.hufield_noise(plan, SEED, 0, bits=bits)
    torch.cuda.synchronize()
    blocks = rng.integers(0, N // 4, size=512)
    got = np_(bits.view(-1, 4)[torch.from_numpy(blocks).cuda()]).view(np.uint32)
    key = [SEED & 0xFFFFFFFF, SEED >> 32]
    for j, row in zip(blocks, got):
        np.testing.assert_array_equal(row, oracle.philox4x32_10([int(j) & 0xFFFFFFFF, int(j) >> 32, 0, 0], key))
    del bits

    # 2. forward spectrum of field 0 at sampled modes, each from its definition
    modes = sample_modes(shape, nmodes, rng, of)
    wsf = plan.workspace(0, 0)
    hf.hufield_forward(plan, SEED, 0, wsf)
    torch.cuda.synchronize()
    spec = wsf[256: 256 + (N // 2) * 8].view(torch.complex64)
    X_gpu = np.array([complex(np_(spec[half_index(shape, m)])) for m in modes])
    X_ref = oracle.noise_dft_at(shape, SEED, 0, modes)
    assert np.abs(X_gpu - X_ref).max() <= 2e-5 * math.sqrt(N)
    del wsf, spec

    # 3. each field: mean 0, variance sigma_f^2 = 1 (Eq. 15)
    for e in range(nf):
        f = out_f[e].double()
        assert abs(float(f.mean())) < 1e-6
        assert abs(float((f * f).mean()) - 1.0) < 2e-5
        del f

    # 4. sign maps are the threshold of the stored field, bit for bit
    for e in range(nf):
        for t, lev in enumerate(levels):
            want = (out_f[e] >= lev).to(torch.int8) * 2 - 1
            assert torch.equal(maps[e, t], want)

    # 5. the field's spectrum at the sampled modes follows |A X|^2 (one common factor, Eq. 8)
    S = torch.empty(N // 2, dtype=torch.float32, device="cuda")
    hf.hufield_spectrum_modes(plan, out_f[0], S, plan.workspace(1, 0))
    torch.cuda.synchronize()
    s_gpu = np.array([float(np_(S[half_index(shape, m)])) for m in modes])
    A = np.array([oracle.filter_value(shape, list(m), of) for m in modes])
    ref = (A * np.abs(X_ref)) ** 2
    ratio = s_gpu / ref
    assert np.abs(ratio / np.median(ratio) - 1.0).max() < 1e-4
    del S

    # 6. bins: the field's power sums to N per field (band-limited, |kappa| < 1 holds it
    # all); the map bins equal the standalone spectrum of the stored maps
    assert abs(float(np_(sf).sum()) / (nf * N) - 1.0) < 1e-5
    counts = np_(cf)
    assert counts.sum() > 0 and np.array_equal(counts, np_(cm)[:nb])
    hm = dev_zeros(nb, torch.float64)
    hc = dev_zeros(nb, torch.int64)
    ws1 = plan.workspace(1, nb)
    for e in range(nf):
        for t in range(nlev):
            hf.hufield_spectrum(plan, maps[e, t], nr, nt, e + t > 0, hm, hc, ws1)
    torch.cuda.synchronize()
    want = np_(hm)
    got = np_(sm).reshape(nlev, nb).sum(axis=0)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-9 * want.max())


def test_bf16_storage_error_512(hf):
    # BF16 field storage (Sec. II.B outputs): its error against the FP32 field, which
    # matches the FP64 oracle to 2e-6 at every parity size, is the rounding of an
    # 8-bit significand, uniform within half an ulp (2^-8 of the binade's base):
    # relative L2 1.6e-3 for a Gaussian field
    shape = (512, 512, 512)
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C2))
    plan = hf.Plan(shape)
    ws = plan.workspace(0, 0)
    f32 = torch.empty(shape, dtype=torch.float32, device="cuda")
    b16 = torch.empty(shape, dtype=torch.bfloat16, device="cuda")
    hf.hufield_generate(plan, gf, 3, 0, f32, ws)
    hf.hufield_generate(plan, gf, 3, 0, b16, ws)
    torch.cuda.synchronize()
    d = (b16.double() - f32.double())
    rel = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(f32.double()))
    assert 1.3e-3 < rel < 2.0e-3, rel
    # round to nearest: every stored value within half an ulp of BF16
    assert float((d.abs() / f32.double().abs().clamp_min(1e-30)).max()) <= 2.0 ** -8


def test_ensemble_bin_sums_against_fp64_accumulation(hf):
    # The binning passes gather each CTA's sums in FP32 over up to four tiles before
    # folding them into FP64.  Against an FP64 sum of the same per-mode map spectra
    # (hufield_spectrum_modes of the stored maps, binned on the host by the oracle's
    # bin of every stored mode, weight 2 off the k_last = 0 plane), the 4096^2
    # ensemble's 64 x 36 map bins agree far inside the 1e-4 gate.
    shape, levels, nr, nt, nf = (4096, 4096), (0.0, 0.5, -0.5), 64, 36, 4
    nb, nlev = nr * nt, len(levels)
    gf, _ = filters(hf, **inputs.filter_kwargs(inputs.C1))
    plan = hf.Plan(shape)
    hf.hufield_plan_set_bins(plan, nr, nt)
    ws = plan.workspace(nlev, nb, lanes=2)
    out_f = torch.empty((nf,) + shape, dtype=torch.float32, device="cuda")
    maps = torch.empty((nf, nlev) + shape, dtype=torch.int8, device="cuda")
    sf, cf = dev_zeros(nb, torch.float64), dev_zeros(nb, torch.int64)
    sm, cm = dev_zeros(nlev * nb, torch.float64), dev_zeros(nlev * nb, torch.int64)
    hf.hufield_ensemble(plan, gf, SEED, 0, nf, out_f, levels, maps, nr, nt, False, sf, cf, sm, cm, ws)
    torch.cuda.synchronize()
    bins = oracle.half_bins(shape, nr, nt)
    keep = bins >= 0
    M = shape[-1] // 2
    w = np.where(np.arange(bins.size) % M == 0, 1.0, 2.0)
    ref = np.zeros((nlev, nb))
    S = torch.empty(bins.size, dtype=torch.float32, device="cuda")
    ws1 = plan.workspace(1, 0)
    for e in range(nf):
        for t in range(nlev):
            hf.hufield_spectrum_modes(plan, maps[e, t], S, ws1)
            s = np_(S).astype(np.float64) * w
            ref[t] += np.bincount(bins[keep], weights=s[keep], minlength=nb)
    got = np_(sm).reshape(nlev, nb)
    sig = ref > 1e-9 * ref.max()
    rel = float(np.max(np.abs(got - ref)[sig] / ref[sig]))
    print(f"\n4096^2 x {nf} map bins against FP64 sums of the per-mode spectra: largest relative difference {rel:.2e}")
    assert rel < 2e-5
