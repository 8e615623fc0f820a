"""Thin ctypes binding of the C ABI in include/hufield.h.

Argument marshalling only: every step of the generator runs in the CUDA
kernels of libhufield.  Tensors are torch CUDA tensors (device memory and
streams come from PyTorch); the functions keep the C names.  A missing
library raises at import time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import platform
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, f"libhufield_{platform.machine()}.so")

(OK, ERR_INVALID_ARG, ERR_UNSUPPORTED_DIMS, ERR_WS_TOO_SMALL, ERR_CUDA, ERR_TIMEOUT, ERR_TOO_LARGE,
 ERR_NO_POWER) = range(8)
F32, BF16, I8 = 0, 1, 2
PLAN_PROFILE = 1
PLAN_INJECT_TIMEOUT = 2
PLAN_KSPACE_NOISE = 4
MAX_LEVELS = 8

_DTYPES = {torch.float32: F32, torch.bfloat16: BF16, torch.int8: I8}


class HufieldError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class _Dims(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("reserved", C.c_int32), ("n", C.c_int64 * 3)]


class _Filter(C.Structure):
    _fields_ = [("p", C.c_float), ("axes", C.c_float * 3), ("rot", C.c_float), ("k0", C.c_float),
                ("width", C.c_float), ("supp", C.c_float), ("sigma_f", C.c_float), ("form", C.c_int32),
                ("nyquist", C.c_int32)]


class _BatchItem(C.Structure):
    _fields_ = [("dims", _Dims), ("filt", _Filter), ("seed", C.c_uint64), ("field_idx", C.c_uint32),
                ("level", C.c_float), ("nr", C.c_int32)]


@dataclass
class Filter:
    """hufield_filter: wavenumbers in units of the Nyquist wavenumber."""

    p: float = 2.0
    axes: tuple = (1.0, 1.0, 1.0)
    rot: float = 0.0
    k0: float = 0.25
    width: float = 0.05
    supp: float = 2.0
    sigma_f: float = 1.0
    form: int = 0
    nyquist: int = 0

    def _c(self) -> _Filter:
        ax = tuple(float(a) for a in self.axes) + (1.0,) * (3 - len(self.axes))
        return _Filter(self.p, (C.c_float * 3)(*ax[:3]), self.rot, self.k0, self.width, self.supp, self.sigma_f,
                       int(self.form), int(self.nyquist))


def paper_filter(alpha: float, sigma: float, p: float, axes, n: int, L: float, sigma_f: float = 1.0) -> Filter:
    """The paper's parameters (Eq. 13 with physical sigma on a cube of side L, n points
    per axis) in Nyquist units: width = sigma / k_Nyq with k_Nyq = pi n / L."""
    knyq = math.pi * n / L
    return Filter(p=p, axes=tuple(axes), rot=0.0, k0=0.0, width=sigma / knyq, supp=alpha, sigma_f=sigma_f, form=1)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2509_08675_gb300.build() "
                          "(the CUDA library is required, there is no fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, sz, i32, u32, u64 = C.c_void_p, C.c_size_t, C.c_int32, C.c_uint32, C.c_uint64
    fptr = C.POINTER(_Filter)
    lib.hufield_plan_create.argtypes = [C.POINTER(vp), C.POINTER(_Dims), u32]
    lib.hufield_plan_destroy.argtypes = [vp]
    lib.hufield_workspace_bytes.argtypes = [vp, i32, i32]
    lib.hufield_workspace_bytes.restype = sz
    lib.hufield_noise.argtypes = [vp, u64, u32, vp, vp, vp]
    lib.hufield_forward.argtypes = [vp, u64, u32, vp, sz, vp]
    lib.hufield_generate.argtypes = [vp, fptr, u64, u32, i32, vp, vp, sz, vp]
    lib.hufield_threshold.argtypes = [vp, vp, i32, C.POINTER(C.c_float), i32, vp, vp]
    lib.hufield_binarise.argtypes = [vp, vp, i32, C.c_float, C.c_float, i32, vp, vp, sz, vp]
    lib.hufield_spectrum.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, vp, sz, vp]
    lib.hufield_spectrum_modes.argtypes = [vp, vp, i32, vp, vp, sz, vp]
    lib.hufield_filter_modes.argtypes = [vp, fptr, vp, vp]
    lib.hufield_filter_band_edge.argtypes = [vp, fptr, C.POINTER(C.c_int64)]
    lib.hufield_plan_autotune.argtypes = [vp, fptr, i32, i32, i32]
    lib.hufield_plan_tuning.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.hufield_plan_set_tile.argtypes = [vp, i32]
    lib.hufield_plan_tile.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.hufield_plan_set_order.argtypes = [vp, i32]
    lib.hufield_plan_order.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.hufield_plan_set_maps_format.argtypes = [vp, i32]
    lib.hufield_plan_maps_format.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.hufield_window_variance.argtypes = [vp, vp, i32, i32, C.POINTER(C.c_float), vp, vp, sz, vp]
    lib.hufield_window_variance_filter.argtypes = [vp, fptr, i32, C.POINTER(C.c_float), vp, vp, sz, vp]
    lib.hufield_pipeline.argtypes = [vp, fptr, u64, u32, i32, vp, C.POINTER(C.c_float), i32, vp, i32, i32, i32,
                                     vp, vp, vp, vp, vp, sz, vp]
    lib.hufield_ensemble.argtypes = [vp, fptr, u64, u32, i32, i32, vp, C.POINTER(C.c_float), i32, vp, i32, i32,
                                     i32, vp, vp, vp, vp, vp, sz, vp]
    lib.hufield_bins_mean.argtypes = [vp, vp, i32, vp, vp]
    lib.hufield_spectrum_noalloc.argtypes = [C.POINTER(_Dims), vp, i32, i32, i32, i32, vp, vp, vp]
    lib.hufield_spectrum_noalloc_status.argtypes = [vp]
    lib.hufield_status_string.argtypes = [C.c_int]
    lib.hufield_status_string.restype = C.c_char_p
    lib.hufield_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), i32]
    lib.hufield_workspace_status.argtypes = [vp, vp]
    lib.hufield_plan_set_bins.argtypes = [vp, i32, i32]
    lib.hufield_batch_plan.argtypes = [C.POINTER(vp), C.POINTER(_BatchItem), i32, u32]
    lib.hufield_batch_layout.argtypes = [vp, vp, vp, vp]
    lib.hufield_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.hufield_batch_destroy.argtypes = [vp]
    lib.hufield_batch_set_params.argtypes = [vp, C.POINTER(_BatchItem), i32, vp]
    lib.hufield_batch_launches.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.hufield_bins_group_mean.argtypes = [vp, vp, C.c_int64, i32, i32, vp, vp]
    lib.hufield_profile_names.argtypes = []
    lib.hufield_profile_names.restype = C.c_char_p
    return lib


_lib = _load()


def status_string(status: int) -> str:
    return _lib.hufield_status_string(int(status)).decode()


def _check(rc: int, what: str):
    if rc != OK:
        raise HufieldError(rc, what)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _levels(levels):
    levels = [float(x) for x in levels]
    return (C.c_float * max(len(levels), 1))(*levels), len(levels)


class Plan:
    """hufield_plan for one lattice shape (2D or 3D), created on the current device."""

    def __init__(self, shape, profile: bool = False, inject_timeout: bool = False, kspace: bool = False):
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) not in (2, 3):
            raise HufieldError(ERR_UNSUPPORTED_DIMS, "hufield_plan_create")
        dims = _Dims(len(self.shape), 0, (C.c_int64 * 3)(*(self.shape + (1,) * (3 - len(self.shape)))))
        h = C.c_void_p()
        flags = ((PLAN_PROFILE if profile else 0) | (PLAN_INJECT_TIMEOUT if inject_timeout else 0)
                 | (PLAN_KSPACE_NOISE if kspace else 0))
        _check(_lib.hufield_plan_create(C.byref(h), C.byref(dims), flags), "hufield_plan_create")
        self._h = h
        self.N = math.prod(self.shape)
        self.kspace = kspace

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.hufield_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, nlev: int = 0, nbins: int = 0, device=None, lanes: int = 1) -> torch.Tensor:
        """Workspace for calls with nlev maps and nbins bins; lanes = 2 holds two
        slices, with which hufield_ensemble overlaps consecutive fields."""
        n = hufield_workspace_bytes(self, nlev, nbins)
        if lanes == 2:
            n = 2 * ((n + 255) & ~255)
        elif lanes != 1:
            raise ValueError("lanes must be 1 or 2")
        return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def hufield_plan_create(shape, profile: bool = False, kspace: bool = False) -> Plan:
    return Plan(shape, profile, kspace=kspace)


def hufield_plan_destroy(plan: Plan):
    plan.close()


def hufield_workspace_bytes(plan: Plan, nlev: int, nbins: int) -> int:
    n = _lib.hufield_workspace_bytes(plan.handle, nlev, nbins)
    if n == 0:
        raise HufieldError(ERR_INVALID_ARG, "hufield_workspace_bytes")
    return int(n)


def hufield_noise(plan: Plan, seed: int, field_idx: int, bits=None, z=None, stream=None):
    _check(_lib.hufield_noise(plan.handle, seed, field_idx, _ptr(bits), _ptr(z), _stream(stream)), "hufield_noise")


def hufield_forward(plan: Plan, seed: int, field_idx: int, ws: torch.Tensor, stream=None):
    _check(_lib.hufield_forward(plan.handle, seed, field_idx, _ptr(ws), ws.numel(), _stream(stream)),
           "hufield_forward")


def hufield_generate(plan: Plan, filt: Filter, seed: int, field_idx: int, out_f: torch.Tensor, ws: torch.Tensor,
                     stream=None):
    fc = filt._c()
    _check(_lib.hufield_generate(plan.handle, C.byref(fc), seed, field_idx, _DTYPES[out_f.dtype], _ptr(out_f),
                                 _ptr(ws), ws.numel(), _stream(stream)), "hufield_generate")


def hufield_threshold(plan: Plan, f: torch.Tensor, levels, out_maps: torch.Tensor, stream=None):
    lv, n = _levels(levels)
    _check(_lib.hufield_threshold(plan.handle, _ptr(f), _DTYPES[f.dtype], lv, n, _ptr(out_maps), _stream(stream)),
           "hufield_threshold")


def hufield_binarise(plan: Plan, f: torch.Tensor, out_map: torch.Tensor, level: float = 0.0, gain: float = 0.0,
                     strip: int = 0, ws=None, stream=None):
    """Noise-shaped +-1 map of f (sigma-delta along axis 0, in strips; gain 0:
    1 / max |f - level|, which needs the workspace of hufield_generate)."""
    _check(_lib.hufield_binarise(plan.handle, _ptr(f), _DTYPES[f.dtype], float(level), float(gain), int(strip),
                                 _ptr(out_map), _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream)),
           "hufield_binarise")


def hufield_spectrum(plan: Plan, y: torch.Tensor, nr: int, ntheta: int, accumulate: bool, sums: torch.Tensor,
                     counts: torch.Tensor, ws: torch.Tensor, stream=None):
    _check(_lib.hufield_spectrum(plan.handle, _ptr(y), _DTYPES[y.dtype], nr, ntheta, int(accumulate), _ptr(sums),
                                 _ptr(counts), _ptr(ws), ws.numel(), _stream(stream)), "hufield_spectrum")


def hufield_pipeline(plan: Plan, filt: Filter, seed: int, field_idx: int, out_f, levels, out_maps, nr: int,
                     ntheta: int, accumulate: bool, sums_f, counts_f, sums_m, counts_m, ws, stream=None,
                     out_dtype=None):
    fc = filt._c()
    lv, n = _levels(levels)
    dt = _DTYPES[out_f.dtype] if out_f is not None else (out_dtype if out_dtype is not None else F32)
    _check(_lib.hufield_pipeline(plan.handle, C.byref(fc), seed, field_idx, dt, _ptr(out_f), lv, n, _ptr(out_maps),
                                 nr, ntheta, int(accumulate), _ptr(sums_f), _ptr(counts_f), _ptr(sums_m),
                                 _ptr(counts_m), _ptr(ws), ws.numel(), _stream(stream)), "hufield_pipeline")


def hufield_ensemble(plan: Plan, filt: Filter, seed: int, field0: int, nfields: int, out_f, levels, out_maps,
                     nr: int, ntheta: int, accumulate: bool, sums_f, counts_f, sums_m, counts_m, ws, stream=None,
                     out_dtype=None):
    fc = filt._c()
    lv, n = _levels(levels)
    dt = _DTYPES[out_f.dtype] if out_f is not None else (out_dtype if out_dtype is not None else F32)
    _check(_lib.hufield_ensemble(plan.handle, C.byref(fc), seed, field0, nfields, dt, _ptr(out_f), lv, n,
                                 _ptr(out_maps), nr, ntheta, int(accumulate), _ptr(sums_f), _ptr(counts_f),
                                 _ptr(sums_m), _ptr(counts_m), _ptr(ws), ws.numel(), _stream(stream)),
           "hufield_ensemble")


def hufield_spectrum_modes(plan: Plan, y: torch.Tensor, out: torch.Tensor, ws: torch.Tensor, stream=None):
    """S(n) = |DFT(y)|^2 / N over the stored half spectrum into out (float32, N/2)."""
    _check(_lib.hufield_spectrum_modes(plan.handle, _ptr(y), _DTYPES[y.dtype], _ptr(out), _ptr(ws), ws.numel(),
                                       _stream(stream)), "hufield_spectrum_modes")


def hufield_filter_modes(plan: Plan, filt: Filter, out: torch.Tensor, stream=None):
    """A(n)^2 over the stored half spectrum into out (float32, N/2)."""
    fc = filt._c()
    _check(_lib.hufield_filter_modes(plan.handle, C.byref(fc), _ptr(out), _stream(stream)), "hufield_filter_modes")


def hufield_plan_autotune(plan: Plan, filt: Filter, nlev: int, nr: int, ntheta: int = 1) -> None:
    """Time the strided passes' launch choices on hufield_pipeline calls and keep the fastest."""
    fc = filt._c()
    _check(_lib.hufield_plan_autotune(plan.handle, C.byref(fc), nlev, nr, ntheta), "hufield_plan_autotune")


def hufield_plan_set_tile(plan: Plan, tile: int) -> None:
    """Tile width of the strided passes: 0 by size, 1 wide, 2 two-column (see include/hufield.h)."""
    _check(_lib.hufield_plan_set_tile(plan.handle, int(tile)), "hufield_plan_set_tile")


def hufield_plan_set_order(plan: Plan, order: int) -> None:
    """Tile order of the strided passes: 0 default (interleaved), 1 contiguous chunks, 2 interleaved."""
    _check(_lib.hufield_plan_set_order(plan.handle, int(order)), "hufield_plan_set_order")


def hufield_plan_order(plan: Plan) -> int:
    v = C.c_int32()
    _check(_lib.hufield_plan_order(plan.handle, C.byref(v)), "hufield_plan_order")
    return int(v.value)


MAPS_I8, MAPS_BITS = 0, 1


def hufield_plan_set_maps_format(plan: Plan, fmt: int) -> None:
    """Sign-map storage of the plan's threshold/pipeline/ensemble calls: MAPS_I8 (one int8
    per site) or MAPS_BITS (one bit per site, site i at bit i % 32 of 32-bit word i // 32)."""
    _check(_lib.hufield_plan_set_maps_format(plan.handle, int(fmt)), "hufield_plan_set_maps_format")


def hufield_plan_maps_format(plan: Plan) -> int:
    v = C.c_int32()
    _check(_lib.hufield_plan_maps_format(plan.handle, C.byref(v)), "hufield_plan_maps_format")
    return int(v.value)


def hufield_plan_tile(plan: Plan) -> int:
    v = C.c_int32()
    _check(_lib.hufield_plan_tile(plan.handle, C.byref(v)), "hufield_plan_tile")
    return int(v.value)


def hufield_plan_tuning(plan: Plan) -> dict:
    """The plan's launch choices: CTAs per SM per strided-pass mode and the L2 promotion."""
    out = (C.c_int32 * 5)()
    _check(_lib.hufield_plan_tuning(plan.handle, out), "hufield_plan_tuning")
    return {"cta_cap": {"plain": out[0], "filter": out[1], "bins": out[2], "kspace": out[3]}, "l2_promotion": out[4]}


def hufield_filter_band_edge(plan: Plan, filt: Filter) -> int:
    """First k_last from which the filter is exactly zero (n_last / 2: none)."""
    fc = filt._c()
    kz = C.c_int64(0)
    _check(_lib.hufield_filter_band_edge(plan.handle, C.byref(fc), C.byref(kz)), "hufield_filter_band_edge")
    return int(kz.value)


def _radii(radii):
    r = [float(x) for x in radii]
    return (C.c_float * max(len(r), 1))(*r), len(r)


def hufield_window_variance(plan: Plan, y: torch.Tensor, radii, out: torch.Tensor, ws: torch.Tensor, stream=None):
    """sigma_F^2(R) (Eq. 1) of a stored field or sign map y into out (float64, len(radii))."""
    rv, n = _radii(radii)
    _check(_lib.hufield_window_variance(plan.handle, _ptr(y), _DTYPES[y.dtype], n, rv, _ptr(out), _ptr(ws),
                                        ws.numel(), _stream(stream)), "hufield_window_variance")


def hufield_window_variance_filter(plan: Plan, filt: Filter, radii, out: torch.Tensor, ws: torch.Tensor,
                                   stream=None):
    """Ensemble mean of sigma_F^2(R) for filter filt into out (float64, len(radii))."""
    fc = filt._c()
    rv, n = _radii(radii)
    _check(_lib.hufield_window_variance_filter(plan.handle, C.byref(fc), n, rv, _ptr(out), _ptr(ws), ws.numel(),
                                               _stream(stream)), "hufield_window_variance_filter")


def hufield_bins_mean(sums: torch.Tensor, counts: torch.Tensor, out_mean: torch.Tensor, stream=None):
    _check(_lib.hufield_bins_mean(_ptr(sums), _ptr(counts), sums.numel(), _ptr(out_mean), _stream(stream)),
           "hufield_bins_mean")


def hufield_profile_read(plan: Plan):
    """Per-pass device time (ms) and launch counts recorded since the last read
    (plans created with profile=True); synchronises on the recorded events."""
    names = _lib.hufield_profile_names().decode().split(",")
    ms = (C.c_double * len(names))()
    cnt = (C.c_int64 * len(names))()
    _check(_lib.hufield_profile_read(plan.handle, ms, cnt, len(names)), "hufield_profile_read")
    return {nm: (ms[i], cnt[i]) for i, nm in enumerate(names)}


def hufield_spectrum_noalloc(shape, y: torch.Tensor, nr: int, ntheta: int, accumulate: bool, sums: torch.Tensor,
                             counts: torch.Tensor, stream=None):
    """hufield_spectrum without a plan or workspace: the library's static device
    scratch holds the spectrum (lattices up to 2^20 voxels; see include/hufield.h)."""
    shape = tuple(int(v) for v in shape)
    if len(shape) not in (2, 3):
        raise HufieldError(ERR_UNSUPPORTED_DIMS, "hufield_spectrum_noalloc")
    # the C call sees only pointers: buffers smaller than the lattice and the bins
    # would be read or written out of bounds on the device
    nbins = int(nr) * int(ntheta)
    if y.numel() != math.prod(shape) or y.dtype not in _DTYPES:
        raise HufieldError(ERR_INVALID_ARG, "hufield_spectrum_noalloc: y must hold prod(shape) F32/BF16/I8 values")
    if nbins < 1 or sums.dtype != torch.float64 or counts.dtype != torch.int64 or sums.numel() < nbins \
            or counts.numel() < nbins:
        raise HufieldError(ERR_INVALID_ARG, "hufield_spectrum_noalloc: sums (float64) and counts (int64) need "
                                            "nr * ntheta entries")
    dims = _Dims(len(shape), 0, (C.c_int64 * 3)(*(shape + (1,) * (3 - len(shape)))))
    _check(_lib.hufield_spectrum_noalloc(C.byref(dims), _ptr(y), _DTYPES[y.dtype], nr, ntheta, int(accumulate),
                                         _ptr(sums), _ptr(counts), _stream(stream)), "hufield_spectrum_noalloc")


def hufield_spectrum_noalloc_status(stream=None) -> int:
    """Status of the most recent hufield_spectrum_noalloc call on the current device
    (waits for the stream): OK or ERR_TIMEOUT."""
    return int(_lib.hufield_spectrum_noalloc_status(_stream(stream)))


def hufield_workspace_status(ws: torch.Tensor, stream=None) -> int:
    """Status of the most recent call on `ws` (waits for the stream): OK, ERR_TIMEOUT or ERR_NO_POWER."""
    return int(_lib.hufield_workspace_status(_ptr(ws), _stream(stream)))


def hufield_plan_set_bins(plan: Plan, nr: int, ntheta: int = 1):
    """Cache the bins of (nr, ntheta) in the plan (see include/hufield.h)."""
    _check(_lib.hufield_plan_set_bins(plan.handle, nr, ntheta), "hufield_plan_set_bins")


def _batch_items(items):
    arr = (_BatchItem * len(items))()
    for i, (shape, filt, seed, field_idx, level, nr) in enumerate(items):
        shape = tuple(int(v) for v in shape)
        arr[i].dims = _Dims(len(shape), 0, (C.c_int64 * 3)(*(shape + (1,) * (3 - len(shape)))))
        arr[i].filt = filt._c()
        arr[i].seed = seed
        arr[i].field_idx = field_idx
        arr[i].level = level
        arr[i].nr = nr
    return arr


class Batch:
    """hufield_batch: a ragged batch of fields run as one CUDA graph launch.

    items: sequence of (shape, Filter, seed, field_idx, level, nr); autotune = True
    tunes every size class's plan (HUFIELD_BATCH_AUTOTUNE); lanes (1..8, 0 = the
    default of two) sets the lanes per size class (HUFIELD_BATCH_LANES); per_item =
    True runs every item through its own calls instead of batched chunks
    (HUFIELD_BATCH_PER_ITEM); updatable = True allows set_params
    (HUFIELD_BATCH_UPDATABLE); maps_bits = True writes the sign maps one bit per
    site (HUFIELD_BATCH_MAPS_BITS: total_voxels / 8 bytes)."""

    def __init__(self, items, autotune: bool = False, lanes: int = 0, per_item: bool = False,
                 updatable: bool = False, maps_bits: bool = False):
        arr = _batch_items(items)
        h = C.c_void_p()
        flags = ((1 if autotune else 0) | (2 if per_item else 0) | (4 if updatable else 0) |
                 (8 if maps_bits else 0) | ((int(lanes) & 15) << 8))
        _check(_lib.hufield_batch_plan(C.byref(h), arr, len(items), flags), "hufield_batch_plan")
        self._h = h
        self.n = len(items)
        f_off = (C.c_int64 * self.n)()
        b_off = (C.c_int64 * self.n)()
        tot = (C.c_int64 * 3)()
        _check(_lib.hufield_batch_layout(h, f_off, b_off, tot), "hufield_batch_layout")
        self.f_offset = list(f_off)
        self.bin_offset = list(b_off)
        self.total_voxels, self.total_bins, self.ws_bytes = tot[0], tot[1], tot[2]

    def launches(self) -> int:
        """Kernels one run launches."""
        v = C.c_int64()
        _check(_lib.hufield_batch_launches(self._h, C.byref(v)), "hufield_batch_launches")
        return int(v.value)

    def set_params(self, items, stream=None):
        """Replace every item's filter, seed, index and level (updatable batches)."""
        _check(_lib.hufield_batch_set_params(self._h, _batch_items(items), len(items), _stream(stream)),
               "hufield_batch_set_params")

    def close(self):
        if self._h:
            _lib.hufield_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hufield_bins_group_mean(sums, counts, groups: int, group_size: int, nbins: int, out, stream=None):
    """Mean bins of groups of consecutive items (FP32 out, groups x nbins)."""
    if sums.numel() < groups * group_size * nbins or counts.numel() < groups * group_size * nbins \
            or out.numel() < groups * nbins or out.dtype != torch.float32:
        raise HufieldError(ERR_INVALID_ARG, "hufield_bins_group_mean: buffer sizes")
    _check(_lib.hufield_bins_group_mean(_ptr(sums), _ptr(counts), groups, group_size, nbins, _ptr(out),
                                        _stream(stream)), "hufield_bins_group_mean")


def hufield_batch_run(batch: Batch, out_f, out_maps, sums_f, counts_f, sums_m, counts_m, ws, stream=None):
    _check(_lib.hufield_batch_run(batch._h, _ptr(out_f), _ptr(out_maps), _ptr(sums_f), _ptr(counts_f), _ptr(sums_m),
                                  _ptr(counts_m), _ptr(ws), ws.numel(), _stream(stream)), "hufield_batch_run")
