"""FP64 CPU oracle of the spectral-filtering generator (arXiv 2509.08675, Sec. II.B).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package.  The arithmetic lives in ``hufield_oracle.c`` (plain C,
FP64, OpenMP over independent lines); this module compiles it on first use and
marshals numpy arrays in and out.  Everything is FP64 except the noise-shaped
binarisation, whose site decisions are taken in FP32 as the kernel takes them.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hufield_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None


def library_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, OpenMP) into oracle/_build/."""
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps every product and sum rounded as written
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Filter(C.Structure):
    _fields_ = [
        ("p", C.c_double),
        ("axes", C.c_double * 3),
        ("rot", C.c_double),
        ("k0", C.c_double),
        ("width", C.c_double),
        ("supp", C.c_double),
        ("form", C.c_int32),
    ]


@dataclass
class Filter:
    """Filter parameters (wavenumbers in units of the Nyquist wavenumber).

    p: superellipse exponent (Eq. 12); axes: semi-axes (a, b[, c]);
    rot: rotation of the semi-axes in the 0-1 plane (radians);
    k0, width, supp: band centre, Gaussian width and small-k exponent of
    chi = C K^supp exp(-(K-k0)^2 / (2 width^2)) (Eq. 13 when k0 = 0);
    form: 1 forces k0 = 0 (the paper's own form).
    """

    p: float = 2.0
    axes: tuple = (1.0, 1.0, 1.0)
    rot: float = 0.0
    k0: float = 0.25
    width: float = 0.05
    supp: float = 2.0
    form: int = 0

    def _c(self) -> _Filter:
        ax = tuple(float(a) for a in self.axes) + (1.0,) * (3 - len(self.axes))
        return _Filter(float(self.p), (C.c_double * 3)(*ax[:3]), float(self.rot), float(self.k0),
                       float(self.width), float(self.supp), int(self.form))


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = C.CDLL(build())
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
            fp = C.POINTER(_Filter)
            lib.or_num_threads.restype = C.c_int
            lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.or_noise_bits.argtypes = [C.c_int64, C.c_uint64, C.c_uint32, u32p]
            lib.or_noise.argtypes = [C.c_int64, C.c_uint64, C.c_uint32, f64p]
            lib.or_fftn.argtypes = [C.c_int, i64p, f64p, C.c_int]
            lib.or_kstar.argtypes = [fp]
            lib.or_kstar.restype = C.c_double
            lib.or_superellipse.argtypes = [C.c_int, f64p, fp]
            lib.or_superellipse.restype = C.c_double
            lib.or_filter_value.argtypes = [C.c_int, i64p, i64p, fp]
            lib.or_filter_value.restype = C.c_double
            lib.or_filter_grid.argtypes = [C.c_int, i64p, fp, f64p]
            lib.or_generate.argtypes = [C.c_int, i64p, fp, C.c_uint64, C.c_uint32, C.c_double, f64p, C.c_void_p]
            lib.or_inverse_realness.argtypes = [C.c_int, i64p, fp, C.c_uint64, C.c_uint32,
                                                C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.or_threshold.argtypes = [C.c_int64, f64p, C.c_double, i8p]
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
            lib.or_sd_gain.argtypes = [C.c_int64, f32p, C.c_float]
            lib.or_sd_gain.restype = C.c_float
            lib.or_sigma_delta.argtypes = [C.c_int64, C.c_int64, f32p, C.c_float, C.c_float, C.c_int64, i8p,
                                           C.c_void_p]
            lib.or_angle_table.argtypes = [C.c_int, i64p, i64p]
            lib.or_bin_of.argtypes = [C.c_int, i64p, i64p, C.c_int, C.c_int, i64p, i64p]
            lib.or_bin_of.restype = C.c_int
            lib.or_spectrum_bins.argtypes = [C.c_int, i64p, f64p, C.c_int, C.c_int, f64p, i64p]
            lib.or_half_bins.argtypes = [C.c_int, i64p, C.c_int, C.c_int, np.ctypeslib.ndpointer(np.int32, flags="C")]
            lib.or_spectrum_modes.argtypes = [C.c_int, i64p, f64p, f64p]
            lib.or_pipeline.argtypes = [C.c_int, i64p, fp, C.c_uint64, C.c_uint32, C.c_double, f64p, C.c_int,
                                        C.c_int, C.c_int, f64p, i8p, f64p, i64p, f64p, i64p]
            lib.or_kspace_noise.argtypes = [C.c_int, i64p, C.c_uint64, C.c_uint32, f64p]
            lib.or_generate_kspace.argtypes = [C.c_int, i64p, fp, C.c_uint64, C.c_uint32, C.c_double, f64p,
                                               C.c_void_p]
            lib.or_pipeline_noise.argtypes = [C.c_int, i64p, fp, C.c_uint64, C.c_uint32, C.c_int, C.c_double,
                                              f64p, C.c_int, C.c_int, C.c_int, f64p, i8p, f64p, i64p, f64p, i64p]
            lib.or_window_variance.argtypes = [C.c_int, i64p, f64p, C.c_int, f64p, f64p]
            lib.or_window_variance_filter.argtypes = [C.c_int, i64p, fp, C.c_double, C.c_int, f64p, f64p]
            lib.or_noise_dft_at.argtypes = [C.c_int, i64p, C.c_uint64, C.c_uint32, C.c_int, i64p, f64p]
            _LIB = lib
        return _LIB


def _dims(shape) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(shape, dtype=np.int64))


def num_threads() -> int:
    return int(_lib().or_num_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, np.uint32)
    _lib().or_philox4x32_10(c, k, out)
    return out


def noise_bits(shape, seed: int, field_idx: int = 0) -> np.ndarray:
    N = int(np.prod(shape))
    out = np.zeros(N, np.uint32)
    _lib().or_noise_bits(N, seed, field_idx, out)
    return out.reshape(shape)


def noise(shape, seed: int, field_idx: int = 0) -> np.ndarray:
    N = int(np.prod(shape))
    out = np.zeros(N, np.float64)
    _lib().or_noise(N, seed, field_idx, out)
    return out.reshape(shape)


def fftn(a: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Own radix-2 DFT along every axis (forward: e^{-i}, inverse: e^{+i}, no 1/N)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    buf = a.view(np.float64).reshape(-1).copy()
    _lib().or_fftn(a.ndim, _dims(a.shape), buf, 1 if inverse else -1)
    return buf.view(np.complex128).reshape(a.shape)


def kstar(filt: Filter) -> float:
    return float(_lib().or_kstar(C.byref(filt._c())))


def superellipse(kappa, filt: Filter) -> float:
    k = np.ascontiguousarray(np.asarray(kappa, dtype=np.float64))
    return float(_lib().or_superellipse(len(k), k, C.byref(filt._c())))


def filter_value(shape, idx, filt: Filter) -> float:
    return float(_lib().or_filter_value(len(shape), _dims(shape), _dims(idx), C.byref(filt._c())))


def filter_grid(shape, filt: Filter) -> np.ndarray:
    out = np.zeros(int(np.prod(shape)), np.float64)
    _lib().or_filter_grid(len(shape), _dims(shape), C.byref(filt._c()), out)
    return out.reshape(shape)


def kspace_noise(shape, seed: int, field_idx: int = 0) -> np.ndarray:
    """Hermitian k-space white-noise coefficients on the full lattice (FFT order)."""
    N = int(np.prod(shape))
    out = np.zeros(2 * N, np.float64)
    _lib().or_kspace_noise(len(shape), _dims(shape), seed, field_idx, out)
    return out.view(np.complex128).reshape(shape)


def _noise_mode(noise: str) -> int:
    if noise not in ("real", "kspace"):
        raise ValueError(f"noise must be 'real' or 'kspace', not {noise!r}")
    return 1 if noise == "kspace" else 0


def generate(shape, filt: Filter, seed: int, field_idx: int = 0, sigma_f: float = 1.0,
             return_spectrum: bool = False, noise: str = "real"):
    N = int(np.prod(shape))
    f = np.zeros(N, np.float64)
    spec = np.zeros(2 * N, np.float64) if return_spectrum else None
    fn = _lib().or_generate_kspace if _noise_mode(noise) else _lib().or_generate
    fn(len(shape), _dims(shape), C.byref(filt._c()), seed, field_idx, sigma_f, f,
       spec.ctypes.data if spec is not None else None)
    if return_spectrum:
        return f.reshape(shape), spec.view(np.complex128).reshape(shape)
    return f.reshape(shape)


def inverse_realness(shape, filt: Filter, seed: int, field_idx: int = 0):
    mi, rms = C.c_double(), C.c_double()
    _lib().or_inverse_realness(len(shape), _dims(shape), C.byref(filt._c()), seed, field_idx,
                               C.byref(mi), C.byref(rms))
    return mi.value, rms.value


def threshold(f: np.ndarray, t: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    m = np.zeros(f.size, np.int8)
    _lib().or_threshold(f.size, f.reshape(-1), float(t), m)
    return m.reshape(f.shape)


def sd_gain(f: np.ndarray, t: float = 0.0) -> float:
    """Automatic gain of the noise-shaped binarisation: 1 / max |f - t| in FP32 (0 when f == t)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    return float(_lib().or_sd_gain(f.size, f.reshape(-1), float(t)))


def sigma_delta(f: np.ndarray, t: float = 0.0, gain: float = 0.0, strip: int = 0, return_error: bool = False):
    """Noise-shaped binarisation of a stored FP32 field (first-order sigma-delta
    along axis 0 in strips of ``strip`` rows, 0: min(n0, 256)); ``gain`` 0 asks
    for 1 / max |f - t|.  Returns the +-1 map as int8 (and the error state after
    each site, FP32, with ``return_error``)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    n0 = f.shape[0]
    h = min(n0, 256) if strip == 0 else int(strip)
    if h < 1 or n0 % h:
        raise ValueError("strip must divide the length of axis 0")
    m = np.zeros(f.size, np.int8)
    err = np.zeros(f.size, np.float32) if return_error else None
    _lib().or_sigma_delta(n0, f.size // n0, f.reshape(-1), float(t), float(gain), h, m,
                          err.ctypes.data if return_error else None)
    m = m.reshape(f.shape)
    return (m, err.reshape(f.shape)) if return_error else m


def angle_table(ntheta: int):
    c = np.zeros(ntheta, np.int64)
    s = np.zeros(ntheta, np.int64)
    _lib().or_angle_table(ntheta, c, s)
    return c, s


def bin_of(shape, idx, nr: int, ntheta: int = 1) -> int:
    c, s = angle_table(ntheta)
    return int(_lib().or_bin_of(len(shape), _dims(shape), _dims(idx), nr, ntheta, c, s))


def half_bins(shape, nr: int, ntheta: int = 1) -> np.ndarray:
    """Bin of every mode of the stored half spectrum [..][n_last/2] (-1: dropped)."""
    out = np.zeros(int(np.prod(shape)) // 2, np.int32)
    _lib().or_half_bins(len(shape), _dims(shape), nr, ntheta, out)
    return out


def spectrum_bins(y: np.ndarray, nr: int, ntheta: int = 1):
    y = np.ascontiguousarray(y, dtype=np.float64)
    sums = np.zeros(nr * ntheta, np.float64)
    counts = np.zeros(nr * ntheta, np.int64)
    _lib().or_spectrum_bins(y.ndim, _dims(y.shape), y.reshape(-1), nr, ntheta, sums, counts)
    return sums, counts


def spectrum_modes(y: np.ndarray) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(y.size, np.float64)
    _lib().or_spectrum_modes(y.ndim, _dims(y.shape), y.reshape(-1), out)
    return out.reshape(y.shape)


def pipeline(shape, filt: Filter, seed: int, field_idx: int = 0, levels=(0.0,), nr: int = 128,
             ntheta: int = 1, sigma_f: float = 1.0, noise: str = "real"):
    """Field, sign maps, binned S of the field and of each map (all FP64)."""
    N = int(np.prod(shape))
    nlev = len(levels)
    nb = nr * ntheta
    f = np.zeros(N, np.float64)
    maps = np.zeros(max(nlev, 1) * N, np.int8)
    sf = np.zeros(nb, np.float64)
    cf = np.zeros(nb, np.int64)
    sm = np.zeros(max(nlev, 1) * nb, np.float64)
    cm = np.zeros(max(nlev, 1) * nb, np.int64)
    lev = np.ascontiguousarray(np.asarray(levels, dtype=np.float64).reshape(-1)) if nlev else np.zeros(1)
    _lib().or_pipeline_noise(len(shape), _dims(shape), C.byref(filt._c()), seed, field_idx, _noise_mode(noise),
                             sigma_f, lev, nlev, nr, ntheta, f, maps, sf, cf, sm, cm)
    return {
        "f": f.reshape(shape),
        "maps": maps[: nlev * N].reshape((nlev,) + tuple(shape)),
        "sums_f": sf, "counts_f": cf,
        "sums_m": sm[: nlev * nb].reshape(nlev, nb), "counts_m": cm[: nlev * nb].reshape(nlev, nb),
    }


def window_variance(y: np.ndarray, radii) -> np.ndarray:
    """sigma_F^2(R) of a lattice field, Eq. (1), for each radius (lattice units)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    R = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    out = np.zeros(R.size, np.float64)
    _lib().or_window_variance(y.ndim, _dims(y.shape), y.reshape(-1), R.size, R, out)
    return out


def window_variance_filter(shape, filt: Filter, radii, sigma_f: float = 1.0) -> np.ndarray:
    """Ensemble mean of sigma_F^2(R) for fields generated with `filt`."""
    R = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    out = np.zeros(R.size, np.float64)
    _lib().or_window_variance_filter(len(shape), _dims(shape), C.byref(filt._c()), sigma_f, R.size, R, out)
    return out


def noise_dft_at(shape, seed: int, field_idx: int, modes) -> np.ndarray:
    """Forward DFT of the noise at the given signed modes, each from its definition."""
    m = np.ascontiguousarray(np.asarray(modes, dtype=np.int64).reshape(-1, len(shape)))
    out = np.zeros(2 * len(m), np.float64)
    _lib().or_noise_dft_at(len(shape), _dims(shape), seed, field_idx, len(m), m.reshape(-1), out)
    return out.view(np.complex128)
