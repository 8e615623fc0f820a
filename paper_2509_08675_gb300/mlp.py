"""ctypes binding of the surrogate network's C ABI (include/hufield_surrogate.h).

Argument marshalling only: every step runs in the library's kernels.  Tensors
are CUDA tensors (torch supplies the device memory and the stream)."""
from __future__ import annotations

import ctypes as C

import torch

from .hufield import HufieldError, _check, _lib, _ptr, _stream

NIN = 8
NOUT = 128


class _Sched(C.Structure):
    _fields_ = [("lr", C.c_float), ("lr_min_frac", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("wd", C.c_float), ("total_steps", C.c_int64), ("seed", C.c_uint64)]


def _declare(lib):
    vp, sz, i32, i64, u32, u64, f32 = C.c_void_p, C.c_size_t, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float
    lib.hufield_mlp_param_count.argtypes = []
    lib.hufield_mlp_param_count.restype = i64
    lib.hufield_mlp_workspace_bytes.argtypes = [i64]
    lib.hufield_mlp_workspace_bytes.restype = sz
    lib.hufield_mlp_init.argtypes = [vp, u64, vp]
    lib.hufield_mlp_cast.argtypes = [vp, vp, vp]
    lib.hufield_mlp_encode.argtypes = [vp, i64, vp, vp]
    lib.hufield_mlp_decode.argtypes = [vp, i64, vp, vp]
    lib.hufield_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp, sz, vp]
    lib.hufield_mlp_backward.argtypes = [vp, vp, vp, i64, vp, vp, vp, sz, vp]
    lib.hufield_mlp_deviance.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
    lib.hufield_mlp_label_stats.argtypes = [vp, i64, vp, vp, vp]
    lib.hufield_mlp_labels.argtypes = [vp, vp, i64, vp, vp]
    lib.hufield_mlp_spectrum.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.hufield_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i64, i32, f32, f32, f32, f32, f32, vp]
    lib.hufield_mlp_gather.argtypes = [vp, vp, i64, i64, u64, i64, vp, vp, vp]
    lib.hufield_mlp_design_loss.argtypes = [vp, vp, vp, vp, i64, f32, vp, vp, vp]
    lib.hufield_mlp_design_step.argtypes = [vp, vp, vp, vp, i64, u32, i32, f32, vp]
    lib.hufield_mlp_train_workspace_bytes.argtypes = [i64]
    lib.hufield_mlp_train_workspace_bytes.restype = sz
    lib.hufield_mlp_train_reset.argtypes = [vp, i64, vp]
    lib.hufield_mlp_train_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, i64, vp, vp, C.POINTER(_Sched), vp, vp,
                                           sz, vp]


_declare(_lib)


def param_count() -> int:
    return int(_lib.hufield_mlp_param_count())


def workspace_bytes(rows: int) -> int:
    return int(_lib.hufield_mlp_workspace_bytes(int(rows)))


def _rows(t: torch.Tensor, width: int, what: str) -> int:
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != width:
        raise HufieldError(1, f"{what}: expected a float32 [rows, {width}] tensor")
    return int(t.shape[0])


class Params:
    """FP32 master parameters with their BF16 copy (and Adam's moments when trained)."""

    def __init__(self, seed: int = 0, device="cuda", stream=None):
        n = param_count()
        self.p = torch.empty(n, dtype=torch.float32, device=device)
        self.wq = torch.empty(n, dtype=torch.int16, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.grad = torch.zeros(n, dtype=torch.float32, device=device)
        self.step = 0
        _check(_lib.hufield_mlp_init(_ptr(self.p), seed, _stream(stream)), "hufield_mlp_init")
        self.cast(stream)

    def cast(self, stream=None):
        _check(_lib.hufield_mlp_cast(_ptr(self.p), _ptr(self.wq), _stream(stream)), "hufield_mlp_cast")

    def load(self, flat: torch.Tensor, stream=None):
        self.p.copy_(flat)
        self.cast(stream)


class Workspace:
    def __init__(self, rows: int, device="cuda"):
        self.rows = int(rows)
        self.buf = torch.empty(workspace_bytes(rows), dtype=torch.uint8, device=device)


def encode(theta: torch.Tensor, x: torch.Tensor, stream=None):
    rows = _rows(theta, NIN, "hufield_mlp_encode")
    _check(_lib.hufield_mlp_encode(_ptr(theta), rows, _ptr(x), _stream(stream)), "hufield_mlp_encode")


def decode(x: torch.Tensor, theta: torch.Tensor, stream=None):
    rows = _rows(x, NIN, "hufield_mlp_decode")
    _check(_lib.hufield_mlp_decode(_ptr(x), rows, _ptr(theta), _stream(stream)), "hufield_mlp_decode")


def forward(P: Params, x: torch.Tensor, y: torch.Tensor, ws: Workspace, stream=None):
    rows = _rows(x, NIN, "hufield_mlp_forward")
    if y.shape != (rows, NOUT) or ws.rows < rows:
        raise HufieldError(1, "hufield_mlp_forward: y must be [rows, 128] and the workspace hold rows")
    _check(_lib.hufield_mlp_forward(_ptr(P.p), _ptr(P.wq), _ptr(x), rows, _ptr(y), _ptr(ws.buf), ws.buf.numel(),
                                    _stream(stream)), "hufield_mlp_forward")


def backward(P: Params, dy: torch.Tensor, ws: Workspace, grad: torch.Tensor | None, dx: torch.Tensor | None,
             stream=None):
    rows = _rows(dy, NOUT, "hufield_mlp_backward")
    if dx is not None and dx.shape != (rows, NIN):
        raise HufieldError(1, "hufield_mlp_backward: dx must be [rows, 8]")
    _check(_lib.hufield_mlp_backward(_ptr(P.p), _ptr(P.wq), _ptr(dy), rows, _ptr(grad), _ptr(dx), _ptr(ws.buf),
                                     ws.buf.numel(), _stream(stream)), "hufield_mlp_backward")


def deviance(y_hat, S, mu, sigma, dy, loss_sum, stream=None):
    rows = _rows(y_hat, NOUT, "hufield_mlp_deviance")
    _check(_lib.hufield_mlp_deviance(_ptr(y_hat), _ptr(S), _ptr(mu), _ptr(sigma), rows, _ptr(dy), _ptr(loss_sum),
                                     _stream(stream)), "hufield_mlp_deviance")


def spectrum(y_hat, mu, sigma, S, stream=None):
    rows = _rows(y_hat, NOUT, "hufield_mlp_spectrum")
    _check(_lib.hufield_mlp_spectrum(_ptr(y_hat), _ptr(mu), _ptr(sigma), rows, _ptr(S), _stream(stream)),
           "hufield_mlp_spectrum")


def label_stats(S, mu, sigma, stream=None):
    n = _rows(S, NOUT, "hufield_mlp_label_stats")
    _check(_lib.hufield_mlp_label_stats(_ptr(S), n, _ptr(mu), _ptr(sigma), _stream(stream)),
           "hufield_mlp_label_stats")


def labels(sums: torch.Tensor, counts: torch.Tensor, S: torch.Tensor, stream=None):
    n = _rows(S, NOUT, "hufield_mlp_labels")
    if sums.numel() < n * NOUT or counts.numel() < n * NOUT:
        raise HufieldError(1, "hufield_mlp_labels: sums and counts need rows * 128 entries")
    _check(_lib.hufield_mlp_labels(_ptr(sums), _ptr(counts), n, _ptr(S), _stream(stream)), "hufield_mlp_labels")


def adam(P: Params, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, stream=None):
    P.step += 1
    _check(_lib.hufield_mlp_adam(_ptr(P.p), _ptr(P.m), _ptr(P.v), _ptr(P.grad), _ptr(P.wq), P.p.numel(), P.step,
                                 lr, beta1, beta2, eps, wd, _stream(stream)), "hufield_mlp_adam")


def adam_raw(p, m, v, grad, wq, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, stream=None):
    _check(_lib.hufield_mlp_adam(_ptr(p), _ptr(m), _ptr(v), _ptr(grad), _ptr(wq), p.numel(), step, lr, beta1, beta2,
                                 eps, wd, _stream(stream)), "hufield_mlp_adam")


def gather(x_all, S_all, seed: int, step: int, x_out, S_out, stream=None):
    n = _rows(x_all, NIN, "hufield_mlp_gather")
    rows = _rows(x_out, NIN, "hufield_mlp_gather")
    if S_all.shape != (n, NOUT) or S_out.shape != (rows, NOUT):
        raise HufieldError(1, "hufield_mlp_gather: S arrays must be [rows, 128]")
    _check(_lib.hufield_mlp_gather(_ptr(x_all), _ptr(S_all), n, rows, seed, step, _ptr(x_out), _ptr(S_out),
                                   _stream(stream)), "hufield_mlp_gather")


def design_loss(y_hat, T, mu, sigma, lam: float, dy, loss_rows=None, stream=None):
    rows = _rows(y_hat, NOUT, "hufield_mlp_design_loss")
    _check(_lib.hufield_mlp_design_loss(_ptr(y_hat), _ptr(T), _ptr(mu), _ptr(sigma), rows, lam, _ptr(dy),
                                        _ptr(loss_rows), _stream(stream)), "hufield_mlp_design_loss")


def design_step(x, m, v, dx, frozen_mask: int, step: int, lr: float, stream=None):
    rows = _rows(x, NIN, "hufield_mlp_design_step")
    _check(_lib.hufield_mlp_design_step(_ptr(x), _ptr(m), _ptr(v), _ptr(dx), rows, frozen_mask, step, lr,
                                        _stream(stream)), "hufield_mlp_design_step")


class Trainer:
    """Whole training steps (hufield_mlp_train_step) with the step counter on the
    device: the same call replays for every step, so steps can be captured in a
    CUDA graph."""

    def __init__(self, P: Params, x_all, S_all, mu, sigma, rows: int, total_steps: int, lr: float, seed: int,
                 lr_min_frac=0.02, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, device="cuda"):
        self.n = _rows(x_all, NIN, "hufield_mlp_train_step")
        if S_all.shape != (self.n, NOUT):
            raise HufieldError(1, "hufield_mlp_train_step: S_all must be [n, 128]")
        self.P, self.x_all, self.S_all, self.mu, self.sigma = P, x_all, S_all, mu, sigma
        self.rows = int(rows)
        self.sched = _Sched(lr, lr_min_frac, beta1, beta2, eps, wd, int(total_steps), int(seed))
        self.tws = torch.empty(int(_lib.hufield_mlp_train_workspace_bytes(self.rows)), dtype=torch.uint8,
                               device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)

    def reset(self, step: int = 0, stream=None):
        _check(_lib.hufield_mlp_train_reset(_ptr(self.tws), int(step), _stream(stream)), "hufield_mlp_train_reset")

    def step(self, stream=None):
        P = self.P
        _check(_lib.hufield_mlp_train_step(_ptr(P.p), _ptr(P.wq), _ptr(P.m), _ptr(P.v), _ptr(P.grad),
                                           _ptr(self.x_all), _ptr(self.S_all), self.n, self.rows, _ptr(self.mu),
                                           _ptr(self.sigma), C.byref(self.sched), _ptr(self.loss), _ptr(self.tws),
                                           self.tws.numel(), _stream(stream)), "hufield_mlp_train_step")
