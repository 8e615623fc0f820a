"""FP64 CPU oracle of the surrogate network (test infrastructure only).

The paper (Sec. IV) names optimisation loops over the generator's parameters
as future work; the surrogate is this project's take on them: a multilayer
perceptron from the eight filter and threshold parameters to the log radial
S(k) bins of the thresholded +-1 map, trained on fields the plain generator
makes, then differentiated with respect to its inputs for inverse design.
Nothing here is the paper's; every function is a textbook definition written
out plainly in numpy FP64:

- encode      affine maps of the eight parameters onto [-1, 1]
- forward     z_l = W_l a_{l-1} + b_l, a_l = GELU(z_l) on hidden layers
              (GELU(x) = x Phi(x), the exact Gaussian form), linear output
- backward    the chain rule layer by layer (dW = dz^T a, db = sum dz,
              da = dz W, dz = da GELU'(z)), GELU'(x) = Phi(x) + x phi(x)
- deviance    the exponential negative log-likelihood y + S e^{-y} per bin,
              whose minimiser over y is log E[S]: the network learns the log
              of the mean spectrum from single-field samples
- design loss relative L2 (squared) of e^y against a target spectrum over
              the bins b >= 1, plus a small log-space term
- adam        Kingma & Ba (ICLR 2015) with bias correction and decoupled
              weight decay

`emulate_bf16=True` rounds to BF16 at the points where the GPU kernels store
BF16 (the weights, each layer's input activations and the back-propagated
dz), so that the GPU's FP32-accumulated results can be compared tightly;
without it everything stays FP64 (the reference the BF16 error is stated
against).  Only the test suite, smoke() and bench.py's CPU-baseline leg use
this module.

Parity pins live in tests/test_oracle_mlp.py: finite differences for every
gradient, closed forms of GELU and of Adam's first step, a purely linear
network against a plain matrix product, and round-trip of encode/decode.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

# Architecture of the surrogate: 8 inputs, three hidden layers of 256, 128 outputs.
WIDTHS = (8, 256, 256, 256, 128)
IN_PAD = 32  # the first layer's input width as stored (zero-padded)

# Parameter ranges (the ragged workload's draws) and their encodings onto [-1, 1]:
# p in [1, 8]; semi-axis ratios r1, r2 in [0.5, 2] (as log2 r); rotation in [0, pi);
# k0 in [0.05, 0.4]; width in [0.01, 0.1]; s in {2, 4, 6}; threshold level t in [-1, 1].
NAMES = ("p", "r1", "r2", "rot", "k0", "width", "supp", "level")


def encode(theta: np.ndarray) -> np.ndarray:
    """Raw parameters [rows, 8] -> network inputs [rows, 8] on [-1, 1]."""
    t = np.asarray(theta, np.float64)
    x = np.empty_like(t)
    x[:, 0] = (t[:, 0] - 4.5) / 3.5
    x[:, 1] = np.log2(t[:, 1])
    x[:, 2] = np.log2(t[:, 2])
    x[:, 3] = 2.0 * t[:, 3] / math.pi - 1.0
    x[:, 4] = (t[:, 4] - 0.225) / 0.175
    x[:, 5] = (t[:, 5] - 0.055) / 0.045
    x[:, 6] = (t[:, 6] - 4.0) / 2.0
    x[:, 7] = t[:, 7]
    return x


def decode(x: np.ndarray) -> np.ndarray:
    """Inverse of encode."""
    x = np.asarray(x, np.float64)
    t = np.empty_like(x)
    t[:, 0] = 4.5 + 3.5 * x[:, 0]
    t[:, 1] = np.exp2(x[:, 1])
    t[:, 2] = np.exp2(x[:, 2])
    t[:, 3] = 0.5 * math.pi * (x[:, 3] + 1.0)
    t[:, 4] = 0.225 + 0.175 * x[:, 4]
    t[:, 5] = 0.055 + 0.045 * x[:, 5]
    t[:, 6] = 4.0 + 2.0 * x[:, 6]
    t[:, 7] = x[:, 7]
    return t


def layer_shapes(widths=WIDTHS, in_pad=IN_PAD):
    """(n_out, n_in as stored) of each layer."""
    out = []
    for l in range(len(widths) - 1):
        n_in = widths[l] if l > 0 else max(in_pad, widths[0])
        out.append((widths[l + 1], n_in))
    return out


def param_count(widths=WIDTHS, in_pad=IN_PAD) -> int:
    return sum(o * i + o for o, i in layer_shapes(widths, in_pad))


def unpack(flat: np.ndarray, widths=WIDTHS, in_pad=IN_PAD):
    """Flat parameter vector -> [(W [n_out, n_in], b [n_out])], each layer's W
    (row-major) followed by its b."""
    flat = np.asarray(flat, np.float64)
    out, off = [], 0
    for o, i in layer_shapes(widths, in_pad):
        W = flat[off: off + o * i].reshape(o, i)
        off += o * i
        b = flat[off: off + o]
        off += o
        out.append((W, b))
    assert off == flat.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to BF16 (round to nearest, ties to even) and back to FP64: the
    value's FP32 bit pattern keeps its top 16 bits after adding half of the
    dropped part's unit (plus one when the kept part is odd).  Values are first
    rounded to FP32, as the GPU holds them."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _pad_input(x, n_in):
    x = np.asarray(x, np.float64)
    out = np.zeros((x.shape[0], n_in))
    out[:, : x.shape[1]] = x
    return out


def forward(params, x, emulate_bf16=False, widths=WIDTHS, in_pad=IN_PAD):
    """Network output y [rows, n_out] and the cache backward needs."""
    layers = unpack(params, widths, in_pad)
    rnd = bf16 if emulate_bf16 else (lambda v: v)
    a = rnd(_pad_input(x, layers[0][0].shape[1]))
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ rnd(W).T + b
        zs.append(z)
        if l + 1 < len(layers):
            a = rnd(gelu(z))
            acts.append(a)
        else:
            a = z
    return a, {"acts": acts, "zs": zs}


def backward(params, cache, dy, emulate_bf16=False, widths=WIDTHS, in_pad=IN_PAD):
    """Gradients of sum(dy * y): the flat parameter gradient and dL/dx [rows, 8]."""
    layers = unpack(params, widths, in_pad)
    rnd = bf16 if emulate_bf16 else (lambda v: v)
    grads = [None] * len(layers)
    dz = rnd(np.asarray(dy, np.float64))
    dx = None
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_prev = cache["acts"][l]
        dW = dz.T @ a_prev
        db = dz.sum(axis=0)
        grads[l] = (dW, db)
        da = dz @ rnd(W)
        if l > 0:
            dz = rnd(da * gelu_grad(cache["zs"][l - 1]))
        else:
            dx = da[:, : widths[0]]
    return pack(grads), dx


def deviance(y_hat, S, mu, sigma):
    """Mean of y + S e^{-y} over rows and bins (y = mu + sigma y_hat, the log of the
    predicted mean spectrum) and its gradient with respect to y_hat."""
    y = np.asarray(mu) + np.asarray(sigma) * np.asarray(y_hat, np.float64)
    n = y.size
    e = np.exp(-y)
    loss = float(np.mean(y + S * e))
    grad = np.asarray(sigma) * (1.0 - S * e) / n
    return loss, grad


def design_loss(y_hat, target, mu, sigma, lam=0.01, first_bin=1):
    """Per row: sum_{b >= first_bin} (e^{y_b} - T_b)^2 / sum T_b^2 + lam mean (y_b - log T_b)^2,
    and its gradient with respect to y_hat."""
    y = np.asarray(mu) + np.asarray(sigma) * np.asarray(y_hat, np.float64)
    T = np.asarray(target, np.float64)
    sel = slice(first_bin, None)
    nb = y.shape[1] - first_bin
    ey = np.exp(y[:, sel])
    den = np.sum(T[:, sel] ** 2, axis=1, keepdims=True)
    lt = np.log(T[:, sel])
    loss = np.sum((ey - T[:, sel]) ** 2, axis=1) / den[:, 0] + lam * np.sum((y[:, sel] - lt) ** 2, axis=1) / nb
    g = np.zeros_like(y)
    g[:, sel] = 2.0 * (ey - T[:, sel]) * ey / den + 2.0 * lam * (y[:, sel] - lt) / nb
    return loss, g * np.asarray(sigma)


def adam(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One Adam step (step counts from 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = params - lr * (mh / (np.sqrt(vh) + eps) + wd * params)
    return p, m, v


def init(seed: int, widths=WIDTHS, in_pad=IN_PAD) -> np.ndarray:
    """Initial parameters: W uniform on [-1/sqrt(fan_in), 1/sqrt(fan_in)] with fan_in the
    layer's true input width (the first layer's padding columns are 0), b = 0.  Word i
    of the flat vector comes from Philox4x32-10 block i >> 2 (word i & 3) with counter
    (j lo, j hi, 0x4D4C5031, 0) and key = seed, u = (x + 1/2) 2^-32, w = (2u - 1) bound."""
    from oracle import noise_bits

    n = param_count(widths, in_pad)
    bits = noise_bits((n,), seed, 0x4D4C5031).astype(np.float64)
    u = (bits + 0.5) * 2.0 ** -32
    flat = np.zeros(n)
    off = 0
    for l, (o, i) in enumerate(layer_shapes(widths, in_pad)):
        fan = widths[l]
        bound = 1.0 / math.sqrt(fan)
        w = ((2.0 * u[off: off + o * i] - 1.0) * bound).reshape(o, i)
        w[:, fan:] = 0.0
        flat[off: off + o * i] = w.reshape(-1)
        off += o * i + o  # biases stay 0
    return flat


def labels(sums, counts) -> np.ndarray:
    """Bin means S = sums / counts per item (0 for an empty bin), [items, 128]."""
    s = np.asarray(sums, np.float64).reshape(-1, WIDTHS[-1])
    c = np.asarray(counts, np.float64).reshape(-1, WIDTHS[-1])
    return np.where(c > 0, s / np.maximum(c, 1.0), 0.0)


def label_stats(S):
    """Per-bin mean and standard deviation (at least 0.05) of log(S + 1e-3) over the rows."""
    L = np.log(np.asarray(S, np.float64) + 1e-3)
    return L.mean(axis=0), np.maximum(L.std(axis=0), 0.05)
