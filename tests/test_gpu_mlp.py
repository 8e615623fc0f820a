"""The surrogate network's kernels against the FP64 oracle (oracle/mlp.py).

With `emulate_bf16` the oracle rounds to BF16 where the kernels store BF16
(weights, layer inputs, back-propagated dz), so the two differ only by the
FP32 accumulation order and by the rare value that falls on the other side of
a BF16 rounding boundary: results agree to ~1e-4 relative, and the gates here
are 3e-4 (forward) and 1e-3 (gradients).  Against the oracle without BF16
(the network's exact FP64 value) the error of the BF16 storage is stated and
bounded at 3e-2."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from tests import inputs
from tests.gpu_common import np_, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M(hf):
    from paper_2509_08675_gb300 import mlp

    return mlp


def _params(M, seed):
    flat = inputs.mlp_params(seed)
    P = M.Params(seed=0)
    P.load(torch.from_numpy(flat).cuda())
    return P, flat.astype(np.float64)


def _layer_errors(got, want):
    out = []
    for (gw, gb), (ww, wb) in zip(omlp.unpack(got), omlp.unpack(want)):
        out.append((rel_l2(gw, ww), rel_l2(gb, wb)))
    return out


def test_param_layout_and_init(M):
    assert M.param_count() == omlp.param_count()
    P = M.Params(seed=7)
    torch.cuda.synchronize()
    got = np_(P.p).astype(np.float64)
    want = omlp.init(7)
    assert np.max(np.abs(got - want)) < 1e-7
    # the BF16 copy is the round-to-nearest-even of every entry
    wq = np_(P.wq.view(torch.bfloat16).float()).astype(np.float64)
    np.testing.assert_array_equal(wq, omlp.bf16(got))


@pytest.mark.parametrize("rows", [1, 100, 1000])
def test_forward_matches_oracle(M, rows):
    P, flat = _params(M, 3)
    x = inputs.mlp_rows(rows, 4)
    ws = M.Workspace(rows)
    y = torch.empty((rows, 128), dtype=torch.float32, device="cuda")
    M.forward(P, torch.from_numpy(x).cuda(), y, ws)
    torch.cuda.synchronize()
    got = np_(y).astype(np.float64)
    want, _ = omlp.forward(flat, x, emulate_bf16=True)
    # the FP32 dot products (K = 256) carry ~1e-6 relative error, so about one activation
    # in a few thousand rounds to the other BF16 neighbour than the FP64 value does and
    # moves by 2^-8 of itself: ~1e-4 relative L2 at the output (7.6e-5 measured)
    r = rel_l2(got, want)
    assert r < 3e-4
    # an activation that rounds to the other BF16 neighbour (its FP32 value within
    # FP32 rounding of a BF16 tie) moves by 2^-8 of itself, and an output by about
    # |W| 2^-8 |a|: a few 1e-3 of the output rms at the worst element
    rms = math.sqrt(float(np.mean(want ** 2)))
    m = float(np.abs(got - want).max()) / rms
    assert m < 1e-2
    exact, _ = omlp.forward(flat, x)
    e = rel_l2(got, exact)
    print(f"\nforward, {rows} rows: relative L2 {r:.2e} (max {m:.2e} rms) against the emulated oracle, "
          f"{e:.2e} against the FP64 network (BF16 storage)")
    assert e < 3e-2


@pytest.mark.parametrize("rows", [64, 333])
def test_backward_matches_oracle(M, rows):
    P, flat = _params(M, 5)
    x = inputs.mlp_rows(rows, 6)
    dy = np.random.default_rng(7).standard_normal((rows, 128)).astype(np.float32) / rows
    ws = M.Workspace(rows)
    y = torch.empty((rows, 128), dtype=torch.float32, device="cuda")
    xd = torch.from_numpy(x).cuda()
    M.forward(P, xd, y, ws)
    dx = torch.empty((rows, 8), dtype=torch.float32, device="cuda")
    M.backward(P, torch.from_numpy(dy).cuda(), ws, P.grad, dx)
    torch.cuda.synchronize()
    _, cache = omlp.forward(flat, x, emulate_bf16=True)
    gw, gx = omlp.backward(flat, cache, dy, emulate_bf16=True)
    got = np_(P.grad).astype(np.float64)
    for l, (ew, eb) in enumerate(_layer_errors(got, gw)):
        assert ew < 1e-3 and eb < 1e-3, (l, ew, eb)
    assert rel_l2(np_(dx).astype(np.float64), gx) < 1e-3
    # the first layer's padding columns get exactly zero gradient
    W1 = omlp.unpack(got)[0][0]
    assert np.all(W1[:, 8:] == 0.0)
    # input gradients alone (inverse design) give the same dx
    dx2 = torch.empty_like(dx)
    M.backward(P, torch.from_numpy(dy).cuda(), ws, None, dx2)
    torch.cuda.synchronize()
    assert torch.equal(dx, dx2)
    _, c64 = omlp.forward(flat, x)
    g64, x64 = omlp.backward(flat, c64, dy)
    errs = _layer_errors(got, g64)
    worst = max(max(a, b) for a, b in errs)
    print(f"\nbackward, {rows} rows: worst per-tensor relative L2 against the FP64 network {worst:.2e}, "
          f"dx {rel_l2(np_(dx).astype(np.float64), x64):.2e} (BF16 storage)")
    assert worst < 3e-2


def test_adam_matches_oracle(M):
    n = M.param_count()
    r = np.random.default_rng(8)
    p0 = r.uniform(-1, 1, n).astype(np.float32)
    g1 = r.standard_normal(n).astype(np.float32)
    g2 = r.standard_normal(n).astype(np.float32)
    p = torch.from_numpy(p0).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    wq = torch.empty(n, dtype=torch.int16, device="cuda")
    for step, g in ((1, g1), (2, g2)):
        M.adam_raw(p, m, v, torch.from_numpy(g).cuda(), wq, step, 1e-3, wd=0.01)
    torch.cuda.synchronize()
    want, wm, wv = omlp.adam(p0.astype(np.float64), np.zeros(n), np.zeros(n), g1.astype(np.float64), 1, 1e-3,
                             wd=0.01)
    want, wm, wv = omlp.adam(want, wm, wv, g2.astype(np.float64), 2, 1e-3, wd=0.01)
    assert np.max(np.abs(np_(p) - want)) < 1e-6
    np.testing.assert_array_equal(np_(wq.view(torch.bfloat16).float()).astype(np.float64),
                                  omlp.bf16(np_(p).astype(np.float64)))


def test_losses_match_oracle(M):
    rows = 77
    r = np.random.default_rng(9)
    yh = r.standard_normal((rows, 128)).astype(np.float32)
    S = r.exponential(1.5, (rows, 128)).astype(np.float32)
    mu = r.uniform(-1, 1, 128).astype(np.float32)
    sg = r.uniform(0.5, 2, 128).astype(np.float32)
    c = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    dy = torch.empty((rows, 128), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    M.deviance(c(yh), c(S), c(mu), c(sg), dy, loss)
    torch.cuda.synchronize()
    wl, wg = omlp.deviance(yh.astype(np.float64), S.astype(np.float64), mu.astype(np.float64), sg.astype(np.float64))
    assert abs(float(loss.item()) / (rows * 128) - wl) < 1e-5 * abs(wl)
    assert rel_l2(np_(dy).astype(np.float64), wg) < 1e-5
    T = r.uniform(0.2, 5.0, (rows, 128)).astype(np.float32)
    lr = torch.empty(rows, device="cuda")
    M.design_loss(c(yh * 0.3), c(T), c(mu), c(sg), 0.01, dy, lr)
    torch.cuda.synchronize()
    wl, wg = omlp.design_loss(0.3 * yh.astype(np.float64), T.astype(np.float64), mu.astype(np.float64),
                              sg.astype(np.float64), lam=0.01)
    assert rel_l2(np_(lr).astype(np.float64), wl) < 1e-5
    assert rel_l2(np_(dy).astype(np.float64), wg) < 1e-5


def test_encode_decode_labels_match_oracle(M):
    th = inputs.surrogate_thetas(500, 10)
    x = torch.empty((500, 8), device="cuda")
    M.encode(torch.from_numpy(th).cuda(), x)
    back = torch.empty_like(x)
    M.decode(x, back)
    torch.cuda.synchronize()
    assert np.max(np.abs(np_(x) - omlp.encode(th))) < 2e-6
    # FP32 round trip: within a few units in the last place of each parameter's range
    assert np.max(np.abs(np_(back) - th) / np.maximum(np.abs(th), 1.0)) < 2e-6
    r = np.random.default_rng(11)
    sums = r.exponential(3.0, 40 * 128)
    counts = r.integers(0, 20, 40 * 128)
    S = torch.empty((40, 128), device="cuda")
    M.labels(torch.from_numpy(sums).cuda(), torch.from_numpy(counts).cuda(), S)
    mu = torch.empty(128, device="cuda")
    sg = torch.empty(128, device="cuda")
    M.label_stats(S, mu, sg)
    torch.cuda.synchronize()
    want_S = omlp.labels(sums, counts)
    assert np.max(np.abs(np_(S) - want_S) / np.maximum(want_S, 1e-30)) < 1e-6
    wm, ws_ = omlp.label_stats(np_(S).astype(np.float64))
    assert np.max(np.abs(np_(mu) - wm)) < 1e-5 and np.max(np.abs(np_(sg) - ws_)) < 1e-5


def test_gather_draws_valid_rows(M):
    n, rows = 1000, 256
    xa = torch.from_numpy(inputs.mlp_rows(n, 12)).cuda()
    Sa = torch.arange(n * 128, dtype=torch.float32, device="cuda").view(n, 128)
    xo = torch.empty((rows, 8), device="cuda")
    So = torch.empty((rows, 128), device="cuda")
    M.gather(xa, Sa, 5, 17, xo, So)
    torch.cuda.synchronize()
    idx = (np_(So)[:, 0] / 128).astype(np.int64)
    assert np.all((idx >= 0) & (idx < n))
    np.testing.assert_array_equal(np_(So), np_(Sa)[idx])
    np.testing.assert_array_equal(np_(xo), np_(xa)[idx])
    assert len(set(idx.tolist())) > 200  # sampling with replacement from 1000
    xo2, So2 = torch.empty_like(xo), torch.empty_like(So)
    M.gather(xa, Sa, 5, 17, xo2, So2)
    M.gather(xa, Sa, 5, 18, xo, So)
    torch.cuda.synchronize()
    assert torch.equal(So2, Sa[torch.from_numpy(idx).cuda()]) and not torch.equal(So, So2)


def test_training_step_matches_oracle_and_learns(M):
    # one full step (forward, deviance, backward, Adam) against the oracle's,
    # then a short run on a smooth synthetic target lowers the loss
    rows = 128
    P, flat = _params(M, 13)
    r = np.random.default_rng(14)
    x = inputs.mlp_rows(rows, 15)
    mu = np.zeros(128, np.float32)
    sg = np.ones(128, np.float32)
    # target mean spectrum: a smooth function of the inputs, exponential samples around it
    b = np.arange(128) / 128.0
    mean = np.exp(0.5 * np.sin(3 * b[None, :] + x[:, :1] * 2) + 0.3 * x[:, 1:2])
    S = (mean * r.exponential(1.0, mean.shape)).astype(np.float32)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    xd, Sd, mud, sgd = c(x), c(S), c(mu), c(sg)
    ws = M.Workspace(rows)
    y = torch.empty((rows, 128), device="cuda")
    dy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    M.forward(P, xd, y, ws)
    M.deviance(y, Sd, mud, sgd, dy, loss)
    M.backward(P, dy, ws, P.grad, None)
    M.adam(P, 1e-3)
    torch.cuda.synchronize()
    yo, cache = omlp.forward(flat, x, emulate_bf16=True)
    _, go = omlp.deviance(yo, S.astype(np.float64), mu, sg)
    gw, _ = omlp.backward(flat, cache, go, emulate_bf16=True)
    po, _, _ = omlp.adam(flat, np.zeros_like(flat), np.zeros_like(flat), gw, 1, 1e-3)
    # Adam's first step moves every parameter by lr sign(g) (|g| >> eps): compare the moves
    moved = np_(P.p).astype(np.float64) - flat.astype(np.float32).astype(np.float64)
    agree = np.mean(np.sign(moved) == np.sign(po - flat))
    assert agree > 0.99, agree
    first = None
    for step in range(300):
        loss.zero_()
        M.forward(P, xd, y, ws)
        M.deviance(y, Sd, mud, sgd, dy, loss)
        M.backward(P, dy, ws, P.grad, None)
        M.adam(P, 2e-3)
        if step == 0:
            first = float(loss.item())
    torch.cuda.synchronize()
    last = float(loss.item())
    # the deviance's floor is sum(log S_mean + 1) per element; compare the excess
    floor = float(np.sum(np.log(mean) + 1.0))
    assert (last - floor) < 0.5 * (first - floor), (first, last, floor)


def test_train_step_is_the_explicit_step_and_replays_in_a_graph(M):
    # hufield_mlp_train_step (gather, forward, deviance, backward, scheduled Adam, counter
    # advance) against the same calls made one by one, and a CUDA graph of steps
    # against steps called directly: the graph replays bit for bit
    n, rows, total = 3000, 256, 40
    r = np.random.default_rng(21)
    xa = torch.from_numpy(inputs.mlp_rows(n, 22)).cuda()
    Sa = torch.from_numpy(r.exponential(1.0, (n, 128)).astype(np.float32)).cuda()
    mu = torch.zeros(128, device="cuda")
    sg = torch.ones(128, device="cuda")
    flat = torch.from_numpy(inputs.mlp_params(23)).cuda()
    A, B, C = M.Params(0), M.Params(0), M.Params(0)
    for P in (A, B, C):
        P.load(flat)
    lr, lo = 1e-3, 0.1
    tr = M.Trainer(A, xa, Sa, mu, sg, rows, total, lr, seed=9, lr_min_frac=lo)
    tr.reset(0)
    tr.step()
    # the same step by hand: the learning rate at step 0 is lr, Adam's t is 1
    xb = torch.empty((rows, 8), device="cuda")
    Sb = torch.empty((rows, 128), device="cuda")
    y = torch.empty((rows, 128), device="cuda")
    dy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = M.Workspace(rows)
    M.gather(xa, Sa, 9, 0, xb, Sb)
    M.forward(B, xb, y, ws)
    M.deviance(y, Sb, mu, sg, dy, loss)
    M.backward(B, dy, ws, B.grad, None)
    M.adam(B, lr)
    torch.cuda.synchronize()
    assert torch.equal(A.grad, B.grad)
    assert float((A.p - B.p).abs().max()) < 1e-6 * max(1.0, float(B.p.abs().max()))
    assert abs(float(tr.loss.item()) - float(loss.item())) < 1e-9 * abs(float(loss.item()))
    # ten more steps directly, against a graph of ten steps replayed once on a twin
    trC = M.Trainer(C, xa, Sa, mu, sg, rows, total, lr, seed=9, lr_min_frac=lo)
    trC.reset(0)
    trC.step()
    for _ in range(10):
        tr.step()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(10):
            trC.step()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(A.p, C.p) and torch.equal(A.m, C.m) and torch.equal(A.v, C.v)
    assert torch.equal(A.wq, C.wq)
