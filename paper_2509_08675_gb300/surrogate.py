"""The surrogate workflow: data from the plain generator, training, inverse
design, and the plain generator's verdict on every design.

The paper's closing section (Sec. IV) names optimisation loops over the
generator's parameters as future work.  The plain generator cannot say what
spectrum a parameter set gives the thresholded +-1 map without making fields;
a small network that has seen many such fields can, and its input gradient
turns the question around: which parameters give a target two-phase spectrum.
The plain generator stays the judge: every design is re-made by it and its
binned spectrum compared with the target.

Workload (2D 256^2, 128 radial bins of the map's S(k)):
- parameters theta = (p, r1, r2, rot, k0, width, s, t) drawn uniformly over
  p in [1, 8], semi-axes (r1, r2) in [0.5, 2], rot in [0, pi), k0 in
  [0.05, 0.4], width in [0.01, 0.1], s in {2, 4, 6}, level t in [-1, 1];
- a training field is one realisation (seed, field index) of theta through the
  whole plain path; its label is the map's 128 bin means;
- a target is the 64-field mean spectrum of held-out parameters; a design is
  confirmed when the 64-field mean spectrum the plain generator makes from it
  is within 5% of the target in relative L2 over the bins 1..127 (bin 0 holds
  the map's squared mean, a point mass rather than spectral density).

Every step runs in the library's kernels (include/hufield.h for the fields,
include/hufield_surrogate.h for the network); this module is the host-side
driver loop: it draws parameters, orders the calls and keeps the books.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import hufield as hf
from . import mlp

SHAPE = (256, 256)
NR = 128
N = SHAPE[0] * SHAPE[1]
CONFIRM = 0.05
VERIFY_SEEDS = 64
S_CHOICES = (2.0, 4.0, 6.0)


def draw_thetas(n: int, seed: int) -> np.ndarray:
    """n parameter sets from a host Philox stream (numpy), float32 [n, 8]."""
    rng = np.random.Generator(np.random.Philox(seed))
    t = np.empty((n, 8))
    t[:, 0] = rng.uniform(1.0, 8.0, n)
    t[:, 1] = rng.uniform(0.5, 2.0, n)
    t[:, 2] = rng.uniform(0.5, 2.0, n)
    t[:, 3] = rng.uniform(0.0, math.pi, n)
    t[:, 4] = rng.uniform(0.05, 0.4, n)
    t[:, 5] = rng.uniform(0.01, 0.1, n)
    t[:, 6] = rng.choice(np.array(S_CHOICES), n)
    t[:, 7] = rng.uniform(-1.0, 1.0, n)
    return t.astype(np.float32)


def theta_filter(th) -> hf.Filter:
    """The generator's filter for one parameter row (2D semi-axes (r1, r2))."""
    return hf.Filter(p=float(th[0]), axes=(float(th[1]), float(th[2])), rot=float(th[3]), k0=float(th[4]),
                     width=float(th[5]), supp=float(th[6]))


class Timer:
    """Device time of a phase: CUDA events on the working stream around it (the
    phase's elapsed GPU time, idle gaps between its launches included)."""

    def __init__(self, stream=None):
        self.stream = stream or torch.cuda.current_stream()
        self.ms = 0.0
        self.wall = 0.0

    def __enter__(self):
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)
        self.e0.record(self.stream)
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *exc):
        self.e1.record(self.stream)
        self.e1.synchronize()
        self.ms += self.e0.elapsed_time(self.e1)
        self.wall += time.perf_counter() - self.t0
        return False


@dataclass
class DataSet:
    theta: np.ndarray
    x: torch.Tensor        # [n, 8] encoded
    S: torch.Tensor        # [n, 128] bin means of one map each
    gpu_s: float = 0.0
    wall_s: float = 0.0


def generate_dataset(thetas: np.ndarray, seed: int, field0: int = 0, chunk: int = 20000, lanes: int = 2) -> DataSet:
    """One plain-generator field per parameter row (field index field0 + i): the
    map's 128 radial bin means as labels.  Runs as ragged batches of `chunk`
    items (one CUDA graph launch each); the batch runs its items a chunk of
    fields at a time through the batched passes, on `lanes` lanes."""
    n = len(thetas)
    S = torch.empty((n, NR), dtype=torch.float32, device="cuda")
    x = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    th_dev = torch.from_numpy(np.ascontiguousarray(thetas)).cuda()
    gpu_ms, wall = 0.0, 0.0
    bins = None
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        items = [(SHAPE, theta_filter(thetas[i]), seed, field0 + i, float(thetas[i][7]), NR) for i in range(c0, c1)]
        batch = hf.Batch(items, lanes=lanes)
        nb = batch.total_bins
        if bins is None or bins[0].numel() < nb:
            bins = (torch.empty(nb, dtype=torch.float64, device="cuda"),
                    torch.empty(nb, dtype=torch.int64, device="cuda"),
                    torch.empty(nb, dtype=torch.float64, device="cuda"),
                    torch.empty(nb, dtype=torch.int64, device="cuda"))
            ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
        if ws.numel() < batch.ws_bytes:
            ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
        sf, cf, sm, cm = (b[:nb] for b in bins)
        with Timer() as t:
            hf.hufield_batch_run(batch, None, None, sf, cf, sm, cm, ws)
            mlp.labels(sm, cm, S[c0:c1])
        gpu_ms += t.ms
        wall += t.wall
        batch.close()
    with Timer() as t:
        mlp.encode(th_dev, x)
    return DataSet(thetas, x, S, (gpu_ms + t.ms) / 1e3, wall + t.wall)


def plain_spectra(thetas: np.ndarray, seed: int, nseeds: int = VERIFY_SEEDS, field0: int = 0,
                  timer: "Timer | None" = None) -> torch.Tensor:
    """Mean map spectrum of nseeds plain-generator fields per parameter row
    (fields field0 .. field0 + nseeds - 1 of `seed`), [n, 128] on the device: one
    ragged batch of n x nseeds items (the fields of a row consecutive), run in
    batched chunks, and the group means of their bins.  `timer` (if given)
    brackets the device work only; the batch's planning is host work."""
    n = len(thetas)
    items = [(SHAPE, theta_filter(thetas[i]), seed, field0 + k, float(thetas[i][7]), NR)
             for i in range(n) for k in range(nseeds)]
    batch = hf.Batch(items)
    out = torch.empty((n, NR), dtype=torch.float32, device="cuda")
    nb = batch.total_bins
    bins = [torch.empty(nb, dtype=dt, device="cuda") for dt in (torch.float64, torch.int64, torch.float64, torch.int64)]
    ws = torch.empty(batch.ws_bytes, dtype=torch.uint8, device="cuda")
    with (timer if timer is not None else _NoTimer()):
        hf.hufield_batch_run(batch, None, None, *bins, ws)
        hf.hufield_bins_group_mean(bins[2], bins[3], n, nseeds, NR, out)
    torch.cuda.current_stream().synchronize()
    batch.close()
    return out


class _NoTimer:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class Evaluator:
    """The plain generator as a search evaluates it: the mean map spectrum of
    nseeds fields (common random numbers: the same fields every time) of one
    parameter row, through an updatable batch whose graph is captured once."""

    def __init__(self, seed: int, nseeds: int, field0: int = 1000):
        self.seed, self.nseeds, self.field0 = seed, nseeds, field0
        self.batch = hf.Batch(self._items(draw_thetas(1, 0)[0]), updatable=True)
        nb = self.batch.total_bins
        self.bins = [torch.empty(nb, dtype=dt, device="cuda")
                     for dt in (torch.float64, torch.int64, torch.float64, torch.int64)]
        self.ws = torch.empty(self.batch.ws_bytes, dtype=torch.uint8, device="cuda")
        self.out = torch.empty((1, NR), dtype=torch.float32, device="cuda")
        self.timer = Timer()  # device time of the evaluations' runs
        self.calls = 0

    def _items(self, th):
        f = theta_filter(th)
        return [(SHAPE, f, self.seed, self.field0 + k, float(th[7]), NR) for k in range(self.nseeds)]

    def __call__(self, th) -> torch.Tensor:
        self.batch.set_params(self._items(th))
        with self.timer:
            hf.hufield_batch_run(self.batch, None, None, *self.bins, self.ws)
            hf.hufield_bins_group_mean(self.bins[2], self.bins[3], 1, self.nseeds, NR, self.out)
        self.calls += 1
        return self.out

    def close(self):
        self.batch.close()


def rel_err(S: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Relative L2 error over the bins 1..127, per row."""
    S = np.asarray(S, np.float64).reshape(-1, NR)[:, 1:]
    T = np.asarray(T, np.float64).reshape(-1, NR)[:, 1:]
    return np.linalg.norm(S - T, axis=1) / np.linalg.norm(T, axis=1)


@dataclass
class TrainLog:
    steps: int = 0
    losses: list = field(default_factory=list)
    gpu_s: float = 0.0
    wall_s: float = 0.0


class Surrogate:
    """The network, its label standardisation and the inverse-design loop."""

    def __init__(self, seed: int = 0):
        self.P = mlp.Params(seed)
        self.mu = torch.zeros(NR, dtype=torch.float32, device="cuda")
        self.sigma = torch.ones(NR, dtype=torch.float32, device="cuda")

    def fit_stats(self, data: DataSet, rows: int):
        mlp.label_stats(data.S[:rows], self.mu, self.sigma)

    def train(self, data: DataSet, n_train: int, steps: int, batch: int = 1024, lr: float = 2e-3, seed: int = 1,
              wd: float = 1e-5, log_every: int = 500, graph_steps: int = 50) -> TrainLog:
        """Adam on minibatches drawn with replacement from the first n_train rows;
        the learning rate decays as a half cosine to 2% of lr.  Whole steps
        (hufield_mlp_train_step) are captured `graph_steps` at a time into one
        CUDA graph and replayed; the schedule advances on the device."""
        log = TrainLog()
        tr = mlp.Trainer(self.P, data.x[:n_train], data.S[:n_train], self.mu, self.sigma, batch, steps, lr, seed,
                         wd=wd)
        tr.reset(0)
        graph = None
        if graph_steps > 1 and steps >= graph_steps:
            # the capture runs on a side stream; the captured steps do not execute
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                for _ in range(graph_steps):
                    tr.step()
            torch.cuda.current_stream().wait_stream(s)
        done, since = 0, 0
        with Timer() as t:
            while done < steps:
                if graph is not None and steps - done >= graph_steps:
                    graph.replay()
                    done += graph_steps
                    since += graph_steps
                else:
                    tr.step()
                    done += 1
                    since += 1
                if log_every and since >= log_every:
                    log.losses.append(float(tr.loss.item()) / (since * batch * NR))
                    tr.loss.zero_()
                    since = 0
        log.steps = steps
        log.gpu_s = t.ms / 1e3
        log.wall_s = t.wall
        return log

    def predict(self, x: torch.Tensor) -> torch.Tensor:
        """Predicted mean spectrum e^{mu + sigma y_hat}, [rows, 128]."""
        rows = x.shape[0]
        y = torch.empty((rows, NR), dtype=torch.float32, device="cuda")
        mlp.forward(self.P, x, y, mlp.Workspace(rows))
        S = torch.empty_like(y)
        mlp.spectrum(y, self.mu, self.sigma, S)
        return S

    def design(self, T: torch.Tensor, starts: int = 4, iters: int = 300, lr: float = 0.05, lam: float = 0.01,
               seed: int = 2):
        """Gradient descent on the network's input for each target row of T [n, 128]:
        for every s in {2, 4, 6}, `starts` random starting points (s held fixed,
        the other seven parameters on their ranges).  Returns the decoded
        parameters of each row's best start by the surrogate's loss [n, 8]
        (numpy), that loss, and the device time."""
        n = T.shape[0]
        k = len(S_CHOICES) * starts
        rows = n * k
        rng = np.random.Generator(np.random.Philox(seed))
        x0 = rng.uniform(-1.0, 1.0, (rows, 8)).astype(np.float32)
        x0[:, 6] = np.tile(np.repeat((np.array(S_CHOICES) - 4.0) / 2.0, starts), n)
        x = torch.from_numpy(x0).cuda()
        m = torch.zeros_like(x)
        v = torch.zeros_like(x)
        Tr = T.repeat_interleave(k, dim=0).contiguous()
        y = torch.empty((rows, NR), dtype=torch.float32, device="cuda")
        dy = torch.empty_like(y)
        dx = torch.empty_like(x)
        lossr = torch.empty(rows, dtype=torch.float32, device="cuda")
        ws = mlp.Workspace(rows)
        with Timer() as t:
            for it in range(iters):
                mlp.forward(self.P, x, y, ws)
                mlp.design_loss(y, Tr, self.mu, self.sigma, lam, dy, lossr)
                mlp.backward(self.P, dy, ws, None, dx)
                mlp.design_step(x, m, v, dx, 1 << 6, it + 1, lr)
            mlp.forward(self.P, x, y, ws)
            mlp.design_loss(y, Tr, self.mu, self.sigma, lam, dy, lossr)
            theta = torch.empty_like(x)
            mlp.decode(x, theta)
        L = lossr.view(n, k).cpu().numpy()
        best = L.argmin(axis=1)
        th = theta.view(n, k, 8).cpu().numpy()
        order = np.argsort(L, axis=1)
        return th[np.arange(n), best], L[np.arange(n), best], t.ms / 1e3, th, order


def nelder_mead_search(target: np.ndarray, seed: int, nseeds: int = 16, budget: int = 400, tol: float = CONFIRM,
                       rng_seed: int = 0, evaluator: "Evaluator | None" = None):
    """The plain generator alone: Nelder-Mead over the seven continuous encoded
    parameters (s tried as each of 2, 4, 6 on a sample, the best kept) on the
    relative error of the nseeds-field mean spectrum against the target, from
    the best of a 12-point random sample; stops at `tol` or after `budget`
    evaluations.  Each evaluation is one run of an updatable batch of nseeds
    fields (Evaluator).  Returns (theta, error, evaluations)."""
    rng = np.random.Generator(np.random.Philox(rng_seed))
    evals = [0]
    Tn = np.asarray(target, np.float64)
    ev = evaluator or Evaluator(seed, nseeds)

    def f(xv, s):
        xv = np.clip(xv, -1.0, 1.0)
        th = _decode_host(np.concatenate([xv[:6], [(s - 4.0) / 2.0], xv[6:7]]))
        # common random numbers: every evaluation uses the same nseeds fields
        S = ev(th)
        evals[0] += 1
        return float(rel_err(S.cpu().numpy(), Tn)[0]), th

    best = (np.inf, None, None, None)
    for s in S_CHOICES:
        for _ in range(4):
            xv = rng.uniform(-1.0, 1.0, 7)
            e, th = f(xv, s)
            if e < best[0]:
                best = (e, th, xv, s)
    e0, th0, xv, s = best
    if e0 <= tol:
        return th0, e0, evals[0]
    # simplex around the best sample point
    simplex = [xv] + [np.clip(xv + 0.25 * np.eye(7)[i] * (1 if xv[i] < 0 else -1), -1, 1) for i in range(7)]
    vals = [e0] + [f(p, s)[0] for p in simplex[1:]]
    while evals[0] < budget:
        order = np.argsort(vals)
        simplex = [simplex[i] for i in order]
        vals = [vals[i] for i in order]
        if vals[0] <= tol:
            break
        c = np.mean(simplex[:-1], axis=0)
        xr = c + (c - simplex[-1])
        fr = f(xr, s)[0]
        if fr < vals[0]:
            xe = c + 2.0 * (c - simplex[-1])
            fe = f(xe, s)[0]
            simplex[-1], vals[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < vals[-2]:
            simplex[-1], vals[-1] = xr, fr
        else:
            xc = c + 0.5 * (simplex[-1] - c)
            fc = f(xc, s)[0]
            if fc < vals[-1]:
                simplex[-1], vals[-1] = xc, fc
            else:
                for i in range(1, len(simplex)):
                    simplex[i] = simplex[0] + 0.5 * (simplex[i] - simplex[0])
                    vals[i] = f(simplex[i], s)[0]
    i = int(np.argmin(vals))
    xb = np.clip(simplex[i], -1, 1)
    th = _decode_host(np.concatenate([xb[:6], [(s - 4.0) / 2.0], xb[6:7]]))
    return th, float(vals[i]), evals[0]


def _decode_host(xv: np.ndarray) -> np.ndarray:
    """Decode one encoded row through the library's kernel."""
    x = torch.from_numpy(np.asarray(xv, np.float32).reshape(1, 8)).cuda()
    th = torch.empty_like(x)
    mlp.decode(x, th)
    return th.cpu().numpy()[0]
