"""Learned surrogate of the adhesion observables (N_L, delta p, r) over the
particle / cell parameter space of Sec. 3.1, trained on trajectories the
solver itself generates, with the solver as fallback outside the training hull.

Pieces (all numerical work in the library's kernels; this module only lays
out inputs and drives the C ABI):
  * the parameter space and its sampling (``Point``, ``sample_points``), and
    bond-seed replicates of each point (``replicate``, ``seed_statistics``):
    N_L counts stochastic bond events, so a point's trajectories differ from
    seed to seed; the network is trained on replicate means, and that
    seed-to-seed spread is the noise floor its N_L error is judged against;
  * the capillary each point runs in (``capillary_for``);
  * trajectory generation with batched solver contexts (``generate``);
  * training of ``lbib.Mlp`` on the trajectories (``train``), on one GPU or
    data-parallel over several (``data_parallel_step``: shard gradients summed
    by an all-reduce);
  * ``Surrogate.predict``: the network inside the hull, the solver outside.

Training geometry (a reading; the paper's Table 1 is missing): H = 40 nodes,
160 nodes long, tau = 1, Re = 0.05 (Stokes regime, u_max = 2.08e-4), cell
(7 um, 96 markers) released 40 nodes from the inlet, particle (2 um long,
32 markers) at 75 nodes on the lower wall, 3e5 steps (t u_max / H = 1.56),
observables sampled 512 times; bond stiffness and rates scaled by Re / 0.01
(Stokes scaling of the paper's Re = 1e-2).  The particle's capillary number spans
log10 Ca in [-4, -3] (stiffer membranes exceed the explicit membrane update's
stability limit at this step; they are outside the hull) or rigid.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List, Optional, Sequence

import numpy as np

from . import lbib
from . import workloads as wl

NY, NX = 40, 160
RE = 0.05
RE_PAPER = 0.01  # Sec. 3.1; bond stiffness and rates scale with RE / RE_PAPER (Stokes scaling)
CELL_X, PARTICLE_X = 40.0, 75.0
CELL_MARKERS, PARTICLE_MARKERS = 96, 32
STEPS, SAMPLES = 300000, 512
AR_RANGE = (0.25, 1.0)
LOGCA_RANGE = (-4.0, -3.0)
DENSITY_RANGE = (10.0, 50.0)  # ligand sites per um of particle perimeter
FEATURES = ("aspect_ratio", "log10_ca", "rigid", "globular", "biconcave", "ligand_density", "initial_bonds",
            "inverse_initial_bonds", "t_star")
OUTPUTS = ("n_l", "delta_p", "r")


@dataclasses.dataclass(frozen=True)
class Point:
    """One point of the parameter space."""
    aspect_ratio: float      # particle thickness / length
    log10_ca: float          # particle capillary number (ignored when rigid)
    rigid: bool
    cell: str                # "globular" | "biconcave"
    ligand_density: float    # sites per um of perimeter
    seed: int = 0            # Philox key of the bond kinetics


def sample_points(n: int, seed: int = 0, rigid_fraction: float = 0.2) -> List[Point]:
    """Stratified (Latin hypercube) samples of the continuous axes, rigid
    particles with probability rigid_fraction, both cell shapes alternating."""
    rng = np.random.default_rng(seed)

    def lhs(lo, hi):
        u = (rng.permutation(n) + rng.uniform(0, 1, n)) / n
        return lo + (hi - lo) * u

    ar, lc, dens = lhs(*AR_RANGE), lhs(*LOGCA_RANGE), lhs(*DENSITY_RANGE)
    rig = rng.uniform(0, 1, n) < rigid_fraction
    return [Point(float(ar[i]), float(lc[i]), bool(rig[i]), ("globular", "biconcave")[i % 2], float(dens[i]),
                  seed=int(seed * 100003 + i)) for i in range(n)]


def replicate(points: Sequence[Point], replicates: int) -> List[Point]:
    """Each point `replicates` times, consecutively, with bond seeds
    seed * replicates + j (j < replicates): the same capillary under
    independent Philox streams."""
    return [dataclasses.replace(p, seed=p.seed * replicates + j) for p in points for j in range(replicates)]


def seed_statistics(Y: np.ndarray, replicates: int):
    """Y [n * replicates, samples, 3], the replicates of a point consecutive
    (``replicate``).  Returns the replicate means [n, samples, 3] and, per
    output, the seed-to-seed spread: the root mean square over points and
    times of the sample standard deviation across replicates (the error floor
    of predicting one trajectory), and that divided by sqrt(replicates) (the
    floor of predicting a replicate mean, the uncertainty of the mean itself)."""
    if replicates < 2:
        raise ValueError("the spread needs at least two replicates")
    Yr = Y.reshape(-1, replicates, *Y.shape[1:])
    sd = np.sqrt(np.mean(Yr.var(1, ddof=1), axis=(0, 1)))
    return Yr.mean(1), sd, sd / math.sqrt(replicates)


_POLY = {}  # aspect-ratio nodes and the particle polygons (relative to the centre) at them


def _particle_polygon(ar: np.ndarray) -> np.ndarray:
    """The training particle's marker polygon relative to its centre
    [len(ar), PARTICLE_MARKERS, 2] for aspect ratios inside AR_RANGE: a cubic
    spline in the aspect ratio through the exact polygons (``wl.ellipse``,
    equal arc spacing from 20000 samples) at 193 nodes; the vertices agree with
    the exact construction to about 1e-9 dx."""
    from scipy.interpolate import CubicSpline

    if "spline" not in _POLY:
        a = 0.5 * wl.PARTICLE_LENGTH_UM / (wl.H_UM / NY)
        nodes = np.linspace(AR_RANGE[0], AR_RANGE[1], 193)
        tab = np.stack([wl.ellipse(PARTICLE_MARKERS, 0.0, 0.0, a, r * a) for r in nodes])
        _POLY["spline"] = CubicSpline(nodes, tab, axis=0)
    return _POLY["spline"](ar)


def initial_bonds(points: Sequence[Point]) -> np.ndarray:
    """N_L's normalisation N0 for each point's training capillary: the number of
    ligand sites bonded at t = 0 under the library's rule (include/lbib.h,
    ``lbib_adhesion_params``): n_ligands sites at arc lengths (k + 1/2) P / n
    along the particle's chain (P its polygon perimeter), a site bonded when
    its gap to the nearer wall is below y_cr; n_ligands and y_cr as
    ``capillary_for`` sets them.  N0 is a step function of the aspect ratio
    and the ligand density (whole sites cross the y_cr line), which a smooth
    network fits badly; as an input it lets the network predict N_L = N / N0
    without learning the steps."""
    dx = wl.H_UM / NY
    a = 0.5 * wl.PARTICLE_LENGTH_UM / dx
    y_cr = wl.Y_CR_UM / dx
    ar = np.array([p.aspect_ratio for p in points], np.float64)
    inside = (ar >= AR_RANGE[0]) & (ar <= AR_RANGE[1])
    polys = np.zeros((len(points), PARTICLE_MARKERS, 2))
    if inside.any():
        polys[inside] = _particle_polygon(ar[inside])
    for i in np.flatnonzero(~inside):  # outside the table: the exact construction
        polys[i] = wl.ellipse(PARTICLE_MARKERS, 0.0, 0.0, a, ar[i] * a)
    y = polys[:, :, 1] + (wl.PARTICLE_GAP_UM / dx + ar * a)[:, None]  # centre height as capillary_for places it
    seg = np.hypot(*(np.roll(polys, -1, 1) - polys).transpose(2, 0, 1))
    cum = np.concatenate([np.zeros((len(points), 1)), np.cumsum(seg, 1)], 1)  # [P, markers + 1]
    dens = np.array([p.ligand_density for p in points], np.float64)
    P = cum[:, -1]
    n = np.maximum(4, np.rint(dens * P * dx)).astype(np.int64)
    # Vertex 0 is the lowest point of the convex chain, so y rises from it to the top
    # and falls back: only sites before the first vertex at or above y_cr (arc jf) or
    # after the last one (arc jb) can be bonded.  Those candidates (with one site of
    # margin on each side) go through the same position formula as every site.
    high = y >= y_cr
    jf = np.argmax(high[:, 1:], 1) + 1
    jb = PARTICLE_MARKERS - 1 - np.argmax(high[:, ::-1], 1)
    rows = np.arange(len(points))
    kf = np.minimum(n, np.floor(cum[rows, jf] * n / P + 0.5).astype(np.int64) + 1)
    kb = np.maximum(kf, np.floor(cum[rows, jb] * n / P - 0.5).astype(np.int64))
    width = int(max(kf.max(initial=0), (n - kb).max(initial=0)))
    j = np.arange(width)[None, :]
    k = np.concatenate([np.broadcast_to(j, (len(points), width)), kb[:, None] + j], 1)  # forward, backward
    valid = np.concatenate([j < kf[:, None], kb[:, None] + j < n[:, None]], 1)
    k = np.where(valid, k, 0)
    sk = (k + 0.5) * (P / n)[:, None]
    # segment of each site: the first l with s <= cum[l + 1], at most markers - 1
    l = np.minimum(np.sum(cum[:, None, 1:] < sk[:, :, None], -1), PARTICLE_MARKERS - 1)
    c0 = np.take_along_axis(cum, l, 1)
    c1 = np.take_along_axis(cum, l + 1, 1)
    t = np.clip((sk - c0) / (c1 - c0), 0.0, 1.0)
    y0 = np.take_along_axis(y, l, 1)
    y1 = np.take_along_axis(y, (l + 1) % PARTICLE_MARKERS, 1)
    py = y0 + t * (y1 - y0)
    return np.count_nonzero(valid & (np.minimum(py, NY - py) < y_cr), 1).astype(np.int64)


def features_many(points: Sequence[Point], t_star) -> np.ndarray:
    """Feature rows [len(points) * len(t_star), len(FEATURES)], point-major."""
    t = np.atleast_1d(np.asarray(t_star, np.float64))
    n0 = initial_bonds(points).astype(np.float64)
    rows = np.array([[p.aspect_ratio, LOGCA_RANGE[0] if p.rigid else p.log10_ca, float(p.rigid),
                      float(p.cell == "globular"), float(p.cell == "biconcave"), p.ligand_density]
                     for p in points], np.float64).reshape(len(points), 6)
    rows = np.concatenate([rows, n0[:, None], 1.0 / np.maximum(n0, 1.0)[:, None]], 1)
    X = np.concatenate([np.repeat(rows, t.size, 0), np.tile(t, len(points))[:, None]], 1)
    return X.astype(np.float32)


def features(p: Point, t_star) -> np.ndarray:
    """Feature rows [len(t_star), len(FEATURES)] for point p at the given times."""
    return features_many([p], t_star)


def in_hull(p: Point, t_star_max: float) -> bool:
    """Inside the box the training set covers (per axis; categories always)."""
    ok = AR_RANGE[0] <= p.aspect_ratio <= AR_RANGE[1] and DENSITY_RANGE[0] <= p.ligand_density <= DENSITY_RANGE[1]
    if not p.rigid:
        ok = ok and LOGCA_RANGE[0] <= p.log10_ca <= LOGCA_RANGE[1]
    return ok and t_star_max <= STEPS * u_max() / NY + 1e-12


def u_max(re: float = RE) -> float:
    nu = (1.0 - 0.5) / 3.0
    return re * nu / NY


def capillary_for(p: Point, re: float = RE) -> wl.Capillary:
    """The training capillary of point p (geometry in the module docstring)."""
    dx = wl.H_UM / NY
    if p.cell == "globular":
        c = wl.circle(CELL_MARKERS, CELL_X, 0.5 * NY, wl.CELL_RADIUS_UM / dx)
        body_c = wl.Body(wl.CELL, wl.DEFORMABLE, c, ca=1e-3, beta=0.0)
    else:
        c = wl.biconcave(CELL_MARKERS, CELL_X, 0.5 * NY, wl.CELL_RADIUS_UM / dx)
        body_c = wl.Body(wl.CELL, wl.DEFORMABLE, c, ca=1e-3, beta=1e-2)
    a, b = 0.5 * wl.PARTICLE_LENGTH_UM / dx, 0.5 * p.aspect_ratio * wl.PARTICLE_LENGTH_UM / dx
    part = wl.ellipse(PARTICLE_MARKERS, PARTICLE_X, wl.PARTICLE_GAP_UM / dx + b, a, b)
    perim = float(np.sum(np.hypot(*(np.roll(part, -1, 0) - part).T))) * dx  # um
    y_cr = wl.Y_CR_UM / dx
    # sigma (units rho nu^2 / H) and the per-step rates scaled by Re / Re_paper: the
    # ratios sigma / (rho nu u_max) and k H / u_max stay those of the paper's flow
    f = re / RE_PAPER
    adh = wl.Adhesion(n_lig=max(4, int(round(p.ligand_density * perim))), sigma=1.0 * f, y_cr=y_cr, y_eq=0.5 * y_cr,
                      kf_dt=0.085 * f, kr0_dt=1e-5 * f, xi=1.0 / (0.5 * y_cr) ** 2)
    if p.rigid:
        body_p = wl.Body(wl.PARTICLE, wl.RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1, adhesion=adh)
    else:
        body_p = wl.Body(wl.PARTICLE, wl.DEFORMABLE, part, ca=10.0 ** p.log10_ca, beta=1e-2, density_ratio=1.1,
                         adhesion=adh)
    return wl.Capillary(f"surrogate capillary {p}", NX, NY, 1.0, re, STEPS, "fp32", p.seed, [body_c, body_p])


def generate(points: Sequence[Point], steps: int = STEPS, samples: int = SAMPLES, batch: int = 256, device: int = 0,
             stream: Optional[int] = None, log=None):
    """Runs every point's capillary for `steps` steps in batches of `batch`
    instances and samples the observables `samples` times (every
    steps / samples steps).  Returns t_star [samples], Y [len(points),
    samples, 3] (N_L, delta p, r) and the GPU seconds spent."""
    stride = max(1, steps // samples)
    out = np.zeros((len(points), samples, 3))
    t_star = np.zeros(samples)
    secs = 0.0
    for b0 in range(0, len(points), batch):
        chunk = points[b0:b0 + batch]
        caps = [capillary_for(p) for p in chunk]
        s = lbib.from_capillaries(caps, device=device, stream=stream, obs_capacity=max(64, 2 * stride))
        s.autotune(steps_per_trial=20)
        t0 = time.perf_counter()
        for k in range(samples):
            s.advance(stride)
            rec = s.latest_observables()
            for i, r in enumerate(rec):
                out[b0 + i, k] = (r["n_l"], r["delta_p"], r["r"])
            t_star[k] = rec[0]["t_star"]
        secs += time.perf_counter() - t0
        s.close()
        if log:
            log(f"generated {b0 + len(chunk)}/{len(points)} trajectories, {secs:.1f} s")
    return t_star, out, secs


@dataclasses.dataclass
class Trained:
    net: "lbib.Mlp"
    in_shift: np.ndarray
    in_scale: np.ndarray
    out_shift: np.ndarray
    out_scale: np.ndarray
    t_star_max: float
    losses: List[float]
    stream: object = None  # torch stream the network enqueues on
    seconds_per_step: float = float("nan")  # wall time per step after the first 100 (sampling included)


def normalisation(X: np.ndarray, Y: np.ndarray):
    """Affine maps to roughly unit scale: inputs to [-1, 1] by their range,
    outputs standardised."""
    lo, hi = X.min(0), X.max(0)
    span = np.where(hi > lo, hi - lo, 1.0)
    in_shift, in_scale = 0.5 * (lo + hi), 2.0 / span
    out_shift, out_scale = Y.mean(0), np.where(Y.std(0) > 0, Y.std(0), 1.0)
    return (in_shift.astype(np.float32), in_scale.astype(np.float32), out_shift.astype(np.float32),
            out_scale.astype(np.float32))


def _net_stream():
    """The torch stream the library's calls are enqueued on: the current one,
    or a new side stream when the current one is the legacy default stream
    (handle 0, which the library would replace by a private, unordered one)."""
    import torch

    st = torch.cuda.current_stream()
    return st if st.cuda_stream else torch.cuda.Stream()


def data_parallel_step(net, xb, yb, grad, loss, lr: float, rank: int = 0, world: int = 1, group=None) -> None:
    """One Adam step of ``net`` on the global batch (xb, yb), data-parallel over
    `world` ranks (include/lbib_mlp.h): rank r takes rows [r b, (r + 1) b) with
    b = len(xb) / world, computes its shard's gradient into ``grad`` (float32
    tensor of param_count values on the network's device) and its loss into
    ``loss``, the gradients are summed across ranks (all-reduce over `group`),
    and every rank applies 1 / world times the sum, so the copies stay equal.
    All tensors live on the stream the network enqueues on."""
    B = int(xb.shape[0])
    if B % world:
        raise ValueError("the global batch must split into equal shards")
    b = B // world
    xs = xb[rank * b:(rank + 1) * b].contiguous()
    ys = yb[rank * b:(rank + 1) * b].contiguous()
    net.backward(xs.data_ptr(), ys.data_ptr(), b, grad.data_ptr(), grad.numel(), loss.data_ptr())
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(grad, group=group)
    net.apply_gradient(grad.data_ptr(), grad.numel(), 1.0 / world, lr)


def train(X: np.ndarray, Y: np.ndarray, steps: int = 3000, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          device: int = 0, width: int = 256, n_hidden: int = 3, log=None, rank: int = 0, world: int = 1,
          group=None) -> Trained:
    """Adam on minibatches drawn from (X, Y) by the library's kernels;
    cosine decay of the step size.  With world > 1 (one process per GPU,
    torch.distributed initialised) every rank draws the same global batches
    (same seed) and trains on its shard of each (``data_parallel_step``); the
    networks start from the same seed and stay identical."""
    import torch

    torch.cuda.set_device(device)
    st = _net_stream()
    norm = normalisation(X, Y)
    with torch.cuda.stream(st):
        net = lbib.Mlp(X.shape[1], Y.shape[1], width=width, n_hidden=n_hidden, max_batch=max(batch, 65536),
                       device=device, stream=st.cuda_stream, seed=seed,
                       in_shift=norm[0], in_scale=norm[1], out_shift=norm[2], out_scale=norm[3])
        Xd = torch.as_tensor(X, dtype=torch.float32).cuda()
        Yd = torch.as_tensor(Y, dtype=torch.float32).cuda()
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        loss = torch.zeros(1, device="cuda")
        grad = torch.zeros(net.param_count(), device="cuda") if world > 1 else None
        losses = []
        t_warm, k_warm = None, None
        for k in range(steps):
            idx = torch.randint(0, X.shape[0], (batch,), device="cuda", generator=g)
            xb, yb = Xd[idx].contiguous(), Yd[idx].contiguous()
            eta = max(lr * 0.5 * (1.0 + math.cos(math.pi * k / steps)), lr * 1e-3)
            if world > 1:
                data_parallel_step(net, xb, yb, grad, loss, eta, rank, world, group)
            else:
                net.train_step(xb.data_ptr(), yb.data_ptr(), batch, eta, loss.data_ptr())
            if k % 100 == 0 or k == steps - 1:
                st.synchronize()
                losses.append(float(loss.item()))
                if k == min(100, steps - 1):  # first uses of every kernel are behind this point
                    t_warm, k_warm = time.perf_counter(), k
                if log:
                    log(f"step {k}: loss {losses[-1]:.4e}")
        st.synchronize()
        per_step = (time.perf_counter() - t_warm) / (steps - 1 - k_warm) if steps - 1 > k_warm else float("nan")
    return Trained(net, *norm, t_star_max=float(X[:, -1].max()), losses=losses, stream=st, seconds_per_step=per_step)


def predict_network(tr: Trained, X: np.ndarray) -> np.ndarray:
    """Network outputs for feature rows X (any count; batches of 65536)."""
    import torch

    out = np.zeros((X.shape[0], tr.net.n_out), np.float32)
    st = tr.stream if tr.stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(st):
        Xd = torch.as_tensor(X, dtype=torch.float32).cuda()
        Yd = torch.zeros(X.shape[0], tr.net.n_out, device="cuda")
        for b0 in range(0, X.shape[0], 65536):
            n = min(65536, X.shape[0] - b0)
            tr.net.forward(Xd[b0:].data_ptr(), n, Yd[b0:].data_ptr())
        st.synchronize()
        out[:] = Yd.cpu().numpy()
    return out


class Surrogate:
    """Predicts (N_L, delta p, r) at times t_star for parameter points: the
    trained network inside the hull of its training set, the solver outside
    (flagged)."""

    def __init__(self, trained: Trained, steps: int = STEPS):
        self.tr = trained
        self.steps = steps

    def predict(self, points: Sequence[Point], t_star: np.ndarray):
        t_star = np.asarray(t_star, np.float64)
        inside = [in_hull(p, float(t_star.max())) and float(t_star.max()) <= self.tr.t_star_max + 1e-9
                  for p in points]
        Y = np.zeros((len(points), t_star.size, 3))
        idx_in = [i for i, ok in enumerate(inside) if ok]
        if idx_in:
            X = features_many([points[i] for i in idx_in], t_star)
            Yn = predict_network(self.tr, X).reshape(len(idx_in), t_star.size, 3)
            for j, i in enumerate(idx_in):
                Y[i] = Yn[j]
        idx_out = [i for i, ok in enumerate(inside) if not ok]
        if idx_out:
            Y[idx_out] = solve(points=[points[i] for i in idx_out], t_star=t_star)
        return Y, np.asarray(inside)


def solve(points: Sequence[Point], t_star: np.ndarray, device: int = 0) -> np.ndarray:
    """The solver at the requested times (the fallback).  Points with
    log10 Ca below the range run with u_max lowered to keep the explicit
    membrane update stable (t_star is kept; more steps)."""
    t_star = np.asarray(t_star, np.float64)
    Y = np.zeros((len(points), t_star.size, 3))
    for i, p in enumerate(points):
        re = RE
        if not p.rigid and p.log10_ca < LOGCA_RANGE[0]:
            re = RE * 10.0 ** (p.log10_ca - LOGCA_RANGE[0])
        cap = capillary_for(p, re=re)
        s = lbib.from_capillary(cap, device=device)
        um = u_max(re)
        done = 0
        for k, ts in enumerate(t_star):
            target = int(round(ts * NY / um))
            if target > done:
                s.advance(target - done)
                done = target
            r = s.latest_observables()[0] if done > 0 else None
            Y[i, k] = (r["n_l"], r["delta_p"], r["r"]) if r else (1.0, 0.0, np.nan)
        s.close()
    return Y


def plain_solver_seconds_per_step(points: Sequence[Point], steps: int = 2000, device: int = 0) -> float:
    """Device seconds per step of the one-instance solver (each point alone in
    its own autotuned context), mean over the points."""
    import torch

    out = []
    for p in points:
        st = torch.cuda.Stream()
        s = lbib.from_capillary(capillary_for(p), device=device, stream=st.cuda_stream)
        s.autotune(steps_per_trial=20)
        s.advance(10)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        a.record(st)
        s.advance(steps)
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b) / 1e3 / steps)
        s.close()
    return float(np.mean(out))


def evaluate(tr: Trained, points: Sequence[Point], t_star: np.ndarray, Y: np.ndarray, floor=None):
    """Held-out errors of the network: per output, RMSE, mean absolute error,
    RMSE relative to the output's spread over the held-out set, and the
    time of all (points x times) queries: their features on the host and the
    network on the GPU.  With ``floor`` (per output, the noise floor of the
    targets Y, e.g. of replicate means from ``seed_statistics``) also the
    floor and RMSE / floor."""
    import torch

    predict_network(tr, features_many(points[:1], t_star))  # warm-up
    t0 = time.perf_counter()
    X = features_many(points, t_star)
    P = predict_network(tr, X).reshape(len(points), t_star.size, 3)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    err = {}
    for j, name in enumerate(OUTPUTS):
        e = P[:, :, j] - Y[:, :, j]
        spread = float(Y[:, :, j].std())
        rmse = float(np.sqrt(np.mean(e * e)))
        err[name] = {"rmse": rmse, "mae": float(np.mean(np.abs(e))),
                     "rmse_over_std": rmse / spread if spread > 0 else None, "std": spread}
        if floor is not None:
            err[name]["floor"] = float(floor[j])
            err[name]["rmse_over_floor"] = rmse / float(floor[j]) if floor[j] > 0 else None
    return err, secs, P


def main(argv=None):
    import argparse
    import json
    import os

    import torch

    ap = argparse.ArgumentParser(description="generate solver trajectories, train the surrogate, evaluate it")
    ap.add_argument("--points", type=int, default=512)
    ap.add_argument("--replicates", type=int, default=4, help="bond seeds per point (trajectories = points x this)")
    ap.add_argument("--holdout", type=float, default=0.1)
    ap.add_argument("--steps", type=int, default=STEPS)
    ap.add_argument("--samples", type=int, default=SAMPLES)
    ap.add_argument("--batch", type=int, default=256, help="capillaries per solver context")
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--train-batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="surrogate_run")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    pts = sample_points(args.points, seed=args.seed)
    runs = replicate(pts, args.replicates)
    t_star, Yall, gen_secs = generate(runs, steps=args.steps, samples=args.samples, batch=args.batch,
                                      stream=st.cuda_stream, log=print)
    np.savez_compressed(os.path.join(args.out, "trajectories.npz"), t_star=t_star, Y=Yall,
                        P=np.array([[p.aspect_ratio, p.log10_ca, p.rigid, p.cell == "globular", p.ligand_density,
                                     p.seed] for p in runs]))
    Y, seed_sd, floor = seed_statistics(Yall, args.replicates)
    n_hold = max(1, int(round(args.holdout * len(pts))))
    rng = np.random.default_rng(args.seed + 1)
    order = rng.permutation(len(pts))
    hold, fit = order[:n_hold], order[n_hold:]
    X = features_many([pts[i] for i in fit], t_star)
    T = Y[fit].reshape(-1, 3).astype(np.float32)
    t0 = time.perf_counter()
    tr = train(X, T, steps=args.train_steps, batch=args.train_batch, lr=args.lr, seed=args.seed, log=print)
    train_secs = time.perf_counter() - t0
    err, inf_secs, P = evaluate(tr, [pts[i] for i in hold], t_star, Y[hold], floor=floor)
    # against the single held-out trajectories, whose floor is the seed-to-seed spread itself
    Yh = Yall.reshape(len(pts), args.replicates, *Yall.shape[1:])[hold]
    single = {name: {"rmse": float(np.sqrt(np.mean((P[:, None, :, j] - Yh[:, :, :, j]) ** 2))),
                     "floor": float(seed_sd[j])} for j, name in enumerate(OUTPUTS)}
    # solver costs: the batched sweep that generated the data and the plain one-instance solver
    per_step_plain = plain_solver_seconds_per_step([pts[i] for i in hold[:8]])
    plain_per_traj = per_step_plain * args.steps
    batched_per_traj = gen_secs / len(runs)
    surrogate_per_traj = inf_secs / len(hold)
    # fallback: a particle stiffer than the training range goes to the solver
    stiff = dataclasses.replace(pts[hold[0]], rigid=False, log10_ca=-4.5)
    sur = Surrogate(tr, steps=args.steps)
    short = t_star[: max(2, args.samples // 64)]
    Yf, inside = sur.predict([pts[hold[0]], stiff], short)
    report = {
        "points": len(pts), "replicates": int(args.replicates), "trajectories": len(runs),
        "holdout_points": int(n_hold), "samples_per_trajectory": int(args.samples),
        "steps_per_trajectory": int(args.steps), "t_star_max": float(t_star[-1]),
        "generation_gpu_seconds": gen_secs, "training_seconds": train_secs, "train_steps": args.train_steps,
        "training_seconds_per_step": tr.seconds_per_step,
        "final_training_loss": tr.losses[-1], "holdout_errors": err, "holdout_single_trajectory_errors": single,
        "seconds_per_trajectory": {"plain_solver": plain_per_traj, "batched_solver": batched_per_traj,
                                   "surrogate": surrogate_per_traj},
        "sims_per_hour": {"plain_solver": 3600.0 / plain_per_traj, "batched_solver": 3600.0 / batched_per_traj,
                          "surrogate": 3600.0 / surrogate_per_traj},
        "speedup_vs_plain_solver": plain_per_traj / surrogate_per_traj,
        "fallback": {"inside_hull": [bool(v) for v in inside], "stiff_point_solved": bool(np.isfinite(Yf[1]).all())},
    }
    tr.net.get_params().tofile(os.path.join(args.out, "weights.f32"))
    with open(os.path.join(args.out, "report.json"), "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps(report))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
