"""Training of the learned pair selector (bldtt_setup_learned), on the GPU.

The selector network reads six features of a pair of clusters and predicts,
for every degree of its degree set, the log10 of the relative l2 error that
PC, CP and CC (Eqs. (8), (12), (15)) would make on the pair's contribution.
Its training data are errors the BLDTT itself makes: the pairs are the
interaction-list entries of BLDTT traversals at several MAC parameters
theta (the pairs a traversal actually meets near its accept/reject
boundary), their features and FP64 error labels come from the library's
kernels (bldtt_pair_features, bldtt_pair_errors), and the network is trained
by the library's forward/backward/Adam kernels (bldtt_mlp_gradients,
bldtt_mlp_adam).  The per-pair budget and a cap on the separation feature
are then calibrated on a separate problem against the FP64 direct sum so that
the whole potential meets a global relative-l2 budget.  This module only
orchestrates those calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import binding as B
from . import workloads as W

DEGREES = (3, 4, 5, 6, 7, 8)
LOG_FLOOR = -15.0            # labels below this are rounding noise


def init_params(num_degrees: int, rng: np.random.Generator, out_bias=None) -> np.ndarray:
    """He-initialised float32 master weights in the C ABI's packed order."""
    nout = 3 * num_degrees
    parts = []
    for o, i in ((64, 6), (64, 64), (64, 64), (nout, 64)):
        parts.append((rng.standard_normal(o * i) * math.sqrt(2.0 / i)).astype(np.float32))
        parts.append(np.zeros(o, np.float32))
    if out_bias is not None:
        parts[-1] = np.asarray(out_bias, np.float32)
    return np.concatenate(parts)


@dataclass
class Dataset:
    X: np.ndarray        # (n, 6) float64 features
    Y: np.ndarray        # (n, 3 * len(degrees)) float32 log10 errors
    M: np.ndarray        # (n, 3 * len(degrees)) float32 mask (1 = valid label)

    def __len__(self):
        return self.X.shape[0]

    @staticmethod
    def concat(parts):
        return Dataset(np.concatenate([p.X for p in parts]), np.concatenate([p.Y for p in parts]),
                       np.concatenate([p.M for p in parts]))


def collect_pairs(points, charges, kernel=B.COULOMB, kappa=0.0, leaf=2000, thetas=(0.5, 0.7, 0.85, 0.95),
                  max_pairs=4000, degrees=DEGREES, samples=64, seed=0, sources=None):
    """Labelled pairs of one problem: the list entries of MAC traversals at each
    theta (at most max_pairs per theta, drawn at random), with their features
    and FP64 error labels."""
    import torch
    rng = np.random.default_rng(seed)
    dt = torch.from_numpy(np.ascontiguousarray(points)).cuda()
    ds = dt if sources is None else torch.from_numpy(np.ascontiguousarray(sources)).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(charges)).cuda()
    parts = []
    for theta in thetas:
        with B.Plan(dt, ds, dq, kernel=kernel, kappa=kappa, n=max(degrees), theta=theta, N0=leaf,
                    M0=leaf, precision=B.FP64) as plan:
            pairs = np.concatenate([np.stack([t, s], axis=1) for t, s in plan.export_lists()])
            if pairs.shape[0] > max_pairs:
                pairs = pairs[rng.choice(pairs.shape[0], size=max_pairs, replace=False)]
            dp = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
            f = B.pair_features(plan, dp).cpu().numpy()
            ok = ~np.isnan(f[:, 0])
            if not ok.any():
                continue
            dp = torch.from_numpy(np.ascontiguousarray(pairs[ok], dtype=np.int32)).cuda()
            err = B.pair_errors(plan, dp, degrees, samples=samples).cpu().numpy()
            err = err.reshape(err.shape[0], -1)
            good = np.isfinite(err) & (err > 0)
            y = np.where(good, np.log10(np.maximum(err, 1e-300)), LOG_FLOOR)
            y = np.maximum(y, LOG_FLOOR).astype(np.float32)
            parts.append(Dataset(f[ok], y, good.astype(np.float32)))
    return Dataset.concat(parts)


def train(data: Dataset, degrees=DEGREES, epochs=150, batch=1024, lr=2e-3, seed=0, params=None):
    """Adam on the masked squared error of the log10 labels, all on the GPU.
    Returns (params float32, final loss)."""
    import torch
    rng = np.random.default_rng(seed)
    nout = 3 * len(degrees)
    if params is None:
        mean = (data.Y * data.M).sum(0) / np.maximum(data.M.sum(0), 1.0)
        params = init_params(len(degrees), rng, out_bias=mean)
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    X = torch.from_numpy(data.X.astype(np.float32)).cuda()
    Y = torch.from_numpy(data.Y).cuda()
    Mk = torch.from_numpy(data.M).cuda()
    n = X.shape[0]
    step = 0
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    grads = torch.empty_like(p)
    last = float("nan")
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).cuda()
        rate = lr * (0.5 * (1.0 + math.cos(math.pi * ep / epochs)) * 0.95 + 0.05)   # cosine decay
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = order[b0:b0 + batch]
            if idx.numel() < 2:
                continue
            xb, yb, mb = X[idx].contiguous(), Y[idx].contiguous(), Mk[idx].contiguous()
            B.mlp_gradients(p, nout, xb, yb, mb, grads=grads, loss=loss)
            step += 1
            B.mlp_adam(p, m, v, grads, step, rate)
            if ep == epochs - 1:
                tot += float(loss.item()) * idx.numel()
                cnt += idx.numel()
        if ep == epochs - 1 and cnt:
            last = tot / cnt
    return p.cpu().numpy(), last


def predict(params, X, degrees=DEGREES):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    return B.mlp_forward(torch.from_numpy(params).cuda(), 3 * len(degrees), x).cpu().numpy()


def feature_box(X, pad=0.0):
    """The training box of the features (float32 bounds; bf16 rounding of a
    feature can move it by 2^-9 relative, so the box is widened by that)."""
    lo = X.min(axis=0)
    hi = X.max(axis=0)
    widen = np.abs(np.stack([lo, hi])) * 2.0 ** -8 + pad
    return (lo - widen[0]).astype(np.float32), (hi + widen[1]).astype(np.float32)


def sampled_error(points, charges, phi, sample_idx, kernel=B.COULOMB, kappa=0.0, sources=None):
    """Relative l2 error of phi on sampled targets against the FP64 direct
    sum (computed by bldtt_direct_sum on the samples)."""
    import torch
    src = points if sources is None else sources
    dt = torch.from_numpy(np.ascontiguousarray(points[:, sample_idx])).cuda()
    ds = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(charges)).cuda()
    ref = B.direct_sum(dt, ds, dq, kernel, kappa).cpu().numpy()
    got = phi[sample_idx]
    return float(np.sqrt(np.sum((got - ref) ** 2) / np.sum(ref ** 2)))


SEP = 4                      # index of the separation feature (r_t + r_s)/R


def calibrate(params, lo, hi, points, charges, budget=1e-6, degrees=DEGREES, leaf=2000, theta=0.7,
              candidates=(-5.0, -5.25, -5.5, -5.75, -6.0, -6.25, -6.5, -7.0, -7.5, -8.0),
              sep_caps=(0.8, 0.85, 0.9, 0.95), safety=0.5, samples=2000,
              kernel=B.COULOMB, kappa=0.0, seed=0, precision=B.FP32_BULK):
    """The per-pair log10 budget and the cap on the separation feature that
    do the least work while the whole-potential error on this problem stays
    below safety * budget (FP64 direct sum on sampled targets).  A pair whose
    separation ratio exceeds the cap falls outside the selector's box and
    takes the fixed rule, which for such pairs means descending: the pairs
    near the MAC boundary are the ones whose errors the network extrapolates
    worst (without a cap the whole-potential error jumps by four decades
    between two neighbouring budgets).
    Returns (log_eps, sep_cap, table of (log_eps, error, evaluations) at the
    chosen cap, grid of (sep_cap, log_eps, error, evaluations))."""
    import torch
    rng = np.random.default_rng(seed)
    idx = rng.choice(points.shape[1], size=min(samples, points.shape[1]), replace=False)
    dt = torch.from_numpy(np.ascontiguousarray(points)).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(charges)).cuda()

    def measure(cap, le):
        h = np.array(hi, dtype=np.float32)
        h[SEP] = min(h[SEP], np.float32(cap))
        sel = B.Selector(degrees, params, lo, h, log10_budget=le)
        with B.Plan.learned(dt, dt, dq, sel, kernel=kernel, kappa=kappa, theta=theta, N0=leaf,
                            M0=leaf, precision=precision) as plan:
            phi = plan.compute().cpu().numpy()
            plan.check_error()
            ev = sum(plan.stats()["interactions"])
        return sampled_error(points, charges, phi, idx, kernel, kappa), ev

    return choose_calibration(measure, sep_caps, candidates, safety * budget)


def choose_calibration(measure, sep_caps, candidates, target):
    """The calibration walk: at each cap, budgets from the loosest down to the
    first whose error (measure(cap, log_eps) -> (error, evaluations)) is at most
    `target`; among those, the one with the fewest evaluations.  If none meets
    the target, the tightest budget at the tightest cap.  Returns (log_eps,
    sep_cap, table at the chosen cap, grid)."""
    grid = []
    best = None
    for cap in sep_caps:
        for le in sorted(candidates, reverse=True):
            e, ev = measure(cap, le)
            grid.append((cap, le, e, ev))
            if e <= target:
                if best is None or ev < best[3]:
                    best = (cap, le, e, ev)
                break   # tighter budgets at this cap only cost more
    if best is None:
        best = (min(sep_caps), min(candidates), float("nan"), float("nan"))
    table = [(le, e, ev) for cap, le, e, ev in grid if cap == best[0]]
    return best[1], best[0], table, grid


def training_problems(kind_sizes=(("uniform", 400_000), ("uniform", 150_000), ("plummer", 300_000)),
                      seed=100):
    """Seeded training problems (distinct seeds from every benchmark problem)."""
    out = []
    for i, (kind, m) in enumerate(kind_sizes):
        t, _, q = W.make_problem(kind, m, seed=seed + i)
        out.append((t, q))
    return out


def train_selector(budget=1e-6, degrees=DEGREES, leaf=2000, theta=0.7, kernel=B.COULOMB, kappa=0.0,
                   problems=None, calib=None, max_pairs=4000, epochs=150, seed=0, log=None):
    """The whole procedure: labelled pairs from the training problems, GPU
    training, the feature box, and the calibrated per-pair budget.  Returns a
    binding Selector and a report dict."""
    import time
    t0 = time.time()
    problems = problems if problems is not None else training_problems()
    data = Dataset.concat([collect_pairs(p, q, kernel, kappa, leaf, max_pairs=max_pairs, degrees=degrees,
                                         seed=seed + i) for i, (p, q) in enumerate(problems)])
    t1 = time.time()
    params, loss = train(data, degrees, epochs=epochs, seed=seed)
    t2 = time.time()
    lo, hi = feature_box(data.X)
    if calib is None:
        calib = W.make_problem("uniform", 200_000, seed=seed + 200)[::2]
    cp, cq = calib
    log_eps, cap, table, grid = calibrate(params, lo, hi, cp, cq, budget, degrees, leaf, theta,
                                          kernel=kernel, kappa=kappa, seed=seed)
    hi = hi.copy()
    hi[SEP] = min(hi[SEP], np.float32(cap))
    t3 = time.time()
    report = dict(pairs=len(data), loss=loss, label_seconds=t1 - t0, train_seconds=t2 - t1,
                  calibrate_seconds=t3 - t2, log_eps=log_eps, sep_cap=cap, calibration=table,
                  calibration_grid=grid)
    if log:
        log(report)
    return B.Selector(degrees, params, lo, hi, log10_budget=log_eps), report
