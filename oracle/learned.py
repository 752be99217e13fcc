"""CPU oracle of the learned pair selector and of the multi-degree BLDTT it
drives.  TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product.

The paper fixes one degree n and one rule (Alg. 2): a pair (C_t, C_s) is
approximated when the MAC r_t + r_s < theta R holds, by PC, CP or CC according
to the cluster sizes against n_p = (n+1)^3.  The learned selector replaces the
MAC by a small network that predicts, for each approximation type (PC, CP,
CC; Eqs. (8), (12), (15)) and each degree d of a degree set D, the log10 of
the relative l2 error the approximation would make on the pair's
contribution; the cheapest option predicted to meet a per-pair budget is
taken, the traversal descends when none is.  Everything here is written from
these definitions, in the paper's notation:

Features of a pair (all FP64, then rounded to float32 and to bfloat16):
  R = |c_t - c_s| (box centres), r_t, r_s the radii (reading R6);
  only pairs with R > 0 and (r_t + r_s)/R < 1 are candidates.
  f0 = plog2(|C_t|)/16, f1 = plog2(|C_s|)/16, f2 = r_t/R, f3 = r_s/R,
  f4 = (r_t + r_s)/R, f5 = kappa R/(1 + kappa R),
  plog2(m) = e + (f - 1) for m = f 2^e, 1 <= f < 2 (piecewise-linear log2,
  exact in FP64).

Network (the forward both sides compute bit for bit):
  x = bf16(f); three hidden layers of 64, y = W4 a3 + b4 with 3 |D| outputs
  y[3 i + t], t = 0 PC, 1 CP, 2 CC at degree D[i].  A layer computes
  z_j = b_j + sum_k w_jk a_k in float32, k = 0, 1, ... in order (each product
  of two bfloat16 values is exact in float32), a_j = bf16(max(z_j, 0)).
  Weights are bf16 of float32 master weights; biases stay float32.

Decision (integers and float32 compares):
  feasible options: y[3i + t] <= log_eps;  cost PC = |C_t| n_p(d),
  CP = n_p(d) |C_s|, CC = n_p(d)^2, PP = |C_t| |C_s|; the cheapest feasible
  option (lowest class index on ties) is taken unless PP costs no more; no
  feasible option means no approximation (split, or PP for two leaves).
  Features outside the training box [lo, hi] fall back to the MAC of Alg. 2
  at degree max(D).

List classes: 0 = PP, 1 + 3 i + t = (PC, CP, CC)[t] at degree D[i].
"""
from __future__ import annotations

import math

import numpy as np

from . import bldtt_oracle as O

HIDDEN = 64
NFEAT = 6
NO_APPROX = -2
FALLBACK = -1
TYPE_PC, TYPE_CP, TYPE_CC = 0, 1, 2


# --------------------------------------------------------------------------
# bfloat16
# --------------------------------------------------------------------------

def bf16(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even),
    returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


# --------------------------------------------------------------------------
# Features
# --------------------------------------------------------------------------

def plog2(m: int) -> float:
    """Piecewise-linear log2: e + (f - 1) for m = f 2^e, 1 <= f < 2."""
    f, e = math.frexp(float(m))        # m = f 2^e, 0.5 <= f < 1
    return (e - 1) + (2.0 * f - 1.0)


def pair_features(tt: O.Tree, t: int, st: O.Tree, s: int, kappa: float):
    """The six features of pair (t, s) as FP64, or None if the pair cannot be
    approximated (R = 0 or (r_t + r_s)/R >= 1)."""
    ct, cs = tt.center(t), st.center(s)
    dx, dy, dz = ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]
    R = math.sqrt(dx * dx + dy * dy + dz * dz)
    if not R > 0.0:
        return None
    rt, rs = tt.radius(t), st.radius(s)
    sep = (rt + rs) / R
    if not sep < 1.0:
        return None
    kr = kappa * R
    return np.array([plog2(tt.count(t)) / 16.0, plog2(st.count(s)) / 16.0, rt / R, rs / R, sep,
                     kr / (1.0 + kr)])


# --------------------------------------------------------------------------
# Network: bf16 forward (bit-exact), FP64 backward
# --------------------------------------------------------------------------

def init_params(n_out: int, rng: np.random.Generator):
    """He-style random float32 master weights."""
    def lin(o, i):
        return (rng.standard_normal((o, i)) * math.sqrt(2.0 / i)).astype(np.float32)
    return {"W1": lin(HIDDEN, NFEAT), "b1": np.zeros(HIDDEN, np.float32),
            "W2": lin(HIDDEN, HIDDEN), "b2": np.zeros(HIDDEN, np.float32),
            "W3": lin(HIDDEN, HIDDEN), "b3": np.zeros(HIDDEN, np.float32),
            "W4": lin(n_out, HIDDEN), "b4": np.zeros(n_out, np.float32)}


def _layer_f32(W, b, a):
    """z = b + sum_k W[:, k] a[:, k] in float32, k in increasing order."""
    z = np.broadcast_to(b.astype(np.float32), (a.shape[0], W.shape[0])).copy()
    for k in range(W.shape[1]):
        z = (z + a[:, k:k + 1] * W[None, :, k]).astype(np.float32)
    return z


def forward_bf16(params, X):
    """The selector's forward: X (B, 6) float64 features.  Returns float32
    outputs (B, n_out) and the cache the backward pass needs."""
    Wb = {k: bf16(params[k]) for k in ("W1", "W2", "W3", "W4")}
    a0 = bf16(np.asarray(X, dtype=np.float64).astype(np.float32))
    z1 = _layer_f32(Wb["W1"], params["b1"], a0)
    a1 = bf16(np.maximum(z1, 0.0))
    z2 = _layer_f32(Wb["W2"], params["b2"], a1)
    a2 = bf16(np.maximum(z2, 0.0))
    z3 = _layer_f32(Wb["W3"], params["b3"], a2)
    a3 = bf16(np.maximum(z3, 0.0))
    y = _layer_f32(Wb["W4"], params["b4"], a3)
    return y, dict(W=Wb, a=(a0, a1, a2, a3), z=(z1, z2, z3))


def forward_f64(params, X):
    """The same network in plain FP64 without any rounding (for checking the
    backward formulas by finite differences)."""
    a = np.asarray(X, dtype=np.float64)
    acts, zs = [a], []
    for l in (1, 2, 3):
        z = a @ params[f"W{l}"].astype(np.float64).T + params[f"b{l}"]
        zs.append(z)
        a = np.maximum(z, 0.0)
        acts.append(a)
    y = a @ params["W4"].astype(np.float64).T + params["b4"]
    W = {k: params[k].astype(np.float64) for k in ("W1", "W2", "W3", "W4")}
    return y, dict(W=W, a=tuple(acts), z=tuple(zs))


def loss_and_grad_out(y, T, mask):
    """L = sum mask (y - T)^2 / max(1, sum mask) and dL/dy."""
    y = np.asarray(y, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    cnt = max(1.0, float(m.sum()))
    d = (y - T) * m
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def backward(cache, gy):
    """Gradients of the loss for every parameter, in FP64, from the cached
    activations (bf16 values for the selector's forward); the rounding of an
    activation is passed through (derivative 1), ReLU' = [z > 0]."""
    W, (a0, a1, a2, a3), (z1, z2, z3) = cache["W"], cache["a"], cache["z"]
    a0, a1, a2, a3 = (np.asarray(v, dtype=np.float64) for v in (a0, a1, a2, a3))
    g = {}
    g["W4"] = gy.T @ a3
    g["b4"] = gy.sum(axis=0)
    ga = gy @ W["W4"].astype(np.float64)
    for l, (z, a_prev) in zip((3, 2, 1), ((z3, a2), (z2, a1), (z1, a0))):
        gz = ga * (np.asarray(z) > 0.0)
        g[f"W{l}"] = gz.T @ a_prev
        g[f"b{l}"] = gz.sum(axis=0)
        ga = gz @ W[f"W{l}"].astype(np.float64)
    return g


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) on the float32 master weights, FP64 here."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        mk = beta1 * m[k] + (1.0 - beta1) * grads[k]
        vk = beta2 * v[k] + (1.0 - beta2) * grads[k] ** 2
        mh = mk / (1.0 - beta1 ** step)
        vh = vk / (1.0 - beta2 ** step)
        out_p[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


# --------------------------------------------------------------------------
# Decision and traversal
# --------------------------------------------------------------------------

def n_p(d: int) -> int:
    return (d + 1) ** 3


def decide(y, cnt_t: int, cnt_s: int, degrees, log_eps: float) -> int:
    """Class of the cheapest feasible option, 0 (PP) if PP costs no more, or
    NO_APPROX."""
    thr = np.float32(log_eps)
    best, best_cost = NO_APPROX, None
    for i, d in enumerate(degrees):
        npd = n_p(d)
        for t, cost in ((TYPE_PC, cnt_t * npd), (TYPE_CP, npd * cnt_s), (TYPE_CC, npd * npd)):
            if np.float32(y[3 * i + t]) <= thr and (best_cost is None or cost < best_cost):
                best, best_cost = 1 + 3 * i + t, cost
    if best == NO_APPROX:
        return NO_APPROX
    return 0 if cnt_t * cnt_s <= best_cost else best


class Selector:
    """A trained (or given) network with its degree set, budget and
    feature box."""

    def __init__(self, params, degrees, log_eps, lo, hi, theta_fallback=0.7):
        self.params = params
        self.degrees = list(degrees)
        self.log_eps = float(log_eps)
        self.lo = np.asarray(lo, dtype=np.float32)
        self.hi = np.asarray(hi, dtype=np.float32)
        self.theta = theta_fallback

    def choose(self, tt, t, st, s, kappa):
        f = pair_features(tt, t, st, s, kappa)
        if f is None:
            return NO_APPROX
        x = bf16(f.astype(np.float32))
        if self.params is None or np.any(x < self.lo) or np.any(x > self.hi):
            return FALLBACK
        y, _ = forward_bf16(self.params, f[None, :])
        return decide(y[0], tt.count(t), st.count(s), self.degrees, self.log_eps)


def mac_class(tt, t, st, s, theta, degrees):
    """Alg. 2's rule at degree max(D): the class of a well-separated pair,
    or None."""
    if not O.well_separated(tt, t, st, s, theta):
        return None
    i = len(degrees) - 1
    npd = n_p(degrees[i])
    big_t, big_s = tt.count(t) > npd, st.count(s) > npd
    if big_t and big_s:
        return 1 + 3 * i + TYPE_CC
    if big_t:
        return 1 + 3 * i + TYPE_CP
    if big_s:
        return 1 + 3 * i + TYPE_PC
    return 0


def learned_traversal(tt: O.Tree, st: O.Tree, sel: Selector, kappa: float):
    """Alg. 2 with the selector in place of the MAC.  Returns the entries
    (class, t, s) in traversal order."""
    entries = []

    def visit(t, s):
        c = sel.choose(tt, t, st, s, kappa)
        if c == FALLBACK:
            c = mac_class(tt, t, st, s, sel.theta, sel.degrees)
            if c is None:
                c = NO_APPROX
        if c >= 0:
            entries.append((c, t, s))
            return
        leaf_t, leaf_s = tt.is_leaf(t), st.is_leaf(s)
        if leaf_t and leaf_s:
            entries.append((0, t, s))
        elif leaf_s:
            for ch in tt.children[t]:
                visit(ch, s)
        elif leaf_t:
            for ch in st.children[s]:
                visit(t, ch)
        elif st.count(s) < tt.count(t):
            for ch in tt.children[t]:
                visit(ch, s)
        else:
            for ch in st.children[s]:
                visit(t, ch)

    if tt.num_clusters and st.num_clusters:
        visit(0, 0)
    return entries


# --------------------------------------------------------------------------
# Multi-degree BLDTT (the paper's sums, each at its entry's degree)
# --------------------------------------------------------------------------

def bldtt_entries(targets, sources, charges, tt, st, entries, degrees, kernel=O.COULOMB,
                  kappa=0.0):
    """Potentials (input order) of the interaction entries (class, t, s):
    PP by Eq. (6); at degree d: PC by Eq. (8), CP by Eq. (12), CC by Eq. (15),
    with the proxy charges of Eq. (9) computed directly from the cluster's
    particles and the proxy potentials carried to the targets by Eq. (19)."""
    xs = np.asarray(targets, dtype=np.float64)[:, tt.perm]
    ys = np.asarray(sources, dtype=np.float64)[:, st.perm]
    qs = np.asarray(charges, dtype=np.float64)[st.perm]
    phi = np.zeros(xs.shape[1])
    qhat = {}
    phit = {i: np.zeros((tt.num_clusters, n_p(d))) for i, d in enumerate(degrees)}

    def qh(s, i):
        if (s, i) not in qhat:
            qhat[(s, i)] = O.proxy_charges_direct(st, s, degrees[i], ys, qs)
        return qhat[(s, i)]

    for c, t, s in entries:
        tb, te = tt.begin[t], tt.end[t]
        if c == 0:
            phi[tb:te] += O.interact_pp(kernel, kappa, xs, tb, te, ys, qs, st.begin[s], st.end[s])
            continue
        i, typ = divmod(c - 1, 3)
        d = degrees[i]
        if typ == TYPE_PC:
            gx, gy, gz = O.proxy_grid(st, s, d)
            phi[tb:te] += O._block_sum(kernel, kappa, xs[0, tb:te], xs[1, tb:te], xs[2, tb:te],
                                       gx, gy, gz, qh(s, i).ravel())
        elif typ == TYPE_CP:
            phit[i][t] += O.interact_cp(kernel, kappa, tt, t, d, ys, qs, st.begin[s], st.end[s])
        else:
            tx, ty, tz = O.proxy_grid(tt, t, d)
            sx, sy, sz = O.proxy_grid(st, s, d)
            phit[i][t] += O._block_sum(kernel, kappa, tx, ty, tz, sx, sy, sz, qh(s, i).ravel())
    positions = np.arange(xs.shape[1])
    for i, d in enumerate(degrees):
        if np.any(phit[i] != 0.0):
            P = d + 1
            phi += O.downward_direct(tt, d, xs, phit[i].reshape(-1, P, P, P), positions)
    out = np.empty_like(phi)
    out[tt.perm] = phi
    return out


# --------------------------------------------------------------------------
# Training labels: the error each option makes on one pair
# --------------------------------------------------------------------------

def pair_errors(targets, sources, charges, tt, st, t, s, degrees, positions, kernel=O.COULOMB,
                kappa=0.0):
    """Relative l2 error of PC, CP and CC at each degree against the exact
    pair sum (Eq. (6)), on the target tree positions `positions` of C_t.
    Returns an array (len(degrees), 3).  (The GPU labels represent a source
    cluster of more than 4096 particles by a strided subset; this oracle
    always uses the whole cluster, so it pins clusters up to that size.)"""
    xs = np.asarray(targets, dtype=np.float64)[:, tt.perm]
    ys = np.asarray(sources, dtype=np.float64)[:, st.perm]
    qs = np.asarray(charges, dtype=np.float64)[st.perm]
    px, py, pz = xs[0, positions], xs[1, positions], xs[2, positions]
    sb, se = st.begin[s], st.end[s]
    exact = O._block_sum(kernel, kappa, px, py, pz, ys[0, sb:se], ys[1, sb:se], ys[2, sb:se],
                         qs[sb:se])
    out = np.zeros((len(degrees), 3))
    for i, d in enumerate(degrees):
        P = d + 1
        qhat = O.proxy_charges_direct(st, s, d, ys, qs).ravel()
        gx, gy, gz = O.proxy_grid(st, s, d)
        pc = O._block_sum(kernel, kappa, px, py, pz, gx, gy, gz, qhat)
        B1, B2, B3 = O.tensor_basis(tt, t, d, px, py, pz)

        def interp(phit):
            return np.einsum("im,jm,km,ijk->m", B1, B2, B3, phit.reshape(P, P, P))

        cp = interp(O.interact_cp(kernel, kappa, tt, t, d, ys, qs, sb, se))
        tx, ty, tz = O.proxy_grid(tt, t, d)
        cc = interp(O._block_sum(kernel, kappa, tx, ty, tz, gx, gy, gz, qhat))
        for typ, approx in enumerate((pc, cp, cc)):
            out[i, typ] = O.relative_l2_error(exact, approx)
    return out
