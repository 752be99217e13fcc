"""Pins of the learned-selector oracle (oracle/learned.py) against things other
than itself: a library bfloat16 conversion, exact integer arithmetic, finite
differences, Adam's first-step closed form, the MAC traversal of Alg. 2, the
direct sum, and exact reproduction of a polynomial kernel."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import learned as L
from paper_2012_06925_gb300 import workloads as W


def test_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0]])
    a = a.astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(L.bf16(a), ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert L.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0


def test_piecewise_linear_log2():
    for e in range(0, 30):
        assert L.plog2(2 ** e) == e
    assert L.plog2(3) == 1.5 and L.plog2(6) == 2.5 and L.plog2(1536) == 10.5
    vals = [L.plog2(m) for m in range(1, 5000)]
    assert all(b > a for a, b in zip(vals, vals[1:]))


def test_forward_is_exact_on_small_integers():
    """Integer weights and inputs below 2^8 make every bf16 rounding and
    float32 sum exact, so the forward equals an integer ReLU network."""
    rng = np.random.default_rng(1)
    def sparse(shape):
        return rng.choice([-1, 0, 1], size=shape, p=[0.06, 0.88, 0.06])
    params = {"W1": rng.integers(-2, 3, (64, 6)), "b1": rng.integers(-3, 4, 64),
              "W2": sparse((64, 64)), "b2": rng.integers(-3, 4, 64),
              "W3": sparse((64, 64)), "b3": rng.integers(-3, 4, 64),
              "W4": rng.integers(-1, 2, (9, 64)), "b4": rng.integers(-3, 4, 9)}
    X = rng.integers(0, 4, (50, 6))
    a = X.astype(np.int64)
    for l in (1, 2, 3):
        a = np.maximum(a @ params[f"W{l}"].T + params[f"b{l}"], 0)
        assert np.abs(a).max() < 256          # stays exactly representable in bf16
    want = a @ params["W4"].T + params["b4"]
    y, _ = L.forward_bf16({k: v.astype(np.float32) for k, v in params.items()}, X.astype(np.float64))
    assert np.array_equal(y, want.astype(np.float32))


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = {k: v.astype(np.float64) for k, v in L.init_params(6, rng).items()}
    for k in ("b1", "b2", "b3", "b4"):
        params[k] = rng.standard_normal(params[k].shape) * 0.1
    X = rng.uniform(0, 1, (16, 6))
    T = rng.standard_normal((16, 6))
    mask = (rng.uniform(size=(16, 6)) < 0.8).astype(np.float64)

    def loss(p):
        y, _ = L.forward_f64(p, X)
        return L.loss_and_grad_out(y, T, mask)[0]

    y, cache = L.forward_f64(params, X)
    _, gy = L.loss_and_grad_out(y, T, mask)
    g = L.backward(cache, gy)
    h = 1e-6
    for k in params:
        flat = params[k].ravel()
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            pp = {kk: vv.copy() for kk, vv in params.items()}
            pm = {kk: vv.copy() for kk, vv in params.items()}
            pp[k].ravel()[idx] += h
            pm[k].ravel()[idx] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - g[k].ravel()[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_adam_first_step_moves_by_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    z = {"w": np.zeros(3)}
    out, m, v = L.adam_step(p, g, z, z, step=1, lr=0.01, eps=0.0)
    assert np.allclose(out["w"], p["w"] - 0.01 * np.sign(g["w"]), rtol=0, atol=1e-15)


def test_decide_hand_worked():
    degrees = [4, 8]                       # n_p = 125, 729
    y = np.full(6, 5.0, dtype=np.float32)  # nothing feasible
    assert L.decide(y, 3000, 3000, degrees, -6.0) == L.NO_APPROX
    y[3 * 1 + L.TYPE_CC] = -7.0            # CC at 8: 729^2 = 531441
    assert L.decide(y, 3000, 3000, degrees, -6.0) == 1 + 3 * 1 + L.TYPE_CC
    y[3 * 0 + L.TYPE_PC] = -6.0            # PC at 4: 3000 * 125 = 375000 (cheaper; <= is feasible)
    assert L.decide(y, 3000, 3000, degrees, -6.0) == 1 + L.TYPE_PC
    # PP costs no more than the best option: PP
    assert L.decide(y, 3000, 100, degrees, -6.0) == 0     # PP 300000 <= PC 375000


def _problem(m=2500, seed=3):
    t, s, q = W.make_problem("uniform", m, seed=seed)
    return t, s, q


def test_fallback_only_selector_is_the_mac_traversal():
    t, s, q = _problem()
    tt, st = O.build_tree(t, 60), O.build_tree(s, 60)
    n = 4
    lists = O.dual_tree_traversal(tt, st, n, 0.7)
    sel = L.Selector(None, [n], -6.0, np.zeros(6), np.zeros(6), theta_fallback=0.7)
    ent = L.learned_traversal(tt, st, sel, 0.0)
    got = [sorted((a, b) for c, a, b in ent if c == typ) for typ in range(4)]
    assert got == [sorted(l) for l in lists]


def test_never_feasible_selector_gives_the_direct_sum():
    t, s, q = _problem(1500, seed=4)
    tt, st = O.build_tree(t, 40), O.build_tree(s, 40)
    params = L.init_params(6, np.random.default_rng(5))
    params["W4"][:] = 0.0
    params["b4"][:] = 10.0                 # predicted error 1e10: never feasible
    sel = L.Selector(params, [3, 5], -6.0, np.full(6, -1e9), np.full(6, 1e9))
    ent = L.learned_traversal(tt, st, sel, 0.0)
    assert all(c == 0 and tt.is_leaf(a) and st.is_leaf(b) for c, a, b in ent)
    phi = L.bldtt_entries(t, s, q, tt, st, ent, [3, 5])
    assert O.relative_l2_error(O.direct_sum(t, s, q), phi) <= 1e-14


def test_single_degree_entries_equal_the_standard_driver():
    t, s, q = W.make_problem("uniform", 2200, 1900, seed=6, sources_kind="plummer")
    n, theta = 2, 0.7
    ref = O.bldtt(t, s, q, n=n, theta=theta, N0=30, M0=30)
    ent = [(typ, a, b) for typ in range(4) for a, b in ref.lists[typ]]
    assert len(ref.lists[O.PC]) and len(ref.lists[O.CP]) and len(ref.lists[O.CC])
    phi = L.bldtt_entries(t, s, q, ref.ttree, ref.stree, ent, [n])
    assert O.relative_l2_error(ref.phi, phi) <= 1e-12


def test_random_selector_covers_every_pair_once_and_reproduces_polynomials():
    """A random network with a loose budget mixes all classes and degrees;
    every target-source pair is still covered exactly once, and a kernel of
    degree 2 per coordinate is reproduced exactly at degrees >= 2."""
    t, s, q = W.make_problem("uniform", 1800, 1600, seed=7, sources_kind="plummer")
    tt, st = O.build_tree(t, 30), O.build_tree(s, 30)
    degrees = [2, 3, 4]
    params = L.init_params(9, np.random.default_rng(1))
    sel = L.Selector(params, degrees, 0.0, np.full(6, -1e9), np.full(6, 1e9))
    ent = L.learned_traversal(tt, st, sel, 0.0)
    classes = {c for c, _, _ in ent}
    assert 0 in classes and len(classes) >= 6
    cover = np.zeros((t.shape[1], s.shape[1]), dtype=np.int32)
    for c, a, b in ent:
        cover[tt.begin[a]:tt.end[a], st.begin[b]:st.end[b]] += 1
    assert cover.min() == 1 and cover.max() == 1
    phi = L.bldtt_entries(t, s, q, tt, st, ent, degrees, kernel=O.TEST_POLY)
    ref = O.direct_sum(t, s, q, O.TEST_POLY)
    assert O.relative_l2_error(ref, phi) <= 1e-12


def test_pair_errors_polynomial_exact_and_falling_with_degree():
    t, s, q = W.make_problem("uniform", 4000, seed=9)
    tt, st = O.build_tree(t, 100), O.build_tree(s, 100)
    # a well-separated pair of leaves
    pair = None
    for a in tt.leaves():
        for b in st.leaves():
            ct, cs = np.array(tt.center(a)), np.array(st.center(b))
            R = np.linalg.norm(ct - cs)
            if R > 0 and (tt.radius(a) + st.radius(b)) / R < 0.6:
                pair = (a, b)
                break
        if pair:
            break
    a, b = pair
    pos = np.arange(tt.begin[a], tt.end[a])[::3]
    err_poly = L.pair_errors(t, s, q, tt, st, a, b, [2, 3], pos, kernel=O.TEST_POLY)
    assert err_poly.max() <= 1e-12
    err = L.pair_errors(t, s, q, tt, st, a, b, [2, 4, 6, 8], pos)
    for typ in range(3):
        assert err[0, typ] > err[1, typ] > err[2, typ] > err[3, typ]
    # CC interpolates on both sides: never much better than the one-sided forms
    assert np.all(err[:, 2] >= 0.5 * np.maximum(err[:, 0], err[:, 1]))


# --------------------------------------------------------------------------
# Pair features against hand-worked values
# --------------------------------------------------------------------------

def _feature_examples():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "pair_features_examples.json")
    with open(path) as f:
        return json.load(f)["examples"]


def _cluster_points(spec):
    """lo, hi and m - 2 copies of the box centre (one particle when m = 1)."""
    lo, hi, m = np.array(spec["lo"], float), np.array(spec["hi"], float), spec["m"]
    if m == 1:
        assert np.array_equal(lo, hi)
        return lo[:, None].copy()
    mid = (lo + hi) * 0.5
    return np.concatenate([lo[:, None], hi[:, None], np.repeat(mid[:, None], m - 2, axis=1)],
                          axis=1)


def _fraction(text):
    from fractions import Fraction
    return float(Fraction(text))


def pair_feature_mismatches(features_fn):
    """Names of the hand-worked examples whose features features_fn gets
    wrong (bit for bit: every expected value is a correctly rounded quotient
    of exact operands)."""
    bad = []
    for ex in _feature_examples():
        tpts, spts = _cluster_points(ex["target"]), _cluster_points(ex["source"])
        tt, st = O.build_tree(tpts, ex["target"]["m"]), O.build_tree(spts, ex["source"]["m"])
        assert tt.num_clusters == 1 and st.num_clusters == 1
        assert list(tt.lo[0]) == ex["target"]["lo"] and list(st.hi[0]) == ex["source"]["hi"]
        got = features_fn(tt, 0, st, 0, ex["kappa"])
        want = ex["features"]
        if want is None:
            if got is not None:
                bad.append(ex["name"])
        elif got is None or not np.array_equal(np.asarray(got), [_fraction(v) for v in want]):
            bad.append(ex["name"])
    return bad


def test_pair_features_hand_worked():
    assert pair_feature_mismatches(L.pair_features) == []
