"""Pins of the oracle's upward pass, downward pass and whole pipeline.

Exact identities come from App. A-C (polynomial self-reproduction, the
recursive passes equal the direct ones), from Alg. 2 (theta = 0 leaves only
PP, so the BLDTT is the direct sum of Eq. (1)), and from a test kernel of
degree 2 for which every approximation is exact.  The approximate checks use
the paper's own error figures (tests/golden/paper_errors.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_errors.json")


def _sorted_sources(n_src=2500, N0=40, seed=4, kind="plummer"):
    _, src, q = W.make_problem(kind, 10, n_src, seed=seed, sources_kind=kind)
    st = O.build_tree(src, N0)
    return st, src[:, st.perm], q[st.perm]


@pytest.mark.parametrize("n", [1, 2, 5])
def test_upward_recursive_equals_direct(n):
    """App. B: q-hat from children (Eq. (16)) equals Eq. (9) on the particles."""
    st, ys, qs = _sorted_sources()
    qhat = O.upward_pass(st, n, ys, qs)
    for c in range(st.num_clusters):
        direct = O.proxy_charges_direct(st, c, n, ys, qs)
        scale = np.max(np.abs(direct))
        assert np.max(np.abs(qhat[c] - direct)) <= 1e-12 * max(scale, 1.0)


@pytest.mark.parametrize("n", [1, 3])
def test_upward_conserves_charge_and_first_moments(n):
    st, ys, qs = _sorted_sources()
    qhat = O.upward_pass(st, n, ys, qs)
    for c in range(st.num_clusters):
        b, e = st.begin[c], st.end[c]
        gx, gy, gz = O.proxy_grid(st, c, n)
        qh = qhat[c].ravel()
        assert abs(qh.sum() - qs[b:e].sum()) <= 1e-11 * (1 + np.abs(qs[b:e]).sum())
        for g, y in [(gx, ys[0]), (gy, ys[1]), (gz, ys[2])]:
            assert abs((g * qh).sum() - (y[b:e] * qs[b:e]).sum()) <= 1e-11 * (1 + np.abs(qs[b:e]).sum())


def test_downward_recursive_equals_per_level_direct():
    """App. C: the recursive pass (Eqs. (20)-(21)) equals Eq. (19)."""
    tgt, src, q = W.make_problem("uniform", 2500, seed=9)
    res = O.bldtt(tgt, src, q, n=3, theta=0.8, N0=40, M0=40)
    tt = res.ttree
    xs = tgt[:, tt.perm]
    rec = np.zeros(xs.shape[1])
    for c in tt.leaves():
        rec[tt.begin[c]:tt.end[c]] = O.leaf_to_particles(tt, c, 3, xs, res.phit[c])
    pos = np.arange(0, xs.shape[1], 7)
    direct = O.downward_direct(tt, 3, xs, res.phit_dtt, pos)
    assert np.max(np.abs(rec[pos] - direct)) <= 1e-12 * np.max(np.abs(direct))


@pytest.mark.parametrize("kernel,kappa", [(O.COULOMB, 0.0), (O.YUKAWA, 0.5)])
def test_theta_zero_is_the_direct_sum(kernel, kappa):
    tgt, src, q = W.make_problem("uniform", 1200, 900, seed=1, sources_kind="sphere")
    ref = O.direct_sum(tgt, src, q, kernel, kappa)
    res = O.bldtt(tgt, src, q, kernel=kernel, kappa=kappa, n=4, theta=0.0, N0=50, M0=50)
    assert O.relative_l2_error(ref, res.phi) <= 1e-14


def test_direct_sum_against_brute_force_loops():
    rng = np.random.default_rng(0)
    t = rng.uniform(-1, 1, size=(3, 7))
    s = np.concatenate([t[:, :3], rng.uniform(-1, 1, size=(3, 5))], axis=1)
    q = rng.uniform(-1, 1, size=8)
    for kernel, kappa in [(O.COULOMB, 0.0), (O.YUKAWA, 1.3), (O.TEST_POLY, 0.0)]:
        got = O.direct_sum(t, s, q, kernel, kappa)
        for i in range(7):
            acc = 0.0
            for j in range(8):
                d = t[:, i] - s[:, j]
                r = float(np.sqrt(d @ d))
                if r == 0.0:
                    continue
                if kernel == O.COULOMB:
                    g = 1.0 / r
                elif kernel == O.YUKAWA:
                    g = np.exp(-kappa * r) / r
                else:
                    a, b, c = d
                    g = 1 + a - 2 * b + 3 * c + a * b - b * c + a * a * c * c - 0.5 * b * b
                acc += g * q[j]
            assert abs(got[i] - acc) <= 1e-13 * (1 + abs(acc))


@pytest.mark.parametrize("n,theta,leaf,all_types", [(2, 0.7, 15, True), (2, 0.5, 20, True),
                                                   (3, 0.9, 15, False)])
def test_degree_two_kernel_is_reproduced_exactly(n, theta, leaf, all_types):
    """Every approximation (PC, CP, CC, upward, downward) is exact for a
    kernel of degree <= n in each coordinate of x and of y."""
    tgt, src, q = W.make_problem("uniform", 2500, 2200, seed=6, sources_kind="plummer")
    ref = O.direct_sum(tgt, src, q, O.TEST_POLY)
    res = O.bldtt(tgt, src, q, kernel=O.TEST_POLY, n=n, theta=theta, N0=leaf, M0=leaf)
    if all_types:
        assert all(len(l) > 0 for l in res.lists)
    assert O.relative_l2_error(ref, res.phi) <= 1e-12


def test_error_falls_with_degree_and_with_theta():
    tgt, src, q = W.make_problem("uniform", 4000, seed=0)
    ref = O.direct_sum(tgt, src, q)
    by_n = [O.relative_l2_error(ref, O.bldtt(tgt, src, q, n=n, theta=0.9, N0=20, M0=20).phi)
            for n in (1, 2, 4, 6)]
    assert all(by_n[i + 1] < by_n[i] for i in range(3))
    by_theta = [O.relative_l2_error(ref, O.bldtt(tgt, src, q, n=3, theta=th, N0=20, M0=20).phi)
                for th in (0.9, 0.7, 0.5)]
    assert all(by_theta[i + 1] < by_theta[i] for i in range(2))


def test_sampled_potentials_equal_full_driver():
    tgt, src, q = W.make_problem("uniform", 2000, 1800, seed=12, sources_kind="plummer")
    kw = dict(kernel=O.YUKAWA, kappa=0.7, n=3, theta=0.8, N0=30, M0=30)
    full = O.bldtt(tgt, src, q, **kw)
    samp = O.SampledBLDTT(tgt, src, q, **kw)
    idx = np.arange(0, 2000, 37)
    got = samp.potentials(idx)
    assert np.max(np.abs(got - full.phi[idx])) <= 1e-12 * np.max(np.abs(full.phi))


def test_paper_error_at_1e5():
    """Sec. 4.1: N=1E5, theta=0.7, n=8, leaf size 2000 gives error 1.58E-8 on
    a 0.1% sample; the oracle must land within a factor ~6 of it."""
    with open(GOLDEN) as f:
        row = json.load(f)["rows"][0]
    N = row["N"]
    tgt, src, q = W.make_problem("uniform", N, seed=21)
    samp = O.SampledBLDTT(tgt, src, q, n=8, theta=0.7, N0=2000, M0=2000)
    idx = np.random.default_rng(1).choice(N, size=N // 1000, replace=False)
    got = samp.potentials(idx)
    ref = O.direct_sum(tgt[:, idx], src, q)
    err = O.relative_l2_error(ref, got)
    assert row["bldtt_error"] / 6 <= err <= row["bldtt_error"] * 6


# ---- the other kernels of Sec. 4.6 and the CC+PP-only variant of Sec. 4.3 ----

def test_other_kernels_closed_forms():
    g = O.kernel_values(O.OSCILLATORY, np.pi, np.array([0.5, 0.25, 0.0]), np.zeros(3), np.zeros(3))
    assert abs(g[0] - 2.0) <= 1e-15 and abs(g[1] - np.sin(np.pi / 4) * 4) <= 1e-14 and g[2] == 0.0
    g = O.kernel_values(O.REG_COULOMB, 0.005, np.array([0.3, 0.0]), np.array([0.4, 0.0]), np.zeros(2))
    assert abs(g[0] - 1.0 / np.sqrt(0.25 + 0.005 ** 2)) <= 1e-15 and g[1] == 0.0


@pytest.mark.parametrize("kernel,kappa", [(O.OSCILLATORY, np.pi), (O.REG_COULOMB, 0.005)])
def test_other_kernels_theta_zero_and_convergence(kernel, kappa):
    tgt, src, q = W.make_problem("uniform", 2500, seed=14)
    ref = O.direct_sum(tgt, src, q, kernel, kappa)
    res = O.bldtt(tgt, src, q, kernel=kernel, kappa=kappa, n=3, theta=0.0, N0=60, M0=60)
    assert O.relative_l2_error(ref, res.phi) <= 1e-14
    errs = [O.relative_l2_error(ref, O.bldtt(tgt, src, q, kernel=kernel, kappa=kappa, n=n,
                                            theta=0.8, N0=30, M0=30).phi) for n in (2, 4, 6)]
    assert errs[0] > errs[1] > errs[2]


def test_cc_pp_only_variant():
    """Sec. 4.3 ablation: no PC/CP entries, still every pair covered once, the
    degree-2 kernel still reproduced exactly, and the extra PP work shows up."""
    tgt, src, q = W.make_problem("uniform", 2500, 2200, seed=6, sources_kind="plummer")
    full = O.bldtt(tgt, src, q, kernel=O.TEST_POLY, n=2, theta=0.7, N0=15, M0=15)
    abl = O.bldtt(tgt, src, q, kernel=O.TEST_POLY, n=2, theta=0.7, N0=15, M0=15,
                  variant=O.CC_PP_ONLY)
    assert len(full.lists[O.PC]) > 0 and len(full.lists[O.CP]) > 0
    assert len(abl.lists[O.PC]) == 0 and len(abl.lists[O.CP]) == 0
    assert len(abl.lists[O.CC]) == len(full.lists[O.CC])
    assert abl.counts[0] > full.counts[0]
    ref = O.direct_sum(tgt, src, q, O.TEST_POLY)
    assert O.relative_l2_error(ref, abl.phi) <= 1e-12
    m = tgt.shape[1]
    n = src.shape[1]
    cover = np.zeros((m, n), dtype=np.int32)
    for typ in range(4):
        for t, s in abl.lists[typ]:
            cover[abl.ttree.begin[t]:abl.ttree.end[t], abl.stree.begin[s]:abl.stree.end[s]] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_coulomb_and_yukawa_closed_form_values():
    """Values fixed by arithmetic alone: |(3, 4, 0)| = 5, so 1/r = 0.2; with
    kappa = ln 2, exp(-kappa r)/r is 1/2 at r = 1 and 1/8 at r = 2 (Sec. 4.6)."""
    g = O.kernel_values(O.COULOMB, 0.0, np.array([3.0]), np.array([4.0]), np.array([0.0]))
    assert abs(g[0] - 0.2) <= 1e-16
    y = O.kernel_values(O.YUKAWA, math.log(2.0), np.array([1.0, 0.0]), np.array([0.0, -2.0]),
                        np.zeros(2))
    assert abs(y[0] - 0.5) <= 1e-15 and abs(y[1] - 0.125) <= 1e-15
