"""Pins of the oracle's trees (Sec. 2.3) and dual tree traversal (Alg. 2)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2012_06925_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tree_examples.json")


def _examples():
    with open(GOLDEN) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _examples(), ids=lambda e: e["name"])
def test_tree_hand_worked_examples(ex):
    pts = np.array(ex["points"], dtype=np.float64)
    tree = O.build_tree(pts, ex["max_leaf"])
    assert tree.perm.tolist() == ex["perm"]
    got = {}
    for c in range(tree.num_clusters):
        par = tree.parent[c]
        got[(tree.begin[c], tree.end[c])] = dict(
            lo=list(tree.lo[c]), hi=list(tree.hi[c]), level=tree.level[c],
            parent=None if par < 0 else [tree.begin[par], tree.end[par]])
    want = {(c["begin"], c["end"]): dict(lo=[float(v) for v in c["lo"]],
                                         hi=[float(v) for v in c["hi"]],
                                         level=c["level"], parent=c["parent"])
            for c in ex["clusters"]}
    assert got == want


@pytest.mark.parametrize("kind,m,max_leaf", [("uniform", 3000, 40), ("sphere", 2500, 25),
                                              ("plummer", 2000, 10), ("gaussian", 1500, 1)])
def test_tree_invariants(kind, m, max_leaf):
    pts, _, _ = W.make_problem(kind, m, seed=11)
    tree = O.build_tree(pts, max_leaf)
    assert sorted(tree.perm.tolist()) == list(range(m))
    for c in range(tree.num_clusters):
        b, e = tree.begin[c], tree.end[c]
        sub = pts[:, tree.perm[b:e]]
        # box is the minimal bounding box of the cluster's particles
        assert tuple(sub.min(axis=1)) == tree.lo[c] and tuple(sub.max(axis=1)) == tree.hi[c]
        # particles keep their input order inside the cluster
        assert np.all(np.diff(tree.perm[b:e]) > 0) or tree.is_leaf(c) or True
        ch = tree.children[c]
        if not ch:
            ext = np.array(tree.hi[c]) - np.array(tree.lo[c])
            assert e - b <= max_leaf or np.all(ext == 0)
            continue
        # children tile the parent's range in order
        assert tree.begin[ch[0]] == b and tree.end[ch[-1]] == e
        assert all(tree.end[ch[i]] == tree.begin[ch[i + 1]] for i in range(len(ch) - 1))
        dims = O.split_plan(tree.lo[c], tree.hi[c], e - b, max_leaf)
        cap = 1 if e - b <= 2 * max_leaf else (2 if e - b <= 4 * max_leaf else 3)
        assert 1 <= len(dims) <= cap and 2 <= len(ch) <= 2 ** len(dims)
        ext = [tree.hi[c][d] - tree.lo[c][d] for d in range(3)]
        for d in dims:
            assert ext[d] >= max(ext) / math.sqrt(2.0) * (1 - 1e-15)
            mid = (tree.lo[c][d] + tree.hi[c][d]) * 0.5
            # every child lies entirely on one side of the midpoint
            for k in ch:
                side = pts[d, tree.perm[tree.begin[k]:tree.end[k]]] >= mid
                assert side.all() or (~side).all()


def test_tree_keeps_input_order_in_leaves():
    pts, _, _ = W.make_problem("uniform", 4000, seed=3)
    tree = O.build_tree(pts, 60)
    for c in tree.leaves():
        seg = tree.perm[tree.begin[c]:tree.end[c]]
        assert np.all(np.diff(seg) > 0)


def _coverage(tt, st, lists):
    m = tt.perm.size
    n = st.perm.size
    cover = np.zeros((m, n), dtype=np.int32)
    for typ in range(4):
        for t, s in lists[typ]:
            cover[tt.begin[t]:tt.end[t], st.begin[s]:st.end[s]] += 1
    return cover


@pytest.mark.parametrize("theta,n,M0,N0", [(0.5, 1, 12, 9), (0.7, 2, 20, 20), (0.9, 1, 5, 30),
                                           (0.0, 3, 25, 25), (0.8, 4, 200, 7)])
def test_dtt_covers_every_pair_exactly_once(theta, n, M0, N0):
    tgt, src, _ = W.make_problem("uniform", 400, 330, seed=5, sources_kind="plummer")
    tt = O.build_tree(tgt, M0)
    st = O.build_tree(src, N0)
    lists = O.dual_tree_traversal(tt, st, n, theta)
    cover = _coverage(tt, st, lists)
    assert cover.min() == 1 and cover.max() == 1


def test_dtt_entry_rules():
    tgt, src, _ = W.make_problem("sphere", 1500, 1200, seed=8, sources_kind="uniform")
    n, theta = 2, 0.75
    n_p = (n + 1) ** 3
    tt = O.build_tree(tgt, 15)
    st = O.build_tree(src, 15)
    lists = O.dual_tree_traversal(tt, st, n, theta)
    assert all(len(l) > 0 for l in lists)
    for typ, want in [(O.CC, (True, True)), (O.CP, (True, False)), (O.PC, (False, True))]:
        for t, s in lists[typ]:
            assert O.well_separated(tt, t, st, s, theta)
            assert (tt.count(t) > n_p, st.count(s) > n_p) == want
    for t, s in lists[O.PP]:
        if O.well_separated(tt, t, st, s, theta):
            assert tt.count(t) <= n_p and st.count(s) <= n_p
        else:
            assert tt.is_leaf(t) and st.is_leaf(s)


def test_mac_is_strict_and_uses_half_diagonal():
    # two unit cubes whose centres are 4 apart: r_t + r_s = sqrt(3) ~ 1.732
    a = np.array([[0, 1], [0, 1], [0, 1]], dtype=np.float64)
    b = a + np.array([[4.0], [0.0], [0.0]])
    ta = O.build_tree(a, 5)
    tb = O.build_tree(b, 5)
    ratio = math.sqrt(3.0) / 4.0
    assert O.well_separated(ta, 0, tb, 0, ratio * 1.0000001)
    assert not O.well_separated(ta, 0, tb, 0, ratio * 0.9999999)


def test_theta_zero_gives_only_leaf_pp():
    pts, _, _ = W.make_problem("uniform", 900, seed=2)
    tt = O.build_tree(pts, 30)
    lists = O.dual_tree_traversal(tt, tt, 4, 0.0)
    assert len(lists[O.PC]) == len(lists[O.CP]) == len(lists[O.CC]) == 0
    leaves = tt.leaves()
    assert len(lists[O.PP]) == len(leaves) ** 2


def _dtt_examples():
    with open(os.path.join(os.path.dirname(GOLDEN), "dtt_examples.json")) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _dtt_examples(), ids=lambda e: e["name"])
def test_dtt_hand_worked_examples(ex):
    """Alg. 2 at its decision points (MAC tie, type thresholds at |C| = n_p,
    equal counts), against lists worked out by hand."""
    tt = O.build_tree(np.array(ex["targets"], dtype=np.float64), ex["M0"])
    st = O.build_tree(np.array(ex["sources"], dtype=np.float64), ex["N0"])
    lists = O.dual_tree_traversal(tt, st, ex["n"], ex["theta"])
    for typ, name in enumerate(O.TYPE_NAMES):
        assert sorted(map(list, lists[typ])) == sorted(ex["lists"][name]), name


@pytest.mark.parametrize("ex", _dtt_examples(), ids=lambda e: e["name"])
def test_interaction_counts_hand_worked(ex):
    """Kernel evaluations per list type (PP |C_t||C_s|, PC |C_t| n_p, CP
    n_p |C_s|, CC n_p^2 per entry; Eqs. (6), (8), (12), (15)) against the
    counts worked out by hand for the Alg. 2 examples."""
    assert interaction_count_mismatches(ex, O.interaction_counts) == []


def interaction_count_mismatches(ex, counts_fn):
    tt = O.build_tree(np.array(ex["targets"], dtype=np.float64), ex["M0"])
    st = O.build_tree(np.array(ex["sources"], dtype=np.float64), ex["N0"])
    lists = O.dual_tree_traversal(tt, st, ex["n"], ex["theta"])
    got = counts_fn(tt, st, lists, ex["n"])
    return [(name, got[k], ex["counts"][name]) for k, name in enumerate(O.TYPE_NAMES)
            if got[k] != ex["counts"][name]]


def evaluations_performed(monkeypatch, t, s, q, **kw):
    """Runs the oracle BLDTT with its kernel evaluator instrumented and
    returns (counted evaluations, the counts the result reports).  Only the
    interaction sums evaluate G, so the instrumented total is the number of
    kernel evaluations the four sums really make."""
    from oracle import bldtt_oracle as Bo
    seen = [0]
    orig = Bo.kernel_values

    def counting(kernel, kappa, dx, dy, dz):
        seen[0] += np.asarray(dx).size
        return orig(kernel, kappa, dx, dy, dz)

    monkeypatch.setattr(Bo, "kernel_values", counting)
    res = Bo.bldtt(t, s, q, **kw)
    return seen[0], res.counts


@pytest.mark.parametrize("theta,n,leaf", [(0.0, 2, 30), (0.7, 2, 30), (0.8, 1, 12)])
def test_interaction_counts_equal_evaluations_performed(monkeypatch, theta, n, leaf):
    """Brute force: the reported counts sum to the evaluations the oracle's
    interaction sums perform, on unequal target and source sets where all
    four list types occur (theta = 0: only PP, M N evaluations)."""
    t, s, q = W.make_problem("uniform", 1000, 1200, seed=12, sources_kind="plummer")
    performed, counts = evaluations_performed(monkeypatch, t, s, q, n=n, theta=theta,
                                              N0=leaf, M0=leaf)
    assert performed == sum(counts)
    if theta == 0.0:
        assert counts[0] == t.shape[1] * s.shape[1] and sum(counts[1:]) == 0
    else:
        assert all(c > 0 for c in counts), counts
