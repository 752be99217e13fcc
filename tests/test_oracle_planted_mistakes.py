"""Planted mistakes: each test breaks one step of the oracle (on the CPU, via
monkeypatch) and checks that an independent pin notices.  This shows the pins
constrain the oracle, not only that the oracle passes them."""
import numpy as np
import pytest

import oracle as O
from oracle import bldtt_oracle as B
from paper_2012_06925_gb300 import workloads as W


def _poly_exact_error():
    tgt, src, q = W.make_problem("uniform", 1200, 1100, seed=6, sources_kind="plummer")
    ref = O.direct_sum(tgt, src, q, O.TEST_POLY)
    res = O.bldtt(tgt, src, q, kernel=O.TEST_POLY, n=2, theta=0.7, N0=15, M0=15)
    return O.relative_l2_error(ref, res.phi)


def test_clean_oracle_reproduces_poly_kernel():
    assert _poly_exact_error() <= 1e-12


def test_printed_denominator_typo_is_caught(monkeypatch):
    """Eq. (3) as printed uses w_k (not w_k') inside the sum."""
    def typo(x, nodes, weights):
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        d = x[None, :] - np.asarray(nodes)[:, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            terms = np.asarray(weights)[:, None] / d
            denom = np.asarray(weights)[:, None] * (1.0 / d).sum(axis=0)[None, :]
            return terms / denom
    nodes = O.box_nodes(-1.0, 1.0, 6)
    x = np.linspace(-0.93, 0.97, 11)
    ref = O.lagrange_1d_product_form(x, nodes)
    assert np.max(np.abs(typo(x, nodes, O.chebyshev_weights(6)) - ref)) > 1e-3


def test_sign_dropped_from_weights_is_caught(monkeypatch):
    monkeypatch.setattr(B, "chebyshev_weights", lambda n: np.abs(O.chebyshev_points(n) * 0 + 1.0))
    nodes = O.box_nodes(-1.0, 1.0, 5)
    x = np.linspace(-0.9, 0.9, 13)
    L = B.lagrange_1d(x, nodes, B.chebyshev_weights(5))
    assert np.max(np.abs(L - O.lagrange_1d_product_form(x, nodes))) > 1e-3


def test_transposed_child_to_parent_matrix_is_caught(monkeypatch):
    orig = B.child_to_parent_matrices
    monkeypatch.setattr(B, "child_to_parent_matrices",
                        lambda tree, par, ch, n: [U.T for U in orig(tree, par, ch, n)])
    _, src, q = W.make_problem("plummer", 10, 1500, seed=4, sources_kind="plummer")
    st = B.build_tree(src, 40)
    ys, qs = src[:, st.perm], q[st.perm]
    qhat = B.upward_pass(st, 3, ys, qs)
    worst = max(np.max(np.abs(qhat[c] - B.proxy_charges_direct(st, c, 3, ys, qs)))
                for c in range(st.num_clusters))
    assert worst > 1e-6


def test_dropped_cc_term_is_caught(monkeypatch):
    monkeypatch.setattr(B, "interact_cc", lambda kernel, kappa, tt, t, st, s, n, qhat: np.zeros((n + 1) ** 3))
    assert _poly_exact_error() > 1e-6


def test_wrong_separation_sign_is_caught(monkeypatch):
    """d = y - x instead of x - y flips the odd terms of the test kernel."""
    orig = B.kernel_values
    monkeypatch.setattr(B, "kernel_values",
                        lambda kernel, kappa, dx, dy, dz: orig(kernel, kappa, -np.asarray(dx),
                                                               -np.asarray(dy), -np.asarray(dz)))
    t = np.array([[0.0], [0.0], [0.0]])
    s = np.array([[1.0], [0.0], [0.0]])
    got = B.direct_sum(t, s, np.array([1.0]), O.TEST_POLY)[0]
    # d = x - y = (-1, 0, 0): G = 1 - 1 = 0
    assert got != 0.0


def test_non_strict_leaf_rule_is_caught(monkeypatch):
    """Reading R4 (leaf iff |C| <= M0): a '<' rule changes the hand-worked tree."""
    orig = B.split_plan
    monkeypatch.setattr(B, "split_plan",
                        lambda lo, hi, count, m: orig(lo, hi, count + 1, m))
    pts = np.array([[3, 0, 4, 1, 2], [0] * 5, [0] * 5], dtype=np.float64)
    tree = B.build_tree(pts, 2)
    assert tree.num_clusters != 5


def test_swapped_downward_operands_are_caught(monkeypatch):
    orig = B.parent_to_child
    def swapped(tree, par, ch, n, phit_par):
        D1, D2, D3 = B.child_to_parent_matrices(tree, par, ch, n)
        return np.einsum("ai,bj,ck,abc->ijk", D2, D1, D3, phit_par)
    monkeypatch.setattr(B, "parent_to_child", swapped)
    assert _poly_exact_error() > 1e-8


# ---- Alg. 2's decision points, against the hand-worked lists -------------

def _dtt_example(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "dtt_examples.json")
    with open(path) as f:
        ex = {e["name"]: e for e in json.load(f)["examples"]}[name]
    tt = B.build_tree(np.array(ex["targets"], dtype=np.float64), ex["M0"])
    st = B.build_tree(np.array(ex["sources"], dtype=np.float64), ex["N0"])
    return ex, tt, st


def _lists_match(ex, tt, st):
    lists = B.dual_tree_traversal(tt, st, ex["n"], ex["theta"])
    return all(sorted(map(list, lists[k])) == sorted(ex["lists"][nm])
               for k, nm in enumerate(B.TYPE_NAMES))


def test_non_strict_mac_is_caught(monkeypatch):
    ex, tt, st = _dtt_example("mac_tie_is_not_separated")
    assert _lists_match(ex, tt, st)
    def non_strict(tt_, t, st_, s, theta):
        ct, cs = tt_.center(t), st_.center(s)
        R = float(np.sqrt(sum((a - b) ** 2 for a, b in zip(ct, cs))))
        return tt_.radius(t) + st_.radius(s) <= theta * R
    monkeypatch.setattr(B, "well_separated", non_strict)
    assert not _lists_match(ex, tt, st)


@pytest.mark.parametrize("name", ["eight_points_against_n_p_eight_is_pp",
                                  "nine_sources_against_eight_targets_is_pc",
                                  "nine_targets_against_eight_sources_is_cp"])
def test_non_strict_type_threshold_is_caught(monkeypatch, name):
    """|C| >= n_p in place of |C| > n_p (planted by counting one particle more
    after the trees are built)."""
    ex, tt, st = _dtt_example(name)
    assert _lists_match(ex, tt, st)
    orig = B.Tree.count
    monkeypatch.setattr(B.Tree, "count", lambda self, c: orig(self, c) + 1)
    assert not _lists_match(ex, tt, st)


def test_splitting_the_target_on_equal_counts_is_caught():
    """Split the target iff |C_s| <= |C_t| (planted: the target tree reports
    one particle more, which only changes the equal-count decision here)."""
    ex, tt, st = _dtt_example("equal_counts_split_the_source")
    assert _lists_match(ex, tt, st)
    orig = tt.count
    tt.count = lambda c: orig(c) + 1
    assert not _lists_match(ex, tt, st)


# ---- kernels, interactions and the upward pass ------------------------------

def test_flipped_yukawa_exponent_is_caught(monkeypatch):
    orig = B.kernel_values
    monkeypatch.setattr(B, "kernel_values",
                        lambda kernel, kappa, dx, dy, dz: orig(kernel, -kappa if kernel == B.YUKAWA
                                                               else kappa, dx, dy, dz))
    # one unit charge at distance 1, kappa = ln 2: exp(-ln 2)/1 = 1/2 (the closed-form pin)
    got = B.direct_sum(np.zeros((3, 1)), np.array([[1.0], [0.0], [0.0]]), np.array([1.0]),
                       B.YUKAWA, np.log(2.0))[0]
    assert abs(got - 0.5) > 0.1     # exp(+ln 2)/1 = 2


@pytest.mark.parametrize("term", ["interact_pc", "interact_cp"])
def test_dropped_pc_or_cp_term_is_caught(monkeypatch, term):
    tgt, src, q = W.make_problem("uniform", 1200, 1100, seed=6, sources_kind="plummer")
    res = O.bldtt(tgt, src, q, kernel=O.TEST_POLY, n=2, theta=0.7, N0=15, M0=15)
    assert len(res.lists[B.PC if term == "interact_pc" else B.CP]) > 0
    orig = getattr(B, term)
    monkeypatch.setattr(B, term, lambda *a: np.zeros_like(orig(*a)))
    assert _poly_exact_error() > 1e-6


def test_mixed_up_dimension_in_upward_leaf_is_caught(monkeypatch):
    """Eq. (9) with the y factor evaluated at x: the first moments in y no
    longer match the particles'."""
    _, src, q = W.make_problem("plummer", 10, 1500, seed=4, sources_kind="plummer")
    st = B.build_tree(src, 40)
    ys, qs = src[:, st.perm], q[st.perm]
    orig = B.tensor_basis
    monkeypatch.setattr(B, "tensor_basis",
                        lambda tree, c, n, px, py, pz: orig(tree, c, n, px, px, pz))
    n = 3
    with np.errstate(all="ignore"):    # x far outside a leaf's y interval may overflow
        qhat = B.upward_pass(st, n, ys, qs)
        worst = 0.0
        for c in st.leaves():
            b, e = st.begin[c], st.end[c]
            _, gy, _ = B.proxy_grid(st, c, n)
            diff = abs((gy * qhat[c].ravel()).sum() - (ys[1, b:e] * qs[b:e]).sum())
            worst = max(worst, diff if np.isfinite(diff) else np.inf)
    assert worst > 1e-6


# ---- learned-selector features and the interaction counts -------------------

def _mutant_features(mistake):
    """pair_features with one planted mistake."""
    from oracle import learned as Lm

    def f(tt, t, st, s, kappa):
        out = Lm.pair_features(tt, t, st, s, kappa)
        if mistake == "non_strict_separation":
            ct, cs = np.array(tt.center(t)), np.array(st.center(s))
            R = float(np.sqrt(((ct - cs) ** 2).sum()))
            if out is None and R > 0 and (tt.radius(t) + st.radius(s)) / R <= 1.0:
                kr = kappa * R
                return np.array([Lm.plog2(tt.count(t)) / 16, Lm.plog2(st.count(s)) / 16,
                                 tt.radius(t) / R, st.radius(s) / R,
                                 (tt.radius(t) + st.radius(s)) / R, kr / (1 + kr)])
            return out
        if out is None:
            return None
        out = out.copy()
        if mistake == "swapped_radii":
            out[2], out[3] = out[3], out[2]
        elif mistake == "source_count_twice":
            out[0] = out[1]
        elif mistake == "kappa_feature_without_r":
            ct, cs = np.array(tt.center(t)), np.array(st.center(s))
            R = float(np.sqrt(((ct - cs) ** 2).sum()))
            out[5] = kappa / (1.0 + kappa * R)
        return out
    return f


@pytest.mark.parametrize("mistake", ["swapped_radii", "source_count_twice",
                                     "kappa_feature_without_r", "non_strict_separation"])
def test_pair_feature_mistakes_are_caught(mistake):
    from test_oracle_learned import pair_feature_mismatches
    from oracle import learned as Lm
    assert pair_feature_mismatches(Lm.pair_features) == []
    assert pair_feature_mismatches(_mutant_features(mistake)) != []


_counts = B.interaction_counts


def _counts_pc_by_source(tt, st, lists, n):
    pp, pc, cp, cc = _counts(tt, st, lists, n)
    n_p = (n + 1) ** 3
    return pp, sum(n_p * st.count(s) for t, s in lists[B.PC]), cp, cc


def _counts_cp_by_target(tt, st, lists, n):
    pp, pc, cp, cc = _counts(tt, st, lists, n)
    n_p = (n + 1) ** 3
    return pp, pc, sum(tt.count(t) * n_p for t, s in lists[B.CP]), cc


def _counts_cc_by_particles(tt, st, lists, n):
    pp, pc, cp, cc = _counts(tt, st, lists, n)
    return pp, pc, cp, sum(tt.count(t) * st.count(s) for t, s in lists[B.CC])


@pytest.mark.parametrize("mutant", [_counts_pc_by_source, _counts_cp_by_target,
                                    _counts_cc_by_particles])
def test_interaction_count_mistakes_are_caught(monkeypatch, mutant):
    """PC counted as n_p |C_s|, CP as |C_t| n_p or CC as |C_t||C_s| fails the
    hand-worked counts and the instrumented evaluation count."""
    from test_oracle_tree_dtt import (_dtt_examples, evaluations_performed,
                                      interaction_count_mismatches)
    assert any(interaction_count_mismatches(ex, mutant) for ex in _dtt_examples())
    monkeypatch.setattr(B, "interaction_counts", mutant)
    tgt, src, q = W.make_problem("uniform", 1000, 1200, seed=12, sources_kind="plummer")
    performed, counts = evaluations_performed(monkeypatch, tgt, src, q, n=2, theta=0.7,
                                              N0=30, M0=30)
    assert performed != sum(counts)
