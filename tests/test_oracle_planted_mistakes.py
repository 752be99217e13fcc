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
