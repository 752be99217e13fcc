"""Pins of the oracle's barycentric Lagrange basis (Sec. 2.1, App. A).

Each check compares against something other than the oracle itself: the
textbook product form of the Lagrange polynomials, the general weight formula
of Eq. (3), closed-form Chebyshev points, and exact polynomial reproduction.
"""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 10, 12])
def test_chebyshev_points_closed_form(n):
    s = O.chebyshev_points(n)
    ref = np.cos(np.pi * np.arange(n + 1) / n)
    assert np.max(np.abs(s - ref)) <= 4.5e-16          # a few ulps: the mirror image of cos(pi k/n)
    assert s[0] == 1.0 and s[-1] == -1.0
    assert np.all(s[::-1] == -s)                      # exact symmetry (reading R2)
    assert np.all(np.diff(s) < 0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_weights_match_general_definition(n):
    """Eq. (5) must equal Eq. (3)'s w_k = 1/prod(s_k - s_j) up to one common scale."""
    s = O.chebyshev_points(n)
    w = O.chebyshev_weights(n)
    g = O.general_weights(s)
    ratio = g / w
    assert np.allclose(ratio, ratio[0], rtol=1e-12, atol=0)
    assert np.all(np.sign(w[::2]) > 0) and np.all(np.sign(w[1::2]) < 0)
    assert w[0] == 0.5 and abs(w[-1]) == 0.5


@pytest.mark.parametrize("n", [1, 2, 4, 8, 10])
def test_barycentric_equals_product_form(n):
    rng = np.random.default_rng(n)
    lo, hi = -0.3, 1.7
    nodes = O.box_nodes(lo, hi, n)
    x = rng.uniform(lo - 0.5, hi + 0.5, size=200)
    L = O.lagrange_1d(x, nodes, O.chebyshev_weights(n))
    ref = O.lagrange_1d_product_form(x, nodes)
    assert np.max(np.abs(L - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-12


@pytest.mark.parametrize("n", [1, 3, 8])
def test_partition_of_unity_and_cardinality(n):
    nodes = O.box_nodes(0.25, 0.75, n)
    w = O.chebyshev_weights(n)
    x = np.linspace(0.25, 0.75, 57)
    L = O.lagrange_1d(x, nodes, w)
    assert np.max(np.abs(L.sum(axis=0) - 1.0)) <= 1e-14
    C = O.lagrange_1d(nodes, nodes, w)                # guard fires on every column
    assert np.array_equal(C, np.eye(n + 1))


def test_zero_width_box_puts_weight_on_first_node():
    w = O.chebyshev_weights(4)
    nodes = O.box_nodes(0.3, 0.3, 4)
    L = O.lagrange_1d(np.array([0.3, 0.3]), nodes, w)
    assert np.array_equal(L[:, 0], np.array([1.0, 0, 0, 0, 0]))


@pytest.mark.parametrize("n", [2, 4, 6])
def test_tensor_reproduction_of_polynomials(n):
    """App. A: interpolation of degree n reproduces x^a y^b z^c, a,b,c <= n."""
    rng = np.random.default_rng(7)
    lo = np.array([-0.7, 0.1, -0.2])
    hi = np.array([0.4, 0.9, 0.6])
    w = O.chebyshev_weights(n)
    nodes = [O.box_nodes(lo[d], hi[d], n) for d in range(3)]
    pts = rng.uniform(lo[:, None], hi[:, None], size=(3, 40))
    B = [O.lagrange_1d(pts[d], nodes[d], w) for d in range(3)]
    for a, b, c in [(0, 0, 0), (1, 0, 0), (0, n, 1), (n, n, n), (2, 1, n - 1)]:
        f_nodes = np.einsum("i,j,k->ijk", nodes[0] ** a, nodes[1] ** b, nodes[2] ** c)
        interp = np.einsum("im,jm,km,ijk->m", B[0], B[1], B[2], f_nodes)
        exact = pts[0] ** a * pts[1] ** b * pts[2] ** c
        assert np.max(np.abs(interp - exact)) <= 1e-13 * max(1.0, np.max(np.abs(exact)))


def test_interpolation_error_decreases_with_degree():
    """Chebyshev interpolation of a smooth function converges geometrically."""
    f = lambda x: 1.0 / (2.5 - x)                     # analytic on [-1, 1]
    x = np.linspace(-1, 1, 301)
    errs = []
    for n in [2, 4, 8, 16]:
        nodes = O.chebyshev_points(n)
        L = O.lagrange_1d(x, nodes, O.chebyshev_weights(n))
        errs.append(np.max(np.abs(f(nodes) @ L - f(x))))
    assert all(errs[i + 1] < errs[i] * 0.2 for i in range(3))
    assert errs[-1] < 1e-8


def test_kernel_values_closed_forms():
    g = O.kernel_values(O.COULOMB, 0.0, np.array([2.0, 0.0, 3.0]), np.array([0.0, 0.0, 4.0]),
                        np.array([0.0, 0.0, 0.0]))
    assert np.allclose(g, [0.5, 0.0, 0.2], rtol=1e-15)
    g = O.kernel_values(O.YUKAWA, 0.5, np.array([2.0]), np.array([0.0]), np.array([0.0]))
    assert abs(g[0] - math.exp(-1.0) / 2.0) <= 1e-16
    g = O.kernel_values(O.TEST_POLY, 0.0, np.array([1.0]), np.array([2.0]), np.array([-1.0]))
    # 1 + 1 - 4 - 3 + 2 + 2 + 1 - 2 = -2
    assert g[0] == -2.0
