"""Pins of the Lagrange-node oracle (Appendix, STEP1-STEP5, Eq. 1-2; Sec. 2.2.1) to facts
other than itself: Lagrange interpolation's exactness on polynomials (Eq. 1) and its closed-form
remainder, the exact change of basis of STEP4, closed-form potentials of charges on the vertices
of a square and a cube, and the exactness of both FMM forms when the kernel is a polynomial of
degree < 4 per axis (then the node approximation of Eq. 2 makes no error at all)."""
import math

import numpy as np
import pytest

from paper_2009_00767_gb300 import inputs

A = np.array([-2.0, -1.0, 1.0, 2.0])


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.set_threads(4)
    return oracle


# ---------------------------------------------------------------- Eq. 1: Lagrange interpolation

def test_basis_is_cardinal(orc):
    for j, a in enumerate(A):
        w = orc.lag_weights1(a)
        assert np.array_equal(w, np.eye(4)[j])


@pytest.mark.parametrize("x", [-37.5, -2.2, -0.3, 0.0, 0.71, 1.5, 2.0, 9.0, 41.0])
def test_polynomials_below_degree_four_are_reproduced(orc, x):
    w = orc.lag_weights1(x)
    for deg in range(4):
        # rounding: about eps times the sum of the magnitudes of the terms
        tol = 1e-14 * (np.abs(w) @ np.abs(A) ** deg + abs(x) ** deg)
        assert abs(w @ A ** deg - x ** deg) <= tol


@pytest.mark.parametrize("x", [-37.5, -0.3, 0.71, 2.6, 41.0])
def test_remainder_of_degree_four_is_the_node_polynomial(orc, x):
    # sum_i f_i(x) a_i^4 - x^4 = -prod_i (x - a_i): the interpolant of a monic degree-4 polynomial
    w = orc.lag_weights1(x)
    omega = np.prod(x - A)
    tol = 1e-14 * (np.abs(w) @ A ** 4 + x ** 4 + abs(omega))
    assert abs((w @ A ** 4 - x ** 4) - (-omega)) <= tol


@pytest.mark.parametrize("dim", [2, 3])
def test_node_weights_reproduce_cubics_per_axis(orc, dim):
    # STEP2's tensor-product weights: sum_j w_j g(node_j) = g(pos) for g of degree <= 3 per axis
    rng = np.random.default_rng(3)
    level, box = 3, 5.0
    s = box / 2 ** level
    for _ in range(5):
        cell = rng.integers(0, 2 ** level, size=dim)
        pos = (cell + rng.random(dim)) * s
        w = orc.lag_weights(dim, level, cell, pos, box)
        idx = np.indices((4,) * dim).reshape(dim, -1)[::-1]          # node j = i + 4 j' + 16 k
        nodes = (cell[:, None] + 0.5) * s + (s / 5.0) * A[idx]
        assert w.sum() == pytest.approx(1.0, abs=1e-12)
        g = lambda p: 1.0 + p[0] ** 3 * p[1] ** 2 - 0.5 * p[1] ** 3 * p[0] + (p[2] ** 3 * p[0] if dim == 3 else 0.0)
        assert w @ g(nodes) == pytest.approx(g(pos), rel=1e-10)
        # degree 4 in one axis is not reproduced
        assert abs(w @ nodes[0] ** 4 - pos[0] ** 4) > 1e-8 * s ** 4


# ---------------------------------------------------------------- STEP4: M_m h_{m^0}(c) = h_m(c)

@pytest.mark.parametrize("dim,level", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_change_of_basis_is_exact(orc, dim, level):
    rng = np.random.default_rng(10 + level)
    box = 5.0
    s = box / 2 ** level
    for _ in range(4):
        cell = rng.integers(0, 2 ** level, size=dim)
        pos = (cell + rng.random(dim)) * s
        M = orc.lag_matrix_M(dim, level, cell, box)
        w0 = orc.lag_weights(dim, 0, np.zeros(dim, np.int32), pos, box)
        wm = orc.lag_weights(dim, level, cell, pos, box)
        assert np.max(np.abs(M @ w0 - wm)) < 1e-12 * np.abs(M).max() * 10


# ---------------------------------------------------------------- the direct sums: closed forms

def test_direct_3d_cube_vertices(orc):
    a = 0.7
    v = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float)
    pos = 1.0 + a * v
    ones = np.ones(8)
    same = 3 / a + 3 / (a * math.sqrt(2)) + 1 / (a * math.sqrt(3))
    assert np.allclose(orc.lag_direct(pos, ones), same, rtol=1e-14)
    par = (-1.0) ** v.sum(axis=1)          # rock-salt signs: edges opposite, face diagonals equal
    alt = -3 / a + 3 / (a * math.sqrt(2)) - 1 / (a * math.sqrt(3))
    assert np.allclose(orc.lag_direct(pos, par), par * alt, rtol=1e-14)


def test_direct_2d_square_vertices(orc):
    a = 0.9
    pos = 2.0 + a * np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)
    assert np.allclose(orc.lag_direct(pos, np.ones(4)), 2 * math.log(a) + math.log(a * math.sqrt(2)), rtol=1e-14)


def test_direct_targets_is_a_subset(orc):
    pos, q = inputs.paper_cube(700, 4, 3)
    t = np.array([0, 5, 699, 350])
    assert np.array_equal(orc.lag_direct_targets(pos, q, t), orc.lag_direct(pos, q)[t])


# ---------------------------------------------------------------- both forms: exact on polynomials

POLY_CASES = [(2, 2, 600), (2, 3, 2500), (2, 4, 4000), (3, 2, 1500), (3, 3, 3000)]


@pytest.mark.parametrize("dim,levels,n", POLY_CASES)
def test_node_form_is_exact_for_a_polynomial_kernel(orc, dim, levels, n):
    pos, q = inputs.paper_cube(n, 100 + levels, dim)
    d = orc.lag_direct(pos, q, kernel=1)
    assert rel(orc.lag_node(pos, q, levels, kernel=1), d) < 1e-13


@pytest.mark.parametrize("dim,levels,n", [(2, 2, 600), (2, 3, 2500), (3, 2, 1500)])
def test_literal_form_is_exact_for_a_polynomial_kernel(orc, dim, levels, n):
    pos, q = inputs.paper_cube(n, 200 + levels, dim)
    d = orc.lag_direct(pos, q, kernel=1)
    assert rel(orc.lag_literal(pos, q, levels, kernel=1), d) < 1e-9


def test_polynomial_pin_on_clustered_charges(orc):
    xy, q = inputs.gmm(3000, 77, k=6, sigma_lo=0.05, sigma_hi=0.4)
    d = orc.lag_direct(xy, q, kernel=1)
    assert rel(orc.lag_node(xy, q, 4, kernel=1), d) < 1e-13
    assert rel(orc.lag_literal(xy, q, 3, kernel=1), d) < 1e-9


@pytest.mark.parametrize("form", ["lag_node", "lag_literal"])
@pytest.mark.parametrize("skip", [2, 3])
def test_a_dropped_level_is_caught(orc, form, skip):
    pos, q = inputs.paper_cube(2500, 9, 2)
    d = orc.lag_direct(pos, q, kernel=1)
    assert rel(getattr(orc, form)(pos, q, 3, kernel=1, skip_level=skip), d) > 1e-3


def test_levels_below_two_are_the_direct_sum(orc):
    pos, q = inputs.paper_cube(800, 12, 3)
    d = orc.lag_direct(pos, q)
    for levels in (0, 1):
        assert rel(orc.lag_node(pos, q, levels), d) < 1e-14
        assert rel(orc.lag_literal(pos, q, levels), d) < 1e-14


# ---------------------------------------------------------------- the physical kernels

@pytest.mark.parametrize("dim,levels,n", [(2, 3, 3000), (2, 4, 6000), (3, 2, 3000), (3, 3, 4000)])
def test_method_error_is_small(orc, dim, levels, n):
    # 4 nodes per axis: the approximation error of Eq. 2 for well-separated squares is about 1e-4
    # to 1e-3 of the potential (the paper's Tables 1-3 report averaged relative errors of 1e-3)
    pos, q = inputs.paper_cube(n, 300 + levels, dim)
    err = rel(orc.lag_node(pos, q, levels), orc.lag_direct(pos, q))
    assert 1e-6 < err < 1e-3


def test_literal_equals_node_where_fp64_holds(orc):
    for dim, levels, n in [(2, 2, 1000), (2, 3, 3000), (3, 2, 2000)]:
        pos, q = inputs.paper_cube(n, 400 + levels, dim)
        assert rel(orc.lag_literal(pos, q, levels), orc.lag_node(pos, q, levels)) < 1e-8


def test_literal_form_loses_fp64_digits_with_depth(orc):
    # Sec. 4 Discussion (3): the entries of M_m grow like (2^k)^(3 D) and B = M^T M_b M is formed
    # from them, so the literal form's FP64 rounding grows with the level while the node form's
    # does not: at level 6 in 2D the literal result is dominated by rounding.
    pos, q = inputs.paper_cube(6000, 31, 2)
    d = orc.lag_direct(pos, q)
    node_err = rel(orc.lag_node(pos, q, 6), d)
    lit_err = rel(orc.lag_literal(pos, q, 6), d)
    assert node_err < 1e-3
    assert lit_err > 1e3 * node_err


def test_cells_floor_clamp(orc):
    box, L = 5.0, 3
    pos = np.array([[0.0, 5.0, 2.5], [5.0 / 8 * 3, 5.0 / 8 * 3 - 1e-12, 4.999999]])
    cell = orc.lag_cells(pos, L, box)
    assert cell.tolist() == [[0, 7, 4], [3, 2, 7]]
