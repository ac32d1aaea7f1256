"""Pins of the oracle's reference element: Lagrange bases (two constructions),
W-basis integrals and the collapsed quadrature."""

from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np
import pytest

from oracle import quadrature, refelem


def _rand_points(d, k, seed):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < k:
        x = [Fraction(int(v), 97) for v in rng.integers(0, 97, size=d)]
        if sum(x) <= 1:
            pts.append(tuple(x))
    return pts


@pytest.mark.parametrize("d,q", [(2, q) for q in range(0, 9)] + [(3, q) for q in range(0, 7)])
def test_dirac_property_silvester(d, q):
    """phi^_l(x^_k) = delta_kl at the equispaced nodes (Section 2.1)."""
    X = refelem.nodes(d, q)
    assert len(X) == refelem.dim_P(d, q)
    for k, x in enumerate(X):
        for l in range(len(X)):
            assert refelem.silvester_value(d, q, l, x) == (1 if k == l else 0)


@pytest.mark.parametrize("d,q", [(2, q) for q in range(1, 5)] + [(3, q) for q in range(1, 4)])
def test_two_constructions_agree(d, q):
    """Silvester product form == nodal Vandermonde solution, values and gradients, exactly."""
    X = refelem.nodes(d, q)
    for k, x in enumerate(X):  # Vandermonde basis is Dirac too
        for l in range(len(X)):
            assert refelem.vandermonde_value(d, q, l, x) == (1 if k == l else 0)
    for x in _rand_points(d, 4, q):
        for l in range(len(X)):
            assert refelem.silvester_value(d, q, l, x) == refelem.vandermonde_value(d, q, l, x)
            assert refelem.silvester_grad(d, q, l, x) == refelem.vandermonde_grad(d, q, l, x)


@pytest.mark.parametrize("d,q", [(2, 3), (2, 4), (3, 2), (3, 3)])
def test_polynomial_reproduction(d, q):
    """sum_l x_l^a phi^_l(x) = x^a and its gradient for every monomial |a| <= q."""
    X = refelem.nodes(d, q)
    for x in _rand_points(d, 3, 7 * q + d):
        for a in refelem.multi_indices(d, q):
            mono = lambda y: np.prod([Fraction(yi) ** ai for yi, ai in zip(y, a)])
            val = sum(mono(X[l]) * refelem.silvester_value(d, q, l, x) for l in range(len(X)))
            assert val == mono(x)
            for r in range(d):
                g = sum(mono(X[l]) * refelem.silvester_grad(d, q, l, x)[r] for l in range(len(X)))
                if a[r] == 0:
                    assert g == 0
                else:
                    b = list(a)
                    b[r] -= 1
                    assert g == a[r] * np.prod([Fraction(yi) ** bi for yi, bi in zip(x, b)])


def test_p1_gradient_table():
    """Elliptic P1 (W = P0): B^ holds the constant reference gradients of the hat
    functions; local order (0,0), (0,1), (1,0) is lambda_0, y^, x^."""
    B = refelem.bhat("elliptic", 2, 1)
    assert B.shape == (2, 1, 3)
    assert B[0, 0].tolist() == [-1, 0, 1]
    assert B[1, 0].tolist() == [-1, 1, 0]
    B3 = refelem.bhat("elliptic", 3, 1)
    assert B3.shape == (3, 1, 4)
    assert B3[:, 0, 0].tolist() == [-1, -1, -1]


@pytest.mark.parametrize("d,q", [(2, q) for q in range(0, 9)] + [(3, q) for q in range(0, 9)])
def test_what_sums_to_measure(d, q):
    """sum_j w^_j = |T^| = 1/d! (partition of unity, Lemma 3 with u = v = 1)."""
    assert sum(refelem.what_exact(d, q)) == Fraction(1, factorial(d))


def test_what_textbook_p2():
    """Quadratic Lagrange integrals: 2D vertex 0, edge |T|/3; 3D vertex -|T|/20, edge |T|/5."""
    w2 = refelem.what_exact(2, 2)
    for a, w in zip(refelem.multi_indices(2, 2), w2):
        beta = (2 - sum(a),) + a
        assert w == (0 if 2 in beta else Fraction(1, 2) / 3)
    w3 = refelem.what_exact(3, 2)
    for a, w in zip(refelem.multi_indices(3, 2), w3):
        beta = (2 - sum(a),) + a
        assert w == (Fraction(-1, 6) / 20 if 2 in beta else Fraction(1, 6) / 5)


@pytest.mark.parametrize("d,q", [(2, 4), (2, 6), (3, 4), (3, 6)])
def test_what_matches_quadrature(d, q):
    """w^ (exact barycentric expansion) == Gauss rule on the Vandermonde basis."""
    pts, w = quadrature.simplex_rule(d, q // 2 + 1)
    val, _ = refelem.vandermonde_eval_float(d, q, pts)
    # the float monomial expansion cancels: ~1e-14 absolute rounding at q = 6
    np.testing.assert_allclose(w @ val, refelem.what(d, q), rtol=0, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_quadrature_exactness(d, n):
    """integral_T^ x^a = a! / (|a| + d)! for total degree <= 2n - 1."""
    pts, w = quadrature.simplex_rule(d, n)
    for a in product(range(2 * n), repeat=d):
        if sum(a) > 2 * n - 1:
            continue
        exact = np.prod([factorial(ai) for ai in a]) / factorial(sum(a) + d)
        got = w @ np.prod(pts ** np.array(a), axis=1)
        assert abs(got - exact) <= 1e-15 * max(1.0, exact) + 1e-16


def test_negative_weights_exist():
    """W-basis integrals can be negative (3D q=2 vertices): A_T is sign-indefinite
    node by node although B^* A_T B^ is positive."""
    assert min(refelem.what_exact(3, 2)) < 0
    assert min(refelem.what_exact(2, 4)) < 0
