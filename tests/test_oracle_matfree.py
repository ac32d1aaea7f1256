"""Pins of the quadrature-point matrix-free oracle (oracle/matfree.py): for
element-constant coefficients it must give the Galerkin operator, so it is checked
against the DoGIP oracle (exact rational B^ on the lattice W nodes, exact W-basis
integrals: a route that shares neither the rule nor the basis construction) and
against the assembled CSR matrix, on jittered meshes with tensor coefficients.
A mistake in the rule size, a transposed J^-1 or a dropped weight fails here."""

import numpy as np
import pytest

from oracle import assembly, dogip as odogip, matfree, quadrature
from paper_1710_09913_gb300 import inputs

CASES = [(2, p, f) for p in (1, 2, 3, 4) for f in ("elliptic", "projection")] + \
        [(3, p, f) for p in (1, 2, 3) for f in ("elliptic", "projection")]


def _problem(d, p, form, seed=3):
    coords, cells = inputs.lattice_mesh(d, 3 if d == 2 else 2, 0.2 if d == 2 else 0.1, seed)
    E = len(cells)
    coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed) if form == "elliptic" else \
        inputs.coef_uniform(E, 1.0, 10.0, seed)
    return coords, cells, coef, odogip.Problem(form, p, coords, cells, coef)


@pytest.mark.parametrize("d,p,form", CASES)
def test_matfree_equals_dogip(d, p, form):
    coords, cells, coef, P = _problem(d, p, form)
    u = inputs.rhs_normal(P.n, 2, seed=11)
    y = matfree.apply(form, p, coords, cells, coef, P.conn, u, P.bmask)
    scale = matfree.apply(form, p, coords, cells, coef, P.conn, u, P.bmask, absolute=True)
    assert np.all(np.abs(y - P.apply(u)) <= 1e-12 * scale)


@pytest.mark.parametrize("d,p,form", [(2, 3, "elliptic"), (2, 2, "projection"), (3, 2, "elliptic")])
def test_matfree_equals_assembled(d, p, form):
    coords, cells, coef, P = _problem(d, p, form, seed=4)
    K = assembly.assemble(form, p, coords, cells, P.conn, P.n, coef)
    if P.bmask is not None:
        K = assembly.dirichlet(K, P.bmask)
    u = inputs.rhs_normal(P.n, 1, seed=12)[:, 0]
    y = matfree.apply(form, p, coords, cells, coef, P.conn, u, P.bmask)
    np.testing.assert_allclose(y, K @ u, rtol=0, atol=1e-12 * np.abs(K).dot(np.abs(u)).max())


@pytest.mark.parametrize("form,p,n", [("elliptic", 1, 1), ("elliptic", 4, 4), ("projection", 1, 2),
                                      ("projection", 3, 4)])
def test_rule_size_is_minimal_and_exact(form, p, n):
    """n points per direction: the rule integrates the integrand's degree exactly and
    n - 1 points do not (the monomial x^(2n-1) of degree 2n - 1 in 2D)."""
    assert matfree.points_per_direction(form, p) == n
    deg = 2 * p if form == "projection" else 2 * p - 2
    assert 2 * n - 1 >= deg
    if n > 1:
        assert 2 * (n - 1) - 1 < deg
    pts, w = quadrature.simplex_rule(2, n)
    # int_T x^a y^b = a! b! / (a + b + 2)!
    from math import factorial
    for a in range(deg + 1):
        b = deg - a
        exact = factorial(a) * factorial(b) / factorial(a + b + 2)
        assert abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b) - exact) <= 1e-15


def test_matfree_mistake_is_caught():
    """A transposed J^-1 (a plausible slip) breaks the equality with the DoGIP oracle
    on a sheared mesh, so the pin above would catch it."""
    coords, cells, coef, P = _problem(2, 2, "elliptic")
    u = inputs.rhs_normal(P.n, 1, seed=13)[:, 0]
    _, det, Rinv = odogip.geometry(coords, cells)
    Bq, wq = matfree.tables("elliptic", 2, 2)
    G_bad = np.einsum("esi,iql->eqsl", Rinv, Bq)  # R^-1 grad^ instead of R^-T grad^
    uT = np.where(P.bmask, 0.0, u)[P.conn]
    gu = np.einsum("eqsl,el->eqs", G_bad, uT)
    flux = np.einsum("est,eqt->eqs", coef, gu) * (np.abs(det)[:, None, None] * wq[None, :, None])
    Y = np.einsum("eqsl,eqs->el", G_bad, flux)
    y_bad = np.zeros(P.n)
    np.add.at(y_bad, P.conn, Y)
    y_bad = np.where(P.bmask, u, y_bad)
    scale = matfree.apply("elliptic", 2, coords, cells, coef, P.conn, u, P.bmask, absolute=True)
    assert np.any(np.abs(y_bad - P.apply(u)) > 1e-6 * scale)
