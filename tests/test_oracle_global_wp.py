"""Pins of the global (continuous-W) DoGIP oracle for the weighted projection
(oracle/global_wp.py, §2.2): the same Galerkin matrix as the element-wise
decomposition, both bases' partition of unity, continuity of the V basis across
cells (every cell containing a W node gives the owner's row of B), the total of
A_diag equal to int m, and the lattice count of W nodes."""

import numpy as np
import pytest

from oracle import dogip as odogip, global_wp, refelem
from paper_1710_09913_gb300 import inputs

CASES = [(2, p) for p in (1, 2, 3, 4)] + [(3, p) for p in (1, 2, 3)]


def _mesh(d, N, seed=2):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    coef = inputs.coef_uniform(len(cells), 1.0, 10.0, seed)
    return coords, cells, coef


@pytest.mark.parametrize("d,p", CASES)
def test_global_equals_elementwise(d, p):
    coords, cells, coef = _mesh(d, 3 if d == 2 else 2)
    G = global_wp.GlobalProblem(p, coords, cells, coef)
    P = odogip.Problem("projection", p, coords, cells, coef)
    assert G.n == P.n and np.array_equal(G.conn, P.conn)
    u = inputs.rhs_normal(G.n, 2, seed=4)
    assert np.all(np.abs(G.apply(u) - P.apply(u)) <= 1e-13 * P.apply_abs(u))
    np.testing.assert_allclose(G.diag(), P.diag(), rtol=1e-13)


@pytest.mark.parametrize("d,p", CASES)
def test_identities(d, p):
    coords, cells, coef = _mesh(d, 3 if d == 2 else 2, seed=5)
    G = global_wp.GlobalProblem(p, coords, cells, coef)
    N = 3 if d == 2 else 2
    assert G.nW == (2 * p * N + 1) ** d                       # lattice count of C_{N,2p}
    np.testing.assert_allclose(np.asarray(G.B.sum(axis=1)).ravel(), 1.0, atol=1e-14)  # sum_j phi_j = 1
    _, det, _ = odogip.geometry(coords, cells)
    mass = np.sum(coef * np.abs(det)) / (2 if d == 2 else 6)  # int m = sum m_T |T|
    assert abs(G.A.sum() - mass) <= 1e-13 * mass
    assert G.own.sum() == G.nW and np.all(G.own.sum(axis=0) >= 0)


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2)])
def test_rows_are_continuous_across_cells(d, p):
    """phi_V^j(x_W^i) does not depend on which cell containing x_W^i evaluates it."""
    coords, cells, coef = _mesh(d, 3 if d == 2 else 2, seed=6)
    G = global_wp.GlobalProblem(p, coords, cells, coef)
    Bh = refelem.bhat("projection", d, p)
    Bd = G.B.toarray()
    for e in range(len(cells)):
        for j in range(G.connW.shape[1]):
            row = np.zeros(G.n)
            row[G.conn[e]] = Bh[j]
            assert np.abs(Bd[G.connW[e, j]] - row).max() <= 1e-14


def test_memory_of_the_global_variant():
    """The remark after Tables 1-2: the global A_diag stores one value per W node
    against W_T per cell; on the 512 x 512 lattice at k = 1 that is 3x less."""
    N, p = 512, 1
    E = 2 * N * N
    nW = (2 * p * N + 1) ** 2
    WT = refelem.dim_P(2, 2 * p)
    assert WT == 6 and E * WT / nW > 2.9


def test_planted_mistake_is_caught():
    """Scaling by the element-wise W_T weights without summing over shared nodes
    (dropping the continuity) breaks the equality with the element-wise oracle."""
    coords, cells, coef = _mesh(2, 3, seed=7)
    G = global_wp.GlobalProblem(2, coords, cells, coef)
    P = odogip.Problem("projection", 2, coords, cells, coef)
    bad = np.zeros(G.nW)
    _, det, _ = odogip.geometry(coords, cells)
    w = refelem.what(2, 4)
    vals = (coef * np.abs(det))[:, None] * w[None, :]
    bad[G.connW[G.own]] = vals[G.own]  # owner's share only
    u = inputs.rhs_normal(G.n, 1, seed=8)[:, 0]
    y_bad = G.B.T @ (bad * (G.B @ u))
    assert np.any(np.abs(y_bad - P.apply(u)) > 1e-6 * P.apply_abs(u))
