"""Pins of the oracle's dof map, boundary set and colouring."""

import numpy as np
import pytest

from oracle import topology
from paper_1710_09913_gb300 import inputs


@pytest.mark.parametrize("d,p,N", [(2, 1, 4), (2, 2, 3), (2, 4, 3), (3, 1, 2), (3, 2, 2), (3, 3, 2)])
def test_dofmap_vectorised_equals_loop(d, p, N):
    _, t = inputs.lattice_mesh(d, N)
    a, na = topology.dofmap(t, p)
    b, nb = topology.dofmap_loop(t, p)
    assert na == nb and np.array_equal(a, b)


@pytest.mark.parametrize("d,p,N", [(2, 1, 5), (2, 3, 4), (2, 4, 3), (3, 2, 3), (3, 3, 2)])
def test_dofs_are_lattice_points(d, p, N):
    """Every global dof is one point of the p-refined lattice: same id <=> same
    point, (pN+1)^d dofs, boundary dofs are those with a coordinate in {0, 1}."""
    c, t = inputs.lattice_mesh(d, N)
    conn, n = topology.dofmap(t, p)
    assert n == (p * N + 1) ** d
    X = topology.node_points(c, t, p)
    L = np.rint(X * p * N).astype(np.int64).reshape(-1, d)
    assert np.allclose(X.reshape(-1, d) * p * N, L, atol=1e-9)
    code = L @ ((p * N + 1) ** np.arange(d))
    ids = conn.reshape(-1)
    # same id -> same point, and same point -> same id
    order = np.argsort(ids)
    first = np.unique(ids[order], return_index=True)[1]
    rep = np.empty(n, dtype=np.int64)
    rep[ids[order][first]] = code[order][first]
    assert np.array_equal(rep[ids], code)
    assert len(np.unique(code)) == n
    bm = topology.boundary_mask(t, conn, p, n)
    onb = np.any((L == 0) | (L == p * N), axis=1)
    assert np.array_equal(bm[ids], onb)
    assert bm.sum() == (p * N + 1) ** d - (p * N - 1) ** d


@pytest.mark.parametrize("d,N", [(2, 1), (2, 6), (3, 1), (3, 3)])
def test_colouring(d, N):
    _, t = inputs.lattice_mesh(d, N)
    col = topology.colouring(t)
    assert topology.colouring_is_greedy(t, col)
    # a plainly wrong colouring fails the property check
    bad = col.copy()
    bad[-1] = col.max() + 1
    assert not topology.colouring_is_greedy(t, bad)
    if len(t) > 1:
        bad = col.copy()
        bad[1] = bad[0]
        shares = len(set(t[0]) & set(t[1])) > 0
        assert topology.colouring_is_greedy(t, bad) == (not shares and bad[1] == col[1])
