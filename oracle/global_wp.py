"""Global DoGIP for the weighted projection (§2.2, Theorem "DoGIP for weighted
projection" and the double-grid lemma before it), plain FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and bench.py's CPU
baseline leg; the product path never calls it.

With V = C_{N,k} and the continuous double-grid space W = C_{N,2k}:
  K u . v = B^* A_diag B u . v,   B_ij = phi_V^j(x_W^i)  (W x V),
  A_diag,ii = int_Omega m phi_W^i,
so one apply interpolates u at every global W node once, scales by the diagonal, and
applies the adjoint.  For element-constant m, int_Omega m phi_W^i is the sum over the
cells containing node i of m_T |det R_T| w^_j (w^_j the integral of the reference W
basis function j, as in the element-wise theorem).
W nodes are numbered like the V nodes (first appearance, ``topology.dofmap`` at
order 2k).  Row i of B is taken from the first cell containing node i (its owner);
every other cell containing the node gives the same row (continuity of phi_V), which
is one of the pins.
Parity: pinned against the element-wise DoGIP oracle (an independent decomposition
of the same Galerkin matrix), partition-of-unity identities of both bases and the
lattice count (2kN+1)^d.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import refelem, topology
from .dogip import geometry


def w_dofmap(cells: np.ndarray, p: int):
    """(connW [E, W_T], nW): the global W nodes of order 2p."""
    return topology.dofmap(np.asarray(cells, dtype=np.int64), 2 * p)


def owners(connW: np.ndarray) -> np.ndarray:
    """[E, W_T] bool: True where the cell is the first to contain the node."""
    flat = connW.reshape(-1)
    _, first = np.unique(flat, return_index=True)
    own = np.zeros(flat.size, dtype=bool)
    own[first] = True
    return own.reshape(connW.shape)


def interp_matrix(p: int, d: int, conn, connW, nW: int, n: int) -> sp.csr_matrix:
    """B (W x V) with B_ij = phi_V^j(x_W^i), rows from the owning cells."""
    Bh = refelem.bhat("projection", d, p)  # [W_T, V_T]: phi_l(x_j) on the reference cell
    own = owners(connW)
    e, j = np.nonzero(own)
    rows = np.repeat(connW[e, j], conn.shape[1])
    cols = conn[e].reshape(-1)
    vals = Bh[j].reshape(-1)
    return sp.coo_matrix((vals, (rows, cols)), shape=(nW, n)).tocsr()


def ahat_global(p: int, coords, cells, coef, connW, nW: int) -> np.ndarray:
    """A_diag,ii = int_Omega m phi_W^i for element-constant m."""
    d = cells.shape[1] - 1
    _, det, _ = geometry(coords, cells)
    w = refelem.what(d, 2 * p)
    A = np.zeros(nW)
    np.add.at(A, connW, (np.asarray(coef, dtype=np.float64) * np.abs(det))[:, None] * w[None, :])
    return A


class GlobalProblem:
    """Oracle data of one global-W weighted projection problem."""

    def __init__(self, p, coords, cells, coef):
        self.p = p
        self.coords = np.asarray(coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.d = self.cells.shape[1] - 1
        self.conn, self.n = topology.dofmap(self.cells, p)
        self.connW, self.nW = w_dofmap(self.cells, p)
        self.own = owners(self.connW)
        self.B = interp_matrix(p, self.d, self.conn, self.connW, self.nW, self.n)
        self.A = ahat_global(p, self.coords, self.cells, coef, self.connW, self.nW)

    def apply(self, u):
        """B^* (A_diag (B u)) for u [n] or [n, R]."""
        u = np.asarray(u, dtype=np.float64)
        Bu = self.B @ u
        return self.B.T @ (self.A[:, None] * Bu if Bu.ndim == 2 else self.A * Bu)

    def apply_abs(self, u):
        """|B|^T |A| |B| |u|: the componentwise rounding scale."""
        Ba = abs(self.B)
        u = np.abs(np.asarray(u, dtype=np.float64))
        Bu = Ba @ u
        return Ba.T @ (np.abs(self.A)[:, None] * Bu if Bu.ndim == 2 else np.abs(self.A) * Bu)

    def diag(self):
        """K_ll = sum_i B_il^2 A_ii."""
        return np.asarray((self.B.multiply(self.B)).T @ self.A).reshape(-1)
