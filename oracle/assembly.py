"""Conventional assembled matrices (eqs. linsys_gp and linsys_se), computed
independently of the DoGIP factors.

Element matrices by the collapsed Gauss rule of ``quadrature`` with n = p + 1
points per direction (exact to degree 2p + 1 >= 2p, the degree of the integrands
m u v and M grad u . grad v for element-wise constant coefficients), with the
basis from the Vandermonde construction of ``refelem``:
  projection: M_T,kl = m_T |det R_T| sum_q w_q phi^_k(x_q) phi^_l(x_q)
  elliptic:   K_T,kl = |det R_T| sum_q w_q (R_T^-T grad^ phi^_k)^T M_T (R_T^-T grad^ phi^_l)
(chain rule eq. bas_deriv).  Summed into CSR keeping every structural entry
(unlike the paper's 1e-14 dropping in Section 3, so the nnz is the structural count).
Parity: pinned by exactness checks of the rule, textbook P1 matrices, symmetry,
null space and the measure of the domain.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import quadrature, refelem
from .dogip import geometry


def element_matrices(form: str, p: int, coords, cells, coef) -> np.ndarray:
    d = cells.shape[1] - 1
    pts, wq = quadrature.simplex_rule(d, p + 1)
    val, grad = refelem.vandermonde_eval_float(d, p, pts)  # [q, V], [q, d, V]
    _, det, Rinv = geometry(coords, cells)
    vol = np.abs(det)
    coef = np.asarray(coef, dtype=np.float64)
    if form == "projection":
        Mref = np.einsum("q,qk,ql->kl", wq, val, val)
        return (coef * vol)[:, None, None] * Mref[None]
    M = coef[:, None, None] * np.eye(d)[None] if coef.ndim == 1 else coef
    G = np.einsum("epi,qpl->eqil", Rinv, grad)  # physical gradients [E, q, d, V]
    return vol[:, None, None] * np.einsum("q,eqik,eij,eqjl->ekl", wq, G, M, G)


def assemble(form: str, p: int, coords, cells, conn, n, coef) -> sp.csr_matrix:
    Ke = element_matrices(form, p, coords, cells, coef)
    V = conn.shape[1]
    rows = np.repeat(conn, V, axis=1).reshape(-1)
    cols = np.tile(conn, (1, V)).reshape(-1)
    return sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()


def structural_nnz(conn: np.ndarray, n: int) -> int:
    """Number of (i, j) pairs of dofs sharing an element (the CSR pattern)."""
    V = conn.shape[1]
    rows = np.repeat(conn, V, axis=1).reshape(-1).astype(np.int64)
    cols = np.tile(conn, (1, V)).reshape(-1).astype(np.int64)
    return int(np.unique(rows * n + cols).size)


def dirichlet(K: sp.csr_matrix, bmask: np.ndarray) -> sp.csr_matrix:
    """P K P + (I - P): boundary rows/columns replaced by the identity."""
    P = sp.diags((~bmask).astype(np.float64))
    return (P @ K @ P + sp.diags(bmask.astype(np.float64))).tocsr()


def load(d: int, p: int, coords, cells, conn, n, f) -> np.ndarray:
    """b_i = integral f phi_i by the collapsed rule with p + 3 points per direction."""
    pts, wq = quadrature.simplex_rule(d, p + 3)
    val, _ = refelem.vandermonde_eval_float(d, p, pts)
    R, det, _ = geometry(coords, cells)
    X = coords[cells][:, 0, :][:, None, :] + np.einsum("eij,qj->eqi", R, pts)
    fx = f(X)  # [E, q]
    be = np.abs(det)[:, None] * np.einsum("q,eq,ql->el", wq, fx, val)
    b = np.zeros(n)
    np.add.at(b, conn, be)
    return b
