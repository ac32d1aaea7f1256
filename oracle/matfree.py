"""Conventional quadrature-point matrix-free apply (the approach the paper compares
DoGIP against: §1, "alternative approaches", and §3.3), plain FP64.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and bench.py's CPU
baseline leg; the product path never calls it.

Per element T, following the two formulas of §1:
  grad u(x_q)      = J_T^-T sum_i grad^ phi^_i(x^_q) u_T,i
  (A_T u_T)_l      = sum_q  M_T grad u(x_q) . grad phi_l(x_q)  w_q |det J_T|
(elliptic), and for the weighted projection
  (M_T u_T)_l      = sum_q  m_T u(x_q) phi_l(x_q)  w_q |det J_T|.
The rule is the collapsed Gauss--Jacobi rule of ``quadrature`` with n points per
direction, n = p for the stiffness integrand (degree 2p - 2) and n = p + 1 for the
mass integrand (degree 2p), so for element-constant coefficients the result is the
Galerkin operator itself -- the same operator as Algorithm 1.  Basis values and
reference gradients come from the Vandermonde construction of ``refelem``.
Dirichlet rows as in ``dogip.apply``: K~ u = P K P u + (I - P) u.
Parity: pinned against the DoGIP oracle (exact rational tables on the lattice W
nodes, an independent route) and against the assembled CSR operator.
"""

from __future__ import annotations

import numpy as np

from . import quadrature, refelem
from .dogip import geometry


def points_per_direction(form: str, p: int) -> int:
    """n with 2n - 1 >= the integrand degree (2p mass, 2p - 2 stiffness)."""
    return p + 1 if form == "projection" else p


def tables(form: str, d: int, p: int):
    """(B_q, w_q): values [1, Q, V] or reference gradients [d, Q, V] at the rule's
    points, and the weights [Q]."""
    pts, wq = quadrature.simplex_rule(d, points_per_direction(form, p))
    val, grad = refelem.vandermonde_eval_float(d, p, pts)  # [Q, V], [Q, d, V]
    if form == "projection":
        return val[None], wq
    return grad.transpose(1, 0, 2).copy(), wq


def _prepare(form, p, coords, cells, coef):
    d = cells.shape[1] - 1
    Bq, wq = tables(form, d, p)
    _, det, Rinv = geometry(coords, cells)
    coef = np.asarray(coef, dtype=np.float64)
    return d, Bq, wq, np.abs(det), Rinv, coef


def apply(form: str, p: int, coords, cells, coef, conn, u, bmask=None, absolute=False):
    """y = sum_T P_T^T (A_T u_T) with A_T u_T integrated at the quadrature points.

    ``absolute`` evaluates the same sums with |.| of every factor: the componentwise
    scale of the rounding error of any evaluation order (used for tolerances)."""
    d, Bq, wq, vol, Rinv, coef = _prepare(form, p, coords, cells, coef)
    u = np.asarray(u, dtype=np.float64)
    vec = u.ndim == 1
    U0 = u[:, None] if vec else u
    U = U0 if bmask is None else np.where(bmask[:, None], 0.0, U0)
    f = np.abs if absolute else (lambda x: x)
    uT = f(U)[conn]  # [E, V, R]
    if form == "projection":
        uq = np.einsum("ql,elr->eqr", f(Bq[0]), uT)               # u(x_q)
        hq = (f(coef) * vol)[:, None, None] * wq[None, :, None] * uq
        Y = np.einsum("ql,eqr->elr", f(Bq[0]), hq)                # adjoint interpolation
    else:
        M = coef[:, None, None] * np.eye(d)[None] if coef.ndim == 1 else coef
        Gphys = np.einsum("eis,iql->eqsl", f(Rinv), f(Bq))       # J^-T grad^ phi (physical)
        gu = np.einsum("eqsl,elr->eqsr", Gphys, uT)               # grad u(x_q)
        flux = np.einsum("est,eqtr->eqsr", f(M), gu)              # M grad u
        hq = (vol[:, None, None, None] * wq[None, :, None, None]) * flux
        Y = np.einsum("eqsl,eqsr->elr", Gphys, hq)                # . grad phi_l, summed over q
    v = np.zeros_like(U)
    np.add.at(v, conn, Y)
    if bmask is not None:
        v = np.where(bmask[:, None], f(U0), v)
    return v[:, 0] if vec else v
