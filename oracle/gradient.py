"""Gradient of the compliance J = b^T u, K(A) u = b, with respect to the element
coefficients (not in the paper; the DoGIP structure makes it a per-node outer
product).

Adjoint: K lambda = dJ/du = b, so lambda = u (K symmetric) and
  dJ/dM_T,pq = -lambda^T (dK/dM_T,pq) u.
DoGIP form (Theorem 8 with constant M_T): the element contribution is
  sum_j |det R_T| w^_j (R^-T g_j(u))^T M_T (R^-T g_j(v)),  g_j = B^_{.j.} u_T,
so dJ/dM_T,pq = -sum_j omega_T,j (grad lambda)(x_j)_p (grad u)(x_j)_q with
omega_T,j = |det R_T| w^_j and physical gradients at the W nodes.
Projection (Theorem 4): dJ/dm_T = -sum_j omega_T,j lambda(x_j) u(x_j).
An independent path differentiates the assembled element matrices.  Boundary
dofs carry u = lambda = 0 (zero Dirichlet data), so P K P and K give the same value.
"""

from __future__ import annotations

import numpy as np

from . import assembly, refelem
from .dogip import geometry


def grad_coef_dogip(form, p, coords, cells, conn, u, lam):
    d = cells.shape[1] - 1
    Bh = refelem.bhat(form, d, p)
    w = refelem.what(d, refelem.w_degree(form, p))
    _, det, Rinv = geometry(coords, cells)
    om = np.abs(det)[:, None] * w[None, :]
    uT, lT = u[conn], lam[conn]
    if form == "projection":
        return -np.einsum("ej,ej,ej->e", om, uT @ Bh.T, lT @ Bh.T)
    gu = np.einsum("sjl,el->ejs", Bh, uT)
    gl = np.einsum("sjl,el->ejs", Bh, lT)
    Gu = np.einsum("esp,ejs->ejp", Rinv, gu)  # physical gradient components
    Gl = np.einsum("esp,ejs->ejp", Rinv, gl)
    return -np.einsum("ej,ejp,ejq->epq", om, Gl, Gu)


def grad_coef_assembled(form, p, coords, cells, conn, u, lam):
    """-lambda_T^T (dK_T/dM_pq) u_T from the quadrature element matrices, by
    assembling with unit coefficient tensors e_p e_q^T."""
    d = cells.shape[1] - 1
    E = len(cells)
    uT, lT = u[conn], lam[conn]
    if form == "projection":
        Ke = assembly.element_matrices(form, p, coords, cells, np.ones(E))
        return -np.einsum("ek,ekl,el->e", lT, Ke, uT)
    out = np.zeros((E, d, d))
    for a in range(d):
        for c in range(d):
            unit = np.zeros((E, d, d))
            unit[:, a, c] = 1.0
            Ke = assembly.element_matrices(form, p, coords, cells, unit)
            out[:, a, c] = -np.einsum("ek,ekl,el->e", lT, Ke, uT)
    return out
