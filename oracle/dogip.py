"""DoGIP factors and the element-wise matrix-vector multiplication (Algorithm 1).

Weighted projection (Theorem "Element-wise DoGIP for weighted projection", eq.
wp_dogip_mul): A u . v = sum_T B^* A_T B^ u_T . v_T with
  A_T,jj = integral_T m phi^W_{l_T(j)} = m_T |det R_T| w^_j  (m constant on T),
  B^_jl = phi^_l(x^W_j).
Scalar elliptic (Theorem "Element-wise DoGIP for the elliptic problem", eq.
ep_dogip_mul): per W node j a d x d block
  A_T,rs,j = sum_pq (R_T^-1)_rp (R_T^-1)_sq integral_T M_pq phi^W_j
           = |det R_T| w^_j (R_T^-1 M_T R_T^-T)_rs     (M constant on T),
  B^_rjl = d phi^_l / d x^_r (x^W_j).
The affine map is F_T(x^) = R_T x^ + S_T with R_T = [v_1 - v_0, ..., v_d - v_0]
(Section 2.1).  Readings: the theorem's W = D_{N,k} is read as D_{N,2k-2} (Lemma 7
and Section 3.2); Algorithm 1's "B^ A_T B^ u_T" is read as B^* A_T B^ u_T.

Dirichlet boundary conditions (not in the paper; the solver configs need them):
with P the projector that zeroes boundary dofs, the operator is
K~ = P K P + (I - P): boundary rows and columns replaced by the identity.

Parity: pinned in the tests by the identity with the independently assembled
matrix (1e-12), textbook P1 mass/stiffness, K 1 = 0, 1^T M 1 = |Omega|; the
sub-element quadrature (``ahat_quadrature``) by the exact A_T for constant m and
by the measure of a ball.
"""

from __future__ import annotations

import numpy as np

from . import refelem


def geometry(coords: np.ndarray, cells: np.ndarray):
    """(R [E,d,d] with columns v_i - v_0, det R [E], R^-1 [E,d,d])."""
    X = coords[cells]  # [E, d+1, d]
    R = (X[:, 1:, :] - X[:, :1, :]).transpose(0, 2, 1)
    return R, np.linalg.det(R), np.linalg.inv(R)


def ahat(form: str, p: int, coords: np.ndarray, cells: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """A_T^DoGIP for every element.

    projection: coef [E] (m_T)               -> [E, W_T]
    elliptic:   coef [E] (M_T = m_T I) or [E, d, d] (symmetric M_T) -> [E, W_T, d, d]
    """
    d = cells.shape[1] - 1
    _, det, Rinv = geometry(coords, cells)
    w = refelem.what(d, refelem.w_degree(form, p))
    vol = np.abs(det)
    if form == "projection":
        return (coef * vol)[:, None] * w[None, :]
    coef = np.asarray(coef, dtype=np.float64)
    M = coef[:, None, None] * np.eye(d)[None] if coef.ndim == 1 else coef
    K = np.einsum("erp,epq,esq->ers", Rinv, M, Rinv)  # R^-1 M R^-T
    return vol[:, None, None, None] * w[None, :, None, None] * K[:, None, :, :]


def ahat_quadrature(form: str, p: int, coords: np.ndarray, cells: np.ndarray, m_func, nq: int):
    """A_T^DoGIP of an isotropic coefficient m(x) that varies inside the cells
    (Theorems 4 and 8 with the integral int_T m phi^W_j left to quadrature):
      sigma_T,j = int_That m(F_T(x)) phi^W_j(x) dx ~ sum_q w_q m(F_T(x_q)) phi^W_j(x_q)
    with the collapsed Gauss rule of ``nq`` points per direction, and
      A_T,j = sigma_T,j |det R_T| R_T^-1 R_T^-T (elliptic, M = m I), sigma_T,j |det R_T|
    (projection).  Returns the layout of ``ahat``.
    """
    from . import quadrature
    d = cells.shape[1] - 1
    q = refelem.w_degree(form, p)
    pts, wq = quadrature.simplex_rule(d, nq)
    phi, _ = refelem.vandermonde_eval_float(d, q, pts) if q > 0 else (np.ones((len(pts), 1)), None)
    R, det, Rinv = geometry(coords, cells)
    X = coords[cells][:, 0, :][:, None, :] + np.einsum("eij,qj->eqi", R, pts)
    mq = m_func(X)                                   # [E, nq]
    sig = np.einsum("q,eq,qj->ej", wq, mq, phi)      # [E, W]
    vol = np.abs(det)
    if form == "projection":
        return vol[:, None] * sig
    K = np.einsum("erp,esp->ers", Rinv, Rinv)        # R^-1 R^-T
    return (vol[:, None] * sig)[:, :, None, None] * K[:, None, :, :]


def apply(form: str, Bh: np.ndarray, Ah: np.ndarray, conn: np.ndarray, u: np.ndarray,
          bmask: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 1: v = sum_T P_T^T B^* A_T B^ P_T u  (u is [n] or [n, R]).

    For each cell (vectorised over cells): gather u_T, interpolate onto the W nodes
    (B^ u_T), multiply by the (block-)diagonal A_T, project back with B^*, and add
    into v.  With ``bmask`` the result is K~ u = P K P u + (I - P) u.
    """
    u = np.asarray(u, dtype=np.float64)
    vec = u.ndim == 1
    U0 = u[:, None] if vec else u
    U = U0 if bmask is None else np.where(bmask[:, None], 0.0, U0)
    uT = U[conn]  # [E, V, R]
    if form == "projection":
        G = np.einsum("jl,elr->ejr", Bh, uT)
        H = Ah[:, :, None] * G
        Y = np.einsum("jl,ejr->elr", Bh, H)
    else:
        G = np.einsum("sjl,elr->ejsr", Bh, uT)          # reference gradients at W nodes
        H = np.einsum("ejts,ejsr->ejtr", Ah, G)          # block-diagonal multiply
        Y = np.einsum("tjl,ejtr->elr", Bh, H)            # project back (adjoint)
    v = np.zeros_like(U)
    np.add.at(v, conn, Y)
    if bmask is not None:
        v = np.where(bmask[:, None], U0, v)
    return v[:, 0] if vec else v


def apply_abs(form: str, Bh, Ah, conn, u, bmask=None) -> np.ndarray:
    """|B^|^T |A_T| |B^| |u| summed like Algorithm 1: the componentwise scale of the
    rounding error of any evaluation order of the apply (used for tolerances)."""
    return apply(form, np.abs(Bh), np.abs(Ah), conn, np.abs(u), bmask)


def diag(form: str, Bh: np.ndarray, Ah: np.ndarray, conn: np.ndarray, n: int,
         bmask: np.ndarray | None = None) -> np.ndarray:
    """Jacobi diagonal K_ll = sum_T sum_j B^_{.jl}^T A_T,j B^_{.jl}; 1 on boundary rows."""
    if form == "projection":
        per = np.einsum("jl,ej,jl->el", Bh, Ah, Bh)
    else:
        per = np.einsum("sjl,ejts,tjl->el", Bh, Ah, Bh)
    dg = np.zeros(n)
    np.add.at(dg, conn, per)
    if bmask is not None:
        dg[bmask] = 1.0
    return dg


def element_matrices(form: str, Bh: np.ndarray, Ah: np.ndarray) -> np.ndarray:
    """K_T = B^* A_T B^ as dense [E, V_T, V_T] (for small meshes and tests)."""
    if form == "projection":
        return np.einsum("jk,ej,jl->ekl", Bh, Ah, Bh)
    return np.einsum("tjk,ejts,sjl->ekl", Bh, Ah, Bh)


def load_const(d: int, p: int, coords, cells, conn, n, f_elem) -> np.ndarray:
    """b_i = sum_T f_T integral_T phi_i for element-wise constant f (exact):
    integral_T phi^_l = |det R_T| integral_T^ phi^_l."""
    _, det, _ = geometry(coords, cells)
    iv = refelem.int_phiV(d, p)
    b = np.zeros(n)
    np.add.at(b, conn, (np.asarray(f_elem) * np.abs(det))[:, None] * iv[None, :])
    return b


class Problem:
    """All oracle-side data of one DoGIP problem (mesh, dofs, tables, A_T)."""

    def __init__(self, form, p, coords, cells, coef, dirichlet=None):
        from . import topology
        self.form, self.p = form, p
        self.coords = np.asarray(coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.d = self.cells.shape[1] - 1
        self.conn, self.n = topology.dofmap(self.cells, p)
        if dirichlet is None:
            dirichlet = form == "elliptic"
        self.bmask = topology.boundary_mask(self.cells, self.conn, p, self.n) if dirichlet else None
        self.Bh = refelem.bhat(form, self.d, p)
        self.coef = np.asarray(coef, dtype=np.float64)
        self.Ah = ahat(form, p, self.coords, self.cells, self.coef)

    def apply(self, u):
        return apply(self.form, self.Bh, self.Ah, self.conn, u, self.bmask)

    def apply_abs(self, u):
        return apply_abs(self.form, self.Bh, self.Ah, self.conn, u, self.bmask)

    def diag(self):
        return diag(self.form, self.Bh, self.Ah, self.conn, self.n, self.bmask)
