"""Reference simplex T^ = {x^ >= 0, sum x^ <= 1} in d = 2, 3: Lagrange nodes and bases.

Section 2.1 of the paper: P_k Lagrange bases with the Dirac property
phi^j(x^i) = delta_ij; reference shape functions are pulled back by the affine map
F_T(x^) = R_T x^ + S_T.  Node sets (a reading: the paper relies on FEniCS's
equispaced Lagrange elements; the nnz(B^) columns of Tables 1-4 are reproduced
exactly with them): x^_alpha = alpha / q for multi-indices |alpha| <= q, local
order = itertools.product(range(q+1), repeat=d) filtered by |alpha| <= q (last
coordinate fastest).  The degree-0 space has one node, the centroid.

Two independent constructions of the same basis, both exact (fractions.Fraction):
  * ``silvester``: the closed product form of the equispaced simplex Lagrange basis
    in barycentric coordinates (Silvester 1969);
  * ``vandermonde``: the plain definition -- solve the nodal Vandermonde system of
    the monomials x^a, |a| <= q, for the coefficients of the Dirac basis.
The DoGIP tables use the first; the conventional assembly uses the second, and the
tests check that the two agree exactly.

DoGIP tables (both exact rationals, rounded to float64 once):
  * weighted projection (Theorem 4, element-wise): B^_jl = phi^_l(x^W_j),
    W = P_{2p}, shape [W_T, V_T];
  * scalar elliptic (Theorem 8, element-wise): B^_rjl = d phi^_l / d x^_r at x^W_j,
    W = P_{2p-2} (discontinuous), shape [d, W_T, V_T].  Derivatives are taken with
    respect to the reference coordinates (the theorem's d/dx_r read as d/dx^_r; the
    proof's chain-rule step eq. bas_deriv moves R_T^-1 into A_T).
  * w^_j = integral over T^ of the W basis function phi^W_j, used for
    A_T,j = integral_T m phi^W_j for element-wise constant m.
"""

from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import product
from math import comb, factorial

import numpy as np

# ------------------------------------------------------------------------ nodes


@lru_cache(maxsize=None)
def multi_indices(d: int, q: int):
    """Multi-indices alpha in N^d with |alpha| <= q, last coordinate fastest."""
    return tuple(a for a in product(range(q + 1), repeat=d) if sum(a) <= q)


def dim_P(d: int, q: int) -> int:
    """dim P_q(R^d) = C(q + d, d)."""
    return comb(q + d, d)


@lru_cache(maxsize=None)
def nodes(d: int, q: int):
    """Equispaced Lagrange nodes of degree q (exact); q = 0 gives the centroid."""
    if q == 0:
        return (tuple(Fraction(1, d + 1) for _ in range(d)),)
    return tuple(tuple(Fraction(ai, q) for ai in a) for a in multi_indices(d, q))


def barycentric(x):
    """(lambda_0, ..., lambda_d) of a reference point: lambda_0 = 1 - sum x, lambda_i = x_i."""
    return (1 - sum(x),) + tuple(x)


# -------------------------------------------------------- Silvester construction


def _silv_factor(q: int, b: int, t):
    """P_b(t) = prod_{j<b} (q t - j) / (j + 1)."""
    v = Fraction(1)
    for j in range(b):
        v *= Fraction(q * t - j, j + 1)
    return v


def _silv_factor_deriv(q: int, b: int, t):
    """d/dt P_b(t) by the product rule."""
    s = Fraction(0)
    for m in range(b):
        term = Fraction(q, m + 1)
        for j in range(b):
            if j != m:
                term *= Fraction(q * t - j, j + 1)
        s += term
    return s


def _beta(alpha, q):
    """Barycentric multi-index (q - |alpha|, alpha_1, ..., alpha_d) of a node."""
    return (q - sum(alpha),) + tuple(alpha)


def silvester_value(d: int, q: int, l: int, x) -> Fraction:
    """phi^_l(x) = prod_i P_{beta_i}(lambda_i(x)) for the l-th node of degree q."""
    if q == 0:
        return Fraction(1)
    beta = _beta(multi_indices(d, q)[l], q)
    lam = barycentric(x)
    v = Fraction(1)
    for bi, li in zip(beta, lam):
        v *= _silv_factor(q, bi, li)
    return v


def silvester_grad(d: int, q: int, l: int, x):
    """Reference gradient (d phi^_l / d x^_r)_r; d lambda_0/dx^_r = -1, d lambda_i/dx^_r = delta_ir."""
    if q == 0:
        return tuple(Fraction(0) for _ in range(d))
    beta = _beta(multi_indices(d, q)[l], q)
    lam = barycentric(x)
    dlam = []  # d phi / d lambda_i
    for i in range(d + 1):
        v = _silv_factor_deriv(q, beta[i], lam[i])
        for k in range(d + 1):
            if k != i:
                v *= _silv_factor(q, beta[k], lam[k])
        dlam.append(v)
    return tuple(dlam[r + 1] - dlam[0] for r in range(d))


# ------------------------------------------------------ Vandermonde construction


def _solve_exact(M, rhs):
    """Gauss--Jordan elimination over the rationals: returns X with M X = rhs."""
    n = len(M)
    A = [list(M[i]) + list(rhs[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        inv = 1 / A[c][c]
        A[c] = [v * inv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [row[n:] for row in A]


def _mono(x, a):
    v = Fraction(1)
    for xi, ai in zip(x, a):
        v *= Fraction(xi) ** ai
    return v


@lru_cache(maxsize=None)
def vandermonde_coeffs(d: int, q: int):
    """Monomial coefficients C[a][l] of the Dirac basis: sum_a C[a][l] x_k^a = delta_kl."""
    mons = multi_indices(d, q)
    X = nodes(d, q)
    V = [[_mono(x, a) for a in mons] for x in X]  # V[k][a]
    # phi_l(x) = sum_a C[a][l] x^a;  V C = I
    ident = [[Fraction(int(i == j)) for j in range(len(X))] for i in range(len(X))]
    return tuple(tuple(r) for r in _solve_exact(V, ident))


def vandermonde_value(d: int, q: int, l: int, x) -> Fraction:
    C = vandermonde_coeffs(d, q)
    return sum(C[ia][l] * _mono(x, a) for ia, a in enumerate(multi_indices(d, q)))


def vandermonde_grad(d: int, q: int, l: int, x):
    C = vandermonde_coeffs(d, q)
    out = []
    for r in range(d):
        s = Fraction(0)
        for ia, a in enumerate(multi_indices(d, q)):
            if a[r] == 0 or C[ia][l] == 0:
                continue
            b = list(a)
            b[r] -= 1
            s += C[ia][l] * a[r] * _mono(x, b)
        out.append(s)
    return tuple(out)


def vandermonde_eval_float(d: int, q: int, pts: np.ndarray):
    """Float64 values [n_pts, V_T] and reference gradients [n_pts, d, V_T] of the
    Vandermonde-constructed basis at arbitrary float points (used by assembly)."""
    C = np.array([[float(c) for c in row] for row in vandermonde_coeffs(d, q)])  # [a, l]
    mons = multi_indices(d, q)
    pts = np.asarray(pts, dtype=np.float64)
    P = np.stack([np.prod(pts ** np.array(a), axis=1) for a in mons], axis=1)  # [n, a]
    val = P @ C
    grad = np.zeros((pts.shape[0], d, C.shape[1]))
    for r in range(d):
        cols = []
        for a in mons:
            if a[r] == 0:
                cols.append(np.zeros(pts.shape[0]))
            else:
                b = np.array(a)
                b[r] -= 1
                cols.append(a[r] * np.prod(pts ** b, axis=1))
        grad[:, r, :] = np.stack(cols, axis=1) @ C
    return val, grad


# ------------------------------------------------------------------ DoGIP tables


def w_degree(form: str, p: int) -> int:
    """Degree of the double-grid space: 2p (weighted projection, Lemma 3) or
    2p - 2 (scalar elliptic, Lemma 7: products of two P_{p-1} gradients)."""
    if form == "projection":
        return 2 * p
    if form == "elliptic":
        return 2 * p - 2
    raise ValueError(form)


@lru_cache(maxsize=None)
def bhat_exact(form: str, d: int, p: int):
    """Exact B^ (tuple nest of Fractions).

    projection: [W_T][V_T], B^_jl = phi^_l(x^W_j)                 (Theorem 4)
    elliptic:   [d][W_T][V_T], B^_rjl = d phi^_l/d x^_r (x^W_j)    (Theorem 8)
    """
    q = w_degree(form, p)
    XW = nodes(d, q)
    VT = dim_P(d, p)
    if form == "projection":
        return tuple(tuple(silvester_value(d, p, l, x) for l in range(VT)) for x in XW)
    grads = [[silvester_grad(d, p, l, x) for l in range(VT)] for x in XW]
    return tuple(tuple(tuple(grads[j][l][r] for l in range(VT)) for j in range(len(XW)))
                 for r in range(d))


def bhat(form: str, d: int, p: int) -> np.ndarray:
    """B^ rounded to float64 (each exact rational rounded once)."""
    return np.array(bhat_exact(form, d, p), dtype=object).astype(np.float64)


def _flatten(t):
    if isinstance(t, tuple):
        for s in t:
            yield from _flatten(s)
    else:
        yield t


def nnz_counts(form: str, d: int, p: int):
    """(nnz B^, nnz_{+-1} B^): exactly nonzero entries and entries equal to +-1
    (the latter need no multiplication, eq. comp_eff)."""
    vals = list(_flatten(bhat_exact(form, d, p)))
    return sum(v != 0 for v in vals), sum(abs(v) == 1 for v in vals)


def _poly_P(q: int, b: int):
    """Coefficients (ascending powers of t) of P_b(t) = prod_{j<b} (q t - j)/(j+1)."""
    c = [Fraction(1)]
    for j in range(b):
        new = [Fraction(0)] * (len(c) + 1)
        for k, ck in enumerate(c):
            new[k + 1] += ck * Fraction(q, j + 1)
            new[k] -= ck * Fraction(j, j + 1)
        c = new
    return c


@lru_cache(maxsize=None)
def what_exact(d: int, q: int):
    """w^_j = integral over T^ of phi^W_j (degree q), exactly.

    phi^W_j = prod_i P_{beta_i}(lambda_i) is expanded in barycentric monomials and
    each is integrated with the Dirichlet formula
    integral_T^ lambda^k = d! |T^| prod k_i! / (|k| + d)!,  |T^| = 1/d!.
    """
    if q == 0:
        return (Fraction(1, factorial(d)),)
    out = []
    for alpha in multi_indices(d, q):
        beta = _beta(alpha, q)
        polys = [_poly_P(q, b) for b in beta]
        s = Fraction(0)
        for ks in product(*[range(len(pc)) for pc in polys]):
            coef = Fraction(1)
            for pc, k in zip(polys, ks):
                coef *= pc[k]
            if coef == 0:
                continue
            num = 1
            for k in ks:
                num *= factorial(k)
            s += coef * Fraction(num, factorial(sum(ks) + d))
        out.append(s)
    return tuple(out)


def what(d: int, q: int) -> np.ndarray:
    return np.array([float(v) for v in what_exact(d, q)])


def int_phiV(d: int, p: int) -> np.ndarray:
    """integral over T^ of each V basis function (the load of f = 1)."""
    return what(d, p)
