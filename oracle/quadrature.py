"""Collapsed (conical-product) Gauss--Jacobi quadrature on the reference simplex.

The paper leaves the quadrature of the conventional assembly to FEniCS (Section 3,
Fig. 2 discussion of collapsed rules, Karniadakis & Sherwin); the oracle derives
its own rule so that the assembled matrix of eqs. linsys_gp / linsys_se is
computed independently of the DoGIP factors:

* Gauss--Jacobi nodes/weights for the weight (1-x)^a (1+x)^b on [-1, 1] by the
  Golub--Welsch method (eigen-decomposition of the Jacobi matrix of the monic
  three-term recurrence), mapped to [0, 1] with weight (1-t)^a;
* the Duffy collapse x = s(1-t), y = t (2D, Jacobian 1-t) and
  x = s(1-t)(1-r), y = t(1-r), z = r (3D, Jacobian (1-t)(1-r)^2).
n points per direction integrate total degree 2n - 1 exactly.
Parity: pinned by exact monomial integrals a!b![c!]/(a+b[+c]+d)! in the tests.
"""

from __future__ import annotations

from math import gamma

import numpy as np


def gauss_jacobi(n: int, a: float, b: float):
    """n-point Gauss--Jacobi rule on [-1, 1] for (1-x)^a (1+x)^b (Golub--Welsch)."""
    k = np.arange(n, dtype=np.float64)
    s = 2 * k + a + b
    with np.errstate(divide="ignore", invalid="ignore"):
        alpha = np.where(s * (s + 2) != 0, (b * b - a * a) / (s * (s + 2)), (b - a) / (a + b + 2))
    if n > 0:
        alpha[0] = (b - a) / (a + b + 2)
    kk = np.arange(1, n, dtype=np.float64)
    ss = 2 * kk + a + b
    beta = 4 * kk * (kk + a) * (kk + b) * (kk + a + b) / (ss * ss * (ss + 1) * (ss - 1))
    J = np.diag(alpha) + np.diag(np.sqrt(beta), 1) + np.diag(np.sqrt(beta), -1)
    x, V = np.linalg.eigh(J)
    mu0 = 2 ** (a + b + 1) * gamma(a + 1) * gamma(b + 1) / gamma(a + b + 2)
    return x, mu0 * V[0, :] ** 2


def gauss_jacobi01(n: int, a: float):
    """n-point rule on [0, 1] for the weight (1-t)^a."""
    x, w = gauss_jacobi(n, a, 0.0)
    return (x + 1) / 2, w / 2 ** (a + 1)


def simplex_rule(d: int, n: int):
    """(points [n^d, d], weights [n^d]) on the reference simplex, exact to degree 2n-1."""
    s, ws = gauss_jacobi01(n, 0.0)
    t, wt = gauss_jacobi01(n, 1.0)
    if d == 2:
        S, T = np.meshgrid(s, t, indexing="ij")
        W = np.outer(ws, wt)
        pts = np.stack([S * (1 - T), T], axis=-1).reshape(-1, 2)
        return pts, W.reshape(-1)
    r, wr = gauss_jacobi01(n, 2.0)
    S, T, Rr = np.meshgrid(s, t, r, indexing="ij")
    W = ws[:, None, None] * wt[None, :, None] * wr[None, None, :]
    pts = np.stack([S * (1 - T) * (1 - Rr), T * (1 - Rr), Rr], axis=-1).reshape(-1, 3)
    return pts, W.reshape(-1)
