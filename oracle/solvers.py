"""Solvers around the DoGIP apply (not in the paper; its problem statement
A u = b of Section 1 with a positive definite bilinear form).

* ``pcg``: Jacobi-preconditioned conjugate gradients (Hestenes--Stiefel), x0 given
  or zero, stop when the recursively updated ||r||_2 <= tol ||b||_2.
* ``iterative_refinement``: FP64 outer loop r = b - K u, stop on the true relative
  residual; inner Jacobi-PCG on K d = r / ||r|| in emulated FP32 (every vector and
  A_T rounded to float32 after each operation), u += ||r|| d.
  Parity unpinned: the paper fixes no precision; used only for sanity checks of
  iteration counts.
"""

from __future__ import annotations

import numpy as np


def pcg(apply, b, dinv, tol=1e-8, maxiter=100000, x0=None):
    """Returns (x, iterations, final recursive relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply(x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    if nb == 0:
        return x, 0, 0.0
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    res = np.linalg.norm(r) / nb
    while res > tol and it < maxiter:
        q = apply(p)
        pq = float(p @ q)
        if pq <= 0:
            raise FloatingPointError("CG breakdown: p^T K p <= 0")
        a = rz / pq
        x += a * p
        r -= a * q
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        res = np.linalg.norm(r) / nb
    return x, it, res


def iterative_refinement(apply64, apply32, b, dinv, tol=1e-8, inner_tol=1e-5,
                         inner_maxiter=100000, max_outer=50):
    """FP64 refinement with an emulated-FP32 inner PCG.  Returns
    (u, outer iterations, total inner iterations, true relative residual)."""
    f32 = np.float32
    nb = np.linalg.norm(b)
    u = np.zeros_like(b)
    inner_total = 0
    dinv32 = dinv.astype(f32)
    for outer in range(max_outer + 1):
        r = b - apply64(u)
        rel = np.linalg.norm(r) / nb
        if rel <= tol or outer == max_outer:
            return u, outer, inner_total, rel
        s = np.linalg.norm(r)
        rr = (r / s).astype(f32)
        x = np.zeros_like(rr)
        z = (dinv32 * rr).astype(f32)
        p = z.copy()
        rz = f32(rr @ z)
        n0 = f32(np.linalg.norm(rr))
        for _ in range(inner_maxiter):
            q = apply32(p).astype(f32)
            a = f32(rz / f32(p @ q))
            x = (x + a * p).astype(f32)
            rr = (rr - a * q).astype(f32)
            inner_total += 1
            if np.linalg.norm(rr) <= inner_tol * n0:
                break
            z = (dinv32 * rr).astype(f32)
            rzn = f32(rr @ z)
            p = (z + f32(rzn / rz) * p).astype(f32)
            rz = rzn
        u = u + s * x.astype(np.float64)
    return u, max_outer, inner_total, rel
