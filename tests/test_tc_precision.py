"""Error model of the tensor-core FP32 apply, checked on the CPU against the oracle.

The tensor-core kernel splits every FP32 operand as hi + lo (hi rounded to TF32 by
adding half of the 13 dropped mantissa bits and clearing them; lo = x - hi exactly),
the tensor core reads lo truncated to TF32, and each contraction is the sum of the
products hi.hi + hi.lo + lo.hi accumulated in FP32, eight terms per MMA k-step.  This
file emulates that arithmetic with numpy on the oracle's B^ and A_T:

* the emulated apply stays inside the FP32 parity bound the GPU tests use,
  |y - y_oracle| <= 2e-5 (|B^|^T |A_T| |B^| |u|) componentwise (here below 1e-7 of
  the scale), and its norm-wise error is of the order of the FP32 unit roundoff
  (measured on a GB300: 7.3e-7 at 2D P4);
* a single TF32 product of the unsplit operands (what the tensor core makes of raw
  FP32 values: both truncated to TF32) breaks that bound, which is why the kernel
  pays three MMAs per k-step.
"""

import numpy as np
import pytest

from oracle import dogip as odogip
from paper_1710_09913_gb300 import inputs

TOL32 = 2e-5


def tf32_rn(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def tf32_trunc(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return (b & np.uint32(0xFFFFE000)).view(np.float32)


def split(x):
    hi = tf32_rn(x)
    lo = (x.astype(np.float32) - hi).astype(np.float32)  # exact in FP32
    return hi, tf32_trunc(lo)


def gemm_tc(A, Bm, three=True):
    """A [M, K] . Bm [K, N] as the kernel issues it: per k-step of 8, the TF32
    products (hi.hi + hi.lo + lo.hi, or one product of the truncated unsplit operands)
    summed exactly and added to an FP32 accumulator."""
    K = A.shape[1]
    Kp = (K + 7) // 8 * 8
    A = np.pad(A.astype(np.float32), ((0, 0), (0, Kp - K)))
    Bm = np.pad(Bm.astype(np.float32), ((0, Kp - K), (0, 0)))
    Ah, Al = split(A)
    Bh, Bl = split(Bm)
    pairs = ((Ah, Bh), (Ah, Bl), (Al, Bh)) if three else ((tf32_trunc(A), tf32_trunc(Bm)),)
    acc = np.zeros((A.shape[0], Bm.shape[1]), dtype=np.float32)
    for k0 in range(0, Kp, 8):
        for a, b in pairs:
            part = a[:, k0:k0 + 8].astype(np.float64) @ b[k0:k0 + 8].astype(np.float64)
            acc = (acc.astype(np.float64) + part).astype(np.float32)
    return acc


def apply_tc_emulated(P, u32, three=True):
    """Algorithm 1 as the tensor-core kernel evaluates it, in FP32 / TF32 arithmetic."""
    d, form = P.d, P.form
    Bh = P.Bh.astype(np.float32)
    if form == "projection":
        Bh = Bh[None]  # [NB = 1][W][V]
    NB, W, V = Bh.shape
    # B1[l, c] and B2[c, l] with c = j NB + r
    Bc = np.transpose(Bh, (1, 0, 2)).reshape(W * NB, V)  # [c][l]
    conn = P.conn
    U = u32[conn].copy()
    if P.bmask is not None:
        U[P.bmask[conn]] = 0.0
    G = gemm_tc(U, Bc.T, three).reshape(-1, W, NB)  # [E][j][r]
    A32 = P.Ah.astype(np.float32)
    if form == "projection":
        H = (A32[:, :, None] * G).astype(np.float32)
    else:
        H = np.einsum("ejts,ejs->ejt", A32, G).astype(np.float32)
    Y = gemm_tc(H.reshape(-1, W * NB), Bc, three)  # [E][l]
    y = np.zeros(P.n, dtype=np.float32)
    np.add.at(y, conn, Y)
    if P.bmask is not None:
        y[P.bmask] = u32[P.bmask]
    return y.astype(np.float64)


CASES = [(2, 4, "elliptic", 6), (2, 3, "projection", 6), (3, 2, "elliptic", 2),
         (2, 5, "elliptic", 4)]


@pytest.mark.parametrize("d,p,form,N", CASES, ids=[f"{d}D-P{p}-{f}" for d, p, f, _ in CASES])
def test_three_tf32_products_meet_the_fp32_bound(d, p, form, N):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, 3)
    E = len(cells)
    coef = (inputs.coef_tensor_lognormal(E, d, 1.0, 3) if form == "elliptic"
            else inputs.coef_uniform(E, 1.0, 10.0, 3))
    P = odogip.Problem(form, p, coords, cells, coef)
    u32 = inputs.rhs_normal(P.n, 1, seed=11)[:, 0].astype(np.float32)
    u64 = u32.astype(np.float64)
    ref, scale = P.apply(u64), P.apply_abs(u64)
    y = apply_tc_emulated(P, u32)
    assert np.all(np.abs(y - ref) <= TOL32 * scale)
    assert np.linalg.norm(y - ref) <= 5e-6 * np.linalg.norm(ref)
    # one TF32 product per entry (no hi/lo split) breaks the bound (by 5x to 26x here)
    y1 = apply_tc_emulated(P, u32, three=False)
    assert np.max(np.abs(y1 - ref) / np.maximum(scale, 1e-300)) > TOL32
