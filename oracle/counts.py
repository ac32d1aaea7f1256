"""Memory and multiplication counts of Section 3 (Tables 1-4).

mem A = 2 nnz A + nrows A (CSR, Section 3); memory efficiency (eq. memory_eff) =
nnz A_T^DoGIP |M| / mem A; computational efficiency (eq. comp_eff) =
[2 (nnz B^ - nnz_{+-1} B^) + nnz A_T^DoGIP] |M| / nnz A, where nnz A_T^DoGIP is
W_T (projection) or d^2 W_T (elliptic, the full d x d block per W node as the
tables count it) and |M| = 2 N^2 (2D) or 6 N^3 (3D).
"""

from __future__ import annotations

from . import refelem


def n_cells(d: int, N: int) -> int:
    return 2 * N * N if d == 2 else 6 * N ** 3


def nnz_ahat_T(form: str, d: int, p: int) -> int:
    WT = refelem.dim_P(d, refelem.w_degree(form, p))
    return WT if form == "projection" else d * d * WT


def mem_csr(nnz: int, nrows: int) -> int:
    return 2 * nnz + nrows


def memory_eff(form, d, p, N, nnzA, nrows):
    return nnz_ahat_T(form, d, p) * n_cells(d, N) / mem_csr(nnzA, nrows)


def comp_eff(form, d, p, N, nnzA):
    nb, n1 = refelem.nnz_counts(form, d, p)
    return (2 * (nb - n1) + nnz_ahat_T(form, d, p)) * n_cells(d, N) / nnzA
