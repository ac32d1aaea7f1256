"""Local-to-global dof map l_T, Dirichlet boundary dofs and element colouring.

Section 2.1 of the paper: the P_p Lagrange dofs of the continuous space C_{N,p}
are nodal values; the injective map l_T : {1..V_T} -> {1..V} takes local to global
indices, and u_T = (u_{l_T(l)})_l is the local dof vector (discretisation operator
D_V restricted to T).  The paper fixes no global numbering; the reading used here:

* A node of cell T with local multi-index alpha (barycentric beta =
  (p-|alpha|, alpha)) is the point sum_i beta_i v_i / p.  Its identity is the
  multiset {(vertex id v_i, beta_i) : beta_i > 0}, shared by every cell containing
  the point.
* Global ids are given in order of first appearance, scanning cells in index order
  and local nodes in local order.
* Boundary dofs: nodes lying on a boundary facet (a facet of exactly one cell),
  i.e. for a boundary facet opposite local vertex i, every node with beta_i = 0.
* Colouring: cells in index order, each takes the smallest colour >= 0 not used by
  an earlier cell sharing a vertex (for p >= 1 two cells share a dof iff they
  share a vertex, so same-colour cells never write the same dof).

Parity: pinned by the structural nnz of the SE tables (Tables 3 and 4), the lattice
dof count (pN+1)^d, the geometric position of every node, and brute-force loops in
the tests.
"""

from __future__ import annotations

import numpy as np

from .refelem import dim_P, multi_indices


def local_betas(d: int, p: int) -> np.ndarray:
    """[V_T, d+1] barycentric multi-indices of the local nodes."""
    al = np.array(multi_indices(d, p), dtype=np.int64).reshape(-1, d)
    return np.concatenate([p - al.sum(axis=1, keepdims=True), al], axis=1)


def node_keys(cells: np.ndarray, p: int) -> np.ndarray:
    """[E, V_T, d+1] int64 canonical keys: entries 64*vertex + beta_i for beta_i > 0,
    sorted ascending, absent entries = 2^62 (sorting last)."""
    cells = np.asarray(cells, dtype=np.int64)
    d = cells.shape[1] - 1
    B = local_betas(d, p)  # [V, d+1]
    enc = cells[:, None, :] * 64 + B[None, :, :]
    enc = np.where(B[None, :, :] > 0, enc, np.int64(1) << 62)
    return np.sort(enc, axis=2)


def dofmap(cells: np.ndarray, p: int):
    """Returns (conn int64 [E, V_T], n_dofs): first-appearance global numbering."""
    keys = node_keys(cells, p)
    E, V, k = keys.shape
    flat = keys.reshape(E * V, k)
    uniq, first, inv = np.unique(flat, axis=0, return_index=True, return_inverse=True)
    rank = np.empty(len(uniq), dtype=np.int64)
    rank[np.argsort(first, kind="stable")] = np.arange(len(uniq), dtype=np.int64)
    return rank[inv.reshape(-1)].reshape(E, V), len(uniq)


def dofmap_loop(cells: np.ndarray, p: int):
    """The same numbering by a plain dictionary loop (small meshes only)."""
    d = cells.shape[1] - 1
    B = local_betas(d, p)
    ids = {}
    conn = np.zeros((len(cells), len(B)), dtype=np.int64)
    for e, cv in enumerate(cells):
        for l, beta in enumerate(B):
            key = tuple(sorted((int(v), int(b)) for v, b in zip(cv, beta) if b > 0))
            if key not in ids:
                ids[key] = len(ids)
            conn[e, l] = ids[key]
    return conn, len(ids)


def boundary_facets(cells: np.ndarray) -> np.ndarray:
    """[E, d+1] bool: facet opposite local vertex i of cell e belongs to no other cell."""
    cells = np.asarray(cells, dtype=np.int64)
    E, dp1 = cells.shape
    fac = np.stack([np.sort(np.delete(cells, i, axis=1), axis=1) for i in range(dp1)], axis=1)
    flat = fac.reshape(E * dp1, dp1 - 1)
    _, inv, cnt = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
    return (cnt[inv.reshape(-1)] == 1).reshape(E, dp1)


def boundary_mask(cells: np.ndarray, conn: np.ndarray, p: int, n: int) -> np.ndarray:
    """bool [n]: dof lies on the domain boundary."""
    d = cells.shape[1] - 1
    B = local_betas(d, p)
    bf = boundary_facets(cells)  # [E, d+1]
    on = np.zeros(conn.shape, dtype=bool)
    for i in range(d + 1):
        on |= bf[:, i:i + 1] & (B[None, :, i] == 0)
    mask = np.zeros(n, dtype=bool)
    mask[conn[on]] = True
    return mask


def colouring(cells: np.ndarray) -> np.ndarray:
    """Greedy vertex-sharing colouring in element order (plain loop)."""
    cells = np.asarray(cells, dtype=np.int64)
    nv = int(cells.max()) + 1
    touching = [[] for _ in range(nv)]
    col = np.full(len(cells), -1, dtype=np.int64)
    for e, cv in enumerate(cells):
        used = set()
        for v in cv:
            for f in touching[v]:
                used.add(col[f])
        c = 0
        while c in used:
            c += 1
        col[e] = c
        for v in cv:
            touching[v].append(e)
    return col


def colouring_is_greedy(cells: np.ndarray, col: np.ndarray) -> bool:
    """Checks the defining property of the greedy colouring at any size:
    same-colour cells share no vertex, and every colour c_e is the smallest colour
    not taken by an earlier vertex-sharing cell."""
    cells = np.asarray(cells, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    E, dp1 = cells.shape
    ev = cells.reshape(-1)
    ee = np.repeat(np.arange(E), dp1)
    order = np.argsort(ev, kind="stable")
    ev, ee = ev[order], ee[order]
    start = np.searchsorted(ev, np.arange(ev.max() + 2))
    cnt = np.diff(start)
    # all (e, f) pairs of cells that share a vertex, e != f
    reps = cnt[ev]
    first = np.repeat(start[ev], reps)
    off = np.arange(reps.sum()) - np.repeat(np.cumsum(reps) - reps, reps)
    f = ee[first + off]
    e = np.repeat(ee, reps)
    keep = f < e
    e, f = e[keep], f[keep]
    if np.any(col[e] == col[f]):
        return False
    # colours taken by earlier neighbours of e must cover 0 .. col[e]-1
    pairs = np.unique(np.stack([e, col[f]], axis=1), axis=0)
    below = pairs[pairs[:, 1] < col[pairs[:, 0]]]
    covered = np.bincount(below[:, 0], minlength=E)
    return bool(np.all(covered == col))


def node_points(coords: np.ndarray, cells: np.ndarray, p: int) -> np.ndarray:
    """[E, V_T, d] physical position sum_i beta_i v_i / p of every local node."""
    d = cells.shape[1] - 1
    B = local_betas(d, p).astype(np.float64) / p
    return np.einsum("li,eik->elk", B, coords[cells])
