"""Seeded synthetic inputs: simplex lattice meshes, coefficient fields and loads.

This module is the only code shared by the CUDA path and the CPU oracle.  It holds
none of the DoGIP arithmetic: it only produces the *inputs* of the method (vertex
coordinates, cell-to-vertex lists, per-element coefficients, right-hand sides).

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th
draw of stream s under seed S is the SplitMix64 output of the state
key(S, s) + (k + 1) * GOLDEN, key(S, s) = mix(S * GOLDEN + s).  Uniform variates
are the top 53 bits scaled by 2^-53; normals use the Box--Muller transform.

Meshes follow the paper's structured test meshes (Section 3, "irregular meshes
M_N with N elements per direction"): the N^d lattice of the unit square/cube,
each square cut into 2 triangles along its (0,0)-(1,1) diagonal and each cube
into 6 Kuhn tetrahedra around its main diagonal, optionally with the interior
vertices jittered.
"""

from __future__ import annotations

import itertools

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids, one per kind of draw, so that inputs never share random numbers.
STREAM_JITTER = 1
STREAM_COEF = 2
STREAM_ANGLE = 3
STREAM_EIG = 4
STREAM_INCL_CENTRE = 5
STREAM_INCL_RADIUS = 6
STREAM_RHS = 7
STREAM_PICK = 8
STREAM_PROBLEM = 9


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of stream ``stream`` under ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed % 2**64) * GOLDEN + np.uint64(stream))
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(key + k * GOLDEN)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0, 1) doubles: top 53 bits of each draw times 2^-53."""
    bits = splitmix64(seed, stream, count, offset) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """N(0, 1) doubles by Box--Muller on consecutive uniform pairs."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# --------------------------------------------------------------------------- meshes


def lattice_mesh(d: int, N: int, jitter: float = 0.0, seed: int = 0):
    """Structured simplex mesh of the unit square (d=2) or cube (d=3).

    Vertex (i, j[, l]) has id i + (N+1) j [+ (N+1)^2 l] and sits at (i, j[, l]) / N.
    2D: square (i, j) gives cells 2(i + N j) + t,
        t=0: [v(i,j), v(i+1,j), v(i+1,j+1)],  t=1: [v(i,j), v(i,j+1), v(i+1,j+1)].
    3D: cube (i, j, l) gives cells 6(i + N j + N^2 l) + k, where k enumerates the
        axis permutations pi in lexicographic order and the tetrahedron is the
        lattice path o, o+e_pi0, o+e_pi0+e_pi1, o+(1,1,1).
    Jitter moves every interior vertex coordinate by h*jitter*(2U-1), h = 1/N.

    Returns (coords float64 [n_v, d], cells int32 [E, d+1]).
    """
    if d not in (2, 3):
        raise ValueError("d must be 2 or 3")
    if N < 1:
        raise ValueError("N must be >= 1")
    n1 = N + 1
    grids = np.meshgrid(*([np.arange(n1)] * d), indexing="ij")
    # vertex id = i + n1 j + n1^2 l  -> x index fastest
    ijk = np.stack([g.transpose(tuple(range(d))[::-1]).reshape(-1) for g in grids], axis=1)
    coords = ijk.astype(np.float64) / N
    if jitter:
        interior = np.all((ijk > 0) & (ijk < N), axis=1)
        u = uniform(seed, STREAM_JITTER, coords.size).reshape(coords.shape)
        coords = coords + np.where(interior[:, None], (jitter / N) * (2.0 * u - 1.0), 0.0)

    def vid(*c):
        out = c[0].copy()
        mul = n1
        for ci in c[1:]:
            out = out + mul * ci
            mul *= n1
        return out

    if d == 2:
        j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        i = i.reshape(-1)
        j = j.reshape(-1)
        c0 = np.stack([vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)], axis=1)
        c1 = np.stack([vid(i, j), vid(i, j + 1), vid(i + 1, j + 1)], axis=1)
        cells = np.stack([c0, c1], axis=1).reshape(-1, 3)
    else:
        l, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        o = np.stack([i.reshape(-1), j.reshape(-1), l.reshape(-1)], axis=1)
        tets = []
        for perm in itertools.permutations(range(3)):
            e0 = np.zeros(3, dtype=np.int64)
            e0[perm[0]] = 1
            e1 = e0.copy()
            e1[perm[1]] = 1
            path = [o, o + e0, o + e1, o + 1]
            tets.append(np.stack([vid(p[:, 0], p[:, 1], p[:, 2]) for p in path], axis=1))
        cells = np.stack(tets, axis=1).reshape(-1, 4)
    return coords, cells.astype(np.int32)


def lattice_boundary_vertices(coords: np.ndarray, N: int) -> np.ndarray:
    """uint8 flags of vertices on the boundary of the unit square/cube lattice."""
    ijk = np.rint(coords * N)
    return np.any((ijk <= 0) | (ijk >= N), axis=1).astype(np.uint8)


def centroids(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """Vertex mean of every cell, used to sample cell-wise coefficient fields."""
    return coords[cells].mean(axis=1)


# ------------------------------------------------------------------- coefficients


def coef_uniform(E: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Per-element scalar drawn from U[lo, hi)."""
    return lo + (hi - lo) * uniform(seed, STREAM_COEF, E)


def coef_lognormal(E: int, sigma: float, seed: int, mu: float = 0.0) -> np.ndarray:
    """Per-element scalar exp(mu + sigma * N(0,1))."""
    return np.exp(mu + sigma * normal(seed, STREAM_COEF, E))


def _rotations3(E: int, seed: int) -> np.ndarray:
    """Uniform random rotations from normalised Gaussian quaternions."""
    q = normal(seed, STREAM_ANGLE, 4 * E).reshape(E, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack(
        [
            np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], 1),
            np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], 1),
            np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], 1),
        ],
        axis=1,
    )


def coef_tensor_lognormal(E: int, d: int, sigma: float, seed: int) -> np.ndarray:
    """Per-element SPD d x d tensors Q diag(exp(g)) Q^T, g ~ N(0, sigma^2).

    2D: Q is the rotation by theta ~ U[0, pi).  3D: Q is a uniform random rotation.
    Returns float64 [E, d, d] (exactly symmetric: assembled as Q D Q^T then averaged
    with its transpose).
    """
    g = sigma * normal(seed, STREAM_EIG, d * E).reshape(E, d)
    if d == 2:
        th = np.pi * uniform(seed, STREAM_ANGLE, E)
        c, s = np.cos(th), np.sin(th)
        Q = np.stack([np.stack([c, -s], 1), np.stack([s, c], 1)], axis=1)
    else:
        Q = _rotations3(E, seed)
    A = np.einsum("eik,ek,ejk->eij", Q, np.exp(g), Q)
    return 0.5 * (A + A.transpose(0, 2, 1))


def inclusion_balls(d: int, n_incl: int, rmin: float, rmax: float, seed: int):
    """``n_incl`` balls: centres U[0,1]^d, radii U[rmin, rmax]."""
    ctr = uniform(seed, STREAM_INCL_CENTRE, n_incl * d).reshape(n_incl, d)
    rad = rmin + (rmax - rmin) * uniform(seed, STREAM_INCL_RADIUS, n_incl)
    return ctr, rad


def inclusion_field(centres: np.ndarray, radii: np.ndarray, inside: float, outside: float):
    """The field m(x) = ``inside`` in the union of the balls (|x - c|^2 <= r^2),
    ``outside`` elsewhere, as a function of points [..., d]."""
    def m(X):
        X = np.asarray(X, dtype=np.float64)
        hit = np.zeros(X.shape[:-1], dtype=bool)
        for c, r in zip(centres, radii):
            hit |= np.sum((X - c) ** 2, axis=-1) <= r * r
        return np.where(hit, inside, outside)
    return m


def coef_inclusions(cent: np.ndarray, n_incl: int, rmin: float, rmax: float, seed: int,
                    inside: float = 100.0, outside: float = 1.0) -> np.ndarray:
    """Per-element scalar: the inclusion field of ``inclusion_balls`` at the element
    centroid."""
    ctr, rad = inclusion_balls(cent.shape[1], n_incl, rmin, rmax, seed)
    return inclusion_field(ctr, rad, inside, outside)(cent)


def rhs_normal(n: int, R: int, seed: int) -> np.ndarray:
    """Dof-major [n, R] N(0, 1) nodal loads."""
    return normal(seed, STREAM_RHS, n * R).reshape(n, R)


def pick(seed: int, count: int, upper: int) -> np.ndarray:
    """``count`` indices drawn uniformly from [0, upper) (with replacement)."""
    return np.minimum((uniform(seed, STREAM_PICK, count) * upper).astype(np.int64), upper - 1)


def uneven_problems(count: int, seed: int, nmin: int = 16, nmax: int = 128, pmax: int = 3):
    """Problem list of a batched load: (N_k, p_k, coefficient seed) per problem,
    N_k ~ U{nmin..nmax}, p_k ~ U{1..pmax}."""
    u = uniform(seed, STREAM_PROBLEM, 2 * count).reshape(count, 2)
    Ns = nmin + np.minimum((u[:, 0] * (nmax - nmin + 1)).astype(np.int64), nmax - nmin)
    ps = 1 + np.minimum((u[:, 1] * pmax).astype(np.int64), pmax - 1)
    return [(int(N), int(p), seed * 1000 + k) for k, (N, p) in enumerate(zip(Ns, ps))]
