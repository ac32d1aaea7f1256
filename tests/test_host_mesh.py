"""Host-side mesh preprocessing of the library (dof numbering, Dirichlet boundary,
greedy colouring, W nodes of the global double grid) on the CPU, through the
host-only C ABI, bit-exact against the oracle's independent implementations
(oracle/topology.py, oracle/global_wp.py) — lattice meshes in lattice order and in a
shuffled cell order, 2D p = 1..8 and 3D p = 1..4."""

import numpy as np
import pytest

from oracle import global_wp, topology
from paper_1710_09913_gb300 import inputs

B = pytest.importorskip("paper_1710_09913_gb300.binding")

CASES = [(2, p) for p in range(1, 9)] + [(3, p) for p in range(1, 5)]


def _meshes(d):
    coords, cells = inputs.lattice_mesh(d, 5 if d == 2 else 3, 0.0, 1)
    perm = np.random.default_rng(3).permutation(len(cells))
    # shuffled cells, and each cell's vertices rotated (same simplices, other local order)
    shuffled = np.roll(cells[perm], 1, axis=1)
    return [cells.astype(np.int64), shuffled.astype(np.int64)]


@pytest.mark.parametrize("d,p", CASES)
def test_dofmap_and_boundary_bit_exact(d, p):
    for cells in _meshes(d):
        ids, n = B.mesh_dofmap(cells, p)
        ref, nref = topology.dofmap(cells, p)
        assert n == nref and np.array_equal(ids, ref)
        mask = B.mesh_boundary(cells, p)
        assert np.array_equal(mask, topology.boundary_mask(cells, ref, p, nref))


@pytest.mark.parametrize("d", [2, 3])
def test_colouring_bit_exact_and_greedy(d):
    for cells in _meshes(d):
        col, nc = B.mesh_colouring(cells)
        ref = topology.colouring(cells)
        assert np.array_equal(col, ref) and nc == ref.max() + 1
        assert topology.colouring_is_greedy(cells, col)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)])
def test_wdofmap_and_owners_bit_exact(d, p):
    for cells in _meshes(d):
        ids, own, n = B.mesh_wdofmap(cells, p)
        ref, nref = global_wp.w_dofmap(cells, p)
        assert n == nref and np.array_equal(ids, ref)
        assert np.array_equal(own, global_wp.owners(ref))


def test_dofmap_matches_plain_loop_on_a_small_mesh():
    cells = _meshes(2)[1][:20]
    for p in (1, 3, 6):
        ids, n = B.mesh_dofmap(cells, p)
        ref, nref = topology.dofmap_loop(cells, p)
        assert n == nref and np.array_equal(ids, ref)


def test_host_mesh_rejects_bad_input():
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    for dim, p in ((4, 1), (2, 0), (2, 17)):
        code = B.lib.dogip_mesh_dofmap(dim, p, 1, cells.ctypes.data_as(B._vp), None, None)
        assert code == B.EINVAL
    with pytest.raises(B.DogipError) as e:
        B.mesh_dofmap(np.array([[0, -1, 2]]), 1)
    assert e.value.code == B.EINVAL
