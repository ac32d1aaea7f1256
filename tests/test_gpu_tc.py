"""GPU parity of the tensor-core FP32 apply (tcgen05, variant 3) against the FP64 oracle.

The two contractions with the reference table run as 3xTF32 MMAs (hi.hi + hi.lo +
lo.hi, FP32 accumulation): about 2^-21 relative per product, inside the FP32 apply
tolerance 2e-5 (|B|^T |A_T| |B| |u|) componentwise used for every FP32 kernel.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 2e-5

TC = [(2, p, f) for p in (1, 2, 3, 4) for f in ("elliptic", "projection")] + \
     [(3, p, f) for p in (1, 2) for f in ("elliptic", "projection")]
IDS = [f"{d}D-P{p}-{f}" for d, p, f in TC]


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def make(B, d, p, form, N, seed=1):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    E = len(cells)
    coef = (inputs.coef_tensor_lognormal(E, d, 1.0, seed) if form == "elliptic"
            else inputs.coef_uniform(E, 1.0, 10.0, seed))
    return B.Context(coords, cells, p, form, coef), odogip.Problem(form, p, coords, cells, coef)


# 242 / 1,682 triangles, 162 / 750 tetrahedra: one ragged 128-cell tile, then
# several tiles per CTA with a ragged tail
@pytest.mark.parametrize("N2,N3", [(11, 3), (29, 5)], ids=["one-tile", "many-tiles"])
@pytest.mark.parametrize("d,p,form", TC, ids=IDS)
def test_tc_apply_parity(B, d, p, form, N2, N3, monkeypatch):
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    ctx, P = make(B, d, p, form, N2 if d == 2 else N3)
    u = inputs.rhs_normal(P.n, 1, seed=41)[:, 0].astype(np.float32)
    u64 = u.astype(np.float64)
    for _ in range(2):  # the second call reuses the kernel's tensor memory and tables
        y = ctx.apply(torch.tensor(u, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    ctx.check()


# 165,888 triangles = 1,296 tiles of 128 cells: more tiles than warpgroups on a GB300,
# so every warpgroup loops (next-tile conn and gathers in flight across iterations)
# orders above the compiled tables: B^ from the context's run-time table, split in the
# kernel; 2D N = 7 (98 triangles, one ragged tile) and N = 20 (800 triangles)
HI = [(5, "elliptic"), (5, "projection"), (6, "elliptic"), (6, "projection"), (7, "projection")]


@pytest.mark.parametrize("N", [7, 20])
@pytest.mark.parametrize("p,form", HI, ids=[f"P{p}-{f}" for p, f in HI])
def test_tc_high_order_parity(B, p, form, N, monkeypatch):
    _hi_parity(B, 2, p, form, N, monkeypatch)


# 3D P4 projection (Table 2, k = 4): 48 and 384 tetrahedra
@pytest.mark.parametrize("N", [2, 4])
def test_tc_3d_p4_projection_parity(B, N, monkeypatch):
    _hi_parity(B, 3, 4, "projection", N, monkeypatch)


def _hi_parity(B, d, p, form, N, monkeypatch):
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    ctx, P = make(B, d, p, form, N)
    u = inputs.rhs_normal(P.n, 1, seed=47)[:, 0].astype(np.float32)
    u64 = u.astype(np.float64)
    for _ in range(2):
        y = ctx.apply(torch.tensor(u, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    ctx.check()


def test_tc_high_order_autotune_and_solve(B):
    """The autotuner chooses between the run-time-table kernel and the tensor cores for
    a high order; the mixed solve reaches the FP64 tolerance with its choice."""
    ctx, P = make(B, 2, 5, "elliptic", 8)
    t = ctx.autotune(force=True)
    assert t["fp32"][0] in (1, 3)
    b = ctx.load()
    x, info = ctx.solve(b, mode="mixed", tol=1e-10)
    bb = b.cpu().numpy()
    assert info["status"] == 0
    assert np.linalg.norm(bb - P.apply(x.cpu().numpy())) <= 1.01e-10 * np.linalg.norm(bb)
    ctx.check()


@pytest.mark.parametrize("p,form", [(2, "elliptic"), (3, "projection"), (4, "elliptic")])
def test_tc_apply_parity_looping(B, p, form, monkeypatch):
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    ctx, P = make(B, 2, p, form, 288)
    u = inputs.rhs_normal(P.n, 1, seed=43)[:, 0].astype(np.float32)
    u64 = u.astype(np.float64)
    y = ctx.apply(torch.tensor(u, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    ctx.check()


def test_tc_empty_like_inputs(B, monkeypatch):
    """Zero input gives exactly zero (no stale tensor memory or shared-memory tables
    leak into the result); Dirichlet rows copy u."""
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    ctx, P = make(B, 2, 4, "elliptic", 11)
    y = ctx.apply(torch.zeros(P.n, dtype=torch.float32, device="cuda"), prec="fp32")
    assert torch.count_nonzero(y).item() == 0
    u = torch.ones(P.n, dtype=torch.float32, device="cuda")
    y = ctx.apply(u, prec="fp32").cpu().numpy()
    assert np.array_equal(y[P.bmask], np.ones(P.bmask.sum(), dtype=np.float32))
    ctx.check()


@pytest.mark.parametrize("p", [2, 4])
def test_tc_full_size_against_fp64(B, p, monkeypatch):
    """512 x 512 x 2 jittered triangles with lognormal SPD tensors (the benchmark mesh):
    the tensor-core FP32 apply against the FP64 apply (itself oracle-checked) norm-wise,
    and against the error of the CUDA-core FP32 kernel on the same input."""
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    coords, cells = inputs.lattice_mesh(2, 512, 0.2, 2)
    A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, 2)
    ctx = B.Context(coords, cells, p, "elliptic", A)
    u = torch.randn(ctx.n, dtype=torch.float64, device="cuda")
    y64 = ctx.apply(u)
    y32 = ctx.apply(u.float(), prec="fp32").double()
    rel = (torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)).item()
    assert rel <= 1e-5
    # the staged CUDA-core FP32 kernel on the same input: same error scale
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "1")
    ctx1 = B.Context(coords, cells, p, "elliptic", A)
    y1 = ctx1.apply(u.float(), prec="fp32").double()
    rel1 = (torch.linalg.norm(y1 - y64) / torch.linalg.norm(y64)).item()
    assert rel <= 20 * rel1 + 1e-7
    ctx.check()


@pytest.mark.parametrize("form", ["elliptic", "projection"])
def test_tc_mixed_solve(B, form, monkeypatch):
    """Mixed-precision refinement with the tensor-core inner apply reaches the FP64 tolerance."""
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", "3")
    ctx, P = make(B, 2, 3, form, 16)
    b = ctx.load()
    x, info = ctx.solve(b, mode="mixed", tol=1e-10)
    bb = b.cpu().numpy()
    r = bb - P.apply(x.cpu().numpy())
    assert info["status"] == 0
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)
    ctx.check()
