"""The allocation-free residual-norm entry point (dogip_residual_norms_noalloc).

Callers that cannot allocate device memory -- a framework whose allocator owns
all device memory, a latency-critical loop that cannot afford cudaMalloc/cudaFree,
a process under a fixed memory budget -- get the FP64 relative residual
||b - K u|| / ||b|| from a kernel whose reduction scratch is a fixed array inside
the library.  This test calls it through the C ABI twice in a row and checks each
result against the relative residual that dogip_solve (whose kernel reduces into
memory the library allocated) reports for the same solution.

This file is collected last on purpose: it also has to pass in a fresh process.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_solve():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding as B

    # The first call on the device resolves the scratch address; it comes before the
    # solves below, which capture CUDA graphs (its result is checked too).
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert B.residual_norms_noalloc(z, z).cpu().numpy()[0] == 0.0

    coords, cells = inputs.lattice_mesh(2, 24, 0.2, seed=5)
    A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=5)
    # colour scatter: the solve's final residual and the apply below see the same K u
    ctx = B.Context(coords, cells, 2, "elliptic", A, scatter="colour")
    bmask = torch.tensor(ctx.boundary(), device="cuda")
    b4 = torch.tensor(inputs.rhs_normal(ctx.n, 4, seed=6), device="cuda")
    b4[bmask] = 0.0
    u4, info4 = ctx.solve(b4, mode="mixed", tol=1e-9, scatter="colour")
    Ku4 = ctx.apply(u4, scatter="colour")
    b1 = ctx.load()
    u1, info1 = ctx.solve(b1, mode="fp64", tol=1e-10, scatter="colour")
    Ku1 = ctx.apply(u1, scatter="colour")

    # call 1: four right-hand sides of a mixed-precision solve
    r4 = torch.empty_like(b4)
    rel4 = B.residual_norms_noalloc(b4, Ku4, r4).cpu().numpy()
    np.testing.assert_allclose(rel4, info4["rel_per_rhs"], rtol=1e-12, atol=0)
    assert torch.allclose(r4, b4 - Ku4, rtol=0, atol=0)

    # call 2, right after: one right-hand side of an FP64 solve, no residual output
    rel1 = B.residual_norms_noalloc(b1, Ku1).cpu().numpy()
    np.testing.assert_allclose(rel1, info1["rel_per_rhs"], rtol=1e-12, atol=0)
    assert rel1[0] <= 1e-10 and np.all(rel4 <= 1e-9)

    # sizes beyond the static scratch are refused with a clear error
    with pytest.raises(B.DogipError) as e:
        B.residual_norms_noalloc(torch.zeros((10, 33), dtype=torch.float64, device="cuda"),
                                 torch.zeros((10, 33), dtype=torch.float64, device="cuda"))
    assert e.value.code == B.EINVAL and "32" in str(e.value)


@pytest.mark.parametrize("R", [3, 7, 32])
def test_noalloc_full_grid_against_torch(R):
    """Sizes far above the 256-block grid (every thread loops many times), right-hand
    side counts that do not divide the block size, checked against torch norms; the
    result is the same on a second call (fixed reduction order)."""
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding as B

    g = torch.Generator(device="cuda").manual_seed(11 + R)
    n = 300_001
    b = torch.randn(n, R, dtype=torch.float64, device="cuda", generator=g)
    Ky = b + 1e-3 * torch.randn(n, R, dtype=torch.float64, device="cuda", generator=g)
    r = torch.empty_like(b)
    rel = B.residual_norms_noalloc(b, Ky, r)
    ref = torch.linalg.vector_norm(b - Ky, dim=0) / torch.linalg.vector_norm(b, dim=0)
    torch.testing.assert_close(rel, ref, rtol=1e-13, atol=0)
    assert torch.equal(r, b - Ky)
    assert torch.equal(B.residual_norms_noalloc(b, Ky), rel)


def test_noalloc_empty():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding as B

    e = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    rel = B.residual_norms_noalloc(e, e)
    assert rel.shape == (5,) and torch.all(rel == 0)
