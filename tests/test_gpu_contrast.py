"""High-contrast coefficients in the mixed-precision solve (GPU): spherical inclusions
of contrast 1e2, 1e4 and 1e6 against the matrix value 1 (the paper's niche of rough,
high-contrast coefficients), element values by the centroid rule, 3D P2 elliptic with
zero Dirichlet data and the seeded N(0, 1) loads of the 16-right-hand-side workload
(one right-hand side here).

FP32 stores A_T with FP32's exponent range (about 1e+-38), so contrasts far beyond
1e6 are represented without any per-block scaling: every entry keeps FP32's relative
precision.  What contrast changes is the conditioning; the Jacobi preconditioner
removes the cell-to-cell scale and the FP64 refinement decides convergence.  The test
checks the FP64 true residual with the oracle's own apply, and the solution against
the FP64 PCG solution at the same tolerance."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


@pytest.mark.parametrize("contrast", [1e2, 1e4, 1e6])
def test_mixed_solve_high_contrast(B, contrast):
    coords, cells = inputs.lattice_mesh(3, 10)
    cent = inputs.centroids(coords, cells)
    m = inputs.coef_inclusions(cent, 30, 0.08, 0.2, seed=8, inside=contrast, outside=1.0)
    assert (m == contrast).any() and (m == 1.0).any()
    ctx = B.Context(coords, cells, 2, "elliptic", m)
    P = odogip.Problem("elliptic", 2, coords, cells, m)
    b = inputs.rhs_normal(P.n, 1, seed=9)[:, 0]
    b[P.bmask] = 0.0
    bg = torch.tensor(b, device="cuda")
    x, info = ctx.solve(bg, mode="mixed", tol=1e-8)
    assert info["status"] == 0
    xx = x.cpu().numpy()
    r = b - P.apply(xx)
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(b)
    x64, info64 = ctx.solve(bg, mode="fp64", tol=1e-10)
    assert info64["status"] == 0
    # both solutions are within sqrt(cond) * tol of the exact one in the energy norm
    # (relative); cond(D^-1 K) grows with the contrast, up to ~1e9 here
    e = xx - x64.cpu().numpy()
    assert e @ P.apply(e) <= 1e-6 * (xx @ b)
