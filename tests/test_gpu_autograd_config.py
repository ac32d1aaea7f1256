"""Compliance gradient at the sizes of the differentiation workload: 256 x 256
squares x 2 triangles at P3 (131,072 cells, 591,361 dofs) and the 32^3 cube x 6
tetrahedra at P1 (196,608 cells), FP32 leaf SPD tensors with log-eigenvalues
N(0, 0.5^2), J = b^T u with b from f = 1 and zero Dirichlet data.

* The gradient through torch.autograd (adjoint solve + W-node outer product) is
  compared with the oracle's assembled-matrix adjoint gradient, the oracle taking
  its own solution (sparse LU of its assembled matrix, refined twice in FP64), at
  1e-5 of max |dJ/dA|.
* Central finite differences, step 1e-4 in FP64 on the FP32 leaf values cast up, on
  50 seeded elements (one seeded entry each; off-diagonal entries perturbed
  symmetrically and compared with g_pq + g_qp), of the stationary compliance
  J = 2 b^T x - x^T K x re-solved to 1e-10 from the unperturbed solution (its error
  is quadratic in the solve error, and the part common to both solves cancels in the
  difference; 1e-10 is near the FP64 rounding floor of the residual at P3), at 1e-5
  of max |dJ/dA|.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assembly, dogip as odogip, gradient as ograd  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import autograd, binding
    return binding, autograd


def _oracle_gradient(d, p, coords, cells, A64):
    import scipy.sparse.linalg as spla
    P = odogip.Problem("elliptic", p, coords, cells, A64)
    K = assembly.dirichlet(assembly.assemble("elliptic", p, coords, cells, P.conn, P.n, A64),
                           P.bmask).tocsc()
    b = odogip.load_const(d, p, coords, cells, P.conn, P.n, np.ones(len(cells)))
    b[P.bmask] = 0.0
    lu = spla.splu(K)
    u = lu.solve(b)
    for _ in range(2):  # iterative refinement of the direct solution
        u += lu.solve(b - K @ u)
    assert np.linalg.norm(b - K @ u) <= 1e-10 * np.linalg.norm(b)
    g = ograd.grad_coef_assembled("elliptic", p, coords, cells, P.conn, u, u)
    return 0.5 * (g + g.transpose(0, 2, 1))


@pytest.mark.parametrize("d,p,N", [(2, 3, 256), (3, 1, 32)], ids=["2D-P3-256", "3D-P1-32"])
def test_compliance_gradient_config_size(mods, d, p, N):
    B, AG = mods
    coords, cells = inputs.lattice_mesh(d, N)
    E = len(cells)
    A32 = inputs.coef_tensor_lognormal(E, d, 0.5, 4).astype(np.float32)
    A64 = A32.astype(np.float64)
    ctx = B.Context(coords, cells, p, "elliptic", A64)
    leaf = torch.tensor(A32, device="cuda", requires_grad=True)
    b = ctx.load()
    J = AG.compliance(leaf, b, ctx, mode="mixed", tol=1e-10)
    J.backward()
    g = leaf.grad.double().cpu().numpy()
    ref = _oracle_gradient(d, p, coords, cells, A64)
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max(), np.abs(g - ref).max() / np.abs(ref).max()

    A_dev = torch.tensor(A64, device="cuda")
    ctx.set_coef(A_dev)
    x0, _ = ctx.solve(b, mode="mixed", tol=1e-10)

    def Jst(Ap):
        ctx.set_coef(Ap)
        x, info = ctx.solve(b, x0.clone(), mode="mixed", tol=1e-10, x0=True)
        assert info["status"] == 0
        return float(2 * (b @ x) - x @ ctx.apply(x))

    entries = [(r, s) for r in range(d) for s in range(r, d)]
    rng = np.random.default_rng(23)
    h, gmax = 1e-4, np.abs(g).max()
    for e in inputs.pick(22, 50, E):
        a_, c_ = entries[rng.integers(len(entries))]
        Ap, Am = A_dev.clone(), A_dev.clone()
        Ap[e, a_, c_] += h
        Am[e, a_, c_] -= h
        if a_ != c_:
            Ap[e, c_, a_] += h
            Am[e, c_, a_] -= h
        fd = (Jst(Ap) - Jst(Am)) / (2 * h)
        an = g[e, a_, c_] + (g[e, c_, a_] if a_ != c_ else 0.0)
        assert abs(fd - an) <= 1e-5 * gmax, (e, a_, c_, fd, an, gmax)
    ctx.set_coef(A_dev)
