"""torch.autograd.Function parity (GPU): apply backward, adjoint solve backward and
the W-node outer-product coefficient gradient.

The compliance J(A) = b^T u(A), K(A) u = b, has dJ/dA_T = -(dK/dA_T)[u, u].
Finite differences use the stationary form J = 2 b^T u - u^T K u (its error is
quadratic in the solve error), central steps of 1e-4 on FP32 leaf tensors cast to
FP64, perturbing A_pq and A_qp together; tolerance 1e-5 relative to max |dJ/dA|.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip, gradient as ograd  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import autograd, binding
    return binding, autograd


def _case(B, d, p, N, seed=4):
    coords, cells = inputs.lattice_mesh(d, N)
    E = len(cells)
    A = inputs.coef_tensor_lognormal(E, d, 0.5, seed).astype(np.float32)
    ctx = B.Context(coords, cells, p, "elliptic", A.astype(np.float64))
    return coords, cells, A, ctx


def test_apply_backward_is_symmetric_operator(mods):
    B, AG = mods
    coords, cells, A, ctx = _case(B, 2, 2, 16)
    u = torch.randn(ctx.n, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.randn(ctx.n, dtype=torch.float64, device="cuda")
    y = AG.dogip_apply(u, ctx)
    (w @ y).backward()
    ref = ctx.apply(w).detach()
    assert torch.allclose(u.grad, ref, rtol=0, atol=1e-12 * ref.abs().max().item())


@pytest.mark.parametrize("d,p,N", [(2, 3, 16), (3, 1, 6)])
def test_compliance_gradient_vs_oracle_and_fd(mods, d, p, N):
    B, AG = mods
    coords, cells, A32, ctx = _case(B, d, p, N)
    E = len(cells)
    leaf = torch.tensor(A32, device="cuda", requires_grad=True)
    b = ctx.load()
    J = AG.compliance(leaf, b, ctx, mode="fp64", tol=1e-13)
    J.backward()
    g = leaf.grad.double().cpu().numpy()
    # oracle: its own solve (direct) and its assembled-matrix adjoint gradient
    A64 = A32.astype(np.float64)
    P = odogip.Problem("elliptic", p, coords, cells, A64)
    from oracle import assembly
    import scipy.sparse.linalg as spla
    K = assembly.dirichlet(assembly.assemble("elliptic", p, coords, cells, P.conn, P.n, A64), P.bmask)
    bb = odogip.load_const(d, p, coords, cells, P.conn, P.n, np.ones(E))
    bb[P.bmask] = 0.0
    u = spla.spsolve(K.tocsc(), bb)
    ref = ograd.grad_coef_assembled("elliptic", p, coords, cells, P.conn, u, u)
    ref = 0.5 * (ref + ref.transpose(0, 2, 1))
    # both sides solve K u = b independently (GPU PCG to 1e-13, oracle direct): the
    # gradient inherits the solution error ~ cond(K) * 1e-13 ~ 1e-8; the kernel itself
    # is checked on identical (u, lambda) to 1e-12 in the full-size test below
    assert np.abs(g - ref).max() <= 1e-6 * np.abs(ref).max()
    # central finite differences of the stationary compliance on seeded elements
    A_dev = torch.tensor(A64, device="cuda")
    x0, _ = ctx.solve(b, mode="fp64", tol=1e-13)

    def Jst(Ap):
        ctx.set_coef(Ap)
        x, _ = ctx.solve(b, x0.clone(), mode="fp64", tol=1e-12, x0=True)
        return float(2 * (b @ x) - x @ ctx.apply(x))

    h = 1e-4
    for e in inputs.pick(21, 6, E):
        for a_, c_ in [(0, 0), (0, 1), (d - 1, d - 1)]:
            Ap = A_dev.clone()
            Am = A_dev.clone()
            Ap[e, a_, c_] += h
            Am[e, a_, c_] -= h
            if a_ != c_:
                Ap[e, c_, a_] += h
                Am[e, c_, a_] -= h
            fd = (Jst(Ap) - Jst(Am)) / (2 * h)
            an = g[e, a_, c_] + (g[e, c_, a_] if a_ != c_ else 0.0)
            assert abs(fd - an) <= 1e-5 * np.abs(g).max(), (e, a_, c_, fd, an)
    ctx.set_coef(A_dev)


@pytest.mark.parametrize("d,p,N", [(2, 3, 256), (3, 1, 32)])
def test_coefficient_gradient_full_size(mods, d, p, N):
    """Config sizes (256^2 P3 triangles, 32^3 P1 tetrahedra): the outer-product
    backward on seeded (u, lambda) equals the oracle's W-node and assembled forms."""
    B, AG = mods
    coords, cells, A32, ctx = _case(B, d, p, N)
    E = len(cells)
    u = inputs.rhs_normal(ctx.n, 1, seed=31)[:, 0]
    lam = inputs.rhs_normal(ctx.n, 1, seed=32)[:, 0]
    P = odogip.Problem("elliptic", p, coords, cells, A32.astype(np.float64))
    u[P.bmask] = 0.0
    lam[P.bmask] = 0.0
    g = ctx.grad_coef(torch.tensor(u, device="cuda"), torch.tensor(lam, device="cuda")).cpu().numpy()
    ref = ograd.grad_coef_dogip("elliptic", p, coords, cells, P.conn, u, lam)
    assert np.all(np.abs(g - ref) <= 1e-12 * np.abs(ref).max())
    ref2 = ograd.grad_coef_assembled("elliptic", p, coords, cells, P.conn, u, lam)
    assert np.all(np.abs(g - ref2) <= 1e-11 * np.abs(ref2).max())
    # one adjoint solve at full size satisfies K lambda = g (oracle apply)
    gsrc = torch.tensor(lam, device="cuda")
    x, info = ctx.solve(gsrc, mode="mixed", tol=1e-8)
    r = lam - P.apply(x.cpu().numpy())
    assert info["status"] == 0 and np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(lam)
