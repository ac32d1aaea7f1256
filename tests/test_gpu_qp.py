"""The quadrature-point matrix-free comparator (dogip_apply_qp) against the oracle.

For element-constant coefficients it computes the Galerkin operator, so the
reference is the oracle's DoGIP apply; the componentwise tolerance scale is the
oracle's quadrature-point evaluation with absolute values of every factor
(|B_q|^T |w_q R^-1 M R^-T| |B_q| |u|), the rounding scale of this evaluation order.
FP64 1e-12; FP32 2e-5 of that scale (the geometry is formed in FP32 after FP64
edge vectors: a few extra roundings, well inside the budget)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip, matfree  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

SMALL = [(2, p, f) for p in (1, 2, 3, 4) for f in ("elliptic", "projection")] + \
        [(3, p, f) for p in (1, 2, 3) for f in ("elliptic", "projection")]
IDS = [f"{d}D-P{p}-{f}" for d, p, f in SMALL]
NSMALL = {2: 11, 3: 3}


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def _make(B, d, p, form, N, seed=1):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    E = len(cells)
    coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed) if form == "elliptic" else \
        inputs.coef_uniform(E, 1.0, 10.0, seed)
    ctx = B.Context(coords, cells, p, form, coef)
    P = odogip.Problem(form, p, coords, cells, coef)
    return ctx, P, coords, cells, coef


@pytest.mark.parametrize("R", [1, 3])
@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_qp_apply_parity(B, d, p, form, R):
    ctx, P, coords, cells, coef = _make(B, d, p, form, NSMALL[d])
    u = inputs.rhs_normal(P.n, R, seed=21)
    ref = P.apply(u)
    sc = matfree.apply(form, p, coords, cells, coef, P.conn, u, P.bmask, absolute=True)
    y = ctx.apply_qp(torch.tensor(u if R > 1 else u[:, 0], device="cuda")).cpu().numpy()
    y = y.reshape(P.n, R)
    assert np.all(np.abs(y - ref) <= TOL64 * sc), (np.abs(y - ref) / sc).max()
    u32 = u.astype(np.float32)
    y32 = ctx.apply_qp(torch.tensor(u32 if R > 1 else u32[:, 0], device="cuda"), prec="fp32")
    y32 = y32.cpu().numpy().astype(np.float64).reshape(P.n, R)
    u64 = u32.astype(np.float64)
    sc32 = matfree.apply(form, p, coords, cells, coef, P.conn, u64, P.bmask, absolute=True)
    assert np.all(np.abs(y32 - P.apply(u64)) <= TOL32 * sc32), (np.abs(y32 - P.apply(u64)) / sc32).max()


def test_qp_full_size_2d_p4(B):
    """512 x 512 jittered grid, lognormal SPD tensors, P4: sampled outputs against the
    oracle evaluated on the cells that touch them, FP64 and FP32."""
    coords, cells = inputs.lattice_mesh(2, 512, 0.2, seed=2)
    A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=2)
    ctx = B.Context(coords, cells, 4, "elliptic", A)
    P = odogip.Problem("elliptic", 4, coords, cells, A)
    samples = inputs.pick(17, 3000, P.n)
    touch = np.isin(P.conn, samples).any(axis=1)
    u = inputs.rhs_normal(P.n, 1, seed=22)[:, 0]
    for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
        uu = u if prec == "fp64" else u.astype(np.float32).astype(np.float64)
        ug = torch.tensor(uu if prec == "fp64" else uu.astype(np.float32), device="cuda")
        y = ctx.apply_qp(ug, prec=prec).cpu().numpy().astype(np.float64)
        ref = odogip.apply("elliptic", P.Bh, P.Ah[touch], P.conn[touch], uu, P.bmask)[samples]
        sc = matfree.apply("elliptic", 4, coords, cells[touch], A[touch], P.conn[touch], uu, P.bmask,
                           absolute=True)[samples]
        assert np.all(np.abs(y[samples] - ref) <= tol * sc), prec


def test_qp_rejected_after_inclusions_and_restored(B):
    coords, cells = inputs.lattice_mesh(2, 6, 0.2, 3)
    coef = np.full(len(cells), 2.0)
    ctx = B.Context(coords, cells, 2, "elliptic", coef)
    u = torch.tensor(inputs.rhs_normal(ctx.n, 1, seed=3)[:, 0], device="cuda")
    y0 = ctx.apply_qp(u).cpu().numpy()
    ctr, rad = inputs.inclusion_balls(2, 3, 0.1, 0.2, seed=3)
    ctx.set_coef_inclusions(ctr, rad, 10.0, 1.0, 4)
    with pytest.raises(B.DogipError) as e:
        ctx.apply_qp(u)
    assert e.value.code == B.EUNSUPPORTED
    ctx.set_coef(torch.tensor(coef, device="cuda"))
    y1 = ctx.apply_qp(u).cpu().numpy()  # atomic scatter: equal up to summation order
    assert np.all(np.abs(y1 - y0) <= 1e-13 * np.abs(y0).max())
    with pytest.raises(B.DogipError):  # unknown precision, rejected by the library
        ctx.apply_qp(u.float(), prec=7)
