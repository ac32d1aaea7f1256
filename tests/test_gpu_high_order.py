"""Higher orders (2D p = 5..8, 3D p = 4: the rows of Tables 1-4 above the orders with
compile-time tables), served by the run-time-table kernels, against the FP64 oracle:
A_T and the diagonal to 1e-13, the FP64 apply to 1e-12 and the FP32 apply to 2e-5 of
the rounding scale |B|^T |A_T| |B| |u| (longest FP32 dependency chain W_T*NB + V_T
<= 285 terms here, times the unit roundoff 6e-8 = 1.7e-5), atomic and colour scatter,
one and three right-hand sides; a mixed solve; the operations that are not built for
these orders fail with DOGIP_EUNSUPPORTED."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [(2, p, f) for p in (5, 6, 7, 8) for f in ("elliptic", "projection")] + \
        [(3, 4, f) for f in ("elliptic", "projection")]
IDS = [f"{d}D-P{p}-{f}" for d, p, f in CASES]


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def _make(B, d, p, form, N, seed=1, scatter="atomic"):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    E = len(cells)
    coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed) if form == "elliptic" else \
        inputs.coef_uniform(E, 1.0, 10.0, seed)
    ctx = B.Context(coords, cells, p, form, coef, scatter=scatter)
    return ctx, odogip.Problem(form, p, coords, cells, coef)


def _pack(P):
    if P.form == "projection":
        return P.Ah[:, :, None]
    idx = [(r, s) for r in range(P.d) for s in range(r, P.d)]
    return np.stack([P.Ah[:, :, r, s] for r, s in idx], axis=-1)


@pytest.mark.parametrize("scatter", ["atomic", "colour"])
@pytest.mark.parametrize("d,p,form", CASES, ids=IDS)
def test_high_order_parity(B, d, p, form, scatter):
    ctx, P = _make(B, d, p, form, 7 if d == 2 else 2, scatter=scatter)
    assert ctx.n == P.n and np.array_equal(ctx.dofmap(), P.conn)
    A = ctx.ahat().cpu().numpy()
    ref = _pack(P)
    assert np.all(np.abs(A - ref) <= 1e-13 * np.abs(ref).max(axis=(1, 2), keepdims=True))
    np.testing.assert_allclose(ctx.diag().cpu().numpy(), P.diag(), rtol=1e-13, atol=0)
    for R in (1, 3):
        u = inputs.rhs_normal(P.n, R, seed=5)
        y = ctx.apply(torch.tensor(u if R > 1 else u[:, 0], device="cuda"), scatter=scatter)
        y = y.cpu().numpy().reshape(P.n, R)
        assert np.all(np.abs(y - P.apply(u)) <= 1e-12 * P.apply_abs(u))
        u32 = u.astype(np.float32)
        y32 = ctx.apply(torch.tensor(u32 if R > 1 else u32[:, 0], device="cuda"), prec="fp32",
                        scatter=scatter)
        y32 = y32.cpu().numpy().astype(np.float64).reshape(P.n, R)
        u64 = u32.astype(np.float64)
        assert np.all(np.abs(y32 - P.apply(u64)) <= 2e-5 * P.apply_abs(u64)), \
            (np.abs(y32 - P.apply(u64)) / P.apply_abs(u64)).max()


def test_high_order_solve_and_load(B):
    ctx, P = _make(B, 2, 6, "elliptic", 8, seed=3)
    b = ctx.load()
    bref = odogip.load_const(2, 6, P.coords, P.cells, P.conn, P.n, np.ones(len(P.cells)))
    bref[P.bmask] = 0.0
    assert np.all(np.abs(b.cpu().numpy() - bref) <= 1e-13 * np.abs(bref).max())
    x, info = ctx.solve(b, mode="mixed", tol=1e-9)
    r = b.cpu().numpy() - P.apply(x.cpu().numpy())
    assert info["status"] == 0 and np.linalg.norm(r) <= 1.01e-9 * np.linalg.norm(b.cpu().numpy())


def test_high_order_unbuilt_operations(B):
    ctx, P = _make(B, 2, 5, "elliptic", 4)
    u = torch.tensor(inputs.rhs_normal(P.n, 1, seed=2)[:, 0], device="cuda")
    for call in (lambda: ctx.apply_qp(u), lambda: ctx.grad_coef(u, u),
                 lambda: ctx.set_coef_inclusions(np.full((1, 2), 0.5), np.array([0.1]), 2., 1., 4)):
        with pytest.raises(B.DogipError) as e:
            call()
        assert e.value.code == B.EUNSUPPORTED
    coords, cells = inputs.lattice_mesh(2, 4)
    with pytest.raises(B.DogipError) as e:
        B.Context(coords, cells, 6, "elliptic", np.ones(len(cells)), factorized=True)
    assert e.value.code == B.EUNSUPPORTED
    ctx.autotune()  # the run-time-table kernel against the tensor cores; must not fail
