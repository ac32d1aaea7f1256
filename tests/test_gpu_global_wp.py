"""Global (continuous-W) DoGIP for the weighted projection (global_w contexts)
against the oracle (oracle/global_wp.py): the W-node map and owner flags bit-exact,
A_diag to 1e-13, the FP64 apply to 1e-12 and the FP32 apply to 2e-5 of the rounding
scale |B|^T |A_diag| |B| |u|, a solve to its tolerance, and the rejections."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import global_wp  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [(2, p) for p in (1, 2, 3, 4)] + [(3, p) for p in (1, 2, 3)]
IDS = [f"{d}D-P{p}" for d, p in CASES]


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def _make(B, d, p, N, seed=1):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    coef = inputs.coef_uniform(len(cells), 1.0, 10.0, seed)
    ctx = B.Context(coords, cells, p, "projection", coef, global_w=True)
    G = global_wp.GlobalProblem(p, coords, cells, coef)
    return ctx, G


@pytest.mark.parametrize("R", [1, 3])
@pytest.mark.parametrize("d,p", CASES, ids=IDS)
def test_global_wp_parity(B, d, p, R):
    ctx, G = _make(B, d, p, 11 if d == 2 else 3)
    assert ctx.info.n_wglobal == G.nW
    ids, own = ctx.wdofmap()
    assert np.array_equal(ids, G.connW) and np.array_equal(own, G.own)
    A = ctx.ahat_global().cpu().numpy()
    np.testing.assert_allclose(A, G.A, rtol=1e-13, atol=0)
    np.testing.assert_allclose(ctx.diag().cpu().numpy(), G.diag(), rtol=1e-13, atol=0)
    u = inputs.rhs_normal(G.n, R, seed=9)
    y = ctx.apply(torch.tensor(u if R > 1 else u[:, 0], device="cuda")).cpu().numpy().reshape(G.n, R)
    assert np.all(np.abs(y - G.apply(u)) <= 1e-12 * G.apply_abs(u))
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32 if R > 1 else u32[:, 0], device="cuda"), prec="fp32")
    y32 = y32.cpu().numpy().astype(np.float64).reshape(G.n, R)
    u64 = u32.astype(np.float64)
    assert np.all(np.abs(y32 - G.apply(u64)) <= 2e-5 * G.apply_abs(u64))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_global_wp_solve(B, mode):
    ctx, G = _make(B, 2, 2, 24, seed=4)
    b = ctx.load()
    x, info = ctx.solve(b, mode=mode, tol=1e-10)
    r = b.cpu().numpy() - G.apply(x.cpu().numpy())
    assert info["status"] == 0 and np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())


def test_global_wp_memory_and_rejects(B):
    coords, cells = inputs.lattice_mesh(2, 16)
    coef = np.ones(len(cells))
    g = B.Context(coords, cells, 1, "projection", coef, global_w=True)
    e = B.Context(coords, cells, 1, "projection", coef)
    assert g.info.bytes_ahat_fp64 == g.info.n_wglobal * 8 == (2 * 16 + 1) ** 2 * 8
    assert e.info.bytes_ahat_fp64 == len(cells) * 6 * 8
    for kw in (dict(form="elliptic"), dict(factorized=True), dict(scatter="colour"),
               dict(dirichlet=True)):
        form = kw.pop("form", "projection")
        with pytest.raises(B.DogipError) as ex:
            B.Context(coords, cells, 1, form, coef, global_w=True, **kw)
        assert ex.value.code == B.EINVAL
    with pytest.raises(B.DogipError) as ex:
        g.set_coef_inclusions(np.zeros((1, 2)) + 0.5, np.array([0.1]), 2.0, 1.0, 4)
    assert ex.value.code == B.EUNSUPPORTED
    with pytest.raises(B.DogipError):
        g.ahat()
