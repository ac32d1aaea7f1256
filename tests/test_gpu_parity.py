"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
* integer artefacts (dof map, boundary set, colouring): bit-exact;
* FP64 apply: |y_gpu - y_oracle| <= 1e-12 (|B|^T |A_T| |B| |u|) componentwise, the
  scale of the rounding error of any evaluation order of Algorithm 1;
* FP32 apply: the same scale times 2e-5 (FP32 unit roundoff 6e-8 times the
  length of the longest dependency chain, below ~300 operations here);
* A_T, diagonal, loads: 1e-14 relative (one FP64 evaluation of a closed form);
* solves: true FP64 relative residual <= tol (FP64 PCG and mixed refinement).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import assembly, dogip as odogip, gradient as ograd, topology as otopo  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def make(B, d, p, form, N, seed=1, scatter="atomic", tensor=True, jitter=None):
    if jitter is None:
        jitter = 0.2 if d == 2 else 0.1
    coords, cells = inputs.lattice_mesh(d, N, jitter, seed)
    E = len(cells)
    if form == "elliptic" and tensor:
        coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed)
    else:
        coef = inputs.coef_uniform(E, 1.0, 10.0, seed)
    ctx = B.Context(coords, cells, p, form, coef, scatter=scatter)
    P = odogip.Problem(form, p, coords, cells, coef)
    return ctx, P


def pack(P):
    """Oracle A_T in the packed layout of dogip_get_ahat: [E, W, n_sym]."""
    if P.form == "projection":
        return P.Ah[:, :, None]
    d = P.d
    idx = [(r, s) for r in range(d) for s in range(r, d)]
    return np.stack([P.Ah[:, :, r, s] for r, s in idx], axis=-1)


SMALL = [(2, p, f) for p in (1, 2, 3, 4) for f in ("elliptic", "projection")] + \
        [(3, p, f) for p in (1, 2, 3) for f in ("elliptic", "projection")]
IDS = [f"{d}D-P{p}-{f}" for d, p, f in SMALL]
NSMALL = {2: 11, 3: 3}  # 242 triangles / 162 tetrahedra: several 32-element tiles + ragged tail


@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_topology_bit_exact(B, d, p, form):
    ctx, P = make(B, d, p, form, NSMALL[d])
    assert ctx.n == P.n
    assert np.array_equal(ctx.dofmap(), P.conn)
    col, nc = ctx.colouring()
    assert np.array_equal(col, otopo.colouring(P.cells))
    assert nc == col.max() + 1
    bm = ctx.boundary()
    if P.bmask is None:
        assert not bm.any()
    else:
        assert np.array_equal(bm, P.bmask)


@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_ahat_and_diag(B, d, p, form):
    ctx, P = make(B, d, p, form, NSMALL[d])
    A = ctx.ahat().cpu().numpy()
    ref = pack(P)
    assert np.all(np.abs(A - ref) <= 1e-14 * np.abs(ref).max(axis=(1, 2), keepdims=True))
    dg = ctx.diag().cpu().numpy()
    np.testing.assert_allclose(dg, P.diag(), rtol=1e-13, atol=0)


@pytest.mark.parametrize("scatter", ["atomic", "colour"])
@pytest.mark.parametrize("R", [1, 3, 16])
@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_apply_fp64(B, d, p, form, R, scatter):
    ctx, P = make(B, d, p, form, NSMALL[d], scatter=scatter)
    u = inputs.rhs_normal(P.n, R, seed=5)
    ug = torch.tensor(u if R > 1 else u[:, 0], device="cuda")
    y = ctx.apply(ug, prec="fp64", scatter=scatter).cpu().numpy().reshape(P.n, R)
    ref = P.apply(u)
    scale = P.apply_abs(u)
    assert np.all(np.abs(y - ref) <= TOL64 * scale), np.abs(y - ref).max()


@pytest.mark.parametrize("R", [1, 16])
@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_apply_fp32(B, d, p, form, R):
    ctx, P = make(B, d, p, form, NSMALL[d])
    u = inputs.rhs_normal(P.n, R, seed=6).astype(np.float32)
    ug = torch.tensor(u if R > 1 else u[:, 0], device="cuda")
    y = ctx.apply(ug, prec="fp32").cpu().numpy().astype(np.float64).reshape(P.n, R)
    u64 = u.astype(np.float64)
    ref = P.apply(u64)
    scale = P.apply_abs(u64)
    assert np.all(np.abs(y - ref) <= TOL32 * scale), (np.abs(y - ref) / scale).max()


@pytest.mark.parametrize("d,p,form", [(2, 2, "elliptic"), (2, 3, "projection"), (3, 2, "elliptic")])
def test_load(B, d, p, form):
    ctx, P = make(B, d, p, form, NSMALL[d])
    f = inputs.coef_uniform(len(P.cells), -1.0, 2.0, seed=3)
    b = ctx.load(torch.tensor(f, device="cuda")).cpu().numpy()
    ref = odogip.load_const(d, p, P.coords, P.cells, P.conn, P.n, f)
    if P.bmask is not None:
        ref[P.bmask] = 0.0
    assert np.all(np.abs(b - ref) <= 1e-14 * np.abs(ref).max())
    b1 = ctx.load().cpu().numpy()
    ref1 = odogip.load_const(d, p, P.coords, P.cells, P.conn, P.n, np.ones(len(P.cells)))
    if P.bmask is not None:
        ref1[P.bmask] = 0.0
    assert np.all(np.abs(b1 - ref1) <= 1e-14 * np.abs(ref1).max())


def _direct(P, b):
    import scipy.sparse.linalg as spla
    K = assembly.assemble(P.form, P.p, P.coords, P.cells, P.conn, P.n, P.coef)
    if P.bmask is not None:
        K = assembly.dirichlet(K, P.bmask)
    return spla.spsolve(K.tocsc(), b)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("d,p,form", [(2, 2, "elliptic"), (2, 4, "elliptic"), (2, 2, "projection"),
                                      (3, 2, "elliptic"), (3, 1, "projection"),
                                      (3, 3, "elliptic")])  # 3D P3 FP64: per-cell kernel path
def test_solve(B, d, p, form, mode):
    ctx, P = make(B, d, p, form, NSMALL[d])
    b = ctx.load()
    x, info = ctx.solve(b, mode=mode, tol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    bb = b.cpu().numpy()
    xx = x.cpu().numpy()
    r = bb - P.apply(xx)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)
    ref = _direct(P, bb)
    assert np.linalg.norm(xx - ref) <= 1e-6 * np.linalg.norm(ref)


def test_solve_multi_rhs(B):
    ctx, P = make(B, 2, 2, "elliptic", 12)
    R = 4
    b = inputs.rhs_normal(P.n, R, seed=9)
    b[P.bmask] = 0.0
    bg = torch.tensor(b, device="cuda")
    for mode in ("fp64", "mixed"):
        x, info = ctx.solve(bg, mode=mode, tol=1e-9)
        assert info["status"] == 0
        r = b - P.apply(x.cpu().numpy())
        assert np.all(np.linalg.norm(r, axis=0) <= 1.01e-9 * np.linalg.norm(b, axis=0))
        assert np.all(info["rel_per_rhs"] <= 1e-9)


def test_solve_initial_guess_and_notconv(B):
    ctx, P = make(B, 2, 2, "elliptic", 10)
    b = ctx.load()
    x, info = ctx.solve(b, mode="fp64", tol=1e-12, maxiter=3, allow_notconv=True)
    assert info["status"] == B.ENOTCONV and info["iterations"] == 3
    r_early = info["rel_residual"]
    x2, info2 = ctx.solve(b, x.clone(), mode="fp64", tol=1e-10, x0=True)
    assert info2["status"] == 0 and info2["rel_residual"] <= 1e-10 < r_early


@pytest.mark.parametrize("d,p,form", [(2, 3, "elliptic"), (3, 1, "elliptic"), (2, 2, "projection")])
def test_gradient(B, d, p, form):
    ctx, P = make(B, d, p, form, NSMALL[d])
    b = ctx.load()
    x, _ = ctx.solve(b, mode="fp64", tol=1e-12)
    g = ctx.grad_coef(x, x).cpu().numpy()
    xx = x.cpu().numpy()
    ref = ograd.grad_coef_dogip(form, p, P.coords, P.cells, P.conn, xx, xx)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_set_coef_on_device(B):
    ctx, P = make(B, 2, 2, "elliptic", 9)
    A2 = inputs.coef_tensor_lognormal(len(P.cells), 2, 0.5, seed=77)
    ctx.set_coef(torch.tensor(A2, device="cuda"))
    P2 = odogip.Problem("elliptic", 2, P.coords, P.cells, A2)
    A = ctx.ahat().cpu().numpy()
    ref = pack(P2)
    assert np.all(np.abs(A - ref) <= 1e-14 * np.abs(ref).max(axis=(1, 2), keepdims=True))
    u = inputs.rhs_normal(P.n, 1, 3)[:, 0]
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.all(np.abs(y - P2.apply(u)) <= TOL64 * P2.apply_abs(u))


def test_invalid_inputs_rejected(B):
    coords, cells = inputs.lattice_mesh(2, 3)
    E = len(cells)
    # degenerate cell: collapse one vertex onto another
    bad = coords.copy()
    bad[cells[4, 1]] = bad[cells[4, 0]]
    with pytest.raises(B.DogipError) as e:
        B.Context(bad, cells, 1, "elliptic", np.ones(E))
    assert e.value.code == B.EINVAL
    A = np.repeat(np.eye(2)[None], E, 0)
    A[3] = [[1.0, 2.0], [2.0, 1.0]]  # indefinite
    with pytest.raises(B.DogipError) as e:
        B.Context(coords, cells, 1, "elliptic", A)
    assert e.value.code == B.EINVAL
    A = np.repeat(np.eye(2)[None], E, 0)
    A[3] = [[1.0, 0.1], [0.2, 1.0]]  # not symmetric
    with pytest.raises(B.DogipError):
        B.Context(coords, cells, 1, "elliptic", A)
    m = np.ones(E)
    m[2] = np.nan
    with pytest.raises(B.DogipError):
        B.Context(coords, cells, 1, "projection", m)
    ctx = B.Context(coords, cells, 1, "elliptic", np.ones(E))
    b = ctx.load()
    with pytest.raises(B.DogipError) as e:  # solves take nrhs in {1,2,4,...,32}
        ctx.solve(torch.zeros((ctx.n, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == B.EINVAL
    with pytest.raises(B.DogipError) as e:  # colour scatter needs colour-sorted storage
        ctx.apply(b, scatter="colour")
    assert e.value.code == B.EINVAL
    with pytest.raises(B.DogipError) as e:  # above the orders of Tables 2 and 4
        B.Context(*inputs.lattice_mesh(3, 1), 5, "elliptic", np.ones(6))
    assert e.value.code == B.EUNSUPPORTED


def test_single_cell_and_tiny_meshes(B):
    """Degenerate sizes: one cell (all dofs on the boundary), one cube (6 tets)."""
    for d, N in ((2, 1), (3, 1)):
        coords, cells = inputs.lattice_mesh(d, N)
        for form in ("elliptic", "projection"):
            for p in (1, 2):
                coef = np.full(len(cells), 2.0)
                ctx = B.Context(coords, cells, p, form, coef)
                P = odogip.Problem(form, p, coords, cells, coef)
                u = inputs.rhs_normal(P.n, 1, 4)[:, 0]
                y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
                assert np.all(np.abs(y - P.apply(u)) <= TOL64 * P.apply_abs(u))


# ------------------------------------------------------------ full-size cases


def _sampled_parity(ctx, P, u, y, samples, tol):
    """Oracle values of y at sampled dofs, from the cells containing them only."""
    touch = np.isin(P.conn, samples).any(axis=1)
    conn = P.conn[touch]
    Ah = P.Ah[touch]
    ref = odogip.apply(P.form, P.Bh, Ah, conn, u, P.bmask)
    sc = odogip.apply_abs(P.form, P.Bh, Ah, conn, u, P.bmask)
    ref, sc = ref[samples], sc[samples]
    got = y[samples]
    assert np.all(np.abs(got - ref) <= tol * sc), (np.abs(got - ref) / sc).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_full_size_2d_tensor(B, p):
    """Config: 512 x 512 jittered grid (524,288 triangles), lognormal SPD tensors,
    P1-P4: dof map bit-exact, colouring greedy at full size, sampled apply parity
    (FP64 and FP32) in the launch configuration the benchmark times."""
    coords, cells = inputs.lattice_mesh(2, 512, 0.2, seed=2)
    A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=2)
    ctx = B.Context(coords, cells, p, "elliptic", A)
    P = odogip.Problem("elliptic", p, coords, cells, A)
    assert ctx.n == (512 * p + 1) ** 2 == P.n
    assert np.array_equal(ctx.dofmap(), P.conn)
    col, _ = ctx.colouring()
    assert otopo.colouring_is_greedy(P.cells, col)
    samples = inputs.pick(11, 3000, P.n)
    u = inputs.rhs_normal(P.n, 1, seed=12)[:, 0]
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    _sampled_parity(ctx, P, u, y, samples, TOL64)
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
    _sampled_parity(ctx, P, u32.astype(np.float64), y32, samples, TOL32)


@pytest.mark.parametrize("form", ["elliptic", "projection"])
def test_full_size_3d_multi_rhs(B, form):
    """Config: 64^3 cube (1,572,864 tetrahedra), P2, inclusion coefficient, 16
    right-hand sides in one launch: sampled parity for FP64 and FP32."""
    coords, cells = inputs.lattice_mesh(3, 64)
    cent = inputs.centroids(coords, cells)
    m = inputs.coef_inclusions(cent, 200, 0.03, 0.08, seed=3)
    ctx = B.Context(coords, cells, 2, form, m)
    P = odogip.Problem(form, 2, coords, cells, m)
    assert ctx.n == 129 ** 3 == P.n
    assert np.array_equal(ctx.dofmap(), P.conn)
    R = 16
    u = inputs.rhs_normal(P.n, R, seed=13)
    samples = inputs.pick(14, 1500, P.n)
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    _sampled_parity(ctx, P, u, y, samples, TOL64)
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
    _sampled_parity(ctx, P, u32.astype(np.float64), y32, samples, TOL32)


def test_full_size_mixed_solve_residual(B):
    """Config-2 P2 mixed-precision solve to 1e-8: the oracle's FP64 apply confirms
    the true relative residual at full size."""
    coords, cells = inputs.lattice_mesh(2, 512, 0.2, seed=2)
    A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=2)
    ctx = B.Context(coords, cells, 2, "elliptic", A)
    b = ctx.load()
    x, info = ctx.solve(b, mode="mixed", tol=1e-8)
    assert info["status"] == 0
    P = odogip.Problem("elliptic", 2, coords, cells, A)
    bb = b.cpu().numpy()
    r = bb - P.apply(x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-8 * np.linalg.norm(bb)


@pytest.mark.parametrize("form", ["elliptic", "projection"])
def test_config_small_fp64_pcg(B, form):
    """Config: 32 x 32 squares x 2 triangles (2,048 cells), no jitter, P2 (4,225 dofs),
    per-cell A ~ U[1, 10]; elliptic with f = 1 and zero Dirichlet data, projection with
    f = sin(pi x) sin(pi y) (load by the oracle's quadrature); FP64 Jacobi-PCG to
    1e-10 against the oracle's direct solve of the assembled system."""
    coords, cells = inputs.lattice_mesh(2, 32)
    A = inputs.coef_uniform(len(cells), 1.0, 10.0, seed=1)
    ctx = B.Context(coords, cells, 2, form, A)
    P = odogip.Problem(form, 2, coords, cells, A)
    assert ctx.n == 4225 == P.n
    if form == "elliptic":
        b = odogip.load_const(2, 2, coords, cells, P.conn, P.n, np.ones(len(cells)))
        b[P.bmask] = 0.0
    else:
        f = lambda X: np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1])
        b = assembly.load(2, 2, coords, cells, P.conn, P.n, f)
    x, info = ctx.solve(torch.tensor(b, device="cuda"), mode="fp64", tol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    ref = _direct(P, b)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_autotune_keeps_parity(B):
    """dogip_autotune picks a kernel per precision from the candidates; the tuned
    apply still matches the oracle, and a second context of the same kind reuses
    the cached choice."""
    ctx, P = make(B, 2, 3, "elliptic", 40)
    choice = ctx.autotune()
    for prec in ("fp64", "fp32"):
        var, blk = choice[prec]
        assert (var, blk) in {(3, 256), (2, 256), (1, 256), (0, 64), (0, 128), (0, 256)}
    u = inputs.rhs_normal(P.n, 1, seed=8)[:, 0]
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.all(np.abs(y - P.apply(u)) <= TOL64 * P.apply_abs(u))
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y32 - P.apply(u32.astype(np.float64))) <= TOL32 * P.apply_abs(u32.astype(np.float64)))
    ctx2, _ = make(B, 2, 3, "elliptic", 40, seed=2)
    assert ctx2.autotune() == choice


@pytest.mark.parametrize("R", [1, 4])
@pytest.mark.parametrize("d,p,form", SMALL, ids=IDS)
def test_factorized_storage(B, d, p, form, R):
    """Factorised element factors (A_T,j = w_j K_T, only K_T stored): the exported
    A_T and the FP64 / FP32 applies match the oracle like the per-node storage."""
    jitter = 0.2 if d == 2 else 0.1
    coords, cells = inputs.lattice_mesh(d, NSMALL[d], jitter, 1)
    E = len(cells)
    coef = inputs.coef_tensor_lognormal(E, d, 1.0, 1) if form == "elliptic" else \
        inputs.coef_uniform(E, 1.0, 10.0, 1)
    ctx = B.Context(coords, cells, p, form, coef, factorized=True)
    P = odogip.Problem(form, p, coords, cells, coef)
    assert ctx.info.bytes_ahat_fp64 == E * ctx.info.n_sym * 8
    A = ctx.ahat().cpu().numpy()
    ref = pack(P)
    assert np.all(np.abs(A - ref) <= 1e-14 * np.abs(ref).max(axis=(1, 2), keepdims=True))
    u = inputs.rhs_normal(P.n, R, seed=5)
    ug = torch.tensor(u if R > 1 else u[:, 0], device="cuda")
    y = ctx.apply(ug).cpu().numpy().reshape(P.n, R)
    assert np.all(np.abs(y - P.apply(u)) <= TOL64 * P.apply_abs(u))
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32 if R > 1 else u32[:, 0], device="cuda"), prec="fp32")
    y32 = y32.cpu().numpy().astype(np.float64).reshape(P.n, R)
    u64 = u32.astype(np.float64)
    assert np.all(np.abs(y32 - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    if R == 1 and d == 2 and p == 2:
        b = ctx.load()
        x, info = ctx.solve(b, mode="mixed", tol=1e-10)
        r = b.cpu().numpy() - P.apply(x.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())


def test_factorized_rejects_colour(B):
    coords, cells = inputs.lattice_mesh(2, 4)
    with pytest.raises(B.DogipError) as e:
        B.Context(coords, cells, 2, "elliptic", np.ones(len(cells)), factorized=True,
                  scatter="colour")
    assert e.value.code == B.EINVAL


@pytest.mark.parametrize("d,p,form,nq", [(2, 2, "elliptic", 6), (2, 3, "projection", 5),
                                         (3, 2, "elliptic", 4), (3, 1, "projection", 3),
                                         (2, 1, "elliptic", 8)])
def test_subelement_inclusions(B, d, p, form, nq):
    """A_T of a discontinuous inclusion field integrated per W node by the sub-element
    rule (dogip_set_coef_inclusions) equals the oracle's independent quadrature; the
    apply with it matches the oracle apply; the solve meets its tolerance."""
    N = 12 if d == 2 else 4
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, 6)
    ctr, rad = inputs.inclusion_balls(d, 20, 0.05, 0.2, seed=6)
    ctx = B.Context(coords, cells, p, form, np.ones(len(cells)))
    ctx.set_coef_inclusions(ctr, rad, 100.0, 1.0, nq)
    P = odogip.Problem(form, p, coords, cells, np.ones(len(cells)))
    P.Ah = odogip.ahat_quadrature(form, p, coords, cells,
                                  inputs.inclusion_field(ctr, rad, 100.0, 1.0), nq)
    A = ctx.ahat().cpu().numpy()
    ref = pack(P)
    assert np.all(np.abs(A - ref) <= 1e-12 * np.abs(ref).max(axis=(1, 2), keepdims=True))
    u = inputs.rhs_normal(P.n, 1, seed=7)[:, 0]
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.all(np.abs(y - P.apply(u)) <= TOL64 * P.apply_abs(u))
    b = ctx.load()
    x, info = ctx.solve(b, mode="mixed", tol=1e-9)
    r = b.cpu().numpy() - P.apply(x.cpu().numpy())
    assert info["status"] == 0 and np.linalg.norm(r) <= 1.01e-9 * np.linalg.norm(b.cpu().numpy())
    with pytest.raises(B.DogipError):  # no element-wise coefficient to differentiate
        ctx.grad_coef(x, x)


def test_subelement_constant_field_equals_elementwise(B):
    coords, cells = inputs.lattice_mesh(2, 10, 0.2, 3)
    a = B.Context(coords, cells, 3, "elliptic", np.full(len(cells), 2.5))
    b = B.Context(coords, cells, 3, "elliptic", np.ones(len(cells)))
    b.set_coef_inclusions(np.zeros((0, 2)), np.zeros(0), 7.0, 2.5, 4)
    Aa, Ab = a.ahat().cpu().numpy(), b.ahat().cpu().numpy()
    assert np.abs(Aa - Ab).max() <= 1e-13 * np.abs(Aa).max()
    np.testing.assert_allclose(a.diag().cpu().numpy(), b.diag().cpu().numpy(), rtol=1e-13)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("d,p,form", [(2, 1, "elliptic"), (2, 4, "elliptic"), (2, 3, "projection"),
                                      (3, 2, "elliptic"), (3, 3, "projection")])
def test_apply_variants_parity(B, d, p, form, variant, monkeypatch):
    """Each apply kernel the autotuner can choose — one thread per cell (0), the staged
    producer/consumer ring (1), self-feeding warps (2), tensor cores (3, FP32; the
    staged kernel serves FP64 and instances without a tensor-core kernel) — matches
    the oracle on its own, FP64 and FP32, one right-hand side."""
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", str(variant))
    ctx, P = make(B, d, p, form, NSMALL[d])
    u = inputs.rhs_normal(P.n, 1, seed=31)[:, 0]
    y = ctx.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.all(np.abs(y - P.apply(u)) <= TOL64 * P.apply_abs(u))
    u32 = u.astype(np.float32)
    y32 = ctx.apply(torch.tensor(u32, device="cuda"), prec="fp32").cpu().numpy().astype(np.float64)
    u64 = u32.astype(np.float64)
    assert np.all(np.abs(y32 - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    ctx.check()
