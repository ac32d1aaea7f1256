"""GPU parity of the apply entry points beside dogip_apply: the accumulating
dogip_apply_add (y += K u, one kernel launch) and the TF32 precision (the two
contractions with B on the tensor cores), both against the FP64 CPU oracle.

Tolerances as in test_gpu_parity: FP64 1e-12 and FP32 / TF32 2e-5 of the
componentwise absolute-value scale |B|^T |A_T| |B| |u| (plus |y0| for the added
vector)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dogip as odogip  # noqa: E402
from paper_1710_09913_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
NSMALL = {2: 11, 3: 3}


@pytest.fixture(scope="module")
def B():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding
    return binding


def make(B, d, p, form, N, scatter="atomic", seed=1):
    coords, cells = inputs.lattice_mesh(d, N, 0.2 if d == 2 else 0.1, seed)
    E = len(cells)
    coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed) if form == "elliptic" else \
        inputs.coef_uniform(E, 1.0, 10.0, seed)
    return B.Context(coords, cells, p, form, coef, scatter=scatter), \
        odogip.Problem(form, p, coords, cells, coef)


CASES = [(2, 1, "elliptic"), (2, 4, "elliptic"), (2, 3, "projection"), (3, 2, "elliptic"),
         (3, 3, "projection"), (2, 6, "elliptic")]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("d,p,form", CASES, ids=[f"{d}D-P{p}-{f}" for d, p, f in CASES])
def test_apply_add(B, d, p, form, variant, monkeypatch):
    """y0 + K u through dogip_apply_add for every kernel the autotuner can choose,
    FP64 and FP32; the Dirichlet rows add u_b."""
    monkeypatch.setenv("DOGIP_APPLY_VARIANT", str(variant))
    ctx, P = make(B, d, p, form, NSMALL[d] if p <= 4 else 6)
    u = inputs.rhs_normal(P.n, 1, seed=41)[:, 0]
    y0 = inputs.rhs_normal(P.n, 1, seed=42)[:, 0]
    ref = P.apply(u) + y0
    sc = P.apply_abs(u) + np.abs(y0)
    y = torch.tensor(y0, device="cuda")
    ctx.apply_add(torch.tensor(u, device="cuda"), y)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= TOL64 * sc)
    u32, y032 = u.astype(np.float32), y0.astype(np.float32)
    ref32 = P.apply(u32.astype(np.float64)) + y032
    sc32 = P.apply_abs(u32.astype(np.float64)) + np.abs(y032)
    y = torch.tensor(y032, device="cuda")
    ctx.apply_add(torch.tensor(u32, device="cuda"), y, prec="fp32")
    assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - ref32) <= TOL32 * sc32)
    ctx.check()


@pytest.mark.parametrize("R", [1, 4, 16])
def test_apply_add_colour_and_multi_rhs(B, R):
    ctx, P = make(B, 2, 2, "elliptic", 12, scatter="colour")
    u = inputs.rhs_normal(P.n, R, seed=43)
    y0 = inputs.rhs_normal(P.n, R, seed=44)
    for scat in ("colour", "atomic"):
        y = torch.tensor(y0 if R > 1 else y0[:, 0], device="cuda")
        ctx.apply_add(torch.tensor(u if R > 1 else u[:, 0], device="cuda"), y, scatter=scat)
        got = y.cpu().numpy().reshape(P.n, R)
        assert np.all(np.abs(got - (P.apply(u) + y0)) <= TOL64 * (P.apply_abs(u) + np.abs(y0)))
    # FP32 atomic (16 right-hand sides: the 8-cell x 16-rhs warp units)
    u32, y32 = u.astype(np.float32), y0.astype(np.float32)
    y = torch.tensor(y32 if R > 1 else y32[:, 0], device="cuda")
    ctx.apply_add(torch.tensor(u32 if R > 1 else u32[:, 0], device="cuda"), y, prec="fp32",
                  scatter="atomic")
    got = y.cpu().numpy().astype(np.float64).reshape(P.n, R)
    u64 = u32.astype(np.float64)
    assert np.all(np.abs(got - (P.apply(u64) + y32)) <= TOL32 * (P.apply_abs(u64) + np.abs(y32)))


TF32_CASES = [(2, p, "elliptic") for p in (1, 2, 3, 4)] + [(2, 3, "projection"), (3, 2, "elliptic"),
                                                          (3, 1, "projection"), (2, 5, "elliptic")]


@pytest.mark.parametrize("d,p,form", TF32_CASES, ids=[f"{d}D-P{p}-{f}" for d, p, f in TF32_CASES])
def test_apply_tf32(B, d, p, form):
    """prec = TF32 selects the tensor-core kernel whatever the autotuner chose; its
    3xTF32 products meet the FP32 bound against the oracle."""
    ctx, P = make(B, d, p, form, NSMALL[d] if p <= 4 else 6)
    u32 = inputs.rhs_normal(P.n, 1, seed=45)[:, 0].astype(np.float32)
    y = ctx.apply(torch.tensor(u32, device="cuda"), prec="tf32").cpu().numpy().astype(np.float64)
    u64 = u32.astype(np.float64)
    assert np.all(np.abs(y - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    ctx.check()


TF32_MULTI = [(3, 2, "elliptic", 16), (3, 2, "projection", 32), (2, 3, "elliptic", 16),
              (2, 1, "projection", 16)]


@pytest.mark.parametrize("d,p,form,R", TF32_MULTI,
                         ids=[f"{d}D-P{p}-{f}-R{R}" for d, p, f, R in TF32_MULTI])
def test_apply_tf32_multi_rhs(B, d, p, form, R):
    """Several right-hand sides on the tensor cores: MMA tiles of 8 cells x 16
    right-hand sides (apply and apply_add), against the oracle, FP32 bound."""
    ctx, P = make(B, d, p, form, NSMALL[d])
    u32 = inputs.rhs_normal(P.n, R, seed=46).astype(np.float32)
    u64 = u32.astype(np.float64)
    y = ctx.apply(torch.tensor(u32, device="cuda"), prec="tf32").cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - P.apply(u64)) <= TOL32 * P.apply_abs(u64))
    y0 = inputs.rhs_normal(P.n, R, seed=47).astype(np.float32)
    yg = torch.tensor(y0, device="cuda")
    ctx.apply_add(torch.tensor(u32, device="cuda"), yg, prec="tf32")
    got = yg.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - (P.apply(u64) + y0)) <= TOL32 * (P.apply_abs(u64) + np.abs(y0)))
    ctx.check()


def test_tf32_unsupported_requests(B):
    ctx, P = make(B, 2, 2, "elliptic", 8)
    u = torch.zeros((P.n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.DogipError) as e:  # 1 or a multiple of 16 right-hand sides
        ctx.apply(u, prec="tf32")
    assert e.value.code == B.EUNSUPPORTED
    c8, P8 = make(B, 2, 8, "elliptic", 3)  # no tensor-core instance at 2D P8 elliptic
    with pytest.raises(B.DogipError) as e:
        c8.apply(torch.zeros(P8.n, dtype=torch.float32, device="cuda"), prec="tf32")
    assert e.value.code == B.EUNSUPPORTED


@pytest.mark.parametrize("d,p", [(2, 3), (3, 2)])
def test_mixed_solve_tf32_inner(B, d, p):
    """Mixed solve whose inner FP32 PCG applies run on the tensor cores: the FP64
    true residual, confirmed by the oracle, meets the tolerance."""
    ctx, P = make(B, d, p, "elliptic", NSMALL[d] + 1)
    b = ctx.load()
    x, info = ctx.solve(b, mode="mixed", tol=1e-10, inner_prec="tf32")
    assert info["status"] == 0
    bb = b.cpu().numpy()
    r = bb - P.apply(x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)
