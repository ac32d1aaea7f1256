"""Pins of the oracle's operators, solvers and gradient against what the
mathematics fixes: the DoGIP identity with the independently assembled matrix
(Theorems 4 and 8), textbook P1 matrices, symmetry, null space, measure of the
domain, linear patch test, O(h^{p+1}) convergence, brute-force solves, finite
differences."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, dogip, gradient, refelem, solvers, topology
from paper_1710_09913_gb300 import inputs


def _problem(d, form, p, N, jitter=0.2, seed=1, tensor=True, dirichlet=False):
    c, t = inputs.lattice_mesh(d, N, jitter if d == 2 else 0.5 * jitter, seed)
    E = len(t)
    if form == "elliptic" and tensor:
        coef = inputs.coef_tensor_lognormal(E, d, 1.0, seed)
    else:
        coef = inputs.coef_uniform(E, 1.0, 10.0, seed)
    return dogip.Problem(form, p, c, t, coef, dirichlet=dirichlet)


CASES = [(d, f, p) for d in (2, 3) for f in ("elliptic", "projection") for p in (1, 2, 3, 4)
         if not (d == 3 and p == 4 and f == "projection")]


@pytest.mark.parametrize("d,form,p", CASES)
def test_dogip_equals_assembled(d, form, p):
    """B^* A_T B^ summed over cells == quadrature-assembled matrix (1e-12)."""
    N = {2: 5, 3: 2}[d]
    P = _problem(d, form, p, N)
    K = assembly.assemble(form, p, P.coords, P.cells, P.conn, P.n, P.coef)
    u = inputs.rhs_normal(P.n, 2, 11)
    y = P.apply(u)
    scale = P.apply_abs(u)
    assert np.all(np.abs(y - K @ u) <= 1e-12 * scale)
    assert np.linalg.norm(y - K @ u) <= 1e-13 * np.linalg.norm(K @ u)
    # the diagonal from A_T equals the assembled diagonal
    np.testing.assert_allclose(P.diag(), K.diagonal(), rtol=1e-12, atol=0)
    # element matrices: symmetric
    Ke = dogip.element_matrices(form, P.Bh, P.Ah)
    np.testing.assert_allclose(Ke, Ke.transpose(0, 2, 1), rtol=0, atol=1e-12 * np.abs(Ke).max())


def _bary_grads(coords, cells):
    """Gradients of the barycentric coordinates from the inverse vertex matrix."""
    X = coords[cells]  # [E, d+1, d]
    E, dp1, d = X.shape
    Mv = np.concatenate([np.ones((E, 1, dp1)), X.transpose(0, 2, 1)], axis=1)
    return np.linalg.inv(Mv)[:, :, 1:], np.abs(np.linalg.det(Mv))


@pytest.mark.parametrize("d", [2, 3])
def test_p1_textbook(d):
    """P1 mass |T|(1+delta_ij)/((d+1)(d+2)) and stiffness |T| grad lambda_i . M grad lambda_j."""
    P = _problem(d, "elliptic", 1, 3)
    G, det = _bary_grads(P.coords, P.cells)
    vol = det / (2 if d == 2 else 6)
    # local order of P1 nodes: (0..0) -> lambda_0, then lambda_d, ..., lambda_1
    order = [0] + list(range(d, 0, -1))
    G = G[:, order, :]
    Ke_ref = vol[:, None, None] * np.einsum("eia,eab,ejb->eij", G, P.coef, G)
    Ke = dogip.element_matrices("elliptic", P.Bh, P.Ah)
    np.testing.assert_allclose(Ke, Ke_ref, rtol=1e-12, atol=1e-12 * np.abs(Ke_ref).max())
    Pm = _problem(d, "projection", 1, 3)
    _, detm = _bary_grads(Pm.coords, Pm.cells)
    volm = detm / (2 if d == 2 else 6)
    Me = dogip.element_matrices("projection", Pm.Bh, Pm.Ah)
    ref = (Pm.coef * volm)[:, None, None] * (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    np.testing.assert_allclose(Me, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_stiffness_null_space_and_psd(d, p):
    """K 1 = 0 before boundary conditions; K symmetric positive semidefinite."""
    P = _problem(d, "elliptic", p, 2)
    one = np.ones(P.n)
    assert np.abs(P.apply(one)).max() <= 1e-12 * np.abs(P.apply_abs(one)).max()
    K = dogip.element_matrices("elliptic", P.Bh, P.Ah)
    Kd = np.zeros((P.n, P.n))
    for e in range(len(P.cells)):
        Kd[np.ix_(P.conn[e], P.conn[e])] += K[e]
    np.testing.assert_allclose(Kd, Kd.T, atol=1e-12 * np.abs(Kd).max())
    ev = np.linalg.eigvalsh(Kd)
    assert ev.min() >= -1e-12 * ev.max()
    assert np.sum(ev < 1e-10 * ev.max()) == 1  # only the constants


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_mass_measure(d, p):
    """1^T M 1 = |Omega| = 1 for m = 1 (Lemma 3 with u = v = 1), jittered mesh."""
    c, t = inputs.lattice_mesh(d, 3, 0.2 if d == 2 else 0.1, 5)
    P = dogip.Problem("projection", p, c, t, np.ones(len(t)), dirichlet=False)
    one = np.ones(P.n)
    assert abs(one @ P.apply(one) - 1.0) <= 1e-13
    # the load of f = 1 sums to |Omega| as well, and equals the quadrature load
    b = dogip.load_const(d, p, c, t, P.conn, P.n, np.ones(len(t)))
    assert abs(b.sum() - 1.0) <= 1e-13
    bq = assembly.load(d, p, c, t, P.conn, P.n, lambda X: np.ones(X.shape[:2]))
    np.testing.assert_allclose(b, bq, rtol=0, atol=1e-15)


def _dirichlet_solve(P, b):
    K = assembly.dirichlet(assembly.assemble(P.form, P.p, P.coords, P.cells, P.conn, P.n, P.coef), P.bmask)
    return spla.spsolve(K.tocsc(), b)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_patch_test(d, p):
    """Linear g, Dirichlet data g, f = 0, constant SPD A: u_h = g exactly (jittered mesh)."""
    c, t = inputs.lattice_mesh(d, 4, 0.2 if d == 2 else 0.1, 9)
    A0 = inputs.coef_tensor_lognormal(1, d, 0.7, 3)[0]
    P = dogip.Problem("elliptic", p, c, t, np.repeat(A0[None], len(t), 0), dirichlet=True)
    xn = np.zeros((P.n, d))
    xn[P.conn.reshape(-1)] = topology.node_points(P.coords, P.cells, p).reshape(-1, d)
    g = 0.3 + xn @ np.array([1.0, -2.0, 0.5][:d])
    # K~ u = b with b_boundary = g_b and b_interior = -(K g_b)_interior
    gb = np.where(P.bmask, g, 0.0)
    Kfull = dogip.apply("elliptic", P.Bh, P.Ah, P.conn, gb)
    b = np.where(P.bmask, g, -Kfull)
    u = _dirichlet_solve(P, b)
    np.testing.assert_allclose(u, g, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mms_convergence(p):
    """-div grad u = f, u = sin(pi x) sin(pi y), zero Dirichlet: L2 error O(h^{p+1})."""
    from oracle import quadrature
    errs = []
    Ns = [4, 8, 16]
    for N in Ns:
        c, t = inputs.lattice_mesh(2, N)
        P = dogip.Problem("elliptic", p, c, t, np.ones(len(t)), dirichlet=True)
        f = lambda X: 2 * np.pi ** 2 * np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1])
        b = assembly.load(2, p, c, t, P.conn, P.n, f)
        b[P.bmask] = 0.0
        u = _dirichlet_solve(P, b)
        pts, w = quadrature.simplex_rule(2, p + 3)
        val, _ = refelem.vandermonde_eval_float(2, p, pts)
        R, det, _ = dogip.geometry(c, t)
        X = c[t][:, 0, :][:, None, :] + np.einsum("eij,qj->eqi", R, pts)
        uh = u[P.conn] @ val.T
        ex = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1])
        errs.append(np.sqrt(np.sum(np.abs(det)[:, None] * w[None] * (uh - ex) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] >= p + 1 - 0.15, rates


@pytest.mark.parametrize("d,form,p", [(2, "elliptic", 2), (2, "projection", 2), (3, "elliptic", 2), (2, "elliptic", 3)])
def test_pcg_matches_dense_solve(d, form, p):
    """Jacobi-PCG on the DoGIP operator == dense solve of the assembled system (N <= 4)."""
    P = _problem(d, form, p, 3 if d == 2 else 2, dirichlet=(form == "elliptic"))
    b = inputs.rhs_normal(P.n, 1, 4)[:, 0]
    if P.bmask is not None:
        b[P.bmask] = 0.0
    K = assembly.assemble(form, p, P.coords, P.cells, P.conn, P.n, P.coef)
    if P.bmask is not None:
        K = assembly.dirichlet(K, P.bmask)
    ref = np.linalg.solve(K.toarray(), b)
    x, it, res = solvers.pcg(P.apply, b, 1.0 / P.diag(), tol=1e-13)
    assert res <= 1e-13
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_iterative_refinement_reaches_tolerance():
    """FP64 refinement around an emulated-FP32 inner PCG reaches 1e-10 (parity unpinned:
    sanity of the mixed-precision algorithm only)."""
    P = _problem(2, "elliptic", 2, 8, dirichlet=True)
    b = dogip.load_const(2, 2, P.coords, P.cells, P.conn, P.n, np.ones(len(P.cells)))
    b[P.bmask] = 0.0
    Ah32 = P.Ah.astype(np.float32).astype(np.float64)
    a32 = lambda v: dogip.apply("elliptic", P.Bh, Ah32, P.conn, v.astype(np.float64), P.bmask)
    u, outer, inner, rel = solvers.iterative_refinement(P.apply, a32, b, 1.0 / P.diag(), tol=1e-10)
    assert rel <= 1e-10 and outer <= 6
    ref = _dirichlet_solve(P, b)
    assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,form,p", [(2, "elliptic", 3), (3, "elliptic", 1), (2, "projection", 2), (2, "elliptic", 1)])
def test_gradient(d, form, p):
    """Compliance gradient: W-node outer products == assembled element derivative,
    and == central finite differences of J = b^T u (FP64)."""
    P = _problem(d, form, p, 3 if d == 2 else 2, dirichlet=(form == "elliptic"))
    b = dogip.load_const(d, p, P.coords, P.cells, P.conn, P.n, np.ones(len(P.cells)))
    if P.bmask is not None:
        b[P.bmask] = 0.0

    def solve(coef):
        K = assembly.assemble(form, p, P.coords, P.cells, P.conn, P.n, coef)
        if P.bmask is not None:
            K = assembly.dirichlet(K, P.bmask)
        return spla.spsolve(K.tocsc(), b)

    u = solve(P.coef)
    g1 = gradient.grad_coef_dogip(form, p, P.coords, P.cells, P.conn, u, u)
    g2 = gradient.grad_coef_assembled(form, p, P.coords, P.cells, P.conn, u, u)
    np.testing.assert_allclose(g1, g2, rtol=0, atol=1e-12 * np.abs(g2).max())
    h = 1e-5
    for e in inputs.pick(3, 4, len(P.cells)):
        if form == "projection":
            cp, cm = P.coef.copy(), P.coef.copy()
            cp[e] += h
            cm[e] -= h
            fd = (b @ solve(cp) - b @ solve(cm)) / (2 * h)
            assert abs(fd - g1[e]) <= 1e-6 * abs(g1).max()
        else:
            for a_, c_ in [(0, 0), (0, 1), (1, 1)]:
                cp, cm = P.coef.copy(), P.coef.copy()
                cp[e, a_, c_] += h
                cm[e, a_, c_] -= h
                if a_ != c_:
                    cp[e, c_, a_] += h
                    cm[e, c_, a_] -= h
                fd = (b @ solve(cp) - b @ solve(cm)) / (2 * h)
                an = g1[e, a_, c_] + (g1[e, c_, a_] if a_ != c_ else 0.0)
                assert abs(fd - an) <= 1e-6 * np.abs(g1).max()


@pytest.mark.parametrize("d,form,p", [(2, "elliptic", 2), (2, "projection", 2), (3, "elliptic", 2),
                                      (2, "elliptic", 1), (3, "projection", 1)])
def test_quadrature_ahat_constant_equals_exact(d, form, p):
    """Sub-element quadrature of a constant coefficient reproduces the exact A_T
    (the rule is exact to degree 2 nq - 1 >= the W degree)."""
    c, t = inputs.lattice_mesh(d, 3, 0.2 if d == 2 else 0.1, 4)
    nq = refelem.w_degree(form, p) // 2 + 1
    Aq = dogip.ahat_quadrature(form, p, c, t, lambda X: np.full(X.shape[:-1], 3.5), nq)
    Ae = dogip.ahat(form, p, c, t, np.full(len(t), 3.5))
    np.testing.assert_allclose(Aq, Ae, rtol=0, atol=1e-13 * np.abs(Ae).max())


@pytest.mark.parametrize("d", [2, 3])
def test_quadrature_ahat_measures_a_ball(d):
    """sum over cells and W nodes of sigma_T,j |det R_T| = int m: for one ball of
    radius r inside the domain with m = 1 in it and 0 outside, the measure of the
    ball (pi r^2, 4/3 pi r^3) to the accuracy of the sub-element rule."""
    N, r = (16, 0.3) if d == 2 else (6, 0.3)
    c, t = inputs.lattice_mesh(d, N)
    m = inputs.inclusion_field(np.full((1, d), 0.5), np.array([r]), 1.0, 1e-300)
    A = dogip.ahat_quadrature("projection", 1, c, t, m, 12)
    exact = np.pi * r * r if d == 2 else 4.0 / 3.0 * np.pi * r ** 3
    assert abs(A.sum() - exact) <= 2e-3 * exact
