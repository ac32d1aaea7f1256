"""Batched solves (dogip_batch_solve) of independent uneven problems, in the concurrent
(default), grouped and branch modes, against the oracle's FP64 apply (true relative
residual of every problem) and against the single-problem solver."""

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


def _problems(B, specs):
    out = []
    for N, p, seed in specs:
        coords, cells = inputs.lattice_mesh(2, N)
        m = inputs.coef_lognormal(len(cells), 1.0, seed)
        ctx = B.Context(coords, cells, p, "elliptic", m)
        out.append((ctx, odogip.Problem("elliptic", p, coords, cells, m)))
    return out


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_batch_small_uneven(B, mode):
    specs = [(4, 1, 1), (9, 3, 2), (16, 2, 3), (5, 2, 4), (12, 1, 5), (7, 3, 6), (3, 1, 7)]
    probs = _problems(B, specs)
    bs = [c.load() for c, _ in probs]
    us = [torch.zeros_like(b) for b in bs]
    infos = B.batch_solve([c for c, _ in probs], bs, us, mode=mode, tol=1e-10, check_every=8)
    for (c, P), b, u, inf in zip(probs, bs, us, infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        bb, uu = b.cpu().numpy(), u.cpu().numpy()
        r = bb - P.apply(uu)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)
        u1, _ = c.solve(b, mode=mode, tol=1e-10)
        assert np.linalg.norm(u1.cpu().numpy() - uu) <= 1e-8 * np.linalg.norm(uu)


@pytest.mark.parametrize("order", ["smallest", "largest", "given"])
def test_batch_concurrent_orders_and_single_launch(B, order, monkeypatch):
    """The concurrent mode in each problem order, its solves taking the single-launch
    PCG where it exists (cooperative launches of several problems side by side): every
    problem meets the tolerance the oracle confirms."""
    monkeypatch.setenv("DOGIP_BATCH_MODE", "concurrent")
    monkeypatch.setenv("DOGIP_BATCH_ORDER", order)
    probs = _problems(B, [(12, 1, 21), (20, 2, 22), (6, 3, 23), (16, 1, 24), (9, 2, 25)])
    bs = [c.load() for c, _ in probs]
    us = [torch.zeros_like(b) for b in bs]
    infos = B.batch_solve([c for c, _ in probs], bs, us, mode="mixed", tol=1e-10,
                          single_launch=True)
    for (c, P), b, u, inf in zip(probs, bs, us, infos):
        assert inf["status"] == 0 and inf["seconds"] > 0
        bb = b.cpu().numpy()
        r = bb - P.apply(u.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)


def test_batch_rejects_unknown_mode(B, monkeypatch):
    monkeypatch.setenv("DOGIP_BATCH_MODE", "lockstep")
    probs = _problems(B, [(4, 1, 1), (5, 2, 2)])
    bs = [c.load() for c, _ in probs]
    us = [torch.zeros_like(b) for b in bs]
    with pytest.raises(B.DogipError) as e:
        B.batch_solve([c for c, _ in probs], bs, us, mode="mixed", tol=1e-8)
    assert e.value.code == B.EINVAL
    monkeypatch.setenv("DOGIP_BATCH_MODE", "concurrent")
    monkeypatch.setenv("DOGIP_BATCH_ORDER", "random")
    with pytest.raises(B.DogipError) as e:
        B.batch_solve([c for c, _ in probs], bs, us, mode="mixed", tol=1e-8)
    assert e.value.code == B.EINVAL


@pytest.mark.parametrize("bmode", ["concurrent", "grouped"])
def test_batch_config_uneven_256(B, bmode, monkeypatch):
    """Config: 256 problems, N ~ U{16..128}, p ~ U{1,2,3}, lognormal(0,1) scalar,
    f = 1, mixed precision to 1e-8: every problem's true residual (oracle) meets it."""
    monkeypatch.setenv("DOGIP_BATCH_MODE", bmode)
    specs = inputs.uneven_problems(256, seed=5)
    probs = _problems(B, specs)
    bs = [c.load() for c, _ in probs]
    us = [torch.zeros_like(b) for b in bs]
    infos = B.batch_solve([c for c, _ in probs], bs, us, mode="mixed", tol=1e-8)
    worst = 0.0
    for (c, P), b, u, inf in zip(probs, bs, us, infos):
        assert inf["status"] == 0
        bb = b.cpu().numpy()
        r = bb - P.apply(u.cpu().numpy())
        worst = max(worst, np.linalg.norm(r) / np.linalg.norm(bb))
    assert worst <= 1.01e-8
    times = sorted(i["seconds"] for i in infos)
    assert times[0] > 0 and times[-1] >= times[len(times) // 2]


@pytest.mark.parametrize("bmode", ["concurrent", "grouped", "branches"])
def test_batch_modes_agree(B, bmode, monkeypatch):
    """Independent solves side by side (default), the grouped inner iterations (one
    launch per kernel for the whole batch) and the per-problem graph branches reach the
    same tolerance, confirmed by the oracle; 3D problems and the projection form join
    the 2D elliptic ones in one batch."""
    monkeypatch.setenv("DOGIP_BATCH_MODE", bmode)
    probs = _problems(B, [(6, 2, 11), (10, 1, 12), (4, 3, 13)])
    c3, t3 = inputs.lattice_mesh(3, 3)
    m3 = inputs.coef_uniform(len(t3), 1.0, 5.0, 14)
    for form in ("elliptic", "projection"):
        probs.append((B.Context(c3, t3, 2, form, m3), odogip.Problem(form, 2, c3, t3, m3)))
    bs = [c.load() for c, _ in probs]
    us = [torch.zeros_like(b) for b in bs]
    infos = B.batch_solve([c for c, _ in probs], bs, us, mode="mixed", tol=1e-10, check_every=4)
    for (c, P), b, u, inf in zip(probs, bs, us, infos):
        assert inf["status"] == 0, inf
        bb = b.cpu().numpy()
        r = bb - P.apply(u.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bb)
