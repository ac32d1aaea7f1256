"""Device-side failure detection without a GPU fault: a bounded mbarrier wait runs
out on a copy that is never issued (a test hook, the analogue of a flag that nothing
sets), in the staged apply and in the tensor-core apply (one and 16 right-hand sides
per cell); the kernel drains its other copies, raises its error word and returns
(the tensor-core kernel after its warpgroups leave together and free their tensor
memory); dogip_check reports DOGIP_ETIMEOUT and the CUDA context stays usable."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

CHILD = r"""
import os, sys
sys.path.insert(0, os.environ["DOGIP_ROOT"])
import numpy as np, torch
from paper_1710_09913_gb300 import binding as B, inputs
coords, cells = inputs.lattice_mesh(2, 64, 0.2, seed=3)
A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=3)
ctx = B.Context(coords, cells, 2, "elliptic", A)
R = int(os.environ.get("DOGIP_CHILD_R", "1"))
u = torch.randn(ctx.n, R, dtype=torch.float32, device="cuda").squeeze(1)
ctx.apply(u, prec=os.environ.get("DOGIP_CHILD_PREC", "fp32"))
try:
    ctx.check()
    print("NO-TIMEOUT")
except B.DogipError as e:
    print("TIMEOUT", e.code)
# the context and the device remain usable: a second context without the hook
os.environ.pop("DOGIP_TEST_SKIP_CHUNK")
ok = B.Context(coords, cells, 2, "elliptic", A)
y = ok.apply(u.double()).cpu().numpy()
ok.check()
print("USABLE", np.isfinite(y).all())
"""


@pytest.mark.parametrize("prec,R", [("fp32", 1), ("tf32", 1), ("tf32", 16)],
                         ids=["staged", "tensor-cores", "tensor-cores-16rhs"])
def test_apply_wait_timeout_is_reported(prec, R):
    from paper_1710_09913_gb300 import build
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DOGIP_ROOT=root, DOGIP_TEST_SKIP_CHUNK="0",
               DOGIP_TEST_WAIT_CYCLES="2000000",  # ~1 ms per bounded wait
               DOGIP_CHILD_PREC=prec, DOGIP_CHILD_R=str(R))
    out = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "TIMEOUT 6" in out.stdout, out.stdout
    assert "USABLE True" in out.stdout, out.stdout


CHILD_PCG = r"""
import os, sys
sys.path.insert(0, os.environ["DOGIP_ROOT"])
import numpy as np, torch
from paper_1710_09913_gb300 import binding as B, inputs
coords, cells = inputs.lattice_mesh(2, 64, 0.2, seed=3)
A = inputs.coef_tensor_lognormal(len(cells), 2, 1.0, seed=3)
ctx = B.Context(coords, cells, 1, "elliptic", A)
b = ctx.load()
try:
    # FP64 PCG from u = 0: no apply runs before the single-launch iterations
    ctx.solve(b, mode=os.environ["DOGIP_CHILD_MODE"], tol=1e-8, single_launch=True)
    print("NO-TIMEOUT")
except B.DogipError as e:
    print("TIMEOUT", e.code)
os.environ.pop("DOGIP_TEST_SKIP_CHUNK")
ok = B.Context(coords, cells, 1, "elliptic", A)
u, info = ok.solve(b, mode="fp64", tol=1e-8, single_launch=True)
print("USABLE", info["status"] == 0 and info["rel_residual"] <= 1e-8)
"""


def test_single_launch_barrier_timeout_is_reported():
    """One block of the single-launch PCG never arrives at its first grid barrier (a
    test hook): the other blocks' bounded waits expire, they raise the error word and
    leave; the solve reports DOGIP_ETIMEOUT and a new context solves normally."""
    from paper_1710_09913_gb300 import build
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DOGIP_ROOT=root, DOGIP_TEST_SKIP_CHUNK="0",
               DOGIP_TEST_WAIT_CYCLES="2000000", DOGIP_CHILD_MODE="fp64")
    out = subprocess.run([sys.executable, "-c", CHILD_PCG], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "TIMEOUT 6" in out.stdout, out.stdout
    assert "USABLE True" in out.stdout, out.stdout
