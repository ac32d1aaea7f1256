"""GB300-native DoGIP (double-grid integration with interpolation-projection) for
P_p Lagrange finite elements on simplices (Vondřejc, arXiv 1710.09913).

The hot path -- the element-wise DoGIP operator apply y = sum_T P_T^T B^T A_T B P_T u
(Theorems "Element-wise DoGIP" for the weighted projection and the scalar elliptic
form, Algorithm 1) inside a Jacobi-preconditioned CG -- runs in hand-written CUDA
kernels for sm_103a behind the C ABI declared in ``include/dogip.h``.

Submodules:
  inputs   -- seeded synthetic meshes, coefficient fields and loads (no method arithmetic)
  binding  -- ctypes marshalling onto the C ABI (loads the in-tree shared library)
  autograd -- torch.autograd.Function wrappers (apply, solve, coefficient gradient)
  build    -- nvcc build of the shared library for sm_103a
"""

__all__ = ["inputs", "binding", "autograd", "build"]
