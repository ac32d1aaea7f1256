// Quadrature-point matrix-free apply instances, dimension 2.
#include "apply_qp_inst.cuh"
namespace dogip {
bool apply_qp_d2(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s) {
  switch (c.p * 2 + c.form) {
    DOGIP_QP_CASES(2, 1)
    DOGIP_QP_CASES(2, 2)
    DOGIP_QP_CASES(2, 3)
    DOGIP_QP_CASES(2, 4)
    default:
      return false;
  }
}
}  // namespace dogip
