// Quadrature-point matrix-free apply instances, dimension 3.
#include "apply_qp_inst.cuh"
namespace dogip {
bool apply_qp_d3(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s) {
  switch (c.p * 2 + c.form) {
    DOGIP_QP_CASES(3, 1)
    DOGIP_QP_CASES(3, 2)
    DOGIP_QP_CASES(3, 3)
    default:
      return false;
  }
}
}  // namespace dogip
