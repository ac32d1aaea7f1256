// Apply kernel instances, dimension 2, orders 1 2 3 4.
#include "apply_inst.cuh"
namespace dogip {
int apply_d2(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic,
                 int64_t e0, int64_t e1, cudaStream_t s, const int* skip, bool add) {
  switch (c.p * 2 + c.form) {
    DOGIP_APPLY_CASES(2, 1)
    DOGIP_APPLY_CASES(2, 2)
    DOGIP_APPLY_CASES(2, 3)
    DOGIP_APPLY_CASES(2, 4)
    default:
      return 0;
  }
}
}  // namespace dogip
