// Apply kernel instances, dimension 3, orders 1 2.
#include "apply_inst.cuh"
namespace dogip {
int apply_d3a(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic,
                 int64_t e0, int64_t e1, cudaStream_t s, const int* skip, bool add) {
  switch (c.p * 2 + c.form) {
    DOGIP_APPLY_CASES(3, 1)
    DOGIP_APPLY_CASES(3, 2)
    default:
      return 0;
  }
}
}  // namespace dogip
