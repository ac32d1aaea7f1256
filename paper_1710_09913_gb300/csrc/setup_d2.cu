// Setup-side kernel instances, dimension 2.
#include "setup_inst.cuh"
namespace dogip {
bool setup_d2(Ctx& c, const SetupCall& k, cudaStream_t s) {
  switch (c.p * 2 + c.form) {
    DOGIP_SETUP_CASES(2, 1)
    DOGIP_SETUP_CASES(2, 2)
    DOGIP_SETUP_CASES(2, 3)
    DOGIP_SETUP_CASES(2, 4)
    default:
      return false;
  }
}
}  // namespace dogip
