// Setup-side kernel instances, dimension 3.
#include "setup_inst.cuh"
namespace dogip {
bool setup_d3(Ctx& c, const SetupCall& k, cudaStream_t s) {
  switch (c.p * 2 + c.form) {
    DOGIP_SETUP_CASES(3, 1)
    DOGIP_SETUP_CASES(3, 2)
    DOGIP_SETUP_CASES(3, 3)
    default:
      return false;
  }
}
}  // namespace dogip
