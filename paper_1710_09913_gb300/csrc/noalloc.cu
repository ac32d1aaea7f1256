// FP64 residual norms without any allocation: a variant of the solver's residual
// kernel (r = b - Ky with per-rhs ||r||^2 and ||b||^2, fused grid reduction) whose
// reduction scratch -- one partial sum per block and value, plus the ticket counter
// of the last-block-done pattern -- lives in a fixed file-scope device array instead
// of memory that the library or the caller allocates.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace dogip {
namespace {

constexpr int kNaBlocks = 256;   // maximum grid of the reduction
constexpr int kNaMaxRhs = 32;    // maximum right-hand sides per call
constexpr int kNaThreads = 256;
constexpr size_t kNaPartialBytes = sizeof(double) * kNaBlocks * 2 * kNaMaxRhs;  // 128 KiB
constexpr size_t kNaBytes = kNaPartialBytes + 256;  // + ticket counter (own 256-byte line)

// The scratch.  In host code this name is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

__global__ void __launch_bounds__(kNaThreads) k_residual_norms_static(
    const double* __restrict__ b, const double* __restrict__ Ky, double* __restrict__ r,
    int64_t N, int R, double* __restrict__ out, unsigned char* scratch) {
  double* partial = (double*)scratch;                            // [kNaBlocks][2 R]
  unsigned int* counter = (unsigned int*)(scratch + kNaPartialBytes);
  __shared__ double srr[kNaThreads], sbb[kNaThreads];
  __shared__ bool last;
  // The grid stride is a multiple of R, so every thread stays on one right-hand side
  // (entry i of the dof-major [n x R] arrays belongs to rhs i % R); threads past the
  // rounded stride do no loads.
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x / R) * R;
  double rr = 0.0, bb = 0.0;
  if (t < stride) {
    for (int64_t i = t; i < N; i += stride) {
      const double bi = b[i];
      const double ri = bi - Ky[i];
      if (r != nullptr) r[i] = ri;
      rr += ri * ri;
      bb += bi * bi;
    }
  }
  srr[threadIdx.x] = rr;
  sbb[threadIdx.x] = bb;
  __syncthreads();
  // fixed-order block sums per rhs: thread q (< R) adds the threads of its rhs in order
  const int first = (int)((blockIdx.x * (int64_t)blockDim.x) % R);  // rhs of thread 0
  if (threadIdx.x < R) {
    const int q = threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int k = (q - first + R) % R; k < kNaThreads; k += R) {
      s1 += srr[k];
      s2 += sbb[k];
    }
    partial[(size_t)blockIdx.x * 2 * kNaMaxRhs + 2 * q] = s1;
    partial[(size_t)blockIdx.x * 2 * kNaMaxRhs + 2 * q + 1] = s2;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < R) {  // blocks summed in index order: the result is deterministic
    double trr = 0.0, tbb = 0.0;
    for (unsigned blk = 0; blk < gridDim.x; ++blk) {
      trr += __ldcg(partial + (size_t)blk * 2 * kNaMaxRhs + 2 * threadIdx.x);
      tbb += __ldcg(partial + (size_t)blk * 2 * kNaMaxRhs + 2 * threadIdx.x + 1);
    }
    out[threadIdx.x] = tbb > 0.0 ? sqrt(trr / tbb) : 0.0;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Device address of the scratch on the current device.  Looked up on every call (a
// host call that enqueues nothing), so that it stays valid after the primary context
// of the device has been reset.
unsigned char* scratch_on_current_device() {
  void* p = nullptr;
  cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
  return (unsigned char*)p;
}

}  // namespace
}  // namespace dogip

extern "C" DOGIP_API int dogip_residual_norms_noalloc(const double* b, const double* Ky, double* r,
                                                      int64_t n, int nrhs, double* rel,
                                                      void* stream) {
  try {
    if (!rel || (n > 0 && (!b || !Ky)))
      dogip::fail(DOGIP_EINVAL, "b, Ky and rel are required");
    if (n < 0) dogip::fail(DOGIP_EINVAL, "n must be >= 0");
    if (nrhs < 1 || nrhs > dogip::kNaMaxRhs)
      dogip::fail(DOGIP_EINVAL, "nrhs must be between 1 and 32 (size of the static scratch)");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* scratch = dogip::scratch_on_current_device();
    // the ticket counter must start at zero; the partials are rewritten by every block
    dogip::cuda_check(cudaMemsetAsync(scratch + dogip::kNaPartialBytes, 0, sizeof(unsigned int), s),
                      "clear ticket counter");
    const int64_t N = n * (int64_t)nrhs;
    int64_t blocks = (N + dogip::kNaThreads - 1) / dogip::kNaThreads;
    if (blocks > dogip::kNaBlocks) blocks = dogip::kNaBlocks;
    if (blocks < 1) blocks = 1;
    dogip::k_residual_norms_static<<<(unsigned)blocks, dogip::kNaThreads, 0, s>>>(b, Ky, r, N, nrhs,
                                                                                rel, scratch);
    dogip::cuda_check(cudaGetLastError(), "residual norm kernel launch");
    return DOGIP_OK;
  } catch (const dogip::Failure& e) {
    dogip::set_last_error(e.msg);
    return e.code;
  }
}
