// Global double-grid apply of the weighted projection: instances for 2D P1-P4 and
// 3D P1-P3, and the FP64 -> FP32 copy of A_diag.
#include "kernels.cuh"

namespace dogip {
namespace {

template <int D, int P, typename T>
void gw_run(const Ctx& c, const T* A, const void* u, T* w, void* y, int R, cudaStream_t s,
            const int* skip) {
  GwArgs<T> a{c.d_conn, c.d_connW, A, (const T*)u, w, (T*)y, c.E, R, skip};
  const int64_t nth = c.E * (int64_t)R;
  const unsigned nb = (unsigned)((nth + 255) / 256);
  if (R == 1) {
    k_gw_interp<D, P, T, false><<<nb, 256, 0, s>>>(a);
    k_gw_project<D, P, T, false><<<nb, 256, 0, s>>>(a);
  } else {
    k_gw_interp<D, P, T, true><<<nb, 256, 0, s>>>(a);
    k_gw_project<D, P, T, true><<<nb, 256, 0, s>>>(a);
  }
}

template <int D, int P>
void gw_prec(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s,
             const int* skip) {
  if (prec == DOGIP_FP64) gw_run<D, P, double>(c, c.d_Aw64, u, c.d_w64, y, R, s, skip);
  else gw_run<D, P, float>(c, c.d_Aw32, u, c.d_w32, y, R, s, skip);
}

__global__ void k_narrow_copy(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

}  // namespace

bool apply_gw(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s,
              const int* skip) {
  switch (c.d * 16 + c.p) {
    case 2 * 16 + 1: gw_prec<2, 1>(c, u, y, R, prec, s, skip); return true;
    case 2 * 16 + 2: gw_prec<2, 2>(c, u, y, R, prec, s, skip); return true;
    case 2 * 16 + 3: gw_prec<2, 3>(c, u, y, R, prec, s, skip); return true;
    case 2 * 16 + 4: gw_prec<2, 4>(c, u, y, R, prec, s, skip); return true;
    case 3 * 16 + 1: gw_prec<3, 1>(c, u, y, R, prec, s, skip); return true;
    case 3 * 16 + 2: gw_prec<3, 2>(c, u, y, R, prec, s, skip); return true;
    case 3 * 16 + 3: gw_prec<3, 3>(c, u, y, R, prec, s, skip); return true;
    default: return false;
  }
}

void narrow_copy(const double* a, float* b, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t nb = std::min<int64_t>((n + 255) / 256, 4 * 152);
  k_narrow_copy<<<(unsigned)nb, 256, 0, s>>>(a, b, n);
  cuda_check(cudaGetLastError(), "narrow copy");
}

}  // namespace dogip
