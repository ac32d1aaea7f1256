// Higher orders (2D p = 5..8, 3D p = 4): the same Algorithm 1 and Theorems 4 / 8 with
// the reference tables as run-time data instead of compile-time constants, so that the
// instances compile in seconds whatever the table size.  B (exact rationals rounded
// once, from gen_tables.cpp) is staged in shared memory per CTA and read by broadcast;
// u_T and Y_T stay in registers (V is a compile-time constant); the W-node loop is a
// run-time loop.  Every entry of B is used, zeros included.
#include "kernels.cuh"
#include "tables_hi.h"

namespace dogip {
namespace {

constexpr int binom_c(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

template <int D, int P, int FORM>
struct HiCfg {
  static constexpr int V = binom_c(P + D, D);
  static constexpr int W = binom_c((FORM == DOGIP_PROJECTION ? 2 * P : 2 * P - 2) + D, D);
  static constexpr int NB = FORM == DOGIP_PROJECTION ? 1 : D;
  static constexpr int NS = NSym<D, FORM>::value;
  static constexpr int THREADS = 128;
  template <typename T>
  static constexpr size_t smem() { return sizeof(T) * NB * W * V; }
};

template <typename T>
struct HiArgs {
  const T* B;            // [NB][W][V]
  const T* A;            // AoSoA [Epad/32][W*NS][32]
  const uint32_t* conn;  // AoSoA [Epad/32][V][32]
  const T* u;
  T* y;
  int64_t e0, e1;
  int R;
  const int* skip;
};

template <int D, int P, int FORM, typename T, bool ATOMIC, bool MULTI>
__global__ void __launch_bounds__(128) k_apply_hi(HiArgs<T> a) {
  using C = HiCfg<D, P, FORM>;
  constexpr int V = C::V, W = C::W, NB = C::NB, NS = C::NS;
  extern __shared__ unsigned char smem_raw[];
  T* sB = (T*)smem_raw;
  if (a.skip != nullptr && *a.skip) return;
  for (int k = threadIdx.x; k < NB * W * V; k += blockDim.x) sB[k] = a.B[k];
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t e;
  int r = 0;
  if constexpr (MULTI) {
    const int64_t q = t / a.R;
    e = a.e0 + q;
    r = (int)(t - q * a.R);
  } else {
    e = a.e0 + t;
  }
  if (e >= a.e1) return;
  const int R = MULTI ? a.R : 1;
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  const T* At = a.A + tile * ((int64_t)W * NS * kTile) + lane;
  uint32_t c[V];
  T ul[V], Y[V];
#pragma unroll
  for (int l = 0; l < V; ++l) {
    c[l] = __ldg(ct + l * kTile);
    ul[l] = (c[l] & kBndBit) ? T(0) : __ldg(a.u + (int64_t)(c[l] & kIdMask) * R + r);
    Y[l] = T(0);
  }
#pragma unroll 1
  for (int j = 0; j < W; ++j) {
    T g[NB], h[NB], aj[NS];
#pragma unroll
    for (int rr = 0; rr < NB; ++rr) {
      const T* Bj = sB + ((size_t)rr * W + j) * V;
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < V; ++l) acc = fma(Bj[l], ul[l], acc);
      g[rr] = acc;
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) aj[k] = __ldg(At + (j * NS + k) * kTile);
    block_mul<D, FORM>(aj, g, h);
#pragma unroll
    for (int rr = 0; rr < NB; ++rr) {
      const T* Bj = sB + ((size_t)rr * W + j) * V;
#pragma unroll
      for (int l = 0; l < V; ++l) Y[l] = fma(Bj[l], h[rr], Y[l]);
    }
  }
#pragma unroll
  for (int l = 0; l < V; ++l) {
    if (!(c[l] & kBndBit)) {
      T* dst = a.y + (int64_t)(c[l] & kIdMask) * R + r;
      if constexpr (ATOMIC) atomicAdd(dst, Y[l]);
      else *dst += Y[l];
    }
  }
}

// Step a8 with run-time tables: A_T,j = w_j K_T for every W node, the geometry and the
// Jacobi diagonal sum_j w_j B_{.jl}^T K_T B_{.jl}.
template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_ahat_hi(AhatArgs a, const double* B, const double* w) {
  using C = HiCfg<D, P, FORM>;
  constexpr int V = C::V, W = C::W, NB = C::NB, NS = C::NS;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  double K[NS], Ri[D][D], vol;
  const int err = cell_factor<D, FORM>(a, pos, K, Ri, vol);
  if (err) atomicOr(a.err, err);
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  double* At = a.A64 + tile * ((int64_t)W * NS * kTile) + lane;
  float* At32 = a.A32 ? a.A32 + tile * ((int64_t)W * NS * kTile) + lane : nullptr;
  for (int j = 0; j < W; ++j) {
    const double wj = __ldg(w + j);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double v = wj * K[k];
      At[(j * NS + k) * kTile] = v;
      if (At32) At32[(j * NS + k) * kTile] = (float)v;
    }
  }
  double* g = a.geo + pos * (D * D + 1);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) g[i * D + k] = Ri[i][k];
  g[D * D] = vol;
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  for (int l = 0; l < V; ++l) {
    const uint32_t cl = ct[l * kTile];
    if (cl & kBndBit) continue;
    double acc = 0.0;
    for (int j = 0; j < W; ++j) {
      double q = 0.0;
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        const double br = __ldg(B + ((size_t)r * W + j) * V + l);
#pragma unroll
        for (int s = 0; s < NB; ++s) q += br * __ldg(B + ((size_t)s * W + j) * V + l) * K[sym_idx(D, r, s)];
      }
      acc += __ldg(w + j) * q;
    }
    atomicAdd(a.diag + (cl & kIdMask), acc);
  }
}

// b_l += f_T |det R_T| int_That phi_l with the run-time integrals iv.
template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_load_hi(LoadArgs a, const double* iv) {
  constexpr int V = HiCfg<D, P, FORM>::V;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  const double fv = (a.f ? a.f[a.perm[pos]] : 1.0) * a.geo[pos * (D * D + 1) + D * D];
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  for (int l = 0; l < V; ++l) {
    const uint32_t cl = ct[l * kTile];
    if (!(cl & kBndBit)) atomicAdd(a.b + (cl & kIdMask), fv * __ldg(iv + l));
  }
}

template <int D, int P, int FORM, typename T>
void hi_attr() {
  using C = HiCfg<D, P, FORM>;
  const int sm = (int)C::template smem<T>();
  for (auto k : {k_apply_hi<D, P, FORM, T, true, false>, k_apply_hi<D, P, FORM, T, true, true>,
                 k_apply_hi<D, P, FORM, T, false, false>, k_apply_hi<D, P, FORM, T, false, true>})
    cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
               "high-order apply smem attribute");
}

template <int D, int P, int FORM>
int hi_run(const Ctx& c, int op, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
           int64_t e1, cudaStream_t s, const int* skip, AhatArgs* ah, LoadArgs* ld, bool add) {
  using C = HiCfg<D, P, FORM>;
  if (op == 0) {  // apply
    if (u == nullptr) {  // preparation call (context set-up, outside capture)
      hi_attr<D, P, FORM, double>();
      hi_attr<D, P, FORM, float>();
      apply_tc(c, nullptr, nullptr, nullptr, nullptr);
      return 1;
    }
    // variant 3: the tensor-core kernel (FP32, one right-hand side, whole range)
    const int var = c.apply_variant_prec[prec] >= 0 ? c.apply_variant_prec[prec] : c.apply_variant;
    if (var == 3 && prec == DOGIP_FP32 && R == 1 && atomic && e0 == 0 && e1 == c.E &&
        apply_tc(c, u, y, s, skip, add))
      return 2;
    const int64_t nth = (e1 - e0) * (int64_t)R;
    if (nth <= 0) return 1;
    const unsigned nb = (unsigned)((nth + C::THREADS - 1) / C::THREADS);
    auto go = [&](auto tag) {
      using T = decltype(tag);
      const T* B = std::is_same<T, double>::value ? (const T*)c.d_hiB64 : (const T*)c.d_hiB32;
      const T* A = std::is_same<T, double>::value ? (const T*)c.d_A64 : (const T*)c.d_A32;
      HiArgs<T> a{B, A, c.d_conn, (const T*)u, (T*)y, e0, e1, R, skip};
      const size_t sm = C::template smem<T>();
      if (R == 1) {
        if (atomic) k_apply_hi<D, P, FORM, T, true, false><<<nb, C::THREADS, sm, s>>>(a);
        else k_apply_hi<D, P, FORM, T, false, false><<<nb, C::THREADS, sm, s>>>(a);
      } else {
        if (atomic) k_apply_hi<D, P, FORM, T, true, true><<<nb, C::THREADS, sm, s>>>(a);
        else k_apply_hi<D, P, FORM, T, false, true><<<nb, C::THREADS, sm, s>>>(a);
      }
    };
    if (prec == DOGIP_FP64) go(double{});
    else go(float{});
    return 1;
  }
  const unsigned nb = (unsigned)((c.E + 127) / 128);
  if (op == 1) k_ahat_hi<D, P, FORM><<<nb, 128, 0, s>>>(*ah, c.d_hiB64, c.d_hiW);
  else k_load_hi<D, P, FORM><<<nb, 128, 0, s>>>(*ld, c.d_hiIV);
  return 1;
}

int hi_dispatch(const Ctx& c, int op, const void* u, void* y, int R, int prec, bool atomic,
                int64_t e0, int64_t e1, cudaStream_t s, const int* skip, AhatArgs* ah,
                LoadArgs* ld, bool add = false) {
#define HI_CASE(D, P, F)                                                               \
  if (c.d == D && c.p == P && c.form == F)                                             \
    return hi_run<D, P, F>(c, op, u, y, R, prec, atomic, e0, e1, s, skip, ah, ld, add);
  HI_CASE(2, 5, 0) HI_CASE(2, 5, 1) HI_CASE(2, 6, 0) HI_CASE(2, 6, 1)
  HI_CASE(2, 7, 0) HI_CASE(2, 7, 1) HI_CASE(2, 8, 0) HI_CASE(2, 8, 1)
  HI_CASE(3, 4, 0) HI_CASE(3, 4, 1)
#undef HI_CASE
  return 0;
}

}  // namespace

int apply_hi(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
             int64_t e1, cudaStream_t s, const int* skip, bool add) {
  return hi_dispatch(c, 0, u, y, R, prec, atomic, e0, e1, s, skip, nullptr, nullptr, add);
}

bool ahat_hi(const Ctx& c, AhatArgs& a, cudaStream_t s) {
  return hi_dispatch(c, 1, nullptr, nullptr, 1, 0, true, 0, 0, s, nullptr, &a, nullptr) != 0;
}

bool load_hi(const Ctx& c, LoadArgs& a, cudaStream_t s) {
  return hi_dispatch(c, 2, nullptr, nullptr, 1, 0, true, 0, 0, s, nullptr, nullptr, &a) != 0;
}

bool hi_table(int d, int p, int form, int* NB, int* W, int* V, long long* nnz, long long* nnz1,
              const double** B, const double** w, const double** iv) {
  for (int k = 0; k < dogip_hi::kNumHi; ++k) {
    const auto& t = dogip_hi::kHiTabs[k];
    if (t.d == d && t.p == p && t.form == form) {
      if (NB) *NB = t.NB;
      if (W) *W = t.W;
      if (V) *V = t.V;
      if (nnz) *nnz = t.nnz;
      if (nnz1) *nnz1 = t.nnz1;
      if (B) *B = t.B;
      if (w) *w = t.w;
      if (iv) *iv = t.iv;
      return true;
    }
  }
  return false;
}

}  // namespace dogip
