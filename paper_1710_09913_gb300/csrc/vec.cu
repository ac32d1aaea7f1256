// Vector kernels of the Jacobi-PCG and of the iterative refinement loop.  Every
// reduction is fused into the kernel that produces its terms: each block writes
// its partial sums, and the last block to finish (atomic ticket) adds the
// partials in block order and updates the per-rhs CG scalars on the device, so
// no host round trip is needed inside an iteration.  Vectors are dof-major
// [n x R] with R in {1, 2, 4, 8, 16, 32}: a grid stride that is a multiple of 32
// keeps every lane on one rhs, so warp reductions use xor shuffles over lanes
// with equal lane % R.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace dogip {

namespace {

// See kernels.cuh: first act of a kernel that may be a programmatic dependent.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

constexpr int kNV = 2;  // values reduced per rhs

// 16-byte vector of T (4 floats or 2 doubles) for the one-rhs streaming loops.
template <typename T>
struct alignas(16) Vec16 {
  static constexpr int L = 16 / sizeof(T);
  T v[L];
};
template <typename T>
__device__ __forceinline__ bool aligned16(const T* p) {
  return ((uintptr_t)p & 15u) == 0;
}

struct Red {
  double* partial;
  unsigned int* counter;
  CGScal* scal;
  int* flags;
};

template <int R>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off >= R; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block-reduce acc[0..NV) per rhs, then let the last block combine all partials
// into tot[r * NV + k] (shared) and return true in that block only.
template <int R, int NV>
__device__ bool grid_reduce(const Red& rd, double (&acc)[NV], double* tot) {
  __shared__ double sm[kRedThreads / 32][R * NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double v = warp_sum<R>(acc[k]);
    if (lane < R) sm[wid][lane * NV + k] = v;
  }
  __syncthreads();
  if (threadIdx.x < R * NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) s += sm[w][threadIdx.x];
    rd.partial[(size_t)blockIdx.x * 64 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(rd.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // The last block adds the partials of all blocks: G threads per value, each
  // over a fixed stride of blocks, then a fixed-order tree (deterministic).
  constexpr int RV = R * NV;               // divides kRedThreads
  constexpr int G = kRedThreads / RV;
  __shared__ double fin[kRedThreads];
  {
    const int k = threadIdx.x % RV, g = threadIdx.x / RV;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    unsigned b = g;
    for (; b + 3 * G < gridDim.x; b += 4 * G) {
      s0 += __ldcg(rd.partial + (size_t)b * 64 + k);
      s1 += __ldcg(rd.partial + (size_t)(b + G) * 64 + k);
      s2 += __ldcg(rd.partial + (size_t)(b + 2 * G) * 64 + k);
      s3 += __ldcg(rd.partial + (size_t)(b + 3 * G) * 64 + k);
    }
    for (; b < gridDim.x; b += G) s0 += __ldcg(rd.partial + (size_t)b * 64 + k);
    fin[threadIdx.x] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off * RV) fin[threadIdx.x] += fin[threadIdx.x + off * RV];
    __syncthreads();
  }
  if (threadIdx.x < RV) tot[threadIdx.x] = fin[threadIdx.x];
  __syncthreads();
  return true;
}

__device__ __forceinline__ void set_all_done(const Red& rd, int R) {
  int all = 1, brk = 0, upd = 0;
  for (int r = 0; r < R; ++r) {
    all &= rd.scal[r].done;
    brk |= rd.scal[r].brk;
    upd |= rd.scal[r].upd;
  }
  rd.flags[0] = all | upd;  // stop the chunk: finished, or an FP64 correction is due
  rd.flags[1] = brk;
  rd.flags[2] = all;
  rd.flags[3] = upd;
  *rd.counter = 0u;
}

// CTAs of 256 threads with at least 8 elements per thread: two per SM (152 SMs) for
// vectors that stay in L2 between the kernels of an iteration, four per SM (more
// bytes in flight) from 2^21 entries on, where they stream from HBM.
unsigned red_blocks(int64_t N) {
  int64_t b = (N + 8 * kRedThreads - 1) / (8 * kRedThreads);
  const int64_t cap = N >= (int64_t(1) << 21) ? 4 * 152 : 2 * 152;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// alpha_r = rho_r / (p.q)_r
template <typename T, int R>
__global__ void __launch_bounds__(kRedThreads) k_pq(const T* __restrict__ p, const T* __restrict__ q,
                                                    int64_t N, Red rd) {
  pdl_enter();
  if (rd.flags[0]) return;
  double acc[1] = {0.0};
  T a = T(0);
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t head = 0;
  if constexpr (R == 1) {
    if (aligned16(p) && aligned16(q)) {
      using V = Vec16<T>;
      const int64_t nv = N / V::L;
      const V* p4 = (const V*)p;
      const V* q4 = (const V*)q;
#pragma unroll 2
      for (int64_t k = t0; k < nv; k += stride) {
        const V pv = p4[k], qv = q4[k];
#pragma unroll
        for (int e = 0; e < V::L; ++e) a += pv.v[e] * qv.v[e];
      }
      head = nv * V::L;
    }
  }
  for (int64_t i = head + t0; i < N; i += stride) a += p[i] * q[i];
  acc[0] = (double)a;
  __shared__ double tot[R];
  if (!grid_reduce<R, 1>(rd, acc, tot)) return;
  if (threadIdx.x < R) {
    CGScal& s = rd.scal[threadIdx.x];
    const double v = tot[threadIdx.x];
    if (s.done) {
      s.alpha = 0.0;
    } else if (!(v > 0.0) || !isfinite(v)) {
      s.brk = 1;
      s.done = 1;
      s.alpha = 0.0;
    } else {
      s.pq = v;
      s.alpha = s.rho / v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) set_all_done(rd, R);
}

// x += alpha p, r -= alpha q, rho' = r.(Dinv r), rr = r.r, beta = rho'/rho.
template <typename T, int R>
__global__ void __launch_bounds__(kRedThreads) k_update(T* __restrict__ x, T* __restrict__ r,
                                                        const T* __restrict__ p,
                                                        const T* __restrict__ q,
                                                        const T* __restrict__ dinv, int64_t N,
                                                        double delta, Red rd) {
  pdl_enter();
  if (rd.flags[0]) return;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const T al = (T)rd.scal[t0 % R].alpha;
  T a0 = T(0), a1 = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t head = 0;
  if constexpr (R == 1) {
    if (aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q) && aligned16(dinv)) {
      using V = Vec16<T>;
      const int64_t nv = N / V::L;
      V* x4 = (V*)x;
      V* r4 = (V*)r;
      const V* p4 = (const V*)p;
      const V* q4 = (const V*)q;
      const V* d4 = (const V*)dinv;
#pragma unroll 2
      for (int64_t k = t0; k < nv; k += stride) {
        V xv = x4[k], rv = r4[k];
        const V pv = p4[k], qv = q4[k], dv = d4[k];
#pragma unroll
        for (int e = 0; e < V::L; ++e) {
          xv.v[e] += al * pv.v[e];
          rv.v[e] -= al * qv.v[e];
          a0 += rv.v[e] * (dv.v[e] * rv.v[e]);
          a1 += rv.v[e] * rv.v[e];
        }
        x4[k] = xv;
        r4[k] = rv;
      }
      head = nv * V::L;
    }
  }
  for (int64_t i = head + t0; i < N; i += stride) {
    x[i] += al * p[i];
    const T ri = r[i] - al * q[i];
    r[i] = ri;
    a0 += ri * (dinv[i / R] * ri);
    a1 += ri * ri;
  }
  double acc[2] = {(double)a0, (double)a1};
  __shared__ double tot[R * 2];
  if (!grid_reduce<R, 2>(rd, acc, tot)) return;
  if (threadIdx.x < R) {
    CGScal& s = rd.scal[threadIdx.x];
    if (!s.done) {
      const double rz = tot[threadIdx.x * 2], rr = tot[threadIdx.x * 2 + 1];
      s.beta = rz / s.rho;
      s.rho_prev = s.rho;
      s.rho = rz;
      s.rr = rr;
      s.iters += 1;
      if (sqrt(rr) <= s.tol * s.r0) s.done = 1;
      else if (delta > 0.0 && sqrt(rr) < delta * s.rmax) s.upd = 1;
    } else {
      s.beta = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) set_all_done(rd, R);
}

// p = Dinv r + beta p; also clears q (when given) for the next scatter-add apply
template <typename T, int R>
__global__ void __launch_bounds__(kRedThreads) k_pupdate(T* __restrict__ p, const T* __restrict__ r,
                                                         const T* __restrict__ dinv, int64_t N,
                                                         const CGScal* scal, const int* flags,
                                                         T* __restrict__ qzero) {
  pdl_enter();
  if (flags[0]) return;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const CGScal& s = scal[t0 % R];
  const bool upd = !s.done;
  const T be = (T)s.beta;
  int64_t head = 0;
  if constexpr (R == 1) {
    if (aligned16(p) && aligned16(r) && aligned16(dinv) && (qzero == nullptr || aligned16(qzero))) {
      using V = Vec16<T>;
      const int64_t nv = N / V::L;
      V* p4 = (V*)p;
      const V* r4 = (const V*)r;
      const V* d4 = (const V*)dinv;
      V* q4 = (V*)qzero;
      V zero;
#pragma unroll
      for (int e = 0; e < V::L; ++e) zero.v[e] = T(0);
#pragma unroll 2
      for (int64_t k = t0; k < nv; k += stride) {
        if (q4 != nullptr) q4[k] = zero;
        if (upd) {
          V pv = p4[k];
          const V rv = r4[k], dv = d4[k];
#pragma unroll
          for (int e = 0; e < V::L; ++e) pv.v[e] = dv.v[e] * rv.v[e] + be * pv.v[e];
          p4[k] = pv;
        }
      }
      head = nv * V::L;
    }
  }
  for (int64_t i = head + t0; i < N; i += stride) {
    if (qzero != nullptr) qzero[i] = T(0);
    if (upd) p[i] = dinv[i / R] * r[i] + be * p[i];
  }
}

// Chronopoulos-Gear CG step (one right-hand side, FP32 vectors) before the apply:
//   p = u + beta p,  s = w + beta s  (first step: p = u, s = w),
//   x += alpha p,  r -= alpha s,  u = Dinv r,  w = 0 (for the scatter-add apply),
//   gamma = r.u, rr = r.r; the last block sets beta = gamma / gamma_old and tests
//   convergence.  With s = K p kept by recurrence, one reduction phase (here) and the
//   energy reduction of the apply replace the three of the standard recurrence.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cgcg(T* __restrict__ x, T* __restrict__ r,
                                                      T* __restrict__ u, T* __restrict__ w,
                                                      T* __restrict__ p, T* __restrict__ sv,
                                                      const T* __restrict__ dinv, int64_t N,
                                                      Red rd) {
  pdl_enter();
  if (rd.flags[0]) return;
  const CGScal& s0 = rd.scal[0];
  const bool first = s0.iters == 0;
  const T al = (T)s0.alpha, be = first ? T(0) : (T)s0.beta;
  T a0 = T(0), a1 = T(0);
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto step = [&](T& xv, T& rv, T& uv, T& wv, T& pv, T& svv, T dv) {
    pv = first ? uv : uv + be * pv;
    svv = first ? wv : wv + be * svv;
    xv += al * pv;
    rv -= al * svv;
    uv = dv * rv;
    wv = T(0);
    a0 += rv * uv;
    a1 += rv * rv;
  };
  int64_t head = 0;
  if (aligned16(x) && aligned16(r) && aligned16(u) && aligned16(w) && aligned16(p) &&
      aligned16(sv) && aligned16(dinv)) {
    using V = Vec16<T>;
    const int64_t nv = N / V::L;
    V *x4 = (V*)x, *r4 = (V*)r, *u4 = (V*)u, *w4 = (V*)w, *p4 = (V*)p, *s4 = (V*)sv;
    const V* d4 = (const V*)dinv;
    for (int64_t k = t0; k < nv; k += stride) {
      V xv = x4[k], rv = r4[k], uv = u4[k], wv = w4[k], pv = p4[k], svv = s4[k];
      const V dv = d4[k];
#pragma unroll
      for (int e = 0; e < V::L; ++e) step(xv.v[e], rv.v[e], uv.v[e], wv.v[e], pv.v[e], svv.v[e], dv.v[e]);
      x4[k] = xv;
      r4[k] = rv;
      u4[k] = uv;
      w4[k] = wv;
      p4[k] = pv;
      s4[k] = svv;
    }
    head = nv * V::L;
  }
  for (int64_t i = head + t0; i < N; i += stride) {
    T xv = x[i], rv = r[i], uv = u[i], wv = w[i], pv = p[i], svv = sv[i];
    step(xv, rv, uv, wv, pv, svv, dinv[i]);
    x[i] = xv;
    r[i] = rv;
    u[i] = uv;
    w[i] = wv;
    p[i] = pv;
    sv[i] = svv;
  }
  double acc[2] = {(double)a0, (double)a1};
  __shared__ double tot[2];
  if (!grid_reduce<1, 2>(rd, acc, tot)) return;
  if (threadIdx.x == 0) {
    CGScal& s = rd.scal[0];
    if (!s.done) {
      const double gam = tot[0], rr = tot[1];
      s.beta = gam / s.rho;
      s.rho_prev = s.rho;
      s.rho = gam;
      s.rr = rr;
      s.iters += 1;
      if (sqrt(rr) <= s.tol * s.r0) s.done = 1;
    }
    set_all_done(rd, 1);
  }
}

// Start of a PCG run from the residual r: p = Dinv r, rho = r.p, r0.
template <typename T, int R>
__global__ void __launch_bounds__(kRedThreads) k_init(const T* __restrict__ r, T* __restrict__ p,
                                                      T* __restrict__ x, const T* __restrict__ dinv,
                                                      int64_t N, double tol, int r0_from_bb,
                                                      int zero_x, T* __restrict__ qzero, Red rd) {
  T a0 = T(0), a1 = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const T ri = r[i];
    const T zi = dinv[i / R] * ri;
    p[i] = zi;
    qzero[i] = T(0);
    if (zero_x) x[i] = T(0);
    a0 += ri * zi;
    a1 += ri * ri;
  }
  double acc[2] = {(double)a0, (double)a1};
  __shared__ double tot[R * 2];
  if (!grid_reduce<R, 2>(rd, acc, tot)) return;
  if (threadIdx.x < R) {
    CGScal& s = rd.scal[threadIdx.x];
    s.rho = tot[threadIdx.x * 2];
    s.rr = tot[threadIdx.x * 2 + 1];
    s.r0 = r0_from_bb ? sqrt(s.bb) : sqrt(s.rr);
    s.tol = tol;
    s.alpha = s.beta = s.pq = 0.0;
    s.rho_prev = s.rho;
    s.rmax = sqrt(s.rr);
    s.iters = 0;
    s.brk = 0;
    s.upd = 0;
    s.done = (s.rr == 0.0 || sqrt(s.rr) <= tol * s.r0) ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) set_all_done(rd, R);
}

// r = b - Kx in FP64 with ||r||^2 (and ||b||^2).
template <int R>
__global__ void __launch_bounds__(kRedThreads) k_residual64(const double* __restrict__ b,
                                                            const double* __restrict__ Kx,
                                                            double* __restrict__ r, int64_t N,
                                                            int first, double otol, Red rd) {
  double a0 = 0.0, a1 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const double bi = b[i];
    const double ri = bi - Kx[i];
    r[i] = ri;
    a0 += ri * ri;
    if (first) a1 += bi * bi;
  }
  double acc[2] = {a0, a1};
  __shared__ double tot[R * 2];
  if (!grid_reduce<R, 2>(rd, acc, tot)) return;
  if (threadIdx.x < R) {
    CGScal& s = rd.scal[threadIdx.x];
    const double rr = tot[threadIdx.x * 2];
    if (first) s.bb = tot[threadIdx.x * 2 + 1];
    s.rr = rr;
    s.s = sqrt(rr);
    s.rel = s.bb > 0.0 ? sqrt(rr / s.bb) : 0.0;
    s.otol = otol;
    s.odone = s.rel <= otol ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *rd.counter = 0u;
}

template <int R>
__global__ void k_to32(const double* __restrict__ r64, float* __restrict__ r32, float* __restrict__ x32,
                       int64_t N, const CGScal* scal) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const CGScal& s = scal[t0 % R];
  const double inv = (s.odone || s.s == 0.0) ? 0.0 : 1.0 / s.s;
  for (int64_t i = t0; i < N; i += stride) {
    r32[i] = (float)(r64[i] * inv);
    x32[i] = 0.0f;
  }
}

template <int R>
__global__ void k_correct(double* __restrict__ x64, const float* __restrict__ x32, int64_t N,
                          const CGScal* scal) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const CGScal& s = scal[t0 % R];
  if (s.odone) return;
  for (int64_t i = t0; i < N; i += stride) x64[i] += s.s * (double)x32[i];
}

// r32 = (float) r64, x32 = 0
template <int R>
__global__ void k_narrow(const double* __restrict__ r64, float* __restrict__ r32,
                         float* __restrict__ x32, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    r32[i] = (float)r64[i];
    x32[i] = 0.0f;
  }
}

// x64 += x32, x32 = 0
template <int R>
__global__ void k_fold(double* __restrict__ x64, float* __restrict__ x32, int64_t N) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    x64[i] += (double)x32[i];
    x32[i] = 0.0f;
  }
}

// Residual replacement: r32 = r64 (true FP64 residual), rho' = r32.(Dinv r32),
// beta = rho' / rho_prev; per rhs done iff the true residual meets the tolerance.
template <int R>
__global__ void __launch_bounds__(kRedThreads) k_rel_restart(const double* __restrict__ r64,
                                                             float* __restrict__ r32,
                                                             const float* __restrict__ dinv,
                                                             int64_t N, Red rd) {
  float a0 = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const float ri = (float)r64[i];
    r32[i] = ri;
    a0 += ri * (dinv[i / R] * ri);
  }
  double acc[1] = {(double)a0};
  __shared__ double tot[R];
  if (!grid_reduce<R, 1>(rd, acc, tot)) return;
  if (threadIdx.x < R) {
    CGScal& s = rd.scal[threadIdx.x];
    const double rz = tot[threadIdx.x];
    const double true_rr = s.rr;  // from the FP64 residual kernel just before
    s.done = (sqrt(true_rr) <= s.tol * s.r0) ? 1 : 0;
    s.beta = s.done ? 0.0 : rz / s.rho_prev;
    s.rho = rz;
    s.rmax = sqrt(true_rr);
    s.upd = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) set_all_done(rd, R);
}

Red red_of(SolveWork& w) { return Red{w.partial, w.counter, w.scal, w.flags}; }

#define DOGIP_R_SWITCH(R, CALL) \
  switch (R) {                  \
    case 1: CALL(1); break;     \
    case 2: CALL(2); break;     \
    case 4: CALL(4); break;     \
    case 8: CALL(8); break;     \
    case 16: CALL(16); break;   \
    case 32: CALL(32); break;   \
    default: fail(DOGIP_EINVAL, "nrhs must be 1, 2, 4, 8, 16 or 32 for solves"); \
  }

}  // namespace

void vec_alloc(SolveWork& w, int64_t n, int R) {
  if (w.R == R && w.n == n) return;
  vec_free(w);
  const size_t N = (size_t)n * R;
  auto dm = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      fail(DOGIP_ENOMEM, "device allocation of solver workspace failed");
    }
  };
  dm((void**)&w.x64, N * 8);
  dm((void**)&w.r64, N * 8);
  dm((void**)&w.p64, N * 8);
  dm((void**)&w.q64, N * 8);
  dm((void**)&w.x32, N * 4);
  dm((void**)&w.r32, N * 4);
  dm((void**)&w.p32, N * 4);
  dm((void**)&w.q32, N * 4);
  dm((void**)&w.partial, sizeof(double) * kMaxRedBlocks * 64);
  dm((void**)&w.counter, sizeof(unsigned int) * 4);
  dm((void**)&w.scal, sizeof(CGScal) * 32);
  dm((void**)&w.flags, sizeof(int) * 8);
  cuda_check(cudaMemset(w.counter, 0, sizeof(unsigned int) * 4), "memset counter");
  cuda_check(cudaMemset(w.scal, 0, sizeof(CGScal) * 32), "memset scal");
  cuda_check(cudaMemset(w.flags, 0, sizeof(int) * 8), "memset flags");
  if (cudaMallocHost((void**)&w.h_flags, sizeof(int) * 8) != cudaSuccess ||
      cudaMallocHost((void**)&w.h_scal, sizeof(CGScal) * 32) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "pinned host allocation failed");
  }
  w.R = R;
  w.n = n;
}

void vec_alloc_cgcg(SolveWork& w) {
  if (w.pc32 != nullptr) return;
  const size_t N = (size_t)w.n * w.R;
  if (cudaMalloc((void**)&w.pc32, N * 4) != cudaSuccess ||
      cudaMalloc((void**)&w.sc32, N * 4) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "device allocation of solver workspace failed");
  }
}

void vec_free(SolveWork& w) {
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w.graph = nullptr;
  for (void* p : {(void*)w.x64, (void*)w.r64, (void*)w.p64, (void*)w.q64, (void*)w.x32,
                  (void*)w.r32, (void*)w.p32, (void*)w.q32, (void*)w.partial, (void*)w.counter,
                  (void*)w.scal, (void*)w.flags, (void*)w.pc32, (void*)w.sc32, (void*)w.pb32,
                  (void*)w.pb64})
    if (p) cudaFree(p);
  if (w.h_flags) cudaFreeHost(w.h_flags);
  if (w.h_scal) cudaFreeHost(w.h_scal);
  w = SolveWork{};
}

int vec_residual64(SolveWork& w, const double* b, const double* Kx, bool first, double otol,
                    cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
#define CALL(RR) k_residual64<RR><<<red_blocks(N), kRedThreads, 0, st>>>(b, Kx, w.r64, N, first, otol, rd)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "residual kernel");
  return 1;
}

int vec_inner_init32(SolveWork& w, const float* dinv, double inner_tol, cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
#define CALL(RR)                                                                              \
  k_to32<RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r64, w.r32, w.x32, N, w.scal);          \
  k_init<float, RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r32, w.p32, w.x32, dinv, N,       \
                                                            inner_tol, 0, 0, w.q32, rd)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "inner init kernels");
  return 2;
}

int vec_init64(SolveWork& w, const double* dinv, double tol, cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
#define CALL(RR) \
  k_init<double, RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r64, w.p64, w.x64, dinv, N, tol, 1, 0, \
                                                             w.q64, rd)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "init kernel");
  return 1;
}

int vec_cg_step(SolveWork& w, int prec, double* x64, const void* dinv, double delta,
                cudaStream_t st, bool zero_q, bool with_pq) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
  const unsigned nb = red_blocks(N);
  if (prec == DOGIP_FP64) {
    const double* di = (const double*)dinv;
#define CALL(RR)                                                                           \
  pdl_mark((const void*)k_pq<double, RR>);                                                 \
  pdl_mark((const void*)k_update<double, RR>);                                             \
  pdl_mark((const void*)k_pupdate<double, RR>);                                            \
  k_pq<double, RR><<<nb, kRedThreads, 0, st>>>(w.p64, w.q64, N, rd);                       \
  k_update<double, RR><<<nb, kRedThreads, 0, st>>>(x64, w.r64, w.p64, w.q64, di, N, delta, rd); \
  k_pupdate<double, RR><<<nb, kRedThreads, 0, st>>>(w.p64, w.r64, di, N, w.scal, w.flags,  \
                                                     zero_q ? w.q64 : nullptr)
    DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  } else {
    const float* di = (const float*)dinv;
#define CALL(RR)                                                                           \
  pdl_mark((const void*)k_pq<float, RR>);                                                  \
  pdl_mark((const void*)k_update<float, RR>);                                              \
  pdl_mark((const void*)k_pupdate<float, RR>);                                             \
  if (with_pq) k_pq<float, RR><<<nb, kRedThreads, 0, st>>>(w.p32, w.q32, N, rd);           \
  k_update<float, RR><<<nb, kRedThreads, 0, st>>>(w.x32, w.r32, w.p32, w.q32, di, N, delta, rd); \
  k_pupdate<float, RR><<<nb, kRedThreads, 0, st>>>(w.p32, w.r32, di, N, w.scal, w.flags,   \
                                                    zero_q ? w.q32 : nullptr)
    DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  }
  cuda_check(cudaGetLastError(), "cg step kernels");
  return with_pq || prec == DOGIP_FP64 ? 3 : 2;
}

int vec_rel_init(SolveWork& w, const float* dinv, double tol, cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
#define CALL(RR)                                                                             \
  k_narrow<RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r64, w.r32, w.x32, N);               \
  k_init<float, RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r32, w.p32, w.x32, dinv, N, tol, \
                                                            1, 0, w.q32, rd)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "reliable init kernels");
  return 2;
}

int vec_fold(SolveWork& w, double* x64, cudaStream_t st) {
  const int64_t N = w.n * w.R;
#define CALL(RR) k_fold<RR><<<red_blocks(N), kRedThreads, 0, st>>>(x64, w.x32, N)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "fold kernel");
  return 1;
}

int vec_rel_restart(SolveWork& w, const float* dinv, cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
#define CALL(RR)                                                                              \
  k_rel_restart<RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.r64, w.r32, dinv, N, rd);        \
  k_pupdate<float, RR><<<red_blocks(N), kRedThreads, 0, st>>>(w.p32, w.r32, dinv, N, w.scal,  \
                                                               w.flags, w.q32)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "reliable restart kernels");
  return 2;
}

int vec_correct(SolveWork& w, double* x64, cudaStream_t st) {
  const int64_t N = w.n * w.R;
#define CALL(RR) k_correct<RR><<<red_blocks(N), kRedThreads, 0, st>>>(x64, w.x32, N, w.scal)
  DOGIP_R_SWITCH(w.R, CALL);
#undef CALL
  cuda_check(cudaGetLastError(), "correct kernel");
  return 1;
}

int vec_cgcg_step(SolveWork& w, const float* dinv, cudaStream_t st) {
  const int64_t N = w.n * w.R;
  Red rd = red_of(w);
  pdl_mark((const void*)k_cgcg<float>);
  k_cgcg<float><<<red_blocks(N), kRedThreads, 0, st>>>(w.x32, w.r32, w.p32, w.q32, w.pc32,
                                                       w.sc32, dinv, N, rd);
  cuda_check(cudaGetLastError(), "cg step kernel");
  return 1;
}

}  // namespace dogip
