// Whole-solve persistent PCG for problems whose operator and vectors stay in L2.
//
// At small sizes (2D P1 on 512 x 512 squares: 263 k dofs, 19 MB of A_T, conn and
// vectors) an iteration of the kernel-per-step PCG costs the latency of four kernel
// boundaries and three last-block reductions, not bandwidth.  Here one cooperative
// launch runs the Jacobi-PCG iterations of one solve (R = 1, atomic scatter) with two
// grid-wide barriers per iteration:
//
//   A  q = K p  (Algorithm 1 per cell, one thread per cell, atomic scatter; the
//      Dirichlet rows q_b = p_b), and (p, K p) from the cells' energies
//      sum_T p_T . Y_T plus p_b^2 on the Dirichlet rows.  The search direction of this
//      iteration, p = Dinv r + beta p_old, is formed where it is read (the gathers and
//      the owner of each dof), into the other of two p buffers.
//   -- barrier + reduction: alpha = rho / (p, K p)
//   C  x += alpha p, r -= alpha q, q = 0, rho' = r.(Dinv r), ||r||^2
//   -- barrier + reduction: beta = rho' / rho, convergence test
//
// Every block reduces the per-block partial sums itself, in the same order, so all
// blocks hold bitwise the same CG scalars and take the same branch.  Data written
// by other blocks during the launch is read through L2 (ld.global.cg), never from a
// possibly stale L1 line.  Each barrier wait is bounded by a clock budget: on expiry
// the block raises the kernel error flag and leaves; the others see the flag (or run
// out of budget) at their next wait and leave too.
#include "kernels.cuh"

namespace dogip {

namespace {

// Threads per block: 1024 (one block per SM, fewer arrivals per barrier) where the
// instance fits in 64 registers, else 256.
template <int D, int P, typename T>
constexpr int pcg_threads() {
  return (D == 2 && P == 1) || (sizeof(T) == 4 && ((D == 2 && P == 2) || (D == 3 && P == 1)))
             ? 1024
             : 256;
}

template <typename T>
struct PcgArgs {
  const T* A;            // AoSoA A_T
  const uint32_t* conn;  // AoSoA conn
  int64_t E;             // cells (processing order 0..E-1)
  const int32_t* bnd;    // Dirichlet dofs [nbnd]
  int64_t nbnd;
  T* x;
  T* r;
  T* p0;  // p at entry (and at exit when the iteration limit is reached)
  T* p1;  // second search-direction buffer
  T* q;   // zero at entry
  const T* dinv;
  int64_t n;
  CGScal* scal;
  int* flags;
  double* partial;     // [4 x gridDim]: two halves of two values per block
  unsigned int* bar;   // arrival counter, zero at entry
  int* kerr;           // raised when a barrier wait expires
  long long budget;    // clock cycles per barrier wait
  int maxit;
  int test_skip;       // test hook: this block leaves at its first barrier without
                       // arriving, so the others' bounded waits expire (-1: none)
};

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void arrive_release(unsigned int* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void fence_acquire() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Block sums of NV values in a fixed order: xor shuffles within each warp in the
// working precision T, then warp 0 adds the warps' sums in double (GB300 runs FP64 at
// a small fraction of the FP32 rate, so double arithmetic stays in one warp).  The
// totals land in tot[0..NV-1] (shared), read by every thread after the final barrier.
template <int NV, typename T>
__device__ __forceinline__ void block_sums(const T (&v)[NV], double (*ws)[32], double* tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    w[k] = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], off);
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) ws[k][wid] = (double)w[k];
  __syncthreads();
  if (wid == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? ws[k][lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane == 0) tot[k] = t;
    }
  }
}

// Grid barrier that also sums NV <= 2 values over all blocks: every block stores its
// block sums, arrives, waits (bounded) until all blocks have arrived, then warp 0 of
// every block adds the partial sums of all blocks in the same fixed order, so every
// block holds bitwise the same totals.  Consecutive barriers use alternate halves of
// the partial buffer: a block writes the half of barrier k + 2 only after barrier
// k + 1, by when every block has read the half of barrier k.  fin(tot) runs in thread
// 0 of every block before the block's last barrier (the CG scalar update, kept in
// shared memory).  Returns false when the wait expired.
template <int NV, typename T, class Fin>
__device__ bool grid_sum(const T (&v)[NV], double* partial_all, unsigned int* bar,
                         unsigned int& epoch, int* kerr, long long budget, double (*ws)[32],
                         double* tot, int* s_ok, int test_skip, Fin&& fin) {
  static_assert(NV >= 1 && NV <= 2, "two values per block and barrier at most");
  double* partial = partial_all + (size_t)(epoch & 1u) * 2 * gridDim.x;
  block_sums<NV, T>(v, ws, tot);
  if (threadIdx.x == 0 && (int)blockIdx.x == test_skip) {
    *s_ok = 0;  // test hook: leave without arriving
  } else if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partial[(size_t)blockIdx.x * NV + k] = tot[k];
    // release: the block's writes (ordered before this thread by the block barrier)
    // become visible before the arrival
    arrive_release(bar);
    const unsigned int target = (epoch + 1) * gridDim.x;
    const long long t0 = clock64();
    int ok = 1;
    for (unsigned int spin = 0; ld_relaxed(bar) < target; ++spin) {
      if ((spin & 7u) == 7u && (*(volatile int*)kerr != 0 || clock64() - t0 > budget)) {
        ok = 0;
        atomicExch(kerr, 1);
        break;
      }
      __nanosleep(20);
    }
    fence_acquire();  // the other blocks' writes are visible to this block from here
    *s_ok = ok;
  }
  ++epoch;
  __syncthreads();
  if (!*s_ok) return false;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(partial + (size_t)b * NV + k);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane == 0) tot[k] = t;
    }
    if (lane == 0) fin(tot);
  }
  __syncthreads();
  return true;
}

// The search direction of this iteration at dof d: p_old itself in the first
// iteration of the launch, else Dinv r + beta p_old (one rounding order everywhere, so
// the gathers and the owner of d compute the same value).
template <typename T>
__device__ __forceinline__ T p_at(const PcgArgs<T>& a, const T* pold, bool first, T be, int64_t d) {
  const T po = __ldcg(pold + d);
  if (first) return po;
  const T zr = __ldg(a.dinv + d) * __ldcg(a.r + d);
  return fma(be, po, zr);
}

// Algorithm 1 for cell e in two halves, so that a thread can issue the loads of its
// next cell before the atomics of the current one: cell_gather reads conn, A_T and the
// values formed by p_at; cell_finish interpolates, multiplies, projects, adds Y into q
// (atomics, Dirichlet dofs skipped) and returns the cell's energy p_T . Y_T.
template <int D, int P, int FORM, typename T>
struct CellRegs {
  using TB = dogip_tab::Tab<D, P, FORM>;
  static constexpr int V = TB::V, W = TB::W, NS = NSym<D, FORM>::value;
  uint32_t c[V];
  T ul[V];
  T A[W * NS];
};

template <int D, int P, int FORM, typename T>
__device__ __forceinline__ void cell_gather(const PcgArgs<T>& a, const T* pold, bool first, T be,
                                            int64_t e, CellRegs<D, P, FORM, T>& cr) {
  using CR = CellRegs<D, P, FORM, T>;
  constexpr int V = CR::V, W = CR::W, NS = CR::NS;
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  const T* At = a.A + tile * ((int64_t)W * NS * kTile) + lane;
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    cr.c[l] = __ldg(ct + l * kTile);
  });
  static_for<W * NS>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    cr.A[k] = __ldg(At + k * kTile);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    cr.ul[l] = (cr.c[l] & kBndBit) ? T(0) : p_at(a, pold, first, be, (int64_t)(cr.c[l] & kIdMask));
  });
}

template <int D, int P, int FORM, typename T>
__device__ __forceinline__ T cell_finish(const PcgArgs<T>& a, const CellRegs<D, P, FORM, T>& cr) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V, W = TB::W, NB = TB::NB, NS = NSym<D, FORM>::value;
  T Y[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    if constexpr (col_empty<TB>(l)) Y[l] = T(0);
  });
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    T g[NB], h[NB];
    interp<TB, j>(cr.ul, g);
    block_mul<D, FORM>(cr.A + j * NS, g, h);
    project<TB, j>(h, Y);
  });
  T en = T(0);
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    if (!(cr.c[l] & kBndBit)) {
      atomicAdd(a.q + (cr.c[l] & kIdMask), Y[l]);
      en = fma(cr.ul[l], Y[l], en);
    }
  });
  return en;
}

template <int D, int P, int FORM, typename T, int NT>
__global__ void __launch_bounds__(NT) k_pcg_small(PcgArgs<T> a) {
  // CG scalars: updated by thread 0 (double arithmetic in one thread), read by all
  struct Scal {
    double rho, rr, pq, alpha, beta;
    int iters, state;  // state: 0 iterate, 1 converged, 2 breakdown
  };
  __shared__ double ws[2][32];
  __shared__ double tot[2];
  __shared__ int s_ok;
  __shared__ Scal sc;
  const CGScal s0 = *a.scal;
  if (s0.done) return;
  const double stop = s0.tol * s0.r0;
  if (threadIdx.x == 0) sc = Scal{s0.rho, s0.rr, 0.0, 0.0, 0.0, s0.iters, 0};
  __syncthreads();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned int epoch = 0;
  bool first = true, failed = false;
  T* pold = a.p0;
  T* pnew = a.p0;
  for (int it = 0; it < a.maxit; ++it) {
    // A: q = K p with this iteration's p, the owners storing it in pnew; (p, K p)
    if (!first) pnew = (pold == a.p0) ? a.p1 : a.p0;
    const T be = (T)sc.beta;
    T en = T(0);
    if constexpr (P == 1) {
      for (int64_t e = tid; e < a.E; e += 2 * stride) {  // two cells in flight per thread
        CellRegs<D, P, FORM, T> c0, c1;
        const bool two = e + stride < a.E;
        cell_gather(a, pold, first, be, e, c0);
        if (two) cell_gather(a, pold, first, be, e + stride, c1);
        en += cell_finish(a, c0);
        if (two) en += cell_finish(a, c1);
      }
    } else {  // larger cells: one at a time (registers)
      for (int64_t e = tid; e < a.E; e += stride) {
        CellRegs<D, P, FORM, T> c0;
        cell_gather(a, pold, first, be, e, c0);
        en += cell_finish(a, c0);
      }
    }
    for (int64_t i = tid; i < a.nbnd; i += stride) {
      const int64_t d = a.bnd[i];
      const T pv = p_at(a, pold, first, be, d);
      a.q[d] = pv;
      en = fma(pv, pv, en);
    }
    if (!first)
      for (int64_t i = tid; i < a.n; i += stride) pnew[i] = p_at(a, pold, false, be, i);
    const T e1[1] = {en};
    if (!grid_sum<1, T>(e1, a.partial, a.bar, epoch, a.kerr, a.budget, ws, tot, &s_ok,
                        a.test_skip, [&](const double* t) {
                          sc.pq = t[0];
                          if (!(t[0] > 0.0) || !isfinite(t[0])) {
                            sc.state = 2;
                            sc.alpha = 0.0;
                          } else {
                            sc.alpha = sc.rho / t[0];
                          }
                        })) {
      failed = true;
      break;
    }
    if (sc.state != 0) break;
    // C: x, r update, q cleared for the next apply; rho' and ||r||^2
    const T al = (T)sc.alpha;
    T a0 = T(0), a1 = T(0);
    for (int64_t i = tid; i < a.n; i += stride) {
      const T pi = __ldcg(pnew + i);  // stored by this thread in A (or the entry p)
      a.x[i] += al * pi;
      const T ri = __ldcg(a.r + i) - al * __ldcg(a.q + i);
      a.r[i] = ri;
      a.q[i] = T(0);
      a0 += ri * (__ldg(a.dinv + i) * ri);
      a1 += ri * ri;
    }
    const T e2[2] = {a0, a1};
    if (!grid_sum<2, T>(e2, a.partial, a.bar, epoch, a.kerr, a.budget, ws, tot, &s_ok,
                        a.test_skip, [&](const double* t) {
                          sc.beta = t[0] / sc.rho;
                          sc.rho = t[0];
                          sc.rr = t[1];
                          sc.iters += 1;
                          if (sqrt(t[1]) <= stop) sc.state = 1;
                        })) {
      failed = true;
      break;
    }
    pold = pnew;
    first = false;
    if (sc.state != 0) break;
  }
  if (failed) return;  // the host reports the expired wait; the vectors are undefined
  // Iteration limit: leave p_new = Dinv r + beta p_old in p0, so that the next launch
  // starts from p as it stands.  Each thread touches only its own dofs here.
  if (sc.state == 0 && !first) {
    const T be = (T)sc.beta;
    for (int64_t i = tid; i < a.n; i += stride) a.p0[i] = p_at(a, pold, false, be, i);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int done = sc.state != 0, brk = sc.state == 2;
    CGScal& s = *a.scal;
    s.rho = sc.rho;
    s.rr = sc.rr;
    s.pq = sc.pq;
    s.alpha = sc.alpha;
    s.beta = sc.beta;
    s.iters = sc.iters;
    s.done = done;
    s.brk = brk;
    a.flags[0] = done;
    a.flags[1] = brk;
    a.flags[2] = done;
    a.flags[3] = 0;
  }
}

struct SmallLaunch {
  const void* fn = nullptr;
  int grid = 0;     // blocks: all resident at once
  int threads = 0;  // per block
  int per_sm = 0;   // resident blocks per SM
};

template <int D, int P, int FORM, typename T>
SmallLaunch small_launch() {
  constexpr int NT = pcg_threads<D, P, T>();
  // resident blocks per SM: a property of the kernel and the architecture (cached);
  // the SM count is read for the current device at every call
  static const int per_sm = [] {
    int nb = 0;
    cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pcg_small<D, P, FORM, T, NT>,
                                                             NT, 0),
               "occupancy");
    return std::max(nb, 0);
  }();
  SmallLaunch t;
  t.fn = (const void*)k_pcg_small<D, P, FORM, T, NT>;
  t.threads = NT;
  int dev = 0, sms = 1;
  cuda_check(cudaGetDevice(&dev), "device");
  cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  // every block must be resident at once (cooperative launch); the partial buffer
  // holds 4 doubles per block
  t.per_sm = per_sm;
  t.grid = std::min(per_sm * sms, kMaxRedBlocks);
  return t;
}

SmallLaunch small_dispatch(int d, int p, int form, int prec) {
  const int key = ((d * 10 + p) * 2 + form) * 2 + (prec == DOGIP_FP64 ? 1 : 0);
  switch (key) {
#define DOGIP_SM(D, P, F)                                                             \
  case ((D * 10 + P) * 2 + F) * 2 + 0: return small_launch<D, P, F, float>();         \
  case ((D * 10 + P) * 2 + F) * 2 + 1: return small_launch<D, P, F, double>();
    DOGIP_SM(2, 1, 0) DOGIP_SM(2, 1, 1) DOGIP_SM(2, 2, 0) DOGIP_SM(2, 2, 1)
    DOGIP_SM(2, 3, 0) DOGIP_SM(2, 3, 1)
    DOGIP_SM(3, 1, 0) DOGIP_SM(3, 1, 1) DOGIP_SM(3, 2, 0) DOGIP_SM(3, 2, 1)
#undef DOGIP_SM
    default:
      return SmallLaunch{};
  }
}

template <typename T>
T* second_p(SolveWork& w);
template <>
float* second_p<float>(SolveWork& w) {
  if (!w.pb32 && cudaMalloc((void**)&w.pb32, (size_t)w.n * 4) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "device allocation of solver workspace failed");
  }
  return w.pb32;
}
template <>
double* second_p<double>(SolveWork& w) {
  if (!w.pb64 && cudaMalloc((void**)&w.pb64, (size_t)w.n * 8) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "device allocation of solver workspace failed");
  }
  return w.pb64;
}

template <typename T>
void launch_small(Ctx& c, const SmallLaunch& L, const T* A, T* x, T* r, T* p, T* q, const T* dinv,
                  int maxit, cudaStream_t s) {
  SolveWork& w = c.work;
  PcgArgs<T> a;
  a.A = A;
  a.conn = c.d_conn;
  a.E = c.E;
  a.bnd = c.d_bnd;
  a.nbnd = c.dirichlet ? c.nbnd : 0;
  a.x = x;
  a.r = r;
  a.p0 = p;
  a.p1 = second_p<T>(w);
  a.q = q;
  a.dinv = dinv;
  a.n = c.n;
  a.scal = w.scal;
  a.flags = w.flags;
  a.partial = w.partial;
  a.bar = w.counter + 1;
  a.kerr = c.d_kerr;
  a.budget = c.wait_budget;
  a.maxit = maxit;
  a.test_skip = c.test_skip_chunk >= 0 ? (int)(c.test_skip_chunk % L.grid) : -1;
  cuda_check(cudaMemsetAsync(w.counter + 1, 0, sizeof(unsigned int), s), "barrier reset");
  void* args[] = {&a};
  cuda_check(cudaLaunchCooperativeKernel(L.fn, dim3(L.grid), dim3(L.threads), args, 0, s),
             "single-launch PCG");
}

}  // namespace

bool pcg_small_supported(const Ctx& c, int prec) {
  if (c.work.R != 1 && c.work.R != 0) return false;
  if (c.hi || c.factorized || c.global_w) return false;
  if (prec != DOGIP_FP32 && prec != DOGIP_FP64) return false;
  if (prec == DOGIP_FP32 && !c.keep32) return false;
  return small_dispatch(c.d, c.p, c.form, prec).fn != nullptr;
}

int64_t pcg_small_bytes(const Ctx& c, int prec) {
  const int64_t s = prec == DOGIP_FP64 ? 8 : 4;
  return c.E * ((int64_t)c.WT * c.NS * s + (int64_t)c.VT * 4) + c.n * s * 7;
}

void pcg_small_run(Ctx& c, int prec, double* x64, int maxit) {
  SolveWork& w = c.work;
  cudaStream_t s = c.stream;
  const SmallLaunch L = small_dispatch(c.d, c.p, c.form, prec);
  if (!L.fn || L.grid <= 0) fail(DOGIP_EUNSUPPORTED, "no single-launch PCG for this problem");
  // grid sized to the problem (two cells per thread at least), so that the solves of
  // small problems can run side by side; every grid up to L.grid is co-resident
  SmallLaunch Lp = L;
  const int64_t want = (c.E + 2LL * L.threads - 1) / (2LL * L.threads);
  Lp.grid = (int)std::max<int64_t>(1, std::min<int64_t>(L.grid, want));
  maxit = std::max(0, std::min(maxit, (int)((1u << 31) / (unsigned)(2 * Lp.grid))));
  if (prec == DOGIP_FP64)
    launch_small<double>(c, Lp, c.d_A64, x64, w.r64, w.p64, w.q64, c.d_dinv64, maxit, s);
  else
    launch_small<float>(c, Lp, c.d_A32, w.x32, w.r32, w.p32, w.q32, c.d_dinv32, maxit, s);
  ++c.launches;
  cuda_check(cudaMemcpyAsync(w.h_flags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s),
             "flags copy");
  cuda_check(cudaMemcpyAsync(w.h_flags + 4, c.d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s),
             "kernel flag copy");
  cuda_check(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(CGScal), cudaMemcpyDeviceToHost, s),
             "scal copy");
  cuda_check(cudaStreamSynchronize(s), "single-launch PCG");
  if (w.h_flags[4]) fail(DOGIP_ETIMEOUT, "a bounded wait inside a kernel expired");
}

}  // namespace dogip
