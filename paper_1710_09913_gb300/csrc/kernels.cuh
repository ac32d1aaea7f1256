// Device code of the DoGIP element kernels, templated on (dimension D, order P,
// form FORM).  The reference tables B (interpolation of P_P values or reference
// gradients onto the W nodes) are compile-time constants from tables_gen.h, so
// every zero entry of B costs nothing and every +-1 entry costs an add -- the
// multiplication count of eq. comp_eff.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <utility>

#include "internal.h"
#include "tables_gen.h"

namespace dogip {

template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int D, int FORM>
struct NSym {
  static constexpr int value = FORM == DOGIP_ELLIPTIC ? D * (D + 1) / 2 : 1;
};

// Packed index of the symmetric pair (r, s): (00,01,11) in 2D, (00,01,02,11,12,22) in 3D.
__host__ __device__ constexpr int sym_idx(int D, int r, int s) {
  return r <= s ? r * (2 * D - r - 1) / 2 + s : s * (2 * D - s - 1) / 2 + r;
}

// First l with B[r][j][l] != 0 (row start), and whether (j, r) is the first
// contribution to column l in the order the kernels visit (j outer, r inner).
template <class TB>
__host__ __device__ constexpr int row_first(int r, int j) {
  for (int l = 0; l < TB::V; ++l)
    if (TB::B[r][j][l] != 0.0) return l;
  return -1;
}
template <class TB>
__host__ __device__ constexpr bool col_first(int j, int r, int l) {
  for (int jj = 0; jj < TB::W; ++jj)
    for (int rr = 0; rr < TB::NB; ++rr) {
      if (TB::B[rr][jj][l] != 0.0) return jj == j && rr == r;
    }
  return false;
}
template <class TB>
__host__ __device__ constexpr bool col_empty(int l) {
  for (int jj = 0; jj < TB::W; ++jj)
    for (int rr = 0; rr < TB::NB; ++rr)
      if (TB::B[rr][jj][l] != 0.0) return false;
  return true;
}

// g_r = sum_l B[r][J][l] u_l for one W node J (interpolation, step "B u_T").
template <class TB, int J, typename T>
__device__ __forceinline__ void interp(const T (&ul)[TB::V], T (&g)[TB::NB]) {
  static_for<TB::NB>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    constexpr int L0 = row_first<TB>(r, J);
    if constexpr (L0 < 0) {
      g[r] = T(0);
    } else {
      static_for<TB::V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        constexpr double b = TB::B[r][J][l];
        if constexpr (l == L0) {
          if constexpr (b == 1.0) g[r] = ul[l];
          else if constexpr (b == -1.0) g[r] = -ul[l];
          else g[r] = T(b) * ul[l];
        } else if constexpr (l > L0 && b != 0.0) {
          if constexpr (b == 1.0) g[r] += ul[l];
          else if constexpr (b == -1.0) g[r] -= ul[l];
          else g[r] = fma(T(b), ul[l], g[r]);
        }
      });
    }
  });
}

// Y_l += sum_r B[r][J][l] h_r for one W node J (projection back, step "B^* h").
template <class TB, int J, typename T>
__device__ __forceinline__ void project(const T (&h)[TB::NB], T (&Y)[TB::V]) {
  static_for<TB::NB>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    static_for<TB::V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      constexpr double b = TB::B[r][J][l];
      if constexpr (b != 0.0) {
        if constexpr (col_first<TB>(J, r, l)) {
          if constexpr (b == 1.0) Y[l] = h[r];
          else if constexpr (b == -1.0) Y[l] = -h[r];
          else Y[l] = T(b) * h[r];
        } else {
          if constexpr (b == 1.0) Y[l] += h[r];
          else if constexpr (b == -1.0) Y[l] -= h[r];
          else Y[l] = fma(T(b), h[r], Y[l]);
        }
      }
    });
  });
}

// h = A_j g with A_j the packed symmetric block (elliptic) or the scalar (projection).
template <int D, int FORM, typename T>
__device__ __forceinline__ void block_mul(const T* a, const T* g, T* h) {
  if constexpr (FORM == DOGIP_PROJECTION) {
    h[0] = a[0] * g[0];
  } else {
    static_for<D>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      h[r] = a[sym_idx(D, r, 0)] * g[0];
      static_for<D - 1>([&](auto sc) {
        constexpr int s = decltype(sc)::value + 1;
        h[r] = fma(a[sym_idx(D, r, s)], g[s], h[r]);
      });
    });
  }
}

// Packed FP32x2 forms of interp / block_mul / project for two right-hand sides of the
// same cell (sm_100 family FFMA2): both lanes of a pair share every constant of B and
// every entry of A_T, so one packed instruction does the work of two.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
template <class TB, int J>
__device__ __forceinline__ void interp2(const float2 (&ul)[TB::V], float2 (&g)[TB::NB]) {
  static_for<TB::NB>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    constexpr int L0 = row_first<TB>(r, J);
    if constexpr (L0 < 0) {
      g[r] = f2(0.0f);
    } else {
      static_for<TB::V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        constexpr double b = TB::B[r][J][l];
        if constexpr (l == L0) {
          if constexpr (b == 1.0) g[r] = ul[l];
          else g[r] = __fmul2_rn(f2((float)b), ul[l]);
        } else if constexpr (l > L0 && b != 0.0) {
          if constexpr (b == 1.0) g[r] = __fadd2_rn(g[r], ul[l]);
          else g[r] = __ffma2_rn(f2((float)b), ul[l], g[r]);
        }
      });
    }
  });
}
template <class TB, int J>
__device__ __forceinline__ void project2(const float2 (&h)[TB::NB], float2 (&Y)[TB::V]) {
  static_for<TB::NB>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    static_for<TB::V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      constexpr double b = TB::B[r][J][l];
      if constexpr (b != 0.0) {
        if constexpr (col_first<TB>(J, r, l)) {
          if constexpr (b == 1.0) Y[l] = h[r];
          else Y[l] = __fmul2_rn(f2((float)b), h[r]);
        } else {
          if constexpr (b == 1.0) Y[l] = __fadd2_rn(Y[l], h[r]);
          else Y[l] = __ffma2_rn(f2((float)b), h[r], Y[l]);
        }
      }
    });
  });
}
template <int D, int FORM, typename S>
__device__ __forceinline__ void block_mul2(const S* a, const float2* g, float2* h) {
  if constexpr (FORM == DOGIP_PROJECTION) {
    h[0] = __fmul2_rn(f2((float)a[0]), g[0]);
  } else {
    static_for<D>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      h[r] = __fmul2_rn(f2((float)a[sym_idx(D, r, 0)]), g[0]);
      static_for<D - 1>([&](auto sc) {
        constexpr int s = decltype(sc)::value + 1;
        h[r] = __ffma2_rn(f2((float)a[sym_idx(D, r, s)]), g[s], h[r]);
      });
    });
  }
}

template <typename T>
struct ApplyArgs {
  const T* A;            // AoSoA [Epad/32][W*NS][32]
  const uint32_t* conn;  // AoSoA [Epad/32][V][32]
  const T* u;            // [n x R]
  T* y;                  // [n x R]
  int64_t e0, e1;        // processing-order element range
  int R;
  const int* skip;       // device flag: return at once when set (may be null)
};

// Algorithm 1 for one (element, rhs) per thread: gather u_T, then per W node
// interpolate (B u_T), multiply by A_T,j, project back (B^*), and finally
// scatter-add Y into y.  The W-node loop is fused, so B u_T is never stored.
// Algorithm 1 for cell e (processing order) and right-hand side r of a.
template <int D, int P, int FORM, typename T, bool ATOMIC, bool MULTI>
__device__ __forceinline__ void apply_cell(const ApplyArgs<T>& a, int64_t e, int r) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V, W = TB::W, NB = TB::NB, NS = NSym<D, FORM>::value;
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  const T* At = a.A + tile * ((int64_t)W * NS * kTile) + lane;
  const int R = MULTI ? a.R : 1;

  uint32_t c[V];
  T ul[V], Y[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    c[l] = __ldg(ct + l * kTile);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    ul[l] = (c[l] & kBndBit) ? T(0) : __ldg(a.u + (int64_t)(c[l] & kIdMask) * R + r);
    if constexpr (col_empty<TB>(l)) Y[l] = T(0);
  });
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    T g[NB], h[NB], aj[NS];
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      aj[k] = __ldg(At + (j * NS + k) * kTile);
    });
    interp<TB, j>(ul, g);
    block_mul<D, FORM>(aj, g, h);
    project<TB, j>(h, Y);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    if (!(c[l] & kBndBit)) {
      T* dst = a.y + (int64_t)(c[l] & kIdMask) * R + r;
      if constexpr (ATOMIC) atomicAdd(dst, Y[l]);
      else *dst += Y[l];
    }
  });
}

template <int D, int P, int FORM, typename T, bool ATOMIC, bool MULTI>
__global__ void __launch_bounds__(256) k_apply(ApplyArgs<T> a) {
  if (a.skip != nullptr && *a.skip) return;
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
  apply_cell<D, P, FORM, T, ATOMIC, MULTI>(a, e, r);
}

// ------------------------------------------------- bulk-async staged apply
//
// Persistent variant of Algorithm 1 for the whole cell range: the A_T and conn
// streams are contiguous per 32-cell tile in the AoSoA layout, so chunks of TPC
// tiles are moved HBM -> shared memory by cp.async.bulk (the TMA engine) into an
// S-stage ring.  A producer warp refills a stage as soon as every consumer warp has
// released it (per-stage full/empty mbarriers), so the TPC consumer warps run
// decoupled, one warp per tile (one thread per cell), looping over the right-hand
// sides and reusing A_T from shared memory.  A stage carries the A_T tiles of its
// chunk and the conn tiles of the CTA's next chunk (the first chunk's conn comes in a
// separate prologue copy), so each warp issues the u gathers of its next unit of
// work before the arithmetic of the current one.  The gathers and the atomic
// scatter go to L2; the Dirichlet rows y_b = u_b are written at the end.  Every wait
// is bounded by a clock budget; on expiry the kernel raises an error flag, drains its
// copies in flight (bounded again) and returns.

// Start of a kernel that may run as the programmatic dependent of the previous kernel
// in a CUDA graph: allow the next kernel to be launched, then wait until the previous
// grid has completed and its memory is visible (a no-op without such a dependency).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// The same copy with an L2 cache-eviction policy (createpolicy) attached: streams read
// once per apply (A_T, conn) are marked evict-first so that they do not push the
// gathered u and the scatter-added y out of L2.
__device__ __forceinline__ void bulk_copy_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                                   uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Copy with the evict-first policy when `ef` is set, plain otherwise.
__device__ __forceinline__ void stream_copy(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar, bool ef, uint64_t policy) {
  if (ef) bulk_copy_g2s_hint(dst, src, bytes, bar, policy);
  else bulk_copy_g2s(dst, src, bytes, bar);
}

// Step "add" of Algorithm 1 for one warp (32 cells, RW right-hand sides per lane):
// y[l_T] += Y_T with atomics.  Lanes 2m and 2m+1 that hold the same dof at the same
// local index -- the common edge of two cells adjacent in the processing order, such
// as the two triangles of a split square -- first add their values in registers, so
// one atomic goes to L2 instead of two.  Every lane of the warp must call this (the
// shuffles); inactive lanes pass conn entries with the Dirichlet bit and Y = 0.
// LD: lane distance of the two cells (1 with one cell per lane; 4 when four lanes
// share a cell, each with 4 of its right-hand sides).
template <int V, int RW, typename T, int LD = 1>
__device__ __forceinline__ void scatter_pairs(const uint32_t (&c)[V], T (&Y)[RW][V], int lane,
                                              T* y, int R, int r) {
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    const bool same = __shfl_xor_sync(0xffffffffu, c[l], LD) == c[l];
    static_for<RW>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      const T other = __shfl_xor_sync(0xffffffffu, Y[q][l], LD);
      if (same) Y[q][l] += other;
    });
    if (!(c[l] & kBndBit) && !(same && (lane & LD))) {
      T* dst = y + (int64_t)(c[l] & kIdMask) * R + r;
      if constexpr (RW == 4)
        atomicAdd((float4*)dst, make_float4(Y[0][l], Y[1][l], Y[2][l], Y[3][l]));
      else
        atomicAdd(dst, Y[0][l]);
    }
  });
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Wait for phase `parity` of `bar`, giving up after `budget` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

constexpr long long kWaitBudget = 4000000000LL;  // ~2 s of SM clock per wait

// FACT: factorised element factors (element-wise constant coefficients): the
// stream holds K_T (n_sym values per cell) and A_T,j = w_j K_T is formed in
// registers, w_j a compile-time constant.
template <int D, int P, int FORM, typename T, bool FACT = false>
struct TmaCfg {
  using TB = dogip_tab::Tab<D, P, FORM>;
  static constexpr int V = TB::V, W = TB::W, NS = NSym<D, FORM>::value;
  static constexpr uint32_t A_TILE = (FACT ? 1 : W) * NS * kTile * sizeof(T);
  static constexpr uint32_t C_TILE = V * kTile * 4;
  // shared memory for the ring plus the prologue (227 KB per CTA at most)
  static constexpr uint32_t kBudget = 224 * 1024;
  // consumer warps per CTA: the largest of 8, 4, 2 that leaves a double-buffered ring
  static constexpr uint32_t need(int tpc) { return tpc * (2 * (A_TILE + C_TILE) + C_TILE); }
  static constexpr int TPC = need(8) <= kBudget ? 8 : (need(4) <= kBudget ? 4 : 2);
  // a stage holds the Â tiles of chunk k and the conn tiles of the CTA's next chunk
  static constexpr uint32_t CHUNK = TPC * (A_TILE + C_TILE);
  static constexpr uint32_t PRO = TPC * C_TILE;  // conn of the CTA's first chunk
  static constexpr int S0 = (int)((kBudget - PRO) / CHUNK);
  // pipeline stages: at most 4 (more stages of small tiles raise the shared memory per
  // CTA and lower the CTAs resident per SM: measured slower at P2, no gain at P1)
  static constexpr int S = S0 > 4 ? 4 : (S0 < 2 ? 2 : S0);
  static constexpr uint32_t SMEM = S * CHUNK + PRO + (2 * S + 1) * 8 + 128;  // + bars, align
  static constexpr int THREADS = (TPC + 1) * 32;  // TPC consumer warps + 1 producer warp
  // Instances whose double-buffered 2-warp ring does not fit (3D P3 FP64) use the
  // one-thread-per-cell kernel instead.
  static constexpr bool OK = need(TPC) <= kBudget;
};

template <typename T>
struct TmaArgs {
  const T* A;
  const uint32_t* conn;
  const T* u;
  T* y;
  int64_t E, ntiles, nchunks;
  int R;
  const int* skip;
  int* err;
  const int32_t* bnd;  // Dirichlet dofs: y_b = u_b is written here (no extra kernel)
  int64_t nbnd;
  long long wait_budget;  // clock cycles per bounded mbarrier wait
  int64_t test_skip_chunk;  // test hook: this chunk's copy is never issued (-1: none)
  int r4;                   // 1: FP32, R % 4 == 0, u and y 16-byte aligned
  int evict_first;          // 1: A_T and conn copies carry the L2 evict-first policy
  int add;                  // 1: y += K u (Dirichlet rows y_b += u_b); 0: y_b = u_b
};  // 128 bytes: keep it so (a larger argument block changed the register allocation of
    // the staged kernel and slowed it by a tenth; the energy target is a parameter of
    // its own)
static_assert(sizeof(TmaArgs<float>) <= 128 && sizeof(TmaArgs<double>) <= 128,
              "staged-apply argument block above 128 bytes");

// End of an apply with the energy reduction (one right-hand side): the CTA's
// (y, u) = sum of its cells' u_T . Y_T and Dirichlet rows u_b^2 goes to
// en.partial[CTA]; the last CTA adds the partials -- one per thread, xor-shuffle
// sums per warp, warps in order: a fixed order, so the result is deterministic --
// and sets alpha: rho / delta (standard recurrence, en.mode 0) or gamma / (delta -
// beta gamma / alpha_old) (single-reduction recurrence, en.mode 1), or flags a
// breakdown.
__device__ __forceinline__ void cg_energy_finish(const CGEnergy& en, double e) {
  __shared__ double ws[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  if (lane == 0) ws[wid] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += ws[w];
    en.partial[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(en.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += __ldcg(en.partial + b);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();  // every warp has read ws above
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double delta = 0.0;
  for (int w = 0; w < nw; ++w) delta += ws[w];
  CGScal& sc = en.scal[0];
  if (!sc.done) {
    const double den = en.mode == 0 || sc.beta == 0.0 ? delta : delta - sc.beta * sc.rho / sc.alpha;
    if (!(den > 0.0) || !isfinite(den)) {
      sc.brk = 1;
      sc.done = 1;
      sc.alpha = 0.0;
    } else {
      sc.pq = delta;
      sc.alpha = sc.rho / den;
    }
  }
  en.flags[0] = sc.done | sc.upd;
  en.flags[1] = sc.brk;
  en.flags[2] = sc.done;
  en.flags[3] = sc.upd;
  *en.counter = 0u;
}


// EN: the instance with the energy reduction into en (FP32, one right-hand side) -- a
// separate instance, so that the plain apply is compiled without it.
template <int D, int P, int FORM, typename T, bool FACT, bool EN = false>
__global__ void __launch_bounds__(TmaCfg<D, P, FORM, T, FACT>::THREADS)
    k_apply_tma(TmaArgs<T> a, CGEnergy en) {
  using C = TmaCfg<D, P, FORM, T, FACT>;
  static_assert(C::OK, "stage does not fit in shared memory");
  using TB = typename C::TB;
  constexpr int V = C::V, W = C::W, NB = TB::NB, NS = C::NS;
  // prefetch the next unit's gathers where the extra V live values fit the registers
  constexpr bool PF = sizeof(T) * V <= 64;
  // 4-wide right-hand-side units (FP32, small V)
  constexpr bool Q4 = std::is_same<T, float>::value && V <= 10;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  unsigned char* pro_buf = base + C::S * C::CHUNK;           // conn of the first chunk
  uint64_t* full = (uint64_t*)(pro_buf + C::PRO);            // chunk landed (tx count)
  uint64_t* empty = full + C::S;                             // all consumer warps done with it
  uint64_t* pro = empty + C::S;                              // prologue landed
  pdl_enter();
  if (a.skip != nullptr && *a.skip) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t G = gridDim.x, k0 = blockIdx.x;
  double e_acc = 0.0;  // (y, u) of this thread's cells (energy reduction only)
  if (tid == 0) {
    for (int s = 0; s < C::S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::TPC);
    }
    mbar_init(pro, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == C::TPC) {
    // ---- producer warp: keep the ring full.  Stage s of chunk k receives the Â
    // tiles of k and the conn tiles of k + G (this CTA's next chunk), so that the
    // consumers can start the next chunk's gathers before they compute chunk k.
    if (lane == 0) {
      int failed = 0;
      int64_t issued = 0;  // chunks whose copies were issued
      const bool ef = a.evict_first != 0;
      const uint64_t pol = ef ? l2_policy_evict_first() : 0;
      const bool pro_issued = k0 < a.nchunks;
      if (pro_issued) {
        const int nt0 = (int)min((int64_t)C::TPC, a.ntiles - k0 * C::TPC);
        mbar_expect_tx(pro, (uint32_t)nt0 * C::C_TILE);
        stream_copy(pro_buf, (const unsigned char*)a.conn + k0 * C::TPC * C::C_TILE,
                    (uint32_t)nt0 * C::C_TILE, pro, ef, pol);
      }
      for (int64_t i = 0;; ++i) {
        const int64_t k = k0 + i * G;
        if (k >= a.nchunks) break;
        const int s = (int)(i % C::S);
        if (i >= C::S &&
            !mbar_wait_bounded(&empty[s], (uint32_t)(((i / C::S) - 1) & 1), a.wait_budget)) {
          failed = 1;
          break;
        }
        fence_proxy_async_smem();
        issued = i + 1;
        if (k == a.test_skip_chunk) continue;  // test hook: this chunk never lands
        const int64_t t0 = k * C::TPC, kn = k + G;
        const int nt = (int)min((int64_t)C::TPC, a.ntiles - t0);
        const int ntn = kn < a.nchunks ? (int)min((int64_t)C::TPC, a.ntiles - kn * C::TPC) : 0;
        unsigned char* sa = base + (size_t)s * C::CHUNK;
        unsigned char* sc = sa + C::TPC * C::A_TILE;
        mbar_expect_tx(&full[s], (uint32_t)nt * C::A_TILE + (uint32_t)ntn * C::C_TILE);
        stream_copy(sa, (const unsigned char*)a.A + t0 * C::A_TILE, (uint32_t)nt * C::A_TILE,
                    &full[s], ef, pol);
        if (ntn > 0)
          stream_copy(sc, (const unsigned char*)a.conn + kn * C::TPC * C::C_TILE,
                      (uint32_t)ntn * C::C_TILE, &full[s], ef, pol);
      }
      // drain: wait (bounded) until the last copies issued have landed
      if (pro_issued) mbar_wait_bounded(pro, 0u, a.wait_budget);
      for (int64_t q = issued - C::S; q < issued; ++q) {
        if (q < 0) continue;
        if (k0 + q * G == a.test_skip_chunk) continue;
        mbar_wait_bounded(&full[q % C::S], (uint32_t)((q / C::S) & 1), a.wait_budget);
      }
      if (failed) atomicOr(a.err, 1);
    }
  } else {
    // ---- consumer warps: warp w computes tile w of every chunk.  A unit of work
    // is (chunk, RW right-hand sides); the u gathers of the next unit are issued
    // before the arithmetic of the current one, so their latency hides behind it.
    // FP32 with nrhs a multiple of 4 (r4) takes RW = 4: one 16-byte gather and one
    // 16-byte atomic per dof and unit, A_T read from shared memory once per 4 rhs.
    auto consume = [&](auto rw_tag) {
      constexpr int RW = decltype(rw_tag)::value;
      constexpr bool PFW = PF && RW == 1;
      int failed = 0;
      uint32_t c[V], cn[V];
      T ul[RW][V];
      bool active = false;
      auto gather = [&](const uint32_t(&cc)[V], int r, T(&dst)[RW][V]) {
        static_for<V>([&](auto lc) {
          constexpr int l = decltype(lc)::value;
          if constexpr (RW == 4) {
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (!(cc[l] & kBndBit))
              v = __ldg((const float4*)(a.u + (int64_t)(cc[l] & kIdMask) * a.R + r));
            dst[0][l] = v.x;
            dst[1][l] = v.y;
            dst[2][l] = v.z;
            dst[3][l] = v.w;
          } else {
            dst[0][l] =
                (cc[l] & kBndBit) ? T(0) : __ldg(a.u + (int64_t)(cc[l] & kIdMask) * a.R + r);
          }
        });
      };
      if (k0 < a.nchunks) {
        failed = __any_sync(0xffffffffu, mbar_wait_bounded(pro, 0u, a.wait_budget) ? 0 : 1);
        if (!failed) {
          const int64_t tile = k0 * C::TPC + warp;
          active = tile < a.ntiles && tile * kTile + lane < a.E;
          const uint32_t* sC = (const uint32_t*)(pro_buf + warp * C::C_TILE) + lane;
          static_for<V>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            c[l] = active ? sC[l * kTile] : kBndBit;
          });
          if constexpr (PFW) gather(c, 0, ul);
        }
      }
      for (int64_t i = 0; !failed; ++i) {
        const int64_t k = k0 + i * G;
        if (k >= a.nchunks) break;
        const int s = (int)(i % C::S);
        const uint32_t parity = (uint32_t)((i / C::S) & 1);
        failed = __any_sync(0xffffffffu, mbar_wait_bounded(&full[s], parity, a.wait_budget) ? 0 : 1);
        if (failed) break;
        const T* sA = (const T*)(base + (size_t)s * C::CHUNK + warp * C::A_TILE) + lane;
        const uint32_t* sCn =
            (const uint32_t*)(base + (size_t)s * C::CHUNK + C::TPC * C::A_TILE + warp * C::C_TILE) +
            lane;
        const int64_t kn = k + G, tile_n = kn * C::TPC + warp;
        const bool active_n = kn < a.nchunks && tile_n < a.ntiles && tile_n * kTile + lane < a.E;
        T kf[NS];  // factorised K_T (FACT only)
        if constexpr (FACT) {
          static_for<NS>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            kf[kk] = active ? sA[kk * kTile] : T(0);
          });
        }
        for (int r = 0; r < a.R; r += RW) {
          // next unit: (this chunk, r + RW) or (next chunk, rhs 0)
          T un[RW][V];
          if (r + RW < a.R) {
            if constexpr (PFW) gather(c, r + RW, un);
          } else {
            static_for<V>([&](auto lc) {
              constexpr int l = decltype(lc)::value;
              cn[l] = active_n ? sCn[l * kTile] : kBndBit;
            });
            if constexpr (PFW) gather(cn, 0, un);
          }
          if constexpr (!PFW) gather(c, r, ul);  // this unit (no prefetch: register budget)
          T Y[RW][V];
          if (active) {
            static_for<RW>([&](auto qc) {
              constexpr int q = decltype(qc)::value;
              static_for<V>([&](auto lc) {
                constexpr int l = decltype(lc)::value;
                if constexpr (col_empty<TB>(l)) Y[q][l] = T(0);
              });
            });
            // packed pairs of right-hand sides (RW = 4, FP32)
            constexpr int NP = RW == 4 && std::is_same<T, float>::value ? 2 : 1;
            float2 u2[NP][V], Y2[NP][V];
            if constexpr (NP == 2) {
              static_for<V>([&](auto lc) {
                constexpr int l = decltype(lc)::value;
                u2[0][l] = make_float2(ul[0][l], ul[1][l]);
                u2[1][l] = make_float2(ul[2][l], ul[3][l]);
                if constexpr (col_empty<TB>(l)) Y2[0][l] = Y2[1][l] = f2(0.0f);
              });
            }
            static_for<W>([&](auto jc) {
              constexpr int j = decltype(jc)::value;
              T aj[NS];
              static_for<NS>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                if constexpr (FACT) {
                  constexpr double wj = TB::w[j];
                  aj[kk] = T(wj) * kf[kk];
                } else {
                  aj[kk] = sA[(j * NS + kk) * kTile];
                }
              });
              if constexpr (RW == 4 && std::is_same<T, float>::value) {
                // right-hand sides (0, 1) and (2, 3) as packed pairs
                static_for<2>([&](auto pc) {
                  constexpr int pp = decltype(pc)::value;
                  float2 g2[NB], h2[NB];
                  interp2<TB, j>(u2[pp], g2);
                  block_mul2<D, FORM>(aj, g2, h2);
                  project2<TB, j>(h2, Y2[pp]);
                });
              } else {
                static_for<RW>([&](auto qc) {
                  constexpr int q = decltype(qc)::value;
                  T g[NB], h[NB];
                  interp<TB, j>(ul[q], g);
                  block_mul<D, FORM>(aj, g, h);
                  project<TB, j>(h, Y[q]);
                });
              }
            });
            if constexpr (RW == 4 && std::is_same<T, float>::value) {
              static_for<V>([&](auto lc) {
                constexpr int l = decltype(lc)::value;
                Y[0][l] = Y2[0][l].x;
                Y[1][l] = Y2[0][l].y;
                Y[2][l] = Y2[1][l].x;
                Y[3][l] = Y2[1][l].y;
              });
            }
          } else {
            static_for<RW>([&](auto qc) {
              static_for<V>([&](auto lc) { Y[decltype(qc)::value][decltype(lc)::value] = T(0); });
            });
          }
          if constexpr (EN && RW == 1) {  // this cell's energy u_T . Y_T
            float el = 0.0f;
            static_for<V>([&](auto lc) {
              constexpr int l = decltype(lc)::value;
              el = fmaf(ul[0][l], Y[0][l], el);
            });
            e_acc += (double)el;
          }
          scatter_pairs<V, RW, T>(c, Y, lane, a.y, a.R, r);
          if constexpr (PFW) {
            static_for<V>([&](auto lc) {
              constexpr int l = decltype(lc)::value;
              ul[0][l] = un[0][l];
            });
          }
        }
        static_for<V>([&](auto lc) {
          constexpr int l = decltype(lc)::value;
          c[l] = cn[l];
        });
        active = active_n;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp no longer reads stage s
      }
      if (failed && lane == 0) atomicOr(a.err, 1);
    };
    if constexpr (Q4 && !EN) {
      if (a.r4) consume(std::integral_constant<int, 4>{});
      else consume(std::integral_constant<int, 1>{});
    } else {
      consume(std::integral_constant<int, 1>{});
    }
  }
  __syncthreads();
  // Dirichlet rows: y_b = u_b (the scatter skipped them)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + tid; t < a.nbnd * a.R;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = (int64_t)a.bnd[t / a.R] * a.R + (t % a.R);
    const T ub = a.u[idx];
    a.y[idx] = a.add ? a.y[idx] + ub : ub;
    if constexpr (EN) e_acc += (double)ub * (double)ub;
  }
  if constexpr (EN) cg_energy_finish(en, e_acc);
}

// ------------------------------------------------- self-feeding warps apply
//
// The same Algorithm 1 with the data movement done by each consumer warp for itself:
// a warp processes the tiles w, w + stride, ... and streams, in order, the items of
// each tile -- its conn tile, then its A_T in pieces of JP W nodes -- into a private
// ring of NSLOT shared-memory slots with cp.async.bulk, LA = NSLOT - 1 items ahead.
// A slot is rewritten only after the same warp has consumed it, so no producer warp
// and no cross-warp barrier is needed, and a warp holds only NSLOT small pieces
// instead of whole double-buffered tiles: 12-16 computing warps per SM instead of 8.
// One right-hand side per launch.  Every wait is bounded by the clock budget; on
// expiry the warp raises the error word, drains its copies in flight and stops.

template <int D, int P, int FORM, typename T>
struct SfwCfg {
  using TB = dogip_tab::Tab<D, P, FORM>;
  static constexpr int V = TB::V, W = TB::W, NS = NSym<D, FORM>::value;
  static constexpr uint32_t A_TILE = W * NS * kTile * sizeof(T);
  static constexpr uint32_t C_TILE = V * kTile * 4;
  static constexpr uint32_t PIECE_TARGET = 3072;  // bytes of A_T per item
  static constexpr int JP0 = (int)(PIECE_TARGET / (NS * kTile * sizeof(T)));
  static constexpr int JP = JP0 < 1 ? 1 : (JP0 > W ? W : JP0);  // W nodes per piece
  static constexpr int NPC = (W + JP - 1) / JP;                  // pieces per tile
  static constexpr uint32_t PIECE = JP * NS * kTile * sizeof(T);
  static constexpr uint32_t SLOT0 = PIECE > C_TILE ? PIECE : C_TILE;
  static constexpr uint32_t SLOT = (SLOT0 + 127) / 128 * 128;
  static constexpr int NSLOT = 4, LA = NSLOT - 1;
  static constexpr uint32_t kBudget = 224 * 1024;
  static constexpr uint32_t per_warp() { return NSLOT * (SLOT + 8); }
  static constexpr int NW = 16 * per_warp() + 128 <= kBudget ? 16
                            : (12 * per_warp() + 128 <= kBudget ? 12 : 8);
  static constexpr uint32_t SMEM = NW * NSLOT * SLOT + NW * NSLOT * 8 + 128;
  static constexpr int THREADS = NW * 32;
  static constexpr bool OK = 8 * per_warp() + 128 <= kBudget;
};

template <int D, int P, int FORM, typename T>
__global__ void __launch_bounds__(SfwCfg<D, P, FORM, T>::THREADS)
    k_apply_sfw(TmaArgs<T> a) {
  using C = SfwCfg<D, P, FORM, T>;
  using TB = typename C::TB;
  constexpr int V = C::V, W = C::W, NB = TB::NB, NS = C::NS, JP = C::JP, NPC = C::NPC;
  constexpr int NSLOT = C::NSLOT, LA = C::LA, ITEMS = NPC + 1;  // items per tile
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  if (a.skip != nullptr && *a.skip) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* ring = base + (size_t)warp * NSLOT * C::SLOT;
  uint64_t* bar = (uint64_t*)(base + (size_t)C::NW * NSLOT * C::SLOT) + warp * NSLOT;
  if (lane == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const bool ef = a.evict_first != 0;
  const uint64_t pol = ef ? l2_policy_evict_first() : 0;
  const int64_t w0 = (int64_t)blockIdx.x * C::NW + warp;
  const int64_t wstride = (int64_t)gridDim.x * C::NW;
  // item it of this warp: tile w0 + (it / ITEMS) * wstride, part it % ITEMS
  // (0: conn tile, m >= 1: A_T piece m - 1); returns false past the last tile
  auto issue = [&](int64_t it) -> bool {
    const int64_t t = w0 + (it / ITEMS) * wstride;
    if (t >= a.ntiles) return false;
    const int m = (int)(it % ITEMS);
    const int s = (int)(it % NSLOT);
    if (m == 0 && t == a.test_skip_chunk) return true;  // test hook: never lands
    const unsigned char* src;
    uint32_t bytes;
    if (m == 0) {
      src = (const unsigned char*)a.conn + t * C::C_TILE;
      bytes = C::C_TILE;
    } else {
      const int j0 = (m - 1) * JP;
      const int nj = min(JP, W - j0);
      src = (const unsigned char*)a.A + t * C::A_TILE + (size_t)j0 * NS * kTile * sizeof(T);
      bytes = (uint32_t)nj * NS * kTile * sizeof(T);
    }
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[s], bytes);
    stream_copy(ring + (size_t)s * C::SLOT, src, bytes, &bar[s], ef, pol);
    return true;
  };
  int64_t issued = 0;  // items issued (or skipped by the test hook)
  if (lane == 0)
    for (int64_t it = 0; it < LA; ++it)
      if (issue(it)) issued = it + 1;
  issued = __shfl_sync(0xffffffffu, issued, 0);
  int failed = 0;
  int64_t it = 0;  // next item to consume
  auto wait_item = [&](int64_t i) -> bool {
    const int s = (int)(i % NSLOT);
    const uint32_t parity = (uint32_t)((i / NSLOT) & 1);
    return __any_sync(0xffffffffu, mbar_wait_bounded(&bar[s], parity, a.wait_budget) ? 0 : 1) == 0;
  };
  auto advance = [&]() {  // item it consumed: reuse its slot for item it + LA
    __syncwarp();
    int64_t n = issued;
    if (lane == 0 && it + LA == issued && issue(it + LA)) n = issued + 1;
    issued = __shfl_sync(0xffffffffu, n, 0);
    ++it;
  };
  for (int64_t k = 0;; ++k) {
    const int64_t t = w0 + k * wstride;
    if (t >= a.ntiles) break;
    const int64_t e = t * kTile + lane;
    const bool active = e < a.E;
    // conn tile
    if (!wait_item(it)) { failed = 1; break; }
    uint32_t c[V];
    {
      const uint32_t* sC = (const uint32_t*)(ring + (size_t)(it % NSLOT) * C::SLOT) + lane;
      static_for<V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        c[l] = active ? sC[l * kTile] : kBndBit;
      });
    }
    advance();
    T ul[V], Y[1][V];
    static_for<V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      ul[l] = (c[l] & kBndBit) ? T(0) : __ldg(a.u + (int64_t)(c[l] & kIdMask));
      if constexpr (col_empty<TB>(l)) Y[0][l] = T(0);
    });
    static_for<NPC>([&](auto pc) {
      constexpr int pcv = decltype(pc)::value;
      if (failed) return;
      if (!wait_item(it)) {
        failed = 1;
        return;
      }
      const T* sA = (const T*)(ring + (size_t)(it % NSLOT) * C::SLOT) + lane;
      static_for<JP>([&](auto jc) {
        constexpr int jj = decltype(jc)::value;
        constexpr int j = pcv * JP + jj;
        if constexpr (j < W) {
          T g[NB], h[NB], aj[NS];
          static_for<NS>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            aj[kk] = sA[(jj * NS + kk) * kTile];
          });
          interp<TB, j>(ul, g);
          block_mul<D, FORM>(aj, g, h);
          project<TB, j>(h, Y[0]);
        }
      });
      advance();
    });
    if (failed) break;
    if (!active) static_for<V>([&](auto lc) { Y[0][decltype(lc)::value] = T(0); });
    scatter_pairs<V, 1, T>(c, Y, lane, a.y, 1, 0);
  }
  // drain (bounded): copies issued and not consumed
  for (int64_t i = it; i < issued; ++i) {
    const int s = (int)(i % NSLOT);
    if (lane == 0) mbar_wait_bounded(&bar[s], (uint32_t)((i / NSLOT) & 1), a.wait_budget);
  }
  if (failed && lane == 0) atomicOr(a.err, 1);
  __syncthreads();
  // Dirichlet rows: y_b = u_b (the scatter skipped them)
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + tid; q < a.nbnd; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = a.bnd[q];
    a.y[idx] = a.add ? a.y[idx] + a.u[idx] : a.u[idx];
  }
}

// ------------------------------------------------------------------ setup

struct AhatArgs {
  const double* coords;   // [nv x D]
  int fact;               // 1: write K_T (n_sym per cell) instead of A_T per W node
  const int32_t* cells;   // [E x (D+1)] processing order
  const int64_t* perm;    // processing position -> caller cell
  const double* coef;     // caller order
  int coef_kind;
  const uint32_t* conn;
  double* A64;
  float* A32;             // may be null
  double* geo;            // [E][D*D+1]
  double* diag;           // [n], accumulated (must be zeroed)
  int* err;
  int64_t E;
  double* qp64 = nullptr;  // [E][n_sym] processing order: the cell's coefficient (packed
  float* qp32 = nullptr;   // symmetric part; the scalar for the projection), may be null
  const uint32_t* connW = nullptr;  // global-W projection: AoSoA [Epad/32][W_T][32] W-node ids
  double* aw = nullptr;             // global-W projection: A_diag [n_W], accumulated (zeroed)
};

template <int D, typename F = double>
__device__ __forceinline__ F det_inv(const F (&R)[D][D], F (&Ri)[D][D]) {
  if constexpr (D == 2) {
    const F det = R[0][0] * R[1][1] - R[0][1] * R[1][0];
    const F id = F(1) / det;
    Ri[0][0] = R[1][1] * id;
    Ri[0][1] = -R[0][1] * id;
    Ri[1][0] = -R[1][0] * id;
    Ri[1][1] = R[0][0] * id;
    return det;
  } else {
    const F c00 = R[1][1] * R[2][2] - R[1][2] * R[2][1];
    const F c01 = R[1][2] * R[2][0] - R[1][0] * R[2][2];
    const F c02 = R[1][0] * R[2][1] - R[1][1] * R[2][0];
    const F det = R[0][0] * c00 + R[0][1] * c01 + R[0][2] * c02;
    const F id = F(1) / det;
    Ri[0][0] = c00 * id;
    Ri[1][0] = c01 * id;
    Ri[2][0] = c02 * id;
    Ri[0][1] = (R[0][2] * R[2][1] - R[0][1] * R[2][2]) * id;
    Ri[1][1] = (R[0][0] * R[2][2] - R[0][2] * R[2][0]) * id;
    Ri[2][1] = (R[0][1] * R[2][0] - R[0][0] * R[2][1]) * id;
    Ri[0][2] = (R[0][1] * R[1][2] - R[0][2] * R[1][1]) * id;
    Ri[1][2] = (R[0][2] * R[1][0] - R[0][0] * R[1][2]) * id;
    Ri[2][2] = (R[0][0] * R[1][1] - R[0][1] * R[1][0]) * id;
    return det;
  }
}

// Per-cell factor of Theorems 4 and 8: geometry (R_T^-1, |det R_T|), the validated
// coefficient and K_T = |det R_T| R_T^-1 M_T R_T^-T (packed) or m_T |det R_T|; also
// writes the cell's entry of the quadrature-point comparator's coefficient stream.
// Returns the validation flags.
template <int D, int FORM>
__device__ __forceinline__ int cell_factor(const AhatArgs& a, int64_t pos,
                                           double (&K)[NSym<D, FORM>::value],
                                           double (&Ri)[D][D], double& vol) {
  constexpr int NS = NSym<D, FORM>::value;
  double X[D + 1][D];
  static_for<D + 1>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int64_t v = a.cells[pos * (D + 1) + i];
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      X[i][k] = a.coords[v * D + k];
    });
  });
  double R[D][D];
  static_for<D>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      R[i][k] = X[k + 1][i] - X[0][i];  // column k = v_{k+1} - v_0
    });
  });
  const double det = det_inv<D>(R, Ri);
  vol = fabs(det);
  int err = 0;
  if (!(vol > 0.0) || !isfinite(det)) err |= kErrGeometry;
  const int64_t user = a.perm[pos];
  if constexpr (FORM == DOGIP_PROJECTION) {
    const double m = a.coef[user];
    if (!isfinite(m)) err |= kErrNonFinite;
    if (!(m > 0.0)) err |= kErrNotPos;
    K[0] = m * vol;
    if (a.qp64 != nullptr) {
      a.qp64[pos] = m;
      if (a.qp32) a.qp32[pos] = (float)m;
    }
  } else {
    double M[D][D];
    if (a.coef_kind == DOGIP_COEF_ELEM_SCALAR) {
      const double m = a.coef[user];
      if (!isfinite(m)) err |= kErrNonFinite;
      if (!(m > 0.0)) err |= kErrNotPos;
      static_for<D>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<D>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          M[i][k] = i == k ? m : 0.0;
        });
      });
    } else {
      const double* mp = a.coef + user * D * D;
      double mx = 0.0;
      static_for<D>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<D>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          M[i][k] = mp[i * D + k];
          if (!isfinite(M[i][k])) err |= kErrNonFinite;
          mx = fmax(mx, fabs(M[i][k]));
        });
      });
      static_for<D>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        static_for<D>([&](auto kc) {
          constexpr int k = decltype(kc)::value;
          if (fabs(M[i][k] - M[k][i]) > 1e-14 * mx) err |= kErrSymmetry;
        });
      });
      // positive definiteness by leading principal minors
      if (!(M[0][0] > 0.0)) err |= kErrNotPos;
      const double m2 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
      if (!(m2 > 0.0)) err |= kErrNotPos;
      if constexpr (D == 3) {
        const double m3 = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                          M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        if (!(m3 > 0.0)) err |= kErrNotPos;
      }
    }
    if (a.qp64 != nullptr) {  // coefficient stream of the quadrature-point comparator
      static_for<D>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        static_for<D>([&](auto sc) {
          constexpr int s = decltype(sc)::value;
          if constexpr (r <= s) {
            const double v = 0.5 * (M[r][s] + M[s][r]);
            a.qp64[pos * NS + sym_idx(D, r, s)] = v;
            if (a.qp32) a.qp32[pos * NS + sym_idx(D, r, s)] = (float)v;
          }
        });
      });
    }
    // K = vol * R^-1 M R^-T, symmetric part, packed
    static_for<D>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      static_for<D>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        if constexpr (r <= s) {
          double acc = 0.0;
          static_for<D>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            static_for<D>([&](auto qc) {
              constexpr int q = decltype(qc)::value;
              acc += Ri[r][p] * 0.5 * (M[p][q] + M[q][p]) * Ri[s][q];
            });
          });
          K[sym_idx(D, r, s)] = vol * acc;
        }
      });
    });
  }
  return err;
}

// Step a8: A_T,j = |det R_T| w_j R_T^-1 M_T R_T^-T (elliptic) or m_T |det R_T| w_j
// (projection), written in FP64 (and FP32), plus the element geometry and the
// Jacobi diagonal sum_j B_{.jl}^T A_T,j B_{.jl} scattered into diag.
template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_ahat(AhatArgs a) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V, W = TB::W, NB = TB::NB, NS = NSym<D, FORM>::value;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  double K[NS], Ri[D][D], vol;
  const int err = cell_factor<D, FORM>(a, pos, K, Ri, vol);
  if (err) atomicOr(a.err, err);
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  if (a.aw != nullptr) {
    // global double grid: A_diag,i = sum over the cells containing W node i of K_T w_j
    const uint32_t* cw = a.connW + tile * ((int64_t)W * kTile) + lane;
    static_for<W>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      constexpr double wj = TB::w[j];
      atomicAdd(a.aw + (cw[j * kTile] & kIdMask), wj * K[0]);
    });
  } else if (a.fact) {
    double* Kt = a.A64 + tile * ((int64_t)NS * kTile) + lane;
    float* Kt32 = a.A32 ? a.A32 + tile * ((int64_t)NS * kTile) + lane : nullptr;
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      Kt[k * kTile] = K[k];
      if (Kt32) Kt32[k * kTile] = (float)K[k];
    });
  } else {
    double* At = a.A64 + tile * ((int64_t)W * NS * kTile) + lane;
    float* At32 = a.A32 ? a.A32 + tile * ((int64_t)W * NS * kTile) + lane : nullptr;
    static_for<W>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      static_for<NS>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr double wj = TB::w[j];
        const double v = wj * K[k];
        At[(j * NS + k) * kTile] = v;
        if (At32) At32[(j * NS + k) * kTile] = (float)v;
      });
    });
  }
  double* g = a.geo + pos * (D * D + 1);
  static_for<D>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      g[i * D + k] = Ri[i][k];
    });
  });
  g[D * D] = vol;
  // Jacobi diagonal contributions: sum_j w_j B_{.jl}^T K B_{.jl}
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    const uint32_t cl = ct[l * kTile];
    if (!(cl & kBndBit)) {
      double acc = 0.0;
      static_for<W>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        double q = 0.0;
        static_for<NB>([&](auto rc) {
          constexpr int r = decltype(rc)::value;
          static_for<NB>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            constexpr double br = TB::B[r][j][l], bs = TB::B[s][j][l];
            if constexpr (br != 0.0 && bs != 0.0) q += br * bs * K[sym_idx(D, r, s)];
          });
        });
        constexpr double wj = TB::w[j];
        acc += wj * q;
      });
      atomicAdd(a.diag + (cl & kIdMask), acc);
    }
  });
}


// Sub-element integration of a discontinuous coefficient (the niche the paper
// names for DoGIP: quadrature is done once here, never in the apply).  For an
// isotropic field m(x) given by spherical inclusions (value `inside` in any ball,
// `outside` elsewhere) every W-node integral
//   sigma_j = int_That m(F_T(x)) phi^W_j(x) dx ~ sum_q w_q m(F_T(x_q)) phi^W_j(x_q)
// is taken with a composite collapsed Gauss rule of nq points, and
//   A_T,j = sigma_j |det R_T| R_T^-1 R_T^-T (elliptic) or sigma_j |det R_T| (projection).
struct AhatQuadArgs {
  const double* coords;
  const int32_t* cells;
  const uint32_t* conn;
  double* A64;
  float* A32;
  double* geo;
  double* diag;
  int* err;
  int64_t E;
  const double* qpts;   // [nq x D] reference points
  const double* qw;     // [nq]
  const double* phi;    // [nq x W] W-basis values at the points
  int nq;
  const double* centres;  // [nb x D]
  const double* radii;    // [nb]
  int nb;
  double inside, outside;
};

template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_ahat_quad(AhatQuadArgs a) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V, W = TB::W, NB = TB::NB, NS = NSym<D, FORM>::value;
  constexpr int kMaxCand = 16;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  double X[D + 1][D];
  static_for<D + 1>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int64_t v = a.cells[pos * (D + 1) + i];
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      X[i][k] = a.coords[v * D + k];
    });
  });
  double R[D][D], Ri[D][D];
  static_for<D>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      R[i][k] = X[k + 1][i] - X[0][i];
    });
  });
  const double det = det_inv<D>(R, Ri);
  const double vol = fabs(det);
  if (!(vol > 0.0) || !isfinite(det)) atomicOr(a.err, kErrGeometry);
  // balls that can meet the cell: distance from centre to the bounding box <= r
  double lo[D], hi[D];
  static_for<D>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    lo[k] = hi[k] = X[0][k];
    static_for<D>([&](auto ic) {
      constexpr int i = decltype(ic)::value + 1;
      lo[k] = fmin(lo[k], X[i][k]);
      hi[k] = fmax(hi[k], X[i][k]);
    });
  });
  int cand[kMaxCand];
  int nc = 0;
  bool overflow = false;
  for (int b = 0; b < a.nb; ++b) {
    double dd = 0.0;
    for (int k = 0; k < D; ++k) {
      const double c = a.centres[b * D + k];
      const double e = c < lo[k] ? lo[k] - c : (c > hi[k] ? c - hi[k] : 0.0);
      dd += e * e;
    }
    if (dd <= a.radii[b] * a.radii[b]) {
      if (nc < kMaxCand) cand[nc++] = b;
      else overflow = true;
    }
  }
  double sig[W];
  static_for<W>([&](auto jc) { sig[decltype(jc)::value] = 0.0; });
  for (int q = 0; q < a.nq; ++q) {
    double x[D];
    static_for<D>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      x[i] = X[0][i];
      static_for<D>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        x[i] = fma(R[i][k], a.qpts[q * D + k], x[i]);
      });
    });
    double m = a.outside;
    const int nt = overflow ? a.nb : nc;
    for (int t = 0; t < nt; ++t) {
      const int b = overflow ? t : cand[t];
      double dd = 0.0;
      for (int k = 0; k < D; ++k) {
        const double e = x[k] - a.centres[b * D + k];
        dd += e * e;
      }
      if (dd <= a.radii[b] * a.radii[b]) {
        m = a.inside;
        break;
      }
    }
    const double wm = a.qw[q] * m;
    static_for<W>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      sig[j] = fma(wm, a.phi[q * W + j], sig[j]);
    });
  }
  double K[NS];
  if constexpr (FORM == DOGIP_PROJECTION) {
    K[0] = vol;
  } else {
    static_for<D>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      static_for<D>([&](auto sc) {
        constexpr int s_ = decltype(sc)::value;
        if constexpr (r <= s_) {
          double acc = 0.0;
          static_for<D>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            acc += Ri[r][p] * Ri[s_][p];
          });
          K[sym_idx(D, r, s_)] = vol * acc;
        }
      });
    });
  }
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  double* At = a.A64 + tile * ((int64_t)W * NS * kTile) + lane;
  float* At32 = a.A32 ? a.A32 + tile * ((int64_t)W * NS * kTile) + lane : nullptr;
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const double v = sig[j] * K[k];
      At[(j * NS + k) * kTile] = v;
      if (At32) At32[(j * NS + k) * kTile] = (float)v;
    });
  });
  double* g = a.geo + pos * (D * D + 1);
  static_for<D>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      g[i * D + k] = Ri[i][k];
    });
  });
  g[D * D] = vol;
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    const uint32_t cl = ct[l * kTile];
    if (!(cl & kBndBit)) {
      double acc = 0.0;
      static_for<W>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        double qv = 0.0;
        static_for<NB>([&](auto rc) {
          constexpr int r = decltype(rc)::value;
          static_for<NB>([&](auto sc) {
            constexpr int s_ = decltype(sc)::value;
            constexpr double br = TB::B[r][j][l], bs = TB::B[s_][j][l];
            if constexpr (br != 0.0 && bs != 0.0) qv += br * bs * K[sym_idx(D, r, s_)];
          });
        });
        acc += sig[j] * qv;
      });
      atomicAdd(a.diag + (cl & kIdMask), acc);
    }
  });
}

struct LoadArgs {
  const double* geo;
  const int64_t* perm;
  const double* f;  // caller order or null (f = 1)
  const uint32_t* conn;
  double* b;
  int64_t E;
};

// b_l += f_T |det R_T| int_That phi_l (element-wise constant source).
template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_load(LoadArgs a) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  const double fv = (a.f ? a.f[a.perm[pos]] : 1.0) * a.geo[pos * (D * D + 1) + D * D];
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    const uint32_t cl = ct[l * kTile];
    constexpr double ivl = TB::iv[l];
    if (!(cl & kBndBit)) atomicAdd(a.b + (cl & kIdMask), fv * ivl);
  });
}

struct GradArgs {
  const double* geo;
  const int64_t* perm;
  const uint32_t* conn;
  const double* u;
  const double* lam;
  double* dA;  // caller order
  int coef_kind;
  int64_t E;
};

// dJ/dA_T = -sum_j om_j (grad lam)(x_j) (x) (grad u)(x_j) (elliptic, physical
// gradients R^-T B u_T) or -sum_j om_j lam(x_j) u(x_j) (projection).
template <int D, int P, int FORM>
__global__ void __launch_bounds__(128) k_grad(GradArgs a) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int V = TB::V, W = TB::W, NB = TB::NB;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= a.E) return;
  const int64_t tile = pos >> 5;
  const int lane = (int)(pos & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  double uT[V], lT[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    const uint32_t cl = ct[l * kTile];
    const bool bnd = cl & kBndBit;
    uT[l] = bnd ? 0.0 : a.u[cl & kIdMask];
    lT[l] = bnd ? 0.0 : a.lam[cl & kIdMask];
  });
  const double* g = a.geo + pos * (D * D + 1);
  const double vol = g[D * D];
  double G[NB][NB];
  static_for<NB>([&](auto pc) {
    static_for<NB>([&](auto qc) { G[decltype(pc)::value][decltype(qc)::value] = 0.0; });
  });
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    double gu[NB], gl[NB];
    interp<TB, j>(uT, gu);
    interp<TB, j>(lT, gl);
    double pu[NB], pl[NB];
    if constexpr (FORM == DOGIP_ELLIPTIC) {
      static_for<D>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        pu[p] = 0.0;
        pl[p] = 0.0;
        static_for<D>([&](auto sc) {
          constexpr int s = decltype(sc)::value;
          pu[p] += g[s * D + p] * gu[s];  // (R^-T g)_p = sum_s Ri[s][p] g_s
          pl[p] += g[s * D + p] * gl[s];
        });
      });
    } else {
      pu[0] = gu[0];
      pl[0] = gl[0];
    }
    constexpr double wj = TB::w[j];
    const double om = vol * wj;
    static_for<NB>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      static_for<NB>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        G[p][q] += om * pl[p] * pu[q];
      });
    });
  });
  const int64_t user = a.perm[pos];
  if (FORM == DOGIP_ELLIPTIC && a.coef_kind == DOGIP_COEF_ELEM_TENSOR) {
    static_for<NB>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      static_for<NB>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        a.dA[user * D * D + p * D + q] = -G[p][q];
      });
    });
  } else {
    double tr = 0.0;
    static_for<NB>([&](auto pc) { tr += G[decltype(pc)::value][decltype(pc)::value]; });
    a.dA[user] = -tr;
  }
}

// Factorised K_T (AoSoA [Epad/32][NS][32]) -> A_T,j = w_j K_T as [E][W][NS], caller order.
template <int D, int P, int FORM>
__global__ void k_export_fact(const double* K, const int64_t* perm, double* out, int64_t E) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  constexpr int W = TB::W, NS = NSym<D, FORM>::value;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= E) return;
  const double* Kt = K + (pos >> 5) * ((int64_t)NS * kTile) + (pos & 31);
  double* o = out + perm[pos] * (int64_t)W * NS;
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    constexpr double wj = TB::w[j];
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      o[j * NS + k] = wj * Kt[k * kTile];
    });
  });
}

// A_T (AoSoA, processing order) -> [E][W][NS] caller order; nsw = W * NS.
__global__ void k_export_ahat(const double* A, const int64_t* perm, double* out, int64_t E,
                              int nsw);

// ------------------------------------ quadrature-point matrix-free apply
//
// The conventional matrix-free operator that the paper sets DoGIP against (§1,
// §3.3), on the same GPU as a comparator: per (cell, right-hand side) one thread
// recomputes the geometry R_T, |det R_T|, R_T^-1 from the vertex coordinates at every
// apply, reads the cell's coefficient, and integrates with the collapsed
// Gauss-Jacobi rule of TabQ (exact for element-constant coefficients):
//   Y_T = sum_q B_q^T (w_q K_T) B_q u_T,   K_T = |det R_T| R_T^-1 M_T R_T^-T  (or m_T |det R_T|).
// The edge vectors are formed in FP64 from the FP64 coordinates; everything after
// that runs in T.  Atomic scatter; the Dirichlet rows are written by the caller.

template <typename T>
struct QpArgs {
  const double* coords;  // [nv x D]
  const int32_t* cells;  // [E x (D+1)] processing order
  const T* coef;         // [E][n_sym] processing order
  const uint32_t* conn;  // AoSoA [Epad/32][V][32]
  const T* u;            // [n x R]
  T* y;                  // [n x R]
  int64_t E;
  int R;
};

template <int D, int P, int FORM, typename T, bool MULTI>
__global__ void __launch_bounds__(256) k_apply_qp(QpArgs<T> a) {
  using TQ = dogip_tab::TabQ<D, P, FORM>;
  constexpr int V = TQ::V, Q = TQ::W, NB = TQ::NB, NS = NSym<D, FORM>::value;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t e;
  int r = 0;
  if constexpr (MULTI) {
    const int64_t q = t / a.R;
    e = q;
    r = (int)(t - q * a.R);
  } else {
    e = t;
  }
  if (e >= a.E) return;
  const int R = MULTI ? a.R : 1;
  // geometry of the cell
  double X0[D];
  T Rm[D][D], Ri[D][D];
  const int32_t v0 = __ldg(a.cells + e * (D + 1));
  static_for<D>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    X0[k] = __ldg(a.coords + (int64_t)v0 * D + k);
  });
  static_for<D>([&](auto ic) {
    constexpr int i = decltype(ic)::value;  // column i = v_{i+1} - v_0
    const int32_t vi = __ldg(a.cells + e * (D + 1) + i + 1);
    static_for<D>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      Rm[k][i] = (T)(__ldg(a.coords + (int64_t)vi * D + k) - X0[k]);
    });
  });
  const T vol = fabs(det_inv<D, T>(Rm, Ri));
  T K[NS];
  if constexpr (FORM == DOGIP_PROJECTION) {
    K[0] = __ldg(a.coef + e) * vol;
  } else {
    T M[NS];
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      M[k] = __ldg(a.coef + e * NS + k);
    });
    static_for<D>([&](auto rc) {
      constexpr int rr = decltype(rc)::value;
      static_for<D>([&](auto sc) {
        constexpr int ss = decltype(sc)::value;
        if constexpr (rr <= ss) {
          T acc = T(0);
          static_for<D>([&](auto pc) {
            constexpr int pp = decltype(pc)::value;
            static_for<D>([&](auto qc) {
              constexpr int qq = decltype(qc)::value;
              acc = fma(Ri[rr][pp] * M[sym_idx(D, pp, qq)], Ri[ss][qq], acc);
            });
          });
          K[sym_idx(D, rr, ss)] = vol * acc;
        }
      });
    });
  }
  // gather, quadrature loop, scatter
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  uint32_t c[V];
  T ul[V], Y[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    c[l] = __ldg(ct + l * kTile);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    ul[l] = (c[l] & kBndBit) ? T(0) : __ldg(a.u + (int64_t)(c[l] & kIdMask) * R + r);
    if constexpr (col_empty<TQ>(l)) Y[l] = T(0);
  });
  static_for<Q>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    constexpr double wq = TQ::w[q];
    T g[NB], h[NB], aq[NS];
    static_for<NS>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      aq[k] = T(wq) * K[k];
    });
    interp<TQ, q>(ul, g);
    block_mul<D, FORM>(aq, g, h);
    project<TQ, q>(h, Y);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    if (!(c[l] & kBndBit)) atomicAdd(a.y + (int64_t)(c[l] & kIdMask) * R + r, Y[l]);
  });
}

// ------------------------- global double grid for the weighted projection
//
// §2.2, Theorem "DoGIP for weighted projection": K = B^* A_diag B with the continuous
// W = C_{N,2p}, B_ij = phi_V^j(x_W^i) and A_diag,ii = int m phi_W^i.  Every W node is
// owned by the first cell containing it (bit 31 of its connW entry), so
//   k_gw_interp:  w_i = A_diag,ii (B u)_i, written once by the owner (no atomics),
//   k_gw_project: y  += sum over owned nodes j of the cell of B^_j^T w_i (atomics),
// which counts every pair (i, l) of B exactly once (phi_V^l vanishes at the W nodes of
// a cell that does not contain dof l).  Rows of B are the element-wise tables.

template <typename T>
struct GwArgs {
  const uint32_t* conn;   // AoSoA [Epad/32][V][32]
  const uint32_t* connW;  // AoSoA [Epad/32][W][32], bit 31 = owned by this cell
  const T* A;             // A_diag [n_W]
  const T* u;             // [n x R]
  T* w;                   // [n_W x R] scratch
  T* y;                   // [n x R]
  int64_t E;
  int R;
  const int* skip;        // device flag: return at once when set (may be null)
};

template <int D, int P, typename T, bool MULTI>
__global__ void __launch_bounds__(256) k_gw_interp(GwArgs<T> a) {
  using TB = dogip_tab::Tab<D, P, DOGIP_PROJECTION>;
  constexpr int V = TB::V, W = TB::W;
  if (a.skip != nullptr && *a.skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = MULTI ? t / a.R : t;
  const int r = MULTI ? (int)(t - e * a.R) : 0;
  if (e >= a.E) return;
  const int R = MULTI ? a.R : 1;
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  const uint32_t* cw = a.connW + tile * ((int64_t)W * kTile) + lane;
  T ul[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    ul[l] = __ldg(a.u + (int64_t)(__ldg(ct + l * kTile) & kIdMask) * R + r);
  });
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    const uint32_t cj = __ldg(cw + j * kTile);
    if (cj & kBndBit) {
      T g[1];
      interp<TB, j>(ul, g);
      const int64_t i = (int64_t)(cj & kIdMask);
      a.w[i * R + r] = __ldg(a.A + i) * g[0];
    }
  });
}

template <int D, int P, typename T, bool MULTI>
__global__ void __launch_bounds__(256) k_gw_project(GwArgs<T> a) {
  using TB = dogip_tab::Tab<D, P, DOGIP_PROJECTION>;
  constexpr int V = TB::V, W = TB::W;
  if (a.skip != nullptr && *a.skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = MULTI ? t / a.R : t;
  const int r = MULTI ? (int)(t - e * a.R) : 0;
  if (e >= a.E) return;
  const int R = MULTI ? a.R : 1;
  const int64_t tile = e >> 5;
  const int lane = (int)(e & 31);
  const uint32_t* ct = a.conn + tile * (V * kTile) + lane;
  const uint32_t* cw = a.connW + tile * ((int64_t)W * kTile) + lane;
  T Y[V];
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    if constexpr (col_empty<TB>(l)) Y[l] = T(0);
  });
  static_for<W>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    const uint32_t cj = __ldg(cw + j * kTile);
    T h[1];
    h[0] = (cj & kBndBit) ? __ldg(a.w + (int64_t)(cj & kIdMask) * R + r) : T(0);
    project<TB, j>(h, Y);
  });
  static_for<V>([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    atomicAdd(a.y + (int64_t)(__ldg(ct + l * kTile) & kIdMask) * R + r, Y[l]);
  });
}

}  // namespace dogip
