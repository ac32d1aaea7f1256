// Tensor-core (tcgen05) variant of the FP32 apply, Algorithm 1 with the two
// contractions against the reference table B^ on the 5th-generation tensor cores.
//
// Per tile of 128 cells (one per thread of the four consumer warps):
//   GEMM 1   G[128 x NC] = U[128 x V] . B1[V x NC]        (interpolation B^ u_T,
//            NC = NB * W_T values or reference-gradient components per cell)
//   CUDA     H_j = A^_T,j G_j per W node (scalar or packed symmetric d x d block),
//            A^_T read from the shared-memory ring
//   GEMM 2   Y[128 x V] = H[128 x NC] . B2[NC x V]        (projection B^* h)
//   scatter  y += P_T^T Y_T with FP32 atomics.
// The operands are FP32 values split as hi + lo with hi rounded to TF32; each GEMM
// is three kind::tf32 MMAs (hi.hi + hi.lo + lo.hi) accumulating in FP32 in tensor
// memory, about 21 bits per product (the dropped lo.lo term and the TF32 truncation
// of lo are 2^-21 relative).  The A^_T and conn streams reach shared memory through
// the same producer-warp ring of cp.async.bulk copies as the staged apply.  Every
// wait is bounded: on expiry the warpgroup leaves the loop together (the named
// barriers OR-reduce the failure), the kernel raises the error word, frees its
// tensor memory and returns.
#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace dogip {

template <int D, int P, int FORM>
struct TcCfg {
  using TB = dogip_tab::Tab<D, P, FORM>;
  static constexpr int V = TB::V, W = TB::W, NB = TB::NB, NS = NSym<D, FORM>::value;
  static constexpr int NC = NB * W;
  static constexpr int M = 128, TPC = 4;  // cells per MMA tile; consumer warps (one tile each)
  static constexpr int K1 = (V + 7) / 8 * 8, N1 = (NC + 15) / 16 * 16;
  static constexpr int K2 = (NC + 7) / 8 * 8, N2 = (V + 15) / 16 * 16;
  static constexpr uint32_t TMC = (N1 + N2) <= 32 ? 32u
                                  : (N1 + N2) <= 64 ? 64u
                                  : (N1 + N2) <= 128 ? 128u
                                  : (N1 + N2) <= 256 ? 256u
                                                     : 512u;
  // operand buffers, hi and lo halves of each
  static constexpr uint32_t A1B = M * K1 * 4, A2B = M * K2 * 4, B1B = N1 * K1 * 4, B2B = N2 * K2 * 4;
  static constexpr uint32_t OPS = 2 * (A1B + A2B + B1B + B2B);
  static constexpr uint32_t A_TILE = W * NS * kTile * 4, C_TILE = V * kTile * 4;
  static constexpr uint32_t CHUNK = TPC * (A_TILE + C_TILE), PRO = TPC * C_TILE;
  static constexpr uint32_t kBudget = 224 * 1024;
  static constexpr int S0 = (int)(((long)kBudget - OPS - PRO - 256) / CHUNK);
  static constexpr int S = S0 > 4 ? 4 : S0;
  static constexpr bool OK = S >= 2 && N1 <= 256 && N1 + N2 <= 512;
  static constexpr uint32_t SMEM = OPS + (S < 2 ? 2 : S) * CHUNK + PRO + 256 + 1024;
  static constexpr int THREADS = (TPC + 1) * 32;
};

// B1 and B2 in the operand layout of tc.cuh (FP32; split into hi + lo in the kernel):
// B1 rows c = j NB + r (N1 rows), columns l (K1); B2 rows l (N2), columns c (K2).
template <int D, int P, int FORM>
struct TcTab {
  using C = TcCfg<D, P, FORM>;
  float b1[C::N1 * C::K1];
  float b2[C::N2 * C::K2];
};
template <int D, int P, int FORM>
constexpr TcTab<D, P, FORM> make_tc_tab() {
  using C = TcCfg<D, P, FORM>;
  using TB = typename C::TB;
  TcTab<D, P, FORM> t{};
  for (int r = 0; r < C::NB; ++r)
    for (int j = 0; j < C::W; ++j)
      for (int l = 0; l < C::V; ++l) {
        const int c = j * C::NB + r;
        const float b = (float)TB::B[r][j][l];
        t.b1[tc::op_off(C::N1, c, l) / 4] = b;
        t.b2[tc::op_off(C::N2, l, c) / 4] = b;
      }
  return t;
}
template <int D, int P, int FORM>
__device__ const TcTab<D, P, FORM> kTcTab = make_tc_tab<D, P, FORM>();

template <int D, int P, int FORM>
__global__ void __launch_bounds__(TcCfg<D, P, FORM>::THREADS, 1) k_apply_tc(TmaArgs<float> a) {
  using C = TcCfg<D, P, FORM>;
  static_assert(C::OK, "tensor-core apply does not fit in shared / tensor memory");
  constexpr int V = C::V, W = C::W, NB = C::NB, NS = C::NS, NC = C::NC, M = C::M;
  constexpr int K1 = C::K1, N1 = C::N1, K2 = C::K2, N2 = C::N2, S = C::S, TPC = C::TPC;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* a1h = (float*)base;
  float* a1l = a1h + M * K1;
  float* a2h = a1l + M * K1;
  float* a2l = a2h + M * K2;
  float* b1h = a2l + M * K2;
  float* b1l = b1h + N1 * K1;
  float* b2h = b1l + N1 * K1;
  float* b2l = b2h + N2 * K2;
  unsigned char* ring = base + C::OPS;
  unsigned char* pro_buf = ring + S * C::CHUNK;  // conn of the first chunk
  uint64_t* full = (uint64_t*)(pro_buf + C::PRO);
  uint64_t* empty = full + S;
  uint64_t* pro = empty + S;
  uint64_t* mma1 = pro + 1;
  uint64_t* mma2 = mma1 + 1;
  uint32_t* tslot = (uint32_t*)(mma2 + 1);
  if (a.skip != nullptr && *a.skip) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t G = gridDim.x, k0 = blockIdx.x;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TPC);
    }
    mbar_init(pro, 1);
    mbar_init(mma1, 1);
    mbar_init(mma2, 1);
    mbar_fence_init();
  }
  {  // reference tables -> shared memory, split into TF32 hi + lo
    const TcTab<D, P, FORM>& tab = kTcTab<D, P, FORM>;
    for (int i = tid; i < N1 * K1; i += C::THREADS) tc::split_tf32(tab.b1[i], b1h[i], b1l[i]);
    for (int i = tid; i < N2 * K2; i += C::THREADS) tc::split_tf32(tab.b2[i], b2h[i], b2l[i]);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_alloc(tslot, C::TMC);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == TPC) {
    // ---- producer warp: stage s of chunk k receives the A^ tiles of k and the conn
    // tiles of k + G (this CTA's next chunk).
    if (lane == 0) {
      int failed = 0;
      int64_t issued = 0;
      const bool pro_issued = k0 < a.nchunks;
      if (pro_issued) {
        const int nt0 = (int)min((int64_t)TPC, a.ntiles - k0 * TPC);
        mbar_expect_tx(pro, (uint32_t)nt0 * C::C_TILE);
        bulk_copy_g2s(pro_buf, (const unsigned char*)a.conn + k0 * TPC * C::C_TILE,
                      (uint32_t)nt0 * C::C_TILE, pro);
      }
      for (int64_t i = 0;; ++i) {
        const int64_t k = k0 + i * G;
        if (k >= a.nchunks) break;
        const int s = (int)(i % S);
        if (i >= S && !mbar_wait_bounded(&empty[s], (uint32_t)(((i / S) - 1) & 1), a.wait_budget)) {
          failed = 1;
          break;
        }
        fence_proxy_async_smem();
        issued = i + 1;
        const int64_t t0 = k * TPC, kn = k + G;
        const int nt = (int)min((int64_t)TPC, a.ntiles - t0);
        const int ntn = kn < a.nchunks ? (int)min((int64_t)TPC, a.ntiles - kn * TPC) : 0;
        unsigned char* sa = ring + (size_t)s * C::CHUNK;
        unsigned char* sc = sa + TPC * C::A_TILE;
        mbar_expect_tx(&full[s], (uint32_t)nt * C::A_TILE + (uint32_t)ntn * C::C_TILE);
        bulk_copy_g2s(sa, (const unsigned char*)a.A + t0 * C::A_TILE, (uint32_t)nt * C::A_TILE,
                      &full[s]);
        if (ntn > 0)
          bulk_copy_g2s(sc, (const unsigned char*)a.conn + kn * TPC * C::C_TILE,
                        (uint32_t)ntn * C::C_TILE, &full[s]);
      }
      // drain: wait (bounded) until the last copies issued have landed
      if (pro_issued) mbar_wait_bounded(pro, 0u, a.wait_budget);
      for (int64_t q = issued - S; q < issued; ++q) {
        if (q < 0) continue;
        mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), a.wait_budget);
      }
      if (failed) atomicOr(a.err, 1);
    }
  } else {
    // ---- consumer warpgroup: thread m = 32 warp + lane owns cell m of the tile,
    // i.e. row m of U, G, H, Y and lane m of tensor memory.
    const int m = tid;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t d1 = tmem, d2 = tmem + (uint32_t)N1;
    int failed = 0;
    uint32_t c[V], cn[V];
    float ul[V], un[V];
    bool active = false;
    auto gather = [&](const uint32_t(&cc)[V], float(&dst)[V]) {
      static_for<V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        dst[l] = (cc[l] & kBndBit) ? 0.0f : __ldg(a.u + (cc[l] & kIdMask));
      });
    };
    if (k0 < a.nchunks) {
      failed = mbar_wait_bounded(pro, 0u, a.wait_budget) ? 0 : 1;
      const int64_t tile = k0 * TPC + warp;
      active = !failed && tile < a.ntiles && tile * kTile + lane < a.E;
      const uint32_t* sC = (const uint32_t*)(pro_buf + warp * C::C_TILE) + lane;
      static_for<V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        c[l] = active ? sC[l * kTile] : kBndBit;
      });
      gather(c, ul);
    }
    uint32_t phase = 0;
    const uint32_t s_a1h = smem_addr(a1h), s_a1l = smem_addr(a1l);
    const uint32_t s_a2h = smem_addr(a2h), s_a2l = smem_addr(a2l);
    const uint32_t s_b1h = smem_addr(b1h), s_b1l = smem_addr(b1l);
    const uint32_t s_b2h = smem_addr(b2h), s_b2l = smem_addr(b2l);
    for (int64_t i = 0;; ++i) {
      const int64_t k = k0 + i * G;
      if (k >= a.nchunks) break;  // the same trip count in every consumer warp
      const int s = (int)(i % S);
      const uint32_t parity = (uint32_t)((i / S) & 1);
      int f = failed ? 1 : (mbar_wait_bounded(&full[s], parity, a.wait_budget) ? 0 : 1);
      // U -> A1 (hi, lo); columns V..K1-1 are zero
      static_for<K1 / 4>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        float h[4], l[4];
        static_for<4>([&](auto ec) {
          constexpr int e = decltype(ec)::value;
          constexpr int col = 4 * q + e;
          if constexpr (col < V) tc::split_tf32(ul[col], h[e], l[e]);
          else h[e] = l[e] = 0.0f;
        });
        const uint32_t off = tc::op_off(M, m, 4 * q) / 4;
        *(float4*)(a1h + off) = make_float4(h[0], h[1], h[2], h[3]);
        *(float4*)(a1l + off) = make_float4(l[0], l[1], l[2], l[3]);
      });
      // conn of the CTA's next chunk, and its gathers (in flight during this tile)
      const unsigned char* st = ring + (size_t)s * C::CHUNK;
      const float* sA = (const float*)(st + warp * C::A_TILE) + lane;
      const uint32_t* sCn = (const uint32_t*)(st + TPC * C::A_TILE + warp * C::C_TILE) + lane;
      const int64_t kn = k + G, tile_n = kn * TPC + warp;
      const bool active_n =
          !f && kn < a.nchunks && tile_n < a.ntiles && tile_n * kTile + lane < a.E;
      static_for<V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        cn[l] = active_n ? sCn[l * kTile] : kBndBit;
      });
      gather(cn, un);
      fence_proxy_async_smem();
      tc::fence_before_sync();
      if (tc::bar_or(1, M, f)) {
        failed = 1;
        break;
      }
      if (tid == 0) {  // GEMM 1: G = U B1 (three TF32 products per k-step)
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_tf32(M, N1);
        static_for<K1 / 8>([&](auto sc) {
          constexpr int ks = decltype(sc)::value;
          const uint32_t oa = ks * tc::op_kstep(M), ob = ks * tc::op_kstep(N1);
          const uint64_t ah = tc::smem_desc(s_a1h + oa, tc::op_lbo(M), 128);
          const uint64_t al = tc::smem_desc(s_a1l + oa, tc::op_lbo(M), 128);
          const uint64_t bh = tc::smem_desc(s_b1h + ob, tc::op_lbo(N1), 128);
          const uint64_t bl = tc::smem_desc(s_b1l + ob, tc::op_lbo(N1), 128);
          tc::mma_tf32(d1, ah, bh, idesc, ks > 0 ? 1u : 0u);
          tc::mma_tf32(d1, ah, bl, idesc, 1u);
          tc::mma_tf32(d1, al, bh, idesc, 1u);
        });
        tc::mma_commit(mma1);
      }
      f = __any_sync(0xffffffffu, mbar_wait_bounded(mma1, phase, a.wait_budget) ? 0 : 1);
      tc::fence_after_sync();
      // G (tensor memory) -> H_j = A^_T,j G_j -> A2 (hi, lo); columns NC..K2-1 zero
      {
        float g[N1];
        static_for<N1 / 16>([&](auto bc) {
          constexpr int b = decltype(bc)::value;
          float v[16];
          tc::tmem_ld16(d1 + lane_base + (uint32_t)(16 * b), v);
          static_for<16>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            g[16 * b + e] = v[e];
          });
        });
        float hh[K2];
        static_for<W>([&](auto jc) {
          constexpr int j = decltype(jc)::value;
          float aj[NS];
          static_for<NS>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            aj[kk] = active ? sA[(j * NS + kk) * kTile] : 0.0f;
          });
          block_mul<D, FORM>(aj, g + j * NB, hh + j * NB);
        });
        static_for<K2 - NC>([&](auto ec) { hh[NC + decltype(ec)::value] = 0.0f; });
        static_for<K2 / 4>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          float h[4], l[4];
          static_for<4>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            tc::split_tf32(hh[4 * q + e], h[e], l[e]);
          });
          const uint32_t off = tc::op_off(M, m, 4 * q) / 4;
          *(float4*)(a2h + off) = make_float4(h[0], h[1], h[2], h[3]);
          *(float4*)(a2l + off) = make_float4(l[0], l[1], l[2], l[3]);
        });
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);  // this warp no longer reads stage s
      fence_proxy_async_smem();
      tc::fence_before_sync();
      if (tc::bar_or(1, M, f)) {
        failed = 1;
        break;
      }
      if (tid == 0) {  // GEMM 2: Y = H B2
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_tf32(M, N2);
        static_for<K2 / 8>([&](auto sc) {
          constexpr int ks = decltype(sc)::value;
          const uint32_t oa = ks * tc::op_kstep(M), ob = ks * tc::op_kstep(N2);
          const uint64_t ah = tc::smem_desc(s_a2h + oa, tc::op_lbo(M), 128);
          const uint64_t al = tc::smem_desc(s_a2l + oa, tc::op_lbo(M), 128);
          const uint64_t bh = tc::smem_desc(s_b2h + ob, tc::op_lbo(N2), 128);
          const uint64_t bl = tc::smem_desc(s_b2l + ob, tc::op_lbo(N2), 128);
          tc::mma_tf32(d2, ah, bh, idesc, ks > 0 ? 1u : 0u);
          tc::mma_tf32(d2, ah, bl, idesc, 1u);
          tc::mma_tf32(d2, al, bh, idesc, 1u);
        });
        tc::mma_commit(mma2);
      }
      f = __any_sync(0xffffffffu, mbar_wait_bounded(mma2, phase, a.wait_budget) ? 0 : 1);
      tc::fence_after_sync();
      phase ^= 1u;
      if (!f) {  // Y (tensor memory) -> y += P_T^T Y_T
        static_for<N2 / 16>([&](auto bc) {
          constexpr int b = decltype(bc)::value;
          float v[16];
          tc::tmem_ld16(d2 + lane_base + (uint32_t)(16 * b), v);
          static_for<16>([&](auto ec) {
            constexpr int l = 16 * b + decltype(ec)::value;
            if constexpr (l < V) {
              if (!(c[l] & kBndBit)) atomicAdd(a.y + (c[l] & kIdMask), v[l - 16 * b]);
            }
          });
        });
      }
      tc::fence_before_sync();
      failed = f;
      static_for<V>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        c[l] = cn[l];
        ul[l] = un[l];
      });
      active = active_n;
    }
    if (failed && lane == 0) atomicOr(a.err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, C::TMC);
  }
  // Dirichlet rows: y_b = u_b (the scatter skipped them)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + tid; t < a.nbnd;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = a.bnd[t];
    a.y[idx] = a.u[idx];
  }
}

namespace {

struct TcLaunch {
  int num_sms = 1;
};

template <int D, int P, int FORM>
const TcLaunch& tc_launch() {
  static const TcLaunch info = [] {
    using Cfg = TcCfg<D, P, FORM>;
    TcLaunch t;
    cuda_check(cudaFuncSetAttribute(k_apply_tc<D, P, FORM>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM),
               "tensor-core apply smem attribute");
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "get device");
    cuda_check(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    return t;
  }();
  return info;
}

template <int D, int P, int FORM>
bool run_tc(const Ctx& c, const void* u, void* y, cudaStream_t s, const int* skip) {
  if constexpr (!TcCfg<D, P, FORM>::OK) {
    return false;
  } else {
    using Cfg = TcCfg<D, P, FORM>;
    const TcLaunch& L = tc_launch<D, P, FORM>();  // one CTA per SM (shared memory)
    if (u == nullptr) return true;               // preparation call from context set-up
    const int64_t ntiles = (c.E + kTile - 1) / kTile;
    const int64_t nchunks = (ntiles + Cfg::TPC - 1) / Cfg::TPC;
    if (nchunks == 0) return true;
    const int64_t grid = std::min<int64_t>(nchunks, (int64_t)L.num_sms);
    TmaArgs<float> a{c.d_A32, c.d_conn, (const float*)u, (float*)y, c.E, ntiles, nchunks, 1,
                     skip, c.d_kerr, c.d_bnd, c.dirichlet ? c.nbnd : 0, c.wait_budget, -1, 0};
    k_apply_tc<D, P, FORM><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
    return true;
  }
}

}  // namespace

bool apply_tc_available(int d, int p, int form) {
  auto ok = [&](auto dc, auto pc) {
    constexpr int D = decltype(dc)::value, P = decltype(pc)::value;
    return form == DOGIP_ELLIPTIC ? TcCfg<D, P, DOGIP_ELLIPTIC>::OK
                                  : TcCfg<D, P, DOGIP_PROJECTION>::OK;
  };
  if (d == 2) {
    switch (p) {
      case 1: return ok(std::integral_constant<int, 2>{}, std::integral_constant<int, 1>{});
      case 2: return ok(std::integral_constant<int, 2>{}, std::integral_constant<int, 2>{});
      case 3: return ok(std::integral_constant<int, 2>{}, std::integral_constant<int, 3>{});
      case 4: return ok(std::integral_constant<int, 2>{}, std::integral_constant<int, 4>{});
    }
  } else if (d == 3) {
    switch (p) {
      case 1: return ok(std::integral_constant<int, 3>{}, std::integral_constant<int, 1>{});
      case 2: return ok(std::integral_constant<int, 3>{}, std::integral_constant<int, 2>{});
    }
  }
  return false;
}

// FP32 apply with one right-hand side, atomic scatter over the whole cell range;
// false when no tensor-core instance exists for (d, p, form).  u == nullptr only sets
// the kernel attributes (context set-up, outside any stream capture).
bool apply_tc(const Ctx& c, const void* u, void* y, cudaStream_t s, const int* skip) {
  if (c.hi || c.global_w || c.factorized || !apply_tc_available(c.d, c.p, c.form)) return false;
  const bool ell = c.form == DOGIP_ELLIPTIC;
#define DOGIP_TC_CASE(D, P)                                                          \
  if (c.d == D && c.p == P)                                                          \
    return ell ? run_tc<D, P, DOGIP_ELLIPTIC>(c, u, y, s, skip)                      \
               : run_tc<D, P, DOGIP_PROJECTION>(c, u, y, s, skip);
  DOGIP_TC_CASE(2, 1)
  DOGIP_TC_CASE(2, 2)
  DOGIP_TC_CASE(2, 3)
  DOGIP_TC_CASE(2, 4)
  DOGIP_TC_CASE(3, 1)
  DOGIP_TC_CASE(3, 2)
#undef DOGIP_TC_CASE
  return false;
}

}  // namespace dogip
