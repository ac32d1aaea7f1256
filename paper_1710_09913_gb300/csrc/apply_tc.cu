// Tensor-core (tcgen05) variant of the FP32 apply, Algorithm 1 with the two
// contractions against the reference table B^ on the 5th-generation tensor cores.
//
// Per tile of 128 cells (one per thread of a warpgroup):
//   GEMM 1   G[128 x NC] = U[128 x V] . B1[V x NC]        (interpolation B^ u_T,
//            NC = NB * W_T values or reference-gradient components per cell)
//   CUDA     H_j = A^_T,j G_j per W node (scalar or packed symmetric d x d block),
//            A^_T read from the warpgroup's shared-memory stage
//   GEMM 2   Y[128 x V] = H[128 x NC] . B2[NC x V]        (projection B^* h)
//   scatter  y += P_T^T Y_T with FP32 atomics.
// The operands are FP32 values split as hi + lo with hi rounded to TF32; each GEMM
// is three kind::tf32 MMAs (hi.hi + hi.lo + lo.hi) accumulating in FP32 in tensor
// memory, about 21 bits per product (the dropped lo.lo term and the TF32 truncation
// of lo are 2^-21 relative).  The A operands U and H live in tensor memory next to
// the accumulators, the split tables B1, B2 in shared memory.  Each warpgroup (four
// warps, one 128-cell tile at a time) has its own tensor-memory columns, MMA
// mbarriers and one shared-memory stage of A^_T, refilled by cp.async.bulk for its
// next tile; conn and the u gathers of the next tile are in flight meanwhile.  Every
// wait is bounded: on expiry the warpgroup leaves the loop together (the named
// barriers OR-reduce the failure), the kernel raises the error word, frees its
// tensor memory and returns.
#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace dogip {

constexpr int tc_binom(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

// Kernel arguments; B is the run-time reference table [NB][W][V] of the orders above
// the compiled tables (null otherwise).
struct TcArgs {
  const float* A;
  const uint32_t* conn;
  const float* u;
  float* y;
  int64_t E;
  const int* skip;
  int* err;
  const int32_t* bnd;
  int64_t nbnd;
  long long wait_budget;
  const float* B;
  int add;          // 1: y += K u (Dirichlet rows y_b += u_b); 0: y_b = u_b
  int evict_first;  // 1: the A_T copies carry the L2 evict-first policy
  int R;            // right-hand sides (1, or a multiple of 16 for the MR = 16 kernel)
  int64_t test_skip;  // test hook: the A^_T copy of this work unit is never issued (-1: none)
};

// MR: right-hand sides per cell in one MMA tile (1: 128 cells; 16: 8 cells x 16).
template <int D, int P, int FORM, int MR = 1>
struct TcCfg {
  // RT: B^ comes from the context's run-time table (2D p > 4, 3D p > 3)
  static constexpr bool RT = P > (D == 2 ? 4 : 3);
  static constexpr int V = tc_binom(P + D, D);
  static constexpr int W = tc_binom((FORM == DOGIP_PROJECTION ? 2 * P : 2 * P - 2) + D, D);
  static constexpr int NB = FORM == DOGIP_PROJECTION ? 1 : D;
  static constexpr int NS = NSym<D, FORM>::value;
  static constexpr int NC = NB * W;
  static constexpr int M = 128;  // cells per MMA tile (one per thread of a warpgroup)
  static constexpr int K1 = (V + 7) / 8 * 8, N1 = (NC + 15) / 16 * 16;
  static constexpr int K2 = (NC + 7) / 8 * 8, N2 = (V + 15) / 16 * 16;
  // shared memory: the split tables (per CTA) and, per warpgroup, one stage of A^_T
  // for its 128 cells (four AoSoA tiles, one bulk copy)
  static constexpr uint32_t BTAB = 2 * (N1 * K1 + N2 * K2) * 4;
  static constexpr uint32_t A_TILE = W * NS * kTile * 4;
  static constexpr uint32_t WGB = MR == 1 ? 4 * A_TILE : 2 * A_TILE;
  static constexpr uint32_t kBudget = 224 * 1024;
  // tensor-memory columns of a warpgroup: [0, N1) G = D1, whose first K2 columns then
  // hold the TF32 hi part of H (the A operand of GEMM 2); [K2, 2 K2) the lo part of H;
  // [D2O, D2O + N2) Y = D2; and U (hi, lo), the A operand of GEMM 1, at [N1, N1 + 2 K1)
  // while GEMM 1 runs (columns of the previous tile's H lo and Y, dead by then)
  static constexpr int D2O = (2 * K2 + 15) / 16 * 16;
  static constexpr int TMW0 = D2O + N2 > N1 + 2 * K1 ? D2O + N2 : N1 + 2 * K1;
  static constexpr int TMW = (TMW0 + 15) / 16 * 16;
  static constexpr int NWG0 = (int)(((long)kBudget - BTAB - 256) / WGB);
  static constexpr int NWG1 = NWG0 > 4 ? 4 : NWG0;
  static constexpr int NWG = NWG1 * TMW > 512 ? 512 / TMW : NWG1;  // warpgroups per CTA
  static constexpr uint32_t TMC = NWG * TMW <= 32 ? 32u
                                  : NWG * TMW <= 64 ? 64u
                                  : NWG * TMW <= 128 ? 128u
                                  : NWG * TMW <= 256 ? 256u
                                                     : 512u;
  // D1 columns are read 16 at a time, and a W node's NB values may not straddle two
  // reads: NB = 3 (3D elliptic) reads all N1 <= 32 columns at once
  static constexpr int CH = NB == 3 ? N1 : 16;
  // V <= 36: the cell's conn, u_T and the next tile's must stay in registers
  static constexpr bool OK = NWG >= 1 && N1 <= 256 && (NB != 3 || N1 <= 32) && V <= 36;
  static constexpr uint32_t SMEM = BTAB + (NWG < 1 ? 1 : NWG) * WGB + 256 + 1024;
  static constexpr int THREADS = (NWG < 1 ? 1 : NWG) * M;
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
  using TB = dogip_tab::Tab<D, P, FORM>;
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

template <int D, int P, int FORM, int MR>
__global__ void __launch_bounds__(TcCfg<D, P, FORM, MR>::THREADS, 1) k_apply_tc(TcArgs a) {
  using C = TcCfg<D, P, FORM, MR>;
  static_assert(C::OK, "tensor-core apply does not fit in shared / tensor memory");
  constexpr int V = C::V, W = C::W, NB = C::NB, NS = C::NS, M = C::M;
  constexpr int K1 = C::K1, N1 = C::N1, K2 = C::K2, N2 = C::N2, NWG = C::NWG, CH = C::CH;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* b1h = (float*)base;
  float* b1l = b1h + N1 * K1;
  float* b2h = b1l + N1 * K1;
  float* b2l = b2h + N2 * K2;
  uint64_t* bars = (uint64_t*)(base + C::BTAB + NWG * C::WGB);  // [NWG][4]
  uint32_t* tslot = (uint32_t*)(bars + 4 * NWG);
  if (a.skip != nullptr && *a.skip) return;
  const int tid = threadIdx.x, wg = tid / M, m = tid % M, warp = m >> 5, lane = tid & 31;
  unsigned char* stA = base + C::BTAB + wg * C::WGB;  // A^_T stage(s) of the warpgroup
  uint64_t* mma1 = bars + 4 * wg;
  uint64_t* mma2 = mma1 + 1;
  uint64_t* abar = mma1 + 2;  // [2]: stage barriers (MR = 16 double-buffers one 32-cell tile)
  if (tid == 0) {
    for (int g = 0; g < 4 * NWG; ++g) mbar_init(&bars[g], 1);
    mbar_fence_init();
  }
  if constexpr (!C::RT) {  // reference tables -> shared memory, split into TF32 hi + lo
    const TcTab<D, P, FORM>& tab = kTcTab<D, P, FORM>;
    for (int i = tid; i < N1 * K1; i += C::THREADS) tc::split_tf32(tab.b1[i], b1h[i], b1l[i]);
    for (int i = tid; i < N2 * K2; i += C::THREADS) tc::split_tf32(tab.b2[i], b2h[i], b2l[i]);
  } else {  // the same from the run-time table B[r][j][l]
    for (int i = tid; i < N1 * K1; i += C::THREADS) {
      const int row = i / K1, k = i % K1;  // B1 row c = j NB + r, column l = k
      const float b = row < NB * W && k < V ? a.B[((row % NB) * W + row / NB) * V + k] : 0.0f;
      const uint32_t o = tc::op_off(N1, row, k) / 4;
      tc::split_tf32(b, b1h[o], b1l[o]);
    }
    for (int i = tid; i < N2 * K2; i += C::THREADS) {
      const int l = i / K2, col = i % K2;  // B2 row l, column c = j NB + r
      const float b = l < V && col < NB * W ? a.B[((col % NB) * W + col / NB) * V + l] : 0.0f;
      const uint32_t o = tc::op_off(N2, l, col) / 4;
      tc::split_tf32(b, b2h[o], b2l[o]);
    }
  }
  __syncwarp();
  if (tid < 32) tc::tmem_alloc(tslot, C::TMC);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  // this warpgroup's tensor-memory columns and this warp's lanes
  const uint32_t d1 = tmem + (uint32_t)(wg * C::TMW);  // G, then the hi part of H
  const uint32_t hlo = d1 + (uint32_t)K2;              // lo part of H
  const uint32_t d2 = d1 + (uint32_t)C::D2O;           // Y
  const uint32_t uhi = d1 + (uint32_t)N1, ulo = uhi + (uint32_t)K1;  // U during GEMM 1
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t s_b1h = smem_addr(b1h), s_b1l = smem_addr(b1l);
  const uint32_t s_b2h = smem_addr(b2h), s_b2l = smem_addr(b2l);

  // Work units of warpgroup wg: u = wg + NWG * blockIdx.x + k * step.  MR = 1: a unit
  // is a 128-cell tile (AoSoA tiles 4u .. 4u+3, warp w the cells of tile 4u + w) worked
  // as one item, its A^_T in the warpgroup's single stage.  MR = 16: a unit is one
  // 32-cell AoSoA tile, worked as NI = R / 4 items of 8 cells x 16 right-hand sides
  // (item i = 4 rb + q: thread m takes cell 8 q + m / 16 and right-hand side
  // 16 rb + m % 16), so the 16 threads of a cell gather and scatter-add its dofs'
  // 64-byte rows; its A^_T sits in one of two stages while the next unit's lands.
  const int64_t ntiles32 = (a.E + kTile - 1) / kTile;
  const int64_t nunits = MR == 1 ? (a.E + M - 1) / M : ntiles32;
  const int64_t step = (int64_t)NWG * gridDim.x;
  const int NI = MR == 1 ? 1 : a.R / 4;
  int64_t a_issued = 0, a_waited = 0;  // bulk copies of A^_T (thread m == 0 issues)
  const bool ef = a.evict_first != 0;
  const uint64_t pol = ef ? l2_policy_evict_first() : 0;
  auto issue_a = [&](int64_t tt) {
    if (tt == a.test_skip) {  // test hook: this copy never lands, its bounded wait expires
      ++a_issued;
      return;
    }
    fence_proxy_async_smem();
    if constexpr (MR == 1) {
      const int nt = (int)min((int64_t)4, ntiles32 - 4 * tt);
      mbar_expect_tx(abar, (uint32_t)nt * C::A_TILE);
      stream_copy(stA, (const unsigned char*)a.A + 4 * tt * C::A_TILE, (uint32_t)nt * C::A_TILE,
                  abar, ef, pol);
    } else {
      const int sx = (int)(a_issued & 1);
      mbar_expect_tx(abar + sx, C::A_TILE);
      stream_copy(stA + sx * C::A_TILE, (const unsigned char*)a.A + tt * C::A_TILE, C::A_TILE,
                  abar + sx, ef, pol);
    }
    ++a_issued;
  };
  // the bounded wait for copy number q (its stage and phase)
  auto wait_a = [&](int64_t q) {
    if constexpr (MR == 1) return mbar_wait_bounded(abar, (uint32_t)(q & 1), a.wait_budget);
    else return mbar_wait_bounded(abar + (q & 1), (uint32_t)((q >> 1) & 1), a.wait_budget);
  };
  auto cell32_of = [&](int i) { return MR == 1 ? lane : 8 * (i & 3) + (m >> 4); };
  auto rhs_of = [&](int i) { return MR == 1 ? 0 : 16 * (i >> 2) + (m & 15); };
  auto load_conn = [&](int64_t tt, int i, uint32_t(&cc)[V], bool& act) {
    const int64_t at = MR == 1 ? 4 * tt + warp : tt;
    const int cl = cell32_of(i);
    act = tt < nunits && at * kTile + cl < a.E;
    const uint32_t* src = a.conn + at * (V * kTile) + cl;
    static_for<V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      cc[l] = act ? __ldg(src + l * kTile) : kBndBit;
    });
  };
  auto gather = [&](const uint32_t(&cc)[V], int r, float(&dst)[V]) {
    static_for<V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      dst[l] = (cc[l] & kBndBit) ? 0.0f : __ldg(a.u + (int64_t)(cc[l] & kIdMask) * a.R + r);
    });
  };
  int failed = 0;
  uint32_t phase = 0;
  uint32_t c[V], cn[V];
  float ul[V], un[V];
  bool active, active_n;
  int64_t t = (int64_t)blockIdx.x * NWG + wg;
  int it = 0;
  if (m == 0 && t < nunits) issue_a(t);
  if constexpr (MR != 1)
    if (m == 0 && t + step < nunits) issue_a(t + step);  // the second stage
  load_conn(t, 0, c, active);
  gather(c, rhs_of(0), ul);
  while (t < nunits) {  // the same trip count in the whole warpgroup
    const int64_t tn = it + 1 < NI ? t : t + step;  // next item
    const int itn = it + 1 < NI ? it + 1 : 0;
    // U -> tensor memory (hi, lo); columns V..K1-1 are zero
    static_for<K1 / 8>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      float h[8], l[8];
      static_for<8>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        constexpr int col = 8 * q + e;
        if constexpr (col < V) tc::split_tf32(ul[col], h[e], l[e]);
        else h[e] = l[e] = 0.0f;
      });
      tc::tmem_st8(uhi + lane_base + (uint32_t)(8 * q), h);
      tc::tmem_st8(ulo + lane_base + (uint32_t)(8 * q), l);
    });
    load_conn(tn, itn, cn, active_n);  // next item's conn: in flight during this item
    tc::tmem_st_wait();
    tc::fence_before_sync();
    if (tc::bar_or(1 + wg, M, failed)) {
      failed = 1;
      break;
    }
    if (m == 0) {  // GEMM 1: G = U B1 (three TF32 products per k-step), U from tensor memory
      tc::fence_after_sync();
      constexpr uint32_t idesc = tc::idesc_tf32(M, N1);
      static_for<K1 / 8>([&](auto sc) {
        constexpr int ks = decltype(sc)::value;
        const uint32_t ob = ks * tc::op_kstep(N1);
        const uint64_t bh = tc::smem_desc(s_b1h + ob, tc::op_lbo(N1), 128);
        const uint64_t bl = tc::smem_desc(s_b1l + ob, tc::op_lbo(N1), 128);
        tc::mma_tf32_ts(d1, uhi + 8u * ks, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ts(d1, uhi + 8u * ks, bl, idesc, 1u);
        tc::mma_tf32_ts(d1, ulo + 8u * ks, bh, idesc, 1u);
      });
      tc::mma_commit(mma1);
    }
    int f = __any_sync(0xffffffffu, mbar_wait_bounded(mma1, phase, a.wait_budget) ? 0 : 1);
    if (it == 0) {  // the unit's A^_T stage
      f |= __any_sync(0xffffffffu, wait_a(a_waited) ? 0 : 1);
      ++a_waited;
    }
    tc::fence_after_sync();
    // G (tensor memory) -> H_j = A^_T,j G_j -> H hi over the G columns, H lo at K2.
    // Only the K2 columns GEMM 2 reads are stored: the G columns from K2 on are the
    // zero rows of B1, never used, and may be overwritten by H lo before they are read.
    const float* sA = MR == 1 ? (const float*)(stA + warp * C::A_TILE) + lane
                              : (const float*)(stA + ((a_waited - 1) & 1) * C::A_TILE) + cell32_of(it);
    static_for<N1 / CH>([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      constexpr int j0 = b * CH / NB, j1 = (b + 1) * CH / NB < W ? (b + 1) * CH / NB : W;
      float g[CH];
      static_for<CH / 16>([&](auto hc) {
        constexpr int hb = decltype(hc)::value;
        float v[16];
        tc::tmem_ld16(d1 + lane_base + (uint32_t)(b * CH + 16 * hb), v);
        static_for<16>([&](auto ec) { g[16 * hb + decltype(ec)::value] = v[decltype(ec)::value]; });
      });
      float hh[CH];
      static_for<CH>([&](auto ec) { hh[decltype(ec)::value] = 0.0f; });
      static_for<j1 - j0>([&](auto jc) {
        constexpr int jj = decltype(jc)::value;
        constexpr int o = (j0 + jj) * NB - b * CH;  // first column of node j0 + jj in the chunk
        float aj[NS];
        static_for<NS>([&](auto kc) {
          constexpr int kk = decltype(kc)::value;
          aj[kk] = active ? sA[((j0 + jj) * NS + kk) * kTile] : 0.0f;
        });
        block_mul<D, FORM>(aj, g + o, hh + o);
      });
      static_for<CH / 8>([&](auto hc) {
        constexpr int hb = decltype(hc)::value;
        constexpr int col = b * CH + 8 * hb;
        if constexpr (col < K2) {
          float hi[8], lo[8];
          static_for<8>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            tc::split_tf32(hh[8 * hb + e], hi[e], lo[e]);
          });
          tc::tmem_st8(d1 + lane_base + (uint32_t)col, hi);
          tc::tmem_st8(hlo + lane_base + (uint32_t)col, lo);
        }
      });
    });
    tc::tmem_st_wait();
    gather(cn, rhs_of(itn), un);  // next item's u (its conn has arrived by now)
    tc::fence_before_sync();
    if (tc::bar_or(1 + wg, M, f)) {  // the warpgroup is done with the A^_T stage and H
      failed = 1;
      break;
    }
    if (m == 0) {
      // refill the stage just read: the next unit (MR = 1), or the unit after next once
      // the last item of this one has read its A^_T (MR = 16)
      if constexpr (MR == 1) {
        if (t + step < nunits) issue_a(t + step);
      } else {
        if (it + 1 == NI && t + 2 * step < nunits) issue_a(t + 2 * step);
      }
      tc::fence_after_sync();  // GEMM 2: Y = H B2, H from tensor memory
      constexpr uint32_t idesc = tc::idesc_tf32(M, N2);
      static_for<K2 / 8>([&](auto sc) {
        constexpr int ks = decltype(sc)::value;
        const uint32_t ob = ks * tc::op_kstep(N2);
        const uint64_t bh = tc::smem_desc(s_b2h + ob, tc::op_lbo(N2), 128);
        const uint64_t bl = tc::smem_desc(s_b2l + ob, tc::op_lbo(N2), 128);
        tc::mma_tf32_ts(d2, d1 + 8u * ks, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ts(d2, d1 + 8u * ks, bl, idesc, 1u);
        tc::mma_tf32_ts(d2, hlo + 8u * ks, bh, idesc, 1u);
      });
      tc::mma_commit(mma2);
    }
    f = __any_sync(0xffffffffu, mbar_wait_bounded(mma2, phase, a.wait_budget) ? 0 : 1);
    tc::fence_after_sync();
    phase ^= 1u;
    if (!f) {  // Y (tensor memory) -> y += P_T^T Y_T, shared dofs of paired cells pre-summed
      float Y[1][V];
      static_for<N2 / 16>([&](auto bc) {
        constexpr int b = decltype(bc)::value;
        float v[16];
        tc::tmem_ld16(d2 + lane_base + (uint32_t)(16 * b), v);
        static_for<16>([&](auto ec) {
          constexpr int l = 16 * b + decltype(ec)::value;
          if constexpr (l < V) Y[0][l] = v[l - 16 * b];
        });
      });
      scatter_pairs<V, 1, float, MR == 1 ? 1 : 16>(c, Y, lane, a.y, a.R, rhs_of(it));
    }
    tc::fence_before_sync();
    failed = f;
    static_for<V>([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      c[l] = cn[l];
      ul[l] = un[l];
    });
    active = active_n;
    t = tn;
    it = itn;
  }
  // a copy issued for a unit this warpgroup did not reach (after a failed wait) must
  // land before the shared memory is released
  if (m == 0)
    for (int64_t q = a_waited; q < a_issued; ++q) wait_a(q);
  if (failed && lane == 0) atomicOr(a.err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, C::TMC);
  }
  // Dirichlet rows: y_b = u_b, or y_b += u_b (the scatter skipped them)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < a.nbnd * a.R;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = (int64_t)a.bnd[i / a.R] * a.R + i % a.R;
    a.y[idx] = a.add ? a.y[idx] + a.u[idx] : a.u[idx];
  }
}

namespace {

struct TcLaunch {
  int blocks = 1;  // resident CTAs per SM (shared memory, registers, tensor memory)
  int num_sms = 1;
};

template <int D, int P, int FORM, int MR>
const TcLaunch& tc_launch() {
  static const TcLaunch info = [] {
    using Cfg = TcCfg<D, P, FORM, MR>;
    auto kern = k_apply_tc<D, P, FORM, MR>;
    TcLaunch t;
    cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM),
               "tensor-core apply smem attribute");
    int dev = 0, nb = 0;
    cuda_check(cudaGetDevice(&dev), "get device");
    cuda_check(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Cfg::THREADS, Cfg::SMEM),
               "occupancy");
    // every resident CTA holds TMC of the SM's 512 tensor-memory columns
    t.blocks = std::max(1, std::min(nb, (int)(512 / Cfg::TMC)));
    return t;
  }();
  return info;
}

template <int D, int P, int FORM, int MR>
bool run_tc_mr(const Ctx& c, const void* u, void* y, int R, cudaStream_t s, const int* skip,
               bool add) {
  if constexpr (!TcCfg<D, P, FORM, MR>::OK) {
    return false;
  } else {
    using Cfg = TcCfg<D, P, FORM, MR>;
    const TcLaunch& L = tc_launch<D, P, FORM, MR>();
    if (u == nullptr) return true;  // preparation call from context set-up
    const int64_t units = MR == 1 ? (c.E + Cfg::M - 1) / Cfg::M : (c.E + kTile - 1) / kTile;
    if (units == 0) return true;
    const int64_t grid = std::min<int64_t>((units + Cfg::NWG - 1) / Cfg::NWG,
                                           (int64_t)L.num_sms * L.blocks);
    TcArgs a{c.d_A32, c.d_conn, (const float*)u, (float*)y, c.E, skip, c.d_kerr, c.d_bnd,
             c.dirichlet ? c.nbnd : 0, c.wait_budget, Cfg::RT ? c.d_hiB32 : nullptr, add ? 1 : 0,
             stream_evict_first(c, sizeof(float), Cfg::W * Cfg::NS), R, c.test_skip_chunk};
    k_apply_tc<D, P, FORM, MR><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
    return true;
  }
}

// One right-hand side: 128-cell MMA tiles; a multiple of 16: 8 cells x 16 rhs tiles.
template <int D, int P, int FORM>
bool run_tc(const Ctx& c, const void* u, void* y, int R, cudaStream_t s, const int* skip,
            bool add) {
  if (u == nullptr) {
    const bool a1 = run_tc_mr<D, P, FORM, 1>(c, u, y, R, s, skip, add);
    const bool a16 = run_tc_mr<D, P, FORM, 16>(c, u, y, R, s, skip, add);
    return a1 || a16;
  }
  if (R == 1) return run_tc_mr<D, P, FORM, 1>(c, u, y, R, s, skip, add);
  if (R % 16 == 0) return run_tc_mr<D, P, FORM, 16>(c, u, y, R, s, skip, add);
  return false;
}

}  // namespace

bool apply_tc_available(int d, int p, int form) {
  const bool ell = form == DOGIP_ELLIPTIC;
#define DOGIP_TC_OK(D, P)                                                                  \
  if (d == D && p == P) return ell ? TcCfg<D, P, DOGIP_ELLIPTIC>::OK : TcCfg<D, P, DOGIP_PROJECTION>::OK;
  DOGIP_TC_OK(2, 1) DOGIP_TC_OK(2, 2) DOGIP_TC_OK(2, 3) DOGIP_TC_OK(2, 4)
  DOGIP_TC_OK(2, 5) DOGIP_TC_OK(2, 6) DOGIP_TC_OK(2, 7)
  DOGIP_TC_OK(3, 1) DOGIP_TC_OK(3, 2) DOGIP_TC_OK(3, 4)
#undef DOGIP_TC_OK
  return false;
}

// FP32 apply with R = 1 or a multiple of 16 right-hand sides, atomic scatter over the
// whole cell range; false when no tensor-core instance exists for (d, p, form) or R.
// u == nullptr only sets the kernel attributes (context set-up, outside any capture).
bool apply_tc(const Ctx& c, const void* u, void* y, cudaStream_t s, const int* skip, bool add,
              int R) {
  if (c.global_w || c.factorized || !c.keep32 || !apply_tc_available(c.d, c.p, c.form))
    return false;
  if (c.hi && c.d_hiB32 == nullptr) return false;
  const bool ell = c.form == DOGIP_ELLIPTIC;
#define DOGIP_TC_CASE(D, P)                                                          \
  if (c.d == D && c.p == P)                                                          \
    return ell ? run_tc<D, P, DOGIP_ELLIPTIC>(c, u, y, R, s, skip, add)              \
               : run_tc<D, P, DOGIP_PROJECTION>(c, u, y, R, s, skip, add);
  DOGIP_TC_CASE(2, 1)
  DOGIP_TC_CASE(2, 2)
  DOGIP_TC_CASE(2, 3)
  DOGIP_TC_CASE(2, 4)
  DOGIP_TC_CASE(2, 5)
  DOGIP_TC_CASE(2, 6)
  DOGIP_TC_CASE(2, 7)
  DOGIP_TC_CASE(3, 1)
  DOGIP_TC_CASE(3, 2)
  DOGIP_TC_CASE(3, 4)
#undef DOGIP_TC_CASE
  return false;
}

}  // namespace dogip
