// Host-side launch of the apply kernel for one (D, P, FORM) instance.
#pragma once
#include <algorithm>

#include "kernels.cuh"

namespace dogip {

template <int D, int P, int FORM, typename T>
void run_apply_t(const T* A, const Ctx& c, const void* u, void* y, int R, bool atomic,
                 int64_t e0, int64_t e1, cudaStream_t s, const int* skip) {
  const int64_t nth = (e1 - e0) * (int64_t)R;
  if (nth <= 0) return;
  const int bs = c.apply_block[sizeof(T) == 8 ? DOGIP_FP64 : DOGIP_FP32];  // <= 256
  const unsigned nb = (unsigned)((nth + bs - 1) / bs);
  ApplyArgs<T> a{A, c.d_conn, (const T*)u, (T*)y, e0, e1, R, skip};
  if (R == 1) {
    if (atomic) k_apply<D, P, FORM, T, true, false><<<nb, bs, 0, s>>>(a);
    else k_apply<D, P, FORM, T, false, false><<<nb, bs, 0, s>>>(a);
  } else {
    if (atomic) k_apply<D, P, FORM, T, true, true><<<nb, bs, 0, s>>>(a);
    else k_apply<D, P, FORM, T, false, true><<<nb, bs, 0, s>>>(a);
  }
}

// Persistent bulk-async variant over the whole cell range (atomic scatter).
struct TmaLaunch {
  int blocks_per_sm = 1, num_sms = 1;
};

// Kernel attributes and residency of one instance, set once (thread-safe static);
// first called from context set-up, outside any stream capture.
template <int D, int P, int FORM, typename T, bool FACT, bool EN = false>
const TmaLaunch& tma_launch() {
  static const TmaLaunch info = [] {
    using Cfg = TmaCfg<D, P, FORM, T, FACT>;
    auto kern = k_apply_tma<D, P, FORM, T, FACT, EN>;
    TmaLaunch t;
    cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM),
               "apply smem attribute");
    int dev = 0, nb = 0;
    cuda_check(cudaGetDevice(&dev), "get device");
    cuda_check(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Cfg::THREADS, Cfg::SMEM),
               "occupancy");
    t.blocks_per_sm = nb < 1 ? 1 : nb;
    return t;
  }();
  return info;
}

template <int D, int P, int FORM, typename T, bool FACT>
void run_apply_tma(const T* A, const Ctx& c, const void* u, void* y, int R, cudaStream_t s,
                   const int* skip, bool add) {
  using Cfg = TmaCfg<D, P, FORM, T, FACT>;
  constexpr bool F32 = std::is_same<T, float>::value;
  const bool en = F32 && R == 1 && c.energy != nullptr;
  const TmaLaunch& L = en ? tma_launch<D, P, FORM, T, FACT, F32>() : tma_launch<D, P, FORM, T, FACT>();
  const int blocks_per_sm = L.blocks_per_sm, num_sms = L.num_sms;
  const int64_t ntiles = (c.E + kTile - 1) / kTile;
  const int64_t nchunks = (ntiles + Cfg::TPC - 1) / Cfg::TPC;
  if (nchunks == 0) return;
  const int64_t grid = std::min<int64_t>(nchunks, (int64_t)num_sms * blocks_per_sm);
  const bool r4 = sizeof(T) == 4 && R % 4 == 0 && ((uintptr_t)u & 15u) == 0 &&
                  ((uintptr_t)y & 15u) == 0;
  TmaArgs<T> a{A, c.d_conn, (const T*)u, (T*)y, c.E, ntiles, nchunks, R, skip, c.d_kerr,
                c.d_bnd, c.dirichlet ? c.nbnd : 0, c.wait_budget, c.test_skip_chunk, r4 ? 1 : 0,
                stream_evict_first(c, sizeof(T), FACT ? Cfg::NS : Cfg::W * Cfg::NS), add ? 1 : 0};
  const CGEnergy e = en ? *c.energy : CGEnergy{};
  if (en) {
    pdl_mark((const void*)k_apply_tma<D, P, FORM, T, FACT, F32>);
    k_apply_tma<D, P, FORM, T, FACT, F32><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, e);
  } else {
    pdl_mark((const void*)k_apply_tma<D, P, FORM, T, FACT>);
    k_apply_tma<D, P, FORM, T, FACT><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, e);
  }
}

// Self-feeding warps variant (one right-hand side, atomic scatter, whole range).
template <int D, int P, int FORM, typename T>
const TmaLaunch& sfw_launch() {
  static const TmaLaunch info = [] {
    using Cfg = SfwCfg<D, P, FORM, T>;
    auto kern = k_apply_sfw<D, P, FORM, T>;
    TmaLaunch t;
    cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM),
               "apply smem attribute");
    int dev = 0, nb = 0;
    cuda_check(cudaGetDevice(&dev), "get device");
    cuda_check(cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, Cfg::THREADS, Cfg::SMEM),
               "occupancy");
    t.blocks_per_sm = nb < 1 ? 1 : nb;
    return t;
  }();
  return info;
}

template <int D, int P, int FORM, typename T>
void run_apply_sfw(const T* A, const Ctx& c, const void* u, void* y, cudaStream_t s,
                   const int* skip, bool add) {
  using Cfg = SfwCfg<D, P, FORM, T>;
  const TmaLaunch& L = sfw_launch<D, P, FORM, T>();
  const int64_t ntiles = (c.E + kTile - 1) / kTile;
  if (ntiles == 0) return;
  const int64_t grid = std::min<int64_t>((ntiles + Cfg::NW - 1) / Cfg::NW,
                                         (int64_t)L.num_sms * L.blocks_per_sm);
  TmaArgs<T> a{A, c.d_conn, (const T*)u, (T*)y, c.E, ntiles, 0, 1, skip, c.d_kerr,
                c.d_bnd, c.dirichlet ? c.nbnd : 0, c.wait_budget, c.test_skip_chunk, 0,
                stream_evict_first(c, sizeof(T), Cfg::W * Cfg::NS), add ? 1 : 0};
  k_apply_sfw<D, P, FORM, T><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
}

// Returns 2 when a staged kernel ran (it also wrote the Dirichlet rows), 1 for the
// one-thread-per-cell kernel.
template <int D, int P, int FORM>
int run_apply(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
              int64_t e1, cudaStream_t s, const int* skip, bool add) {
  constexpr bool ok64 = TmaCfg<D, P, FORM, double>::OK, ok32 = TmaCfg<D, P, FORM, float>::OK;
  if (u == nullptr) {  // preparation call from context set-up
    if (c.factorized) {
      tma_launch<D, P, FORM, double, true>();
      tma_launch<D, P, FORM, float, true>();
      tma_launch<D, P, FORM, float, true, true>();
    } else {
      if constexpr (ok64) tma_launch<D, P, FORM, double, false>();
      if constexpr (ok32) tma_launch<D, P, FORM, float, false>();
      if constexpr (ok32) tma_launch<D, P, FORM, float, false, true>();
      if constexpr (SfwCfg<D, P, FORM, double>::OK) sfw_launch<D, P, FORM, double>();
      if constexpr (SfwCfg<D, P, FORM, float>::OK) sfw_launch<D, P, FORM, float>();
      if (c.keep32) apply_tc(c, nullptr, nullptr, nullptr, nullptr);
    }
    return 1;
  }
  if (c.factorized) {  // staged kernel over the whole range, atomic scatter only
    if (prec == DOGIP_FP64) run_apply_tma<D, P, FORM, double, true>(c.d_A64, c, u, y, R, s, skip, add);
    else run_apply_tma<D, P, FORM, float, true>(c.d_A32, c, u, y, R, s, skip, add);
    return 2;
  }
  // variant: 3 tensor cores (FP32), 2 self-feeding warps, 1 staged, 0 one thread per cell
  const int var = c.apply_variant_prec[prec] >= 0 ? c.apply_variant_prec[prec] : c.apply_variant;
  if (var == 3 && prec == DOGIP_FP32 && R == 1 && atomic && e0 == 0 && e1 == c.E &&
      apply_tc(c, u, y, s, skip, add))
    return 2;
  if (var == 2 && R == 1 && atomic && e0 == 0 && e1 == c.E) {
    if (prec == DOGIP_FP64) {
      if constexpr (SfwCfg<D, P, FORM, double>::OK) {
        run_apply_sfw<D, P, FORM, double>(c.d_A64, c, u, y, s, skip, add);
        return 2;
      }
    } else {
      if constexpr (SfwCfg<D, P, FORM, float>::OK) {
        run_apply_sfw<D, P, FORM, float>(c.d_A32, c, u, y, s, skip, add);
        return 2;
      }
    }
  }
  // several right-hand sides in FP32 reuse A_T from shared memory 4 at a time in the
  // staged kernel (the autotuner times one rhs only)
  constexpr bool small_v = dogip_tab::Tab<D, P, FORM>::V <= 10;
  const bool multi4 = small_v && prec == DOGIP_FP32 && R % 4 == 0;
  const bool whole = atomic && e0 == 0 && e1 == c.E && (var >= 1 || multi4);
  if (prec == DOGIP_FP64) {
    if constexpr (ok64) {
      if (whole) {
        run_apply_tma<D, P, FORM, double, false>(c.d_A64, c, u, y, R, s, skip, add);
        return 2;
      }
    }
    run_apply_t<D, P, FORM, double>(c.d_A64, c, u, y, R, atomic, e0, e1, s, skip);
  } else {
    if constexpr (ok32) {
      if (whole) {
        run_apply_tma<D, P, FORM, float, false>(c.d_A32, c, u, y, R, s, skip, add);
        return 2;
      }
    }
    run_apply_t<D, P, FORM, float>(c.d_A32, c, u, y, R, atomic, e0, e1, s, skip);
  }
  return 1;
}

}  // namespace dogip

#define DOGIP_APPLY_CASES(D, P)                                              \
  case P * 2 + 0:                                                            \
    return run_apply<D, P, 0>(c, u, y, R, prec, atomic, e0, e1, s, skip, add); \
  case P * 2 + 1:                                                            \
    return run_apply<D, P, 1>(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
