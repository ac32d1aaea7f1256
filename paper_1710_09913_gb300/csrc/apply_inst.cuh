// Host-side launch of the apply kernel for one (D, P, FORM) instance.
#pragma once
#include "kernels.cuh"

namespace dogip {

template <int D, int P, int FORM, typename T>
void run_apply_t(const T* A, const Ctx& c, const void* u, void* y, int R, bool atomic,
                 int64_t e0, int64_t e1, cudaStream_t s, const int* skip) {
  const int64_t nth = (e1 - e0) * (int64_t)R;
  if (nth <= 0) return;
  constexpr int bs = 256;
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

template <int D, int P, int FORM>
void run_apply(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
               int64_t e1, cudaStream_t s, const int* skip) {
  if (prec == DOGIP_FP64)
    run_apply_t<D, P, FORM, double>(c.d_A64, c, u, y, R, atomic, e0, e1, s, skip);
  else
    run_apply_t<D, P, FORM, float>(c.d_A32, c, u, y, R, atomic, e0, e1, s, skip);
}

}  // namespace dogip

#define DOGIP_APPLY_CASES(D, P)                                              \
  case P * 2 + 0:                                                            \
    run_apply<D, P, 0>(c, u, y, R, prec, atomic, e0, e1, s, skip);          \
    return true;                                                             \
  case P * 2 + 1:                                                            \
    run_apply<D, P, 1>(c, u, y, R, prec, atomic, e0, e1, s, skip);          \
    return true;
