// Host-side launch of the quadrature-point matrix-free apply for one (D, P, FORM).
#pragma once

#include "kernels.cuh"

namespace dogip {

template <int D, int P, int FORM>
void run_apply_qp(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s) {
  const int64_t nth = c.E * (int64_t)R;
  if (nth <= 0) return;
  const unsigned nb = (unsigned)((nth + 255) / 256);
  if (prec == DOGIP_FP64) {
    QpArgs<double> a{c.d_coords, c.d_cells, c.d_qp64, c.d_conn, (const double*)u, (double*)y, c.E, R};
    if (R == 1) k_apply_qp<D, P, FORM, double, false><<<nb, 256, 0, s>>>(a);
    else k_apply_qp<D, P, FORM, double, true><<<nb, 256, 0, s>>>(a);
  } else {
    QpArgs<float> a{c.d_coords, c.d_cells, c.d_qp32, c.d_conn, (const float*)u, (float*)y, c.E, R};
    if (R == 1) k_apply_qp<D, P, FORM, float, false><<<nb, 256, 0, s>>>(a);
    else k_apply_qp<D, P, FORM, float, true><<<nb, 256, 0, s>>>(a);
  }
}

}  // namespace dogip

#define DOGIP_QP_CASES(D, P)                       \
  case P * 2 + 0:                                  \
    run_apply_qp<D, P, 0>(c, u, y, R, prec, s);    \
    return true;                                   \
  case P * 2 + 1:                                  \
    run_apply_qp<D, P, 1>(c, u, y, R, prec, s);    \
    return true;
