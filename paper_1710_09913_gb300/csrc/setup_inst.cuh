// Per-(D, P, FORM) launchers of the setup-side kernels, instantiated once per
// dimension (setup_d2.cu, setup_d3.cu) so that the instances compile in parallel.
#pragma once

#include "kernels.cuh"

namespace dogip {

struct SetupCall {
  int op;  // kSetupAhat, kSetupAhatQuad, kSetupLoad, kSetupGrad, kSetupExportFact
  const double* coef = nullptr;
  int coef_kind = 0;
  const QuadCoef* qc = nullptr;
  const double* f = nullptr;
  double* b = nullptr;
  const double* u = nullptr;
  const double* lam = nullptr;
  double* dA = nullptr;
  double* out = nullptr;
};
constexpr int kSetupAhat = 0, kSetupAhatQuad = 1, kSetupLoad = 2, kSetupGrad = 3,
              kSetupExportFact = 4;

template <int D, int P, int FORM>
void setup_run(Ctx& c, const SetupCall& k, cudaStream_t s) {
  const unsigned nb = (unsigned)((c.E + 127) / 128);
  switch (k.op) {
    case kSetupAhat: {
      AhatArgs a{c.d_coords, c.factorized ? 1 : 0, c.d_cells, c.d_perm, k.coef, k.coef_kind,
                 c.d_conn, c.d_A64, c.keep32 ? c.d_A32 : nullptr, c.d_geo, c.d_diag, c.d_err, c.E};
      a.qp64 = c.d_qp64;
      a.qp32 = c.keep32 ? c.d_qp32 : nullptr;
      if (c.global_w) {
        a.connW = c.d_connW;
        a.aw = c.d_Aw64;
      }
      k_ahat<D, P, FORM><<<nb, 128, 0, s>>>(a);
      break;
    }
    case kSetupAhatQuad: {
      const QuadCoef& qc = *k.qc;
      AhatQuadArgs a{c.d_coords, c.d_cells, c.d_conn, c.d_A64, c.keep32 ? c.d_A32 : nullptr,
                     c.d_geo, c.d_diag, c.d_err, c.E, qc.pts, qc.wts, qc.phi, qc.nq,
                     qc.centres, qc.radii, qc.nb, qc.inside, qc.outside};
      k_ahat_quad<D, P, FORM><<<nb, 128, 0, s>>>(a);
      break;
    }
    case kSetupLoad: {
      LoadArgs a{c.d_geo, c.d_perm, k.f, c.d_conn, k.b, c.E};
      k_load<D, P, FORM><<<nb, 128, 0, s>>>(a);
      break;
    }
    case kSetupGrad: {
      GradArgs a{c.d_geo, c.d_perm, c.d_conn, k.u, k.lam, k.dA, c.coef_kind, c.E};
      k_grad<D, P, FORM><<<nb, 128, 0, s>>>(a);
      break;
    }
    case kSetupExportFact:
      k_export_fact<D, P, FORM><<<nb, 128, 0, s>>>(c.d_A64, c.d_perm, k.out, c.E);
      break;
  }
}

}  // namespace dogip

#define DOGIP_SETUP_CASES(D, P)                 \
  case P * 2 + 0:                               \
    setup_run<D, P, 0>(c, k, s);                \
    return true;                                \
  case P * 2 + 1:                               \
    setup_run<D, P, 1>(c, k, s);                \
    return true;
