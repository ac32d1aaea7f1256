// Launchers of the setup-side element kernels (A_T precompute, load, gradient,
// export) and of the apply dispatcher, plus host access to the static tables.
#include <cstring>

#include "setup_inst.cuh"

namespace dogip {

bool setup_d2(Ctx& c, const SetupCall& k, cudaStream_t s);
bool setup_d3(Ctx& c, const SetupCall& k, cudaStream_t s);

namespace {
void setup_dispatch(Ctx& c, const SetupCall& k, cudaStream_t s, const char* what) {
  if (c.hi) {  // run-time tables: the precompute and the load are built, nothing else
    bool ok = false;
    if (k.op == kSetupAhat) {
      AhatArgs a{c.d_coords, 0, c.d_cells, c.d_perm, k.coef, k.coef_kind, c.d_conn, c.d_A64,
                 c.keep32 ? c.d_A32 : nullptr, c.d_geo, c.d_diag, c.d_err, c.E};
      ok = ahat_hi(c, a, s);
    } else if (k.op == kSetupLoad) {
      LoadArgs a{c.d_geo, c.d_perm, k.f, c.d_conn, k.b, c.E};
      ok = load_hi(c, a, s);
    }
    if (!ok) fail(DOGIP_EUNSUPPORTED, "not built for orders above the compiled tables");
    cuda_check(cudaGetLastError(), what);
    return;
  }
  const bool ok = c.d == 2 ? setup_d2(c, k, s) : setup_d3(c, k, s);
  if (!ok) fail(DOGIP_EUNSUPPORTED, "no compiled instance for this (dim, p, form)");
  cuda_check(cudaGetLastError(), what);
}
}  // namespace

// Apply dispatchers (apply_d*.cu): 0 = not compiled, 1 = per-cell kernel, 2 = staged
// kernel (which also wrote the Dirichlet rows).
int apply_d2(const Ctx&, const void*, void*, int, int, bool, int64_t, int64_t, cudaStream_t,
             const int*, bool);
int apply_d3a(const Ctx&, const void*, void*, int, int, bool, int64_t, int64_t, cudaStream_t,
              const int*, bool);
int apply_d3b(const Ctx&, const void*, void*, int, int, bool, int64_t, int64_t, cudaStream_t,
              const int*, bool);

namespace {
int apply_dispatch(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
                   int64_t e1, cudaStream_t s, const int* skip, bool add = false) {
  if (c.hi) return apply_hi(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
  if (c.d == 2) return apply_d2(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
  if (c.p <= 2) return apply_d3a(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
  if (c.p == 3) return apply_d3b(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
  return 0;
}
}  // namespace

__global__ void k_export_ahat(const double* A, const int64_t* perm, double* out, int64_t E,
                              int nsw) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= E * nsw) return;
  const int64_t pos = t / nsw;
  const int k = (int)(t - pos * nsw);
  out[perm[pos] * nsw + k] = A[(pos >> 5) * ((int64_t)nsw * kTile) + k * kTile + (pos & 31)];
}

// Dirichlet rows of K~ = P K P + (I - P): y_b = u_b, or y_b += u_b (add).
template <typename T>
__global__ void k_dirichlet_copy(const T* u, T* y, const int32_t* bnd, int64_t nb, int R,
                                 const int* skip, int add) {
  if (skip != nullptr && *skip) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nb * R) return;
  const int64_t i = (int64_t)bnd[t / R] * R + (t % R);
  y[i] = add ? y[i] + u[i] : u[i];
}

__global__ void k_diag_finish(double* diag, double* dinv64, float* dinv32, const int32_t* bnd,
                              int64_t nb, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nb) diag[bnd[t]] = 1.0;
}

__global__ void k_diag_inv(const double* diag, double* dinv64, float* dinv32, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = 1.0 / diag[t];
  dinv64[t] = v;
  dinv32[t] = (float)v;
}

namespace {

template <int D, int P, int FORM>
void info_one(int* NB, int* W, int* V, long long* nnz, long long* nnz1) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  *NB = TB::NB;
  *W = TB::W;
  *V = TB::V;
  *nnz = TB::NNZ;
  *nnz1 = TB::NNZ1;
}

template <int D, int P, int FORM>
void copy_one(double* B, double* w, double* iv) {
  using TB = dogip_tab::Tab<D, P, FORM>;
  if (B) std::memcpy(B, TB::B, sizeof(TB::B));
  if (w) std::memcpy(w, TB::w, sizeof(TB::w));
  if (iv) std::memcpy(iv, TB::iv, sizeof(TB::iv));
}

// Calls F<D,P,FORM>::run(args...) for the runtime triple; false if not compiled.
#define DOGIP_DISPATCH(d, p, form, CALL)                                    \
  do {                                                                     \
    const int key_ = (d) * 100 + (p) * 2 + (form);                         \
    switch (key_) {                                                        \
      case 202: CALL(2, 1, 0); break;                                      \
      case 203: CALL(2, 1, 1); break;                                      \
      case 204: CALL(2, 2, 0); break;                                      \
      case 205: CALL(2, 2, 1); break;                                      \
      case 206: CALL(2, 3, 0); break;                                      \
      case 207: CALL(2, 3, 1); break;                                      \
      case 208: CALL(2, 4, 0); break;                                      \
      case 209: CALL(2, 4, 1); break;                                      \
      case 302: CALL(3, 1, 0); break;                                      \
      case 303: CALL(3, 1, 1); break;                                      \
      case 304: CALL(3, 2, 0); break;                                      \
      case 305: CALL(3, 2, 1); break;                                      \
      case 306: CALL(3, 3, 0); break;                                      \
      case 307: CALL(3, 3, 1); break;                                      \
      default: ok_ = false;                                                \
    }                                                                      \
  } while (0)

}  // namespace

void launch_ahat(Ctx& c, const double* coef, int coef_kind, cudaStream_t s) {
  cuda_check(cudaMemsetAsync(c.d_diag, 0, sizeof(double) * c.n, s), "memset diag");
  if (c.global_w) cuda_check(cudaMemsetAsync(c.d_Aw64, 0, sizeof(double) * c.nW, s), "memset A_diag");
  SetupCall k;
  k.op = kSetupAhat;
  k.coef = coef;
  k.coef_kind = coef_kind;
  setup_dispatch(c, k, s, "ahat kernel launch");
  if (c.global_w && c.keep32) narrow_copy(c.d_Aw64, c.d_Aw32, c.nW, s);
  c.launches += 1;
  launch_diag_finish(c, s);
}

void launch_ahat_quad(Ctx& c, const QuadCoef& qc, cudaStream_t s) {
  cuda_check(cudaMemsetAsync(c.d_diag, 0, sizeof(double) * c.n, s), "memset diag");
  SetupCall k;
  k.op = kSetupAhatQuad;
  k.qc = &qc;
  setup_dispatch(c, k, s, "quadrature ahat kernel launch");
  c.launches += 1;
  launch_diag_finish(c, s);
}

void launch_diag_finish(Ctx& c, cudaStream_t s) {
  if (c.nbnd > 0)
    k_diag_finish<<<(unsigned)((c.nbnd + 255) / 256), 256, 0, s>>>(c.d_diag, c.d_dinv64,
                                                                  c.d_dinv32, c.d_bnd, c.nbnd,
                                                                  c.n);
  k_diag_inv<<<(unsigned)((c.n + 255) / 256), 256, 0, s>>>(c.d_diag, c.d_dinv64, c.d_dinv32, c.n);
  cuda_check(cudaGetLastError(), "diag kernels launch");
  c.launches += (c.nbnd > 0 ? 2 : 1);
}

void launch_load(Ctx& c, const double* f, double* b, cudaStream_t s) {
  cuda_check(cudaMemsetAsync(b, 0, sizeof(double) * c.n, s), "memset load");
  SetupCall k;
  k.op = kSetupLoad;
  k.f = f;
  k.b = b;
  setup_dispatch(c, k, s, "load kernel launch");
  c.launches += 1;
}

void launch_grad(Ctx& c, const double* u, const double* lam, double* dA, cudaStream_t s) {
  SetupCall k;
  k.op = kSetupGrad;
  k.u = u;
  k.lam = lam;
  k.dA = dA;
  setup_dispatch(c, k, s, "gradient kernel launch");
  c.launches += 1;
}

void launch_export_ahat(const Ctx& c, double* out, cudaStream_t s) {
  if (c.factorized) {
    SetupCall k;
    k.op = kSetupExportFact;
    k.out = out;
    setup_dispatch(const_cast<Ctx&>(c), k, s, "export kernel launch");
    return;
  }
  const int nsw = c.WT * c.NS;
  const int64_t tot = c.E * nsw;
  if (tot == 0) return;
  k_export_ahat<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c.d_A64, c.d_perm, out, c.E, nsw);
  cuda_check(cudaGetLastError(), "export kernel launch");
}

void launch_dirichlet_copy(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s,
                           const int* skip, bool add) {
  if (c.nbnd == 0) return;
  const int64_t tot = c.nbnd * R;
  const unsigned nb = (unsigned)((tot + 255) / 256);
  if (prec == DOGIP_FP64)
    k_dirichlet_copy<double><<<nb, 256, 0, s>>>((const double*)u, (double*)y, c.d_bnd, c.nbnd, R,
                                                 skip, add ? 1 : 0);
  else
    k_dirichlet_copy<float><<<nb, 256, 0, s>>>((const float*)u, (float*)y, c.d_bnd, c.nbnd, R,
                                                skip, add ? 1 : 0);
}

void prepare_apply(Ctx& c) {
  if (!apply_dispatch(c, nullptr, nullptr, 1, 0, true, 0, 0, nullptr, nullptr))
    fail(DOGIP_EUNSUPPORTED, "no compiled apply instance for this (dim, p, form)");
}

void launch_apply_cg(Ctx& c, const void* p, void* q, int R, int prec, int scatter, cudaStream_t s,
                     SolveWork& w) {
  if (c.global_w) {  // q was cleared by the previous p update (atomic scatter)
    if (R > c.w_cap) fail(DOGIP_EINVAL, "global double-grid scratch too small for nrhs");
    if (!apply_gw(c, p, q, R, prec, s, w.flags))
      fail(DOGIP_EUNSUPPORTED, "no compiled global double-grid instance for this (dim, p)");
    cuda_check(cudaGetLastError(), "global double-grid apply launch");
    c.launches += 2;
    return;
  }
  if (prec == DOGIP_TF32) {  // tensor-core kernel; it writes the Dirichlet rows itself
    if ((R != 1 && R % 16 != 0) || scatter != DOGIP_SCATTER_ATOMIC ||
        !apply_tc(c, p, q, s, w.flags, false, R))
      fail(DOGIP_EUNSUPPORTED, "no tensor-core apply for this context and request");
    cuda_check(cudaGetLastError(), "tensor-core apply launch");
    c.launches += 1;
    return;
  }
  if (scatter == DOGIP_SCATTER_ATOMIC) {
    const int k = apply_dispatch(c, p, q, R, prec, true, 0, c.E, s, w.flags);
    if (!k) fail(DOGIP_EUNSUPPORTED, "no compiled apply instance for this (dim, p, form)");
    cuda_check(cudaGetLastError(), "apply kernel launch");
    c.launches += 1;
    if (k == 1 && c.dirichlet && c.nbnd > 0) {  // the staged kernel writes these itself
      launch_dirichlet_copy(c, p, q, R, prec, s, w.flags);
      c.launches += 1;
    }
    return;
  }
  launch_apply(c, p, q, R, prec, scatter, s, w.flags);  // colour passes (memset inside)
}

bool cgcg_eligible(const Ctx& c, int R, int prec, int scatter) {
  if (R != 1 || prec != DOGIP_FP32 || scatter != DOGIP_SCATTER_ATOMIC || c.hi || c.global_w ||
      !c.keep32)
    return false;
  const int var = c.apply_variant_prec[DOGIP_FP32] >= 0 ? c.apply_variant_prec[DOGIP_FP32]
                                                         : c.apply_variant;
  return c.factorized || var == 1;  // the staged kernel carries the energy reduction
}

void launch_apply_energy(Ctx& c, const float* u, float* w, cudaStream_t s, SolveWork& wk,
                         int mode) {
  const CGEnergy en{wk.partial, wk.counter, wk.scal, wk.flags, mode};
  c.energy = &en;  // copied into the kernel arguments by the staged launcher
  int k = 0;
  try {
    k = apply_dispatch(c, u, w, 1, DOGIP_FP32, true, 0, c.E, s, wk.flags);
  } catch (...) {
    c.energy = nullptr;
    throw;
  }
  c.energy = nullptr;
  if (k != 2) fail(DOGIP_EUNSUPPORTED, "the fused p.Kp reduction needs the staged apply kernel");
  cuda_check(cudaGetLastError(), "apply kernel launch");
  c.launches += 1;
}

void launch_apply(Ctx& c, const void* u, void* y, int R, int prec, int scatter, cudaStream_t s,
                  const int* skip, bool add) {
  const size_t es = prec == DOGIP_FP64 ? sizeof(double) : sizeof(float);
  if (prec == DOGIP_TF32) {
    if ((R != 1 && R % 16 != 0) || scatter != DOGIP_SCATTER_ATOMIC ||
        !apply_tc_available(c.d, c.p, c.form) || c.global_w || c.factorized)
      fail(DOGIP_EUNSUPPORTED,
           "no tensor-core apply for this request (1 or a multiple of 16 right-hand sides, "
           "atomic scatter, element-wise A_T, and an instance for this dimension, order and "
           "form)");
    if (!add) cuda_check(cudaMemsetAsync(y, 0, es * c.n * R, s), "memset y");
    if (!apply_tc(c, u, y, s, skip, add, R))
      fail(DOGIP_EUNSUPPORTED, "no tensor-core apply for this context");
    c.launches += 1;
    cuda_check(cudaGetLastError(), "tensor-core apply launch");
    return;
  }
  if (!add) cuda_check(cudaMemsetAsync(y, 0, es * c.n * R, s), "memset y");
  if (c.global_w) {
    if (R > c.w_cap) fail(DOGIP_EINVAL, "global double-grid scratch too small for nrhs");
    if (!apply_gw(c, u, y, R, prec, s, skip))
      fail(DOGIP_EUNSUPPORTED, "no compiled global double-grid instance for this (dim, p)");
    c.launches += 2;
    cuda_check(cudaGetLastError(), "global double-grid apply launch");
    return;
  }
  bool staged = false;
  auto run = [&](bool atomic, int64_t e0, int64_t e1) {
    const int k = apply_dispatch(c, u, y, R, prec, atomic, e0, e1, s, skip, add);
    if (!k) fail(DOGIP_EUNSUPPORTED, "no compiled apply instance for this (dim, p, form)");
    staged = staged || k == 2;
  };
  if (scatter == DOGIP_SCATTER_COLOUR) {
    for (int k = 0; k < c.ncolours; ++k) run(false, c.colour_start[k], c.colour_start[k + 1]);
    c.launches += c.ncolours;
  } else {
    run(true, 0, c.E);
    c.launches += 1;
  }
  if (c.dirichlet && c.nbnd > 0 && !staged) {
    launch_dirichlet_copy(c, u, y, R, prec, s, skip, add);
    c.launches += 1;
  }
  cuda_check(cudaGetLastError(), "apply kernel launch");
}

bool apply_qp_d2(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s);
bool apply_qp_d3(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s);

void launch_apply_qp(Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s) {
  const size_t es = prec == DOGIP_FP64 ? sizeof(double) : sizeof(float);
  cuda_check(cudaMemsetAsync(y, 0, es * c.n * R, s), "memset y");
  const bool ok = c.d == 2 ? apply_qp_d2(c, u, y, R, prec, s) : apply_qp_d3(c, u, y, R, prec, s);
  if (!ok) fail(DOGIP_EUNSUPPORTED, "no compiled quadrature-point instance for this (dim, p, form)");
  c.launches += 1;
  if (c.dirichlet && c.nbnd > 0) {
    launch_dirichlet_copy(c, u, y, R, prec, s, nullptr);
    c.launches += 1;
  }
  cuda_check(cudaGetLastError(), "quadrature-point apply launch");
}

bool table_info(int d, int p, int form, int* NB, int* W, int* V, long long* nnz, long long* nnz1) {
  bool ok_ = true;
#define CALL(D, P, F) info_one<D, P, F>(NB, W, V, nnz, nnz1)
  DOGIP_DISPATCH(d, p, form, CALL);
#undef CALL
  if (!ok_) return hi_table(d, p, form, NB, W, V, nnz, nnz1, nullptr, nullptr, nullptr);
  return ok_;
}

bool table_copy(int d, int p, int form, double* B, double* w, double* iv) {
  bool ok_ = true;
#define CALL(D, P, F) copy_one<D, P, F>(B, w, iv)
  DOGIP_DISPATCH(d, p, form, CALL);
#undef CALL
  if (!ok_) {
    int NB, W, V;
    const double *hB, *hw, *hiv;
    if (!hi_table(d, p, form, &NB, &W, &V, nullptr, nullptr, &hB, &hw, &hiv)) return false;
    if (B) std::memcpy(B, hB, sizeof(double) * NB * W * V);
    if (w) std::memcpy(w, hw, sizeof(double) * W);
    if (iv) std::memcpy(iv, hiv, sizeof(double) * V);
  }
  return true;
}

bool table_is_compiled(int d, int p, int form) {
  bool ok_ = true;
#define CALL(D, P, F) (void)0
  DOGIP_DISPATCH(d, p, form, CALL);
#undef CALL
  return ok_;
}

}  // namespace dogip
