// Internal state of a DoGIP context and the launch interface between the host
// driver (host.cpp) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dogip.h"

namespace dogip {

// conn entry: bits 0..29 global dof id, bit 31 = dof on a Dirichlet boundary
// (gather reads 0 there, scatter skips it).
constexpr uint32_t kBndBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x3FFFFFFFu;
constexpr int kTile = 32;  // elements per AoSoA tile (one warp)

// Validation flags raised by the setup kernel.
constexpr int kErrGeometry = 1;   // |det R_T| not positive or not finite
constexpr int kErrNonFinite = 2;  // coefficient not finite
constexpr int kErrSymmetry = 4;   // tensor not symmetric
constexpr int kErrNotPos = 8;     // coefficient not positive (definite)

// Per-rhs scalars of a CG iteration (device memory).
struct CGScal {
  double rho, pq, alpha, beta, rr, r0, bb, s, rel, tol, otol;
  double rho_prev;  // rho before the last update (reliable-update restarts of beta)
  double rmax;      // residual norm at the last FP64 correction (reliable updates)
  int done, iters, brk, odone;
  int upd, pad0, pad1, pad2;  // upd: FP64 correction requested
};

struct SolveWork {
  int R = 0;
  int64_t n = 0;
  // FP64 vectors [n x R]
  double *x64 = nullptr, *r64 = nullptr, *p64 = nullptr, *q64 = nullptr;
  // FP32 vectors [n x R]
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  // Chronopoulos-Gear inner CG (R = 1): search direction p and s = K p; u (= M r) and
  // w (= K u) live in p32 and q32
  float *pc32 = nullptr, *sc32 = nullptr;
  // second search-direction buffers of the single-launch PCG (pcg_small_run)
  float* pb32 = nullptr;
  double* pb64 = nullptr;
  // reductions
  double* partial = nullptr;     // [kMaxRedBlocks x 32 x 2]
  unsigned int* counter = nullptr;
  CGScal* scal = nullptr;        // [R]
  int* flags = nullptr;          // [0] stop chunk, [1] breakdown, [2] all done, [3] correction wanted
  int* h_flags = nullptr;        // pinned host mirror: flags[0..3], [4] kernel wait timeout
  CGScal* h_scal = nullptr;      // pinned host mirror of scal
  // graph cache of the inner iteration chunk
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
  int graph_chunk = 0, graph_prec = -1, graph_scatter = -1;
  double graph_delta = -1.0;
  int graph_fused = -1;
  int64_t graph_kernels = 0;  // kernel nodes in the captured chunk
};

// Reduction target of the energy form of the apply (CG with one right-hand side): the
// apply kernel adds (y, u) = sum_T u_T . Y_T (+ the Dirichlet rows) per CTA into
// partial[CTA], and its last CTA sets alpha in scal: rho / (p, K p) for the standard
// recurrence (mode 0), the single-reduction formula of Chronopoulos and Gear (mode 1).
struct CGEnergy {
  double* partial;
  unsigned int* counter;
  CGScal* scal;
  int* flags;
  int mode;
};

constexpr int kMaxRedBlocks = 1216;  // 8 blocks of 256 threads on each of 152 SMs
constexpr int kRedThreads = 256;

}  // namespace dogip

// The opaque context of the C ABI.
struct dogip_ctx {
  int d = 0, p = 0, form = 0, coef_kind = 0;
  int VT = 0, WT = 0, NB = 0, NS = 0;
  bool dirichlet = false, keep32 = true;
  int scatter = DOGIP_SCATTER_ATOMIC;
  int device = 0;
  int64_t E = 0, Epad = 0, n = 0, nv = 0, nbnd = 0;
  int ncolours = 0;
  long long nnzb = 0, nnzb1 = 0;
  std::vector<int64_t> colour_start;  // processing-order ranges [ncolours + 1]
  std::vector<int32_t> dofmap;        // caller order [E x VT]
  std::vector<int32_t> colour;        // caller order [E]
  std::vector<uint8_t> bmask;         // [n]
  std::vector<int64_t> perm;          // processing position -> caller cell
  // device memory (processing order unless noted)
  double* d_coords = nullptr;  // [nv x d]
  int32_t* d_cells = nullptr;  // [E x (d+1)]
  int64_t* d_perm = nullptr;   // [E]
  uint32_t* d_conn = nullptr;  // AoSoA [Epad/32][VT][32]
  double* d_A64 = nullptr;     // AoSoA [Epad/32][WT*NS][32]
  float* d_A32 = nullptr;
  double* d_geo = nullptr;     // [E][d*d + 1]: R^-1 row-major, |det R|
  double* d_diag = nullptr;    // [n]
  double* d_dinv64 = nullptr;  // [n]
  float* d_dinv32 = nullptr;   // [n]
  int32_t* d_bnd = nullptr;    // [nbnd] boundary dof list
  double* d_coef = nullptr;    // caller order copy of the setup coefficients
  double* d_qp64 = nullptr;    // [E][NS] processing order: coefficient stream of the
  float* d_qp32 = nullptr;     //   quadrature-point comparator (dogip_apply_qp)
  bool qp_ok = false;          // element-constant coefficients are set (not sub-element)
  // orders above the compiled tables (2D p 5..8, 3D p 4): run-time tables
  bool hi = false;
  double* d_hiB64 = nullptr;  // [NB][W][V]
  float* d_hiB32 = nullptr;
  double* d_hiW = nullptr;    // [W]
  double* d_hiIV = nullptr;   // [V]
  // global double grid for the weighted projection (dogip_opts.global_w)
  bool global_w = false;
  int64_t nW = 0;                   // W nodes (continuous P_2p space)
  std::vector<int32_t> wdofmap;     // [E x W_T] caller order
  std::vector<uint8_t> wowner;      // [E x W_T] 1 where the cell owns the node
  uint32_t* d_connW = nullptr;      // AoSoA [Epad/32][W_T][32], bit 31 = owner
  double* d_Aw64 = nullptr;         // A_diag [nW]
  float* d_Aw32 = nullptr;
  double* d_w64 = nullptr;          // scratch [nW x w_cap]
  float* d_w32 = nullptr;
  int w_cap = 0;
  int* d_err = nullptr;        // validation flags
  int* d_kerr = nullptr;       // kernel wait timeouts (bounded mbarrier waits)
  int apply_variant = 1;       // 3: tensor cores (FP32); 2: self-feeding warps; 1: bulk-async staged; 0: one thread per cell
  bool factorized = false;     // store K_T per cell; A_T,j = w_j K_T formed in the kernel
  int apply_variant_prec[2] = {-1, -1};  // per precision (autotuner), -1: apply_variant
  int apply_block[2] = {256, 256};       // cells per CTA of the per-cell kernel
  long long wait_budget = 4000000000LL;  // clock cycles per bounded wait in kernels
  int64_t l2_bytes = 0;        // L2 size of the device: streams larger than half of it
                               // are copied with the L2 evict-first policy
  int64_t test_skip_chunk = -1;  // test hook (see DOGIP_TEST_SKIP_CHUNK)
  bool graph_pdl = true;          // programmatic edges in captured CG chunks (DOGIP_GRAPH_PDL)
  // set around one launch by launch_apply_energy (host, one thread per context): the
  // staged kernel then also reduces (w, u) and sets alpha
  mutable const dogip::CGEnergy* energy = nullptr;
  dogip::SolveWork work;
  int64_t launches = 0;           // kernels launched (graph replays count every node)
  cudaStream_t stream = nullptr;  // private stream for graph-captured solves
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace dogip {

using Ctx = ::dogip_ctx;

// Thrown inside the library, turned into a status code at the ABI.
struct Failure {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void set_last_error(const std::string& msg);  // message of dogip_last_error()
void cuda_check(cudaError_t e, const char* what);

// Device arrays of the sub-element quadrature of an inclusion coefficient.
struct QuadCoef {
  const double* pts;      // [nq x d] reference points
  const double* wts;      // [nq]
  const double* phi;      // [nq x W_T] W-basis values
  int nq;
  const double* centres;  // [nb x d]
  const double* radii;    // [nb]
  int nb;
  double inside, outside;
};

// 1 when the A_T and conn streams of one apply (element size es, A_T entries per cell
// nsw or, factorised, n_sym) exceed half of L2: such streams are read with the L2
// evict-first policy so that u and y stay in L2; smaller ones may stay resident
// between the applies of a solve and are copied without a policy.
inline int stream_evict_first(const Ctx& c, size_t es, int nsw) {
  const int64_t bytes = c.Epad * ((int64_t)nsw * (int64_t)es + 4 * (int64_t)c.VT);
  return c.l2_bytes > 0 && 2 * bytes > c.l2_bytes ? 1 : 0;
}

// ---- kernel launchers (implemented in the .cu translation units) ----------
// All take the processing-order state of ctx and enqueue on `s`.
void launch_ahat(Ctx& c, const double* coef, int coef_kind, cudaStream_t s);
void launch_ahat_quad(Ctx& c, const QuadCoef& qc, cudaStream_t s);
// add: y += K u (no clearing of y; Dirichlet rows y_b += u_b) instead of y = K u.
// prec DOGIP_TF32: FP32 data, the contractions with B on the tensor cores (the
// tensor-core kernel; EUNSUPPORTED where no instance exists).
void launch_apply(Ctx& c, const void* u, void* y, int R, int prec, int scatter,
                  cudaStream_t s, const int* skip, bool add = false);
// The apply inside a CG iteration, q = K p.  With atomic scatter q must already be
// zero (the previous p update clears it); colour scatter clears it itself.
void launch_apply_cg(Ctx& c, const void* p, void* q, int R, int prec, int scatter,
                     cudaStream_t s, SolveWork& w);
void launch_load(Ctx& c, const double* f, double* b, cudaStream_t s);
void launch_grad(Ctx& c, const double* u, const double* lam, double* dA,
                 cudaStream_t s);
void launch_export_ahat(const Ctx& c, double* out, cudaStream_t s);
// Run-time-table kernels of the higher orders (apply_hi.cu).
struct AhatArgs;
struct LoadArgs;
int apply_hi(const Ctx& c, const void* u, void* y, int R, int prec, bool atomic, int64_t e0,
             int64_t e1, cudaStream_t s, const int* skip, bool add = false);
bool ahat_hi(const Ctx& c, AhatArgs& a, cudaStream_t s);
bool load_hi(const Ctx& c, LoadArgs& a, cudaStream_t s);
bool hi_table(int d, int p, int form, int* NB, int* W, int* V, long long* nnz, long long* nnz1,
              const double** B, const double** w, const double** iv);
bool table_is_compiled(int d, int p, int form);
// Tensor-core FP32 apply (apply_tc.cu): R = 1 or a multiple of 16 right-hand sides,
// atomic scatter over the whole cell range.  false when no instance exists for
// (d, p, form) or R; u == nullptr only sets the kernel attributes (context set-up).
bool apply_tc(const Ctx& c, const void* u, void* y, cudaStream_t s, const int* skip,
              bool add = false, int R = 1);
bool apply_tc_available(int d, int p, int form);
// Global double-grid apply of the weighted projection (two kernels); false when no
// instance exists.  The scratch must hold R right-hand sides (ensure_w_scratch).
bool apply_gw(const Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s,
              const int* skip);
void ensure_w_scratch(Ctx& c, int R);
void narrow_copy(const double* a, float* b, int64_t n, cudaStream_t s);
// Quadrature-point matrix-free apply (comparator): y = K~ u, atomic scatter.
void launch_apply_qp(Ctx& c, const void* u, void* y, int R, int prec, cudaStream_t s);
void launch_dirichlet_copy(const Ctx& c, const void* u, void* y, int R, int prec,
                           cudaStream_t s, const int* skip, bool add = false);
void launch_diag_finish(Ctx& c, cudaStream_t s);
// One-time kernel attributes of the apply instances of this context (host only).
void prepare_apply(Ctx& c);

// ---- grouped kernels of the batched mixed solve (batch.cu) ----------------------
// One problem of a batch as the grouped kernels see it (device memory, FP32 inner CG).
struct BProb {
  const float* A;           // A_T, AoSoA, processing order = caller order
  const uint32_t* conn;
  int64_t E, n;
  float *x, *r, *p, *q;     // inner CG vectors
  const float* dinv;
  const int32_t* bnd;       // Dirichlet rows
  int64_t nbnd;
  CGScal* scal;
  int* flags;
  double* partial;          // per-problem reduction buffer
  unsigned int* counter;
  int nvblocks;             // vector work items of this problem
};
// Items are (problem, block) pairs; cells per apply item and dofs per vector item:
int64_t batch_cells_per_item();
int64_t batch_dofs_per_item();
bool batch_apply_compiled(int d, int p, int form);
void batch_apply_group(int d, int p, int form, const BProb* probs, const int2* items, int nitems,
                       cudaStream_t s);
// Dirichlet rows (bitems: blocks of 256 boundary dofs), then p.q, x/r update, p update.
void batch_vec_step(const BProb* probs, const int2* bitems, int nbitems, const int2* vitems,
                    int nvitems, cudaStream_t s);
void batch_status(const BProb* probs, int np, CGScal* scal_out, int* flags_out, cudaStream_t s);

// Programmatic dependent launch inside captured CG chunks: kernels whose first act
// is griddepcontrol.launch_dependents + griddepcontrol.wait (they touch nothing of the
// previous kernel before the wait) are marked by their launchers; run_chunk turns the
// graph edges between two marked kernels into programmatic ones, so the next kernel
// is launched while the previous one drains.  Edges to or from any other node keep
// full serialisation.
void pdl_mark(const void* kernel);
bool pdl_marked(const void* kernel);

// Static table access for the host (dogip_get_tables, info).
bool table_info(int d, int p, int form, int* NB, int* W, int* V, long long* nnz,
                long long* nnz1);
bool table_copy(int d, int p, int form, double* B, double* w, double* iv);

// ---- solver vector kernels (vec.cu); each returns the number of kernels it launched
void vec_alloc(SolveWork& w, int64_t n, int R);
void vec_free(SolveWork& w);
// r64 <- b - Kx (FP64) with per-rhs ||r||^2 (and ||b||^2 when first); sets
// rel = ||r||/||b||, s = ||r||, odone = rel <= otol.
int vec_residual64(SolveWork& w, const double* b, const double* Kx, bool first,
                    double otol, cudaStream_t st);
// Inner FP32 start: r32 = r64 / s (0 for finished rhs), x32 = 0, p = Dinv r,
// rho = r.z, r0 = ||r32||, tol = inner_tol.
int vec_inner_init32(SolveWork& w, const float* dinv, double inner_tol, cudaStream_t st);
// FP64 PCG start from r64 = b - K x0: p = Dinv r, rho, r0 = ||b||, tol.
int vec_init64(SolveWork& w, const double* dinv, double tol, cudaStream_t st);
// The CG iteration after q = K p: alpha = rho / p.q, x += alpha p, r -= alpha q,
// rho' = r.Dinv r, beta, p = Dinv r + beta p; per-rhs convergence test.
// zero_q: clear q for the next scatter-add apply (every atomic-scatter iteration;
// colour passes clear it themselves).
int vec_cg_step(SolveWork& w, int prec, double* x64, const void* dinv, double delta,
                cudaStream_t st, bool zero_q, bool with_pq = true);
// Chronopoulos-Gear FP32 inner CG (R = 1), two kernels per iteration:
//   vec_cgcg_step: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = Dinv r,
//                  w = 0, gamma = r.u, rr = r.r; beta = gamma / gamma_old; convergence test
//   launch_apply_energy: w = K u with (w, u) reduced in the apply; alpha = gamma /
//                  ((w, u) - beta gamma / alpha_old)
// false from launch_apply_energy when the context's FP32 apply is not the staged kernel.
int vec_cgcg_step(SolveWork& w, const float* dinv, cudaStream_t st);
void vec_alloc_cgcg(SolveWork& w);
bool cgcg_eligible(const Ctx& c, int R, int prec, int scatter);
void launch_apply_energy(Ctx& c, const float* u, float* w, cudaStream_t s, SolveWork& wk,
                         int mode);
// Reliable-update mixed CG (FP32 recursion, FP64 corrections):
// start: r32 = r64, x32 = 0, p = Dinv r32, rho, r0 = ||b||, rmax = ||r64||.
int vec_rel_init(SolveWork& w, const float* dinv, double tol, cudaStream_t st);
// x64 += x32, x32 = 0 (all rhs).
int vec_fold(SolveWork& w, double* x64, cudaStream_t st);
// after r64 = b - K x64: r32 = r64, rho' = r32.Dinv r32, beta = rho'/rho_prev,
// done = ||r64|| <= tol ||b||, rmax = ||r64||, then p = Dinv r32 + beta p.
int vec_rel_restart(SolveWork& w, const float* dinv, cudaStream_t st);
// x64 += s * x32 for rhs still refining.
int vec_correct(SolveWork& w, double* x64, cudaStream_t st);

// Single-launch PCG (one cooperative kernel runs up to maxit iterations of the PCG
// started by vec_init64 / vec_inner_init32, nrhs 1, atomic scatter): FP64 iterates x64,
// FP32 iterates x32.  Leaves scal, flags and their host mirrors as run_chunk does.
bool pcg_small_supported(const Ctx& c, int prec);
int64_t pcg_small_bytes(const Ctx& c, int prec);  // operator + vectors it streams
void pcg_small_run(Ctx& c, int prec, double* x64, int maxit);

}  // namespace dogip
