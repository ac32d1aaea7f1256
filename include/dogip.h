/*
 * dogip.h -- C ABI of the GB300-native DoGIP library.
 *
 * DoGIP (double-grid integration with interpolation-projection; Vondrejc,
 * arXiv 1710.09913) writes the Galerkin matrix of the weighted projection
 * (Section 2.2, eq. linsys_gp) or of the scalar elliptic problem (Section 2.3,
 * eq. linsys_se) on a simplex mesh with continuous P_p Lagrange elements as
 *
 *     A u . v = sum_T  B^* A_T B u_T . v_T
 *
 * (Theorems "Element-wise DoGIP for weighted projection" and "Element-wise
 * DoGIP for the elliptic problem", eqs. wp_dogip_mul and ep_dogip_mul), where
 * B interpolates the local P_p dofs u_T (their reference gradients for the
 * elliptic form) onto the nodes of the double-grid space W (P_2p resp.
 * discontinuous P_{2p-2}) of the reference simplex, and A_T is diagonal
 * (projection) or block-diagonal with symmetric d x d blocks that carry the
 * element Jacobian (elliptic).  dogip_apply evaluates Algorithm 1
 * ("Matrix-vector multiplication for element-wise DoGIP") on the GPU;
 * dogip_solve runs a Jacobi-preconditioned CG around it.
 *
 * Conventions for every entry point below:
 *  - Return value: DOGIP_OK (0) or one of the DOGIP_E* codes; the message of
 *    the last failure on the calling thread is dogip_last_error().  No C++
 *    exception crosses this interface.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the context's device (e.g. torch CUDA tensors).  The
 *    caller owns every pointer it passes; the library copies what it keeps.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Calls
 *    documented as asynchronous only enqueue work on it.
 *  - Vectors with several right-hand sides are dof-major: entry (i, r) of an
 *    [n x nrhs] array is at i * nrhs + r.
 *  - Element numbering is the caller's cell order; dof numbering is the
 *    library's (dogip_get_dofmap): dofs are numbered in order of first
 *    appearance scanning cells in order and local nodes in local order.
 *  - Local node order of P_q on the reference simplex: multi-indices alpha,
 *    |alpha| <= q, in lexicographic order with the last coordinate fastest;
 *    node alpha sits at sum_i (alpha_i / q) (v_i - v_0) + v_0.
 *
 * Environment variables read by dogip_setup (none is required):
 *  - DOGIP_APPLY_VARIANT: apply kernel until dogip_autotune decides (3 tensor cores
 *    for FP32 single-rhs applies where an instance exists (2D p <= 6, 2D p = 7
 *    projection, 3D p <= 2, 3D p = 4 projection), else as 1; 2 self-feeding warps, 1 staged kernel
 *    (default), 0 one thread per cell; the orders above the compiled tables have
 *    one CUDA-core kernel, taken for every value but 3).
 *  - DOGIP_TUNE_CACHE: file of autotuner choices (see dogip_autotune).
 *  - DOGIP_GRAPH_PDL: 1 (default) launches the kernels of a captured CG chunk as
 *    programmatic dependents of each other where they are written for it (the next
 *    kernel starts while the previous one drains); 0 keeps full serialisation.
 *  - DOGIP_BATCH_MODE, DOGIP_BATCH_ORDER, DOGIP_BATCH_THREADS: how dogip_batch_solve
 *    runs its problems (see there).
 *  - DOGIP_TEST_WAIT_CYCLES, DOGIP_TEST_SKIP_CHUNK: test hooks of the device-side
 *    failure path (a shorter bound on the kernels' waits; one chunk of the staged
 *    apply, or one tile of the tensor-core apply, whose copy is never issued, and
 *    one block of the single-launch PCG that never arrives at its first grid
 *    barrier, so that the bounded waits of the others expire).
 */
#ifndef DOGIP_H
#define DOGIP_H

#include <stdint.h>

#if defined(__GNUC__)
#define DOGIP_API __attribute__((visibility("default")))
#else
#define DOGIP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define DOGIP_OK 0
#define DOGIP_EINVAL 1      /* invalid argument, mesh or coefficient            */
#define DOGIP_ENOMEM 2      /* device or host allocation failed                 */
#define DOGIP_ECUDA 3       /* a CUDA runtime call failed                       */
#define DOGIP_ENOTCONV 4    /* solver hit its iteration limit (result written)  */
#define DOGIP_EBREAKDOWN 5  /* CG breakdown: p^T K p <= 0 or not finite         */
#define DOGIP_ETIMEOUT 6    /* a time limit expired: a solve's host wall-clock
                               limit (timeout_ms), or a bounded wait inside a
                               kernel (copy or tensor-core completion), which
                               then returned without finishing its work      */
#define DOGIP_EUNSUPPORTED 7 /* valid request outside the compiled instances    */

/* ------------------------------------------------------------ enumerations */
#define DOGIP_PROJECTION 0  /* a(u,v) = int m u v            (Section 2.2)     */
#define DOGIP_ELLIPTIC 1    /* a(u,v) = int M grad u . grad v (Section 2.3)    */

#define DOGIP_COEF_ELEM_SCALAR 0 /* one scalar per cell: m_T, or M_T = m_T I   */
#define DOGIP_COEF_ELEM_TENSOR 1 /* one symmetric d x d tensor M_T per cell    */
#define DOGIP_COEF_INCLUSIONS 2  /* isotropic field with spherical inclusions,
                                    integrated per W node (dogip_set_coef_inclusions) */

#define DOGIP_FP64 0        /* FP64 storage and arithmetic                     */
#define DOGIP_FP32 1        /* FP32 A_T, vectors and arithmetic                */
#define DOGIP_TF32 2        /* FP32 A_T and vectors; the two contractions with B
                               (interpolation B u_T, projection B^* h) on the
                               tensor cores as three TF32 products each (hi*hi +
                               hi*lo + lo*hi of a split FP32 operand, FP32
                               accumulation, about 2^-21 relative per product);
                               one right-hand side, atomic scatter, element-wise
                               A_T, instances 2D p <= 6 (p = 7: projection) and
                               3D p <= 2 (p = 4: projection)                    */

#define DOGIP_SCATTER_ATOMIC 0 /* one pass, atomic adds (order not fixed)      */
#define DOGIP_SCATTER_COLOUR 1 /* one pass per element colour, plain adds      */

#define DOGIP_SOLVE_FP64 0  /* FP64 Jacobi-PCG                                 */
#define DOGIP_SOLVE_MIXED 1 /* FP64 iterative refinement around restarted FP32
                               PCG solves of K d = r / ||r||                   */
#define DOGIP_SOLVE_MIXED_RELIABLE 2 /* one FP32 PCG recursion with FP64 residual
                                        replacement (reliable updates)        */

typedef struct dogip_ctx dogip_ctx;

/* Simplex mesh, host memory, caller order.  The library copies it.  There is no
 * per-vertex boundary flag: the boundary is derived from the cells (a facet that
 * belongs to exactly one cell is on the boundary, and so are the dofs on it), which
 * is the boundary of the meshed domain for any conforming simplex mesh. */
typedef struct {
  int dim;                 /* 2 (triangles) or 3 (tetrahedra)                  */
  int64_t n_vertices;
  const double* coords;    /* host [n_vertices x dim]                          */
  int64_t n_cells;
  const int32_t* cells;    /* host [n_cells x (dim+1)] vertex ids              */
} dogip_mesh;

typedef struct {
  int dirichlet;   /* -1 default (1 for elliptic, 0 for projection); 1: zero
                      Dirichlet rows/columns on boundary dofs (facets of one
                      cell), i.e. the operator P K P + (I - P)                 */
  int scatter;     /* DOGIP_SCATTER_*: element storage order (COLOUR sorts the
                      cells by colour) and the default scatter of solves      */
  int keep_fp32;   /* 1 (default): also keep an FP32 copy of A_T              */
  int device;      /* CUDA device ordinal, -1 = current device                */
  int factorized;  /* 0 (default): store A_T per W node (eqs. wp_dogip_mul,
                      ep_dogip_mul).  1: the coefficients are constant per cell
                      (they are, for every coefficient kind of this ABI), so
                      A_T,j = w_j K_T with K_T = |det R_T| R_T^-1 M_T R_T^-T (or
                      m_T |det R_T|): only K_T is stored (d(d+1)/2 or 1 values
                      per cell) and w_j is applied inside the kernel.  Needs
                      scatter = ATOMIC.                                         */
  int global_w;    /* 0 (default): element-wise DoGIP.  1 (projection only): the
                      global double grid of §2.2, Theorem "DoGIP for weighted
                      projection": W = C_{N,2p} continuous, K = B^* A_diag B with
                      A_diag,ii = int m phi_W^i stored once per global W node
                      (instead of W_T values per cell); needs factorized = 0,
                      scatter = ATOMIC and no Dirichlet rows.                    */
} dogip_opts;

/* Fill *o with the defaults above.  Never fails for o != NULL. */
DOGIP_API int dogip_opts_default(dogip_opts* o);

/*
 * Build a context: dof map l_T (Section 2.1), boundary set, greedy element
 * colouring, reference tables B and w (Theorems above), and -- on the device --
 * the element factors A_T (dogip_set_coef) and the Jacobi diagonal.
 *   m       : mesh (host), copied.
 *   p       : polynomial order: 1..8 on triangles, 1..4 on tetrahedra (2D p <= 4
 *             and 3D p <= 3 with compile-time tables, the higher orders with the
 *             run-time-table kernels, which build the apply, precompute, load and
 *             both solvers only).
 *   form    : DOGIP_PROJECTION or DOGIP_ELLIPTIC.
 *   coef_kind, coef : host coefficients in caller cell order, [n_cells] for
 *             DOGIP_COEF_ELEM_SCALAR or [n_cells x dim x dim] for
 *             DOGIP_COEF_ELEM_TENSOR (elliptic only); copied.
 *   o       : options or NULL for defaults.
 *   out     : receives the context; the caller frees it with dogip_destroy.
 * Errors: EINVAL (bad sizes, vertex ids out of range, degenerate or
 * non-finite cell, non-symmetric / non-positive coefficient), ENOMEM, ECUDA,
 * EUNSUPPORTED (p outside the compiled range).  Synchronous.
 */
DOGIP_API int dogip_setup(const dogip_mesh* m, int p, int form, int coef_kind,
                const double* coef, const dogip_opts* o, dogip_ctx** out);

/* Free a context and all memory it owns (synchronises its device). */
DOGIP_API void dogip_destroy(dogip_ctx* ctx);

/*
 * Recompute A_T (eq. ep_dogip_mul: A_T,j = |det R_T| w_j R_T^-1 M_T R_T^-T;
 * eq. wp_dogip_mul: A_T,j = m_T |det R_T| w_j) and the Jacobi diagonal from new
 * coefficients, keeping mesh, dofs and tables.  coef is DEVICE memory in caller
 * cell order with the layout of dogip_setup.  Enqueued on cuda_stream; the
 * call then synchronises that stream to report invalid coefficients (EINVAL).
 */
DOGIP_API int dogip_set_coef(dogip_ctx* ctx, int coef_kind, const double* coef,
                   void* cuda_stream);

/*
 * Element factors of a discontinuous isotropic coefficient m(x) -- `inside` in the
 * union of n_incl balls (host centres [n_incl x dim], radii [n_incl]), `outside`
 * elsewhere -- integrated per W node with a sub-element rule (Section 3.3: DoGIP
 * takes the quadrature of rough coefficients out of the operator apply):
 *   A_T,j = sigma_j |det R_T| R_T^-1 R_T^-T (elliptic, M = m I) or sigma_j |det R_T|
 *   (projection), sigma_j = sum_q w_q m(F_T(x_q)) phi^W_j(x_q),
 * with the collapsed Gauss rule of nq points per direction on the reference simplex
 * (exact to degree 2 nq - 1; nq in 1..16).  Recomputes A_T and the Jacobi diagonal;
 * the apply is unchanged.  Needs factorized = 0.  Synchronises cuda_stream.
 */
DOGIP_API int dogip_set_coef_inclusions(dogip_ctx* ctx, int n_incl, const double* centres,
                                        const double* radii, double inside, double outside,
                                        int nq, void* cuda_stream);

/* ----------------------------------------------------------------- queries */
typedef struct {
  int dim, p, form, coef_kind, dirichlet, scatter;
  int64_t n_cells, n_dofs, n_boundary;
  int v_loc;        /* V_T = dim P_p                                          */
  int w_loc;        /* W_T = dim P_2p (projection) or dim P_{2p-2} (elliptic) */
  int n_sym;        /* stored entries per W node: 1 or dim(dim+1)/2           */
  int n_colours;
  int64_t nnz_b, nnz_pm1_b; /* nonzero / +-1 entries of B (eq. comp_eff)     */
  int64_t bytes_ahat_fp64, bytes_ahat_fp32, bytes_conn;
  int64_t kernel_launches; /* kernels this context has launched so far,
                              counting every node of replayed CUDA graphs   */
  int64_t n_wglobal;       /* global W nodes (global_w), else 0; then the
                              bytes_ahat_* fields count A_diag and bytes_conn
                              includes the W-node map                        */
} dogip_info;

DOGIP_API int dogip_get_info(const dogip_ctx* ctx, dogip_info* info);
DOGIP_API int64_t dogip_ndofs(const dogip_ctx* ctx); /* -1 on NULL ctx */

/* Dof map l_T: host [n_cells x V_T] global dof ids, caller cell order. */
DOGIP_API int dogip_get_dofmap(const dogip_ctx* ctx, int32_t* host_out);
/* Colour of every cell: host [n_cells]; *n_colours receives the count. */
DOGIP_API int dogip_get_colouring(const dogip_ctx* ctx, int32_t* host_out, int* n_colours);
/* Boundary flags: host [n_dofs], 1 on dofs of boundary facets. */
DOGIP_API int dogip_get_boundary(const dogip_ctx* ctx, uint8_t* host_out);
/* A_T in FP64: device [n_cells x W_T x n_sym], caller cell order; symmetric
 * blocks packed as (00,01,11) in 2D and (00,01,02,11,12,22) in 3D.  Async. */
DOGIP_API int dogip_get_ahat(const dogip_ctx* ctx, double* dev_out, void* cuda_stream);
/* Jacobi diagonal of the operator (1 on Dirichlet rows): device [n_dofs]. Async. */
DOGIP_API int dogip_get_diag(const dogip_ctx* ctx, double* dev_out, void* cuda_stream);

/*
 * Host-only mesh preprocessing (no CUDA call, no context; the routines dogip_setup
 * uses).  cells: host int32 [n_cells x (dim+1)] vertex ids >= 0.
 *  dogip_mesh_dofmap : ids [n_cells x V_T] (may be NULL) and the dof count of the
 *                      continuous P_p space, numbered by first appearance (§2.1).
 *  dogip_mesh_boundary: mask [n_dofs], 1 on the dofs of facets of one cell.
 *  dogip_mesh_colouring: greedy cell colouring, cells in order, smallest colour not
 *                      used by an earlier cell sharing a vertex; colour [n_cells].
 *  dogip_mesh_wdofmap: the W nodes of order 2p (global double grid): ids
 *                      [n_cells x W_T], owner flags [n_cells x W_T], count.
 * Errors: DOGIP_EINVAL (dim, p outside 1..16, empty or negative ids).
 */
DOGIP_API int dogip_mesh_dofmap(int dim, int p, int64_t n_cells, const int32_t* cells,
                                int32_t* ids, int64_t* n_dofs);
DOGIP_API int dogip_mesh_boundary(int dim, int p, int64_t n_cells, const int32_t* cells,
                                  uint8_t* mask);
DOGIP_API int dogip_mesh_colouring(int dim, int64_t n_cells, const int32_t* cells,
                                   int32_t* colour, int* n_colours);
DOGIP_API int dogip_mesh_wdofmap(int dim, int p, int64_t n_cells, const int32_t* cells,
                                 int32_t* ids, uint8_t* owner, int64_t* n_w);

/* Global double grid only (global_w = 1):
 * A_diag: device double [n_W] (n_W = info.n_wglobal).  Async.
 * W-node map: host int32 [n_cells x W_T] global W-node ids (first appearance,
 * like the dof map, at order 2p) and host uint8 [n_cells x W_T] owner flags (1 in
 * the first cell containing the node); either pointer may be NULL. */
DOGIP_API int dogip_get_ahat_global(const dogip_ctx* ctx, double* dev_out, void* cuda_stream);
DOGIP_API int dogip_get_wdofmap(const dogip_ctx* ctx, int32_t* host_ids, uint8_t* host_owner);

/*
 * Reference tables of the library, independent of any context (host):
 *   bhat : [NB x W_T x V_T], NB = 1 (projection) or dim (elliptic), may be NULL
 *   what : [W_T] integrals of the W basis over the reference simplex, may be NULL
 *   sizes: [3] receives NB, W_T, V_T, may be NULL.
 */
DOGIP_API int dogip_get_tables(int dim, int p, int form, double* bhat, double* what,
                     int* sizes);

/* ------------------------------------------------------------------- apply */
/*
 * y = K u  (Algorithm 1: gather u_T, interpolate B u_T, multiply by A_T, project
 * back B^*, scatter-add), with K = P K P + (I - P) when Dirichlet rows are on.
 *   u, y  : DEVICE [n_dofs x nrhs], double (DOGIP_FP64) or float (DOGIP_FP32);
 *           y is overwritten; u and y must not overlap.
 *   nrhs  : >= 1.
 *   prec  : DOGIP_FP64, DOGIP_FP32 or DOGIP_TF32 (the latter two need keep_fp32;
 *           TF32 returns DOGIP_EUNSUPPORTED outside its instances, see above).
 *   scatter: DOGIP_SCATTER_ATOMIC, or DOGIP_SCATTER_COLOUR (needs a context
 *           set up with scatter = COLOUR), or -1 for the context default.
 * Asynchronous on cuda_stream; no host synchronisation.  A global_w context keeps
 * an [n_W x nrhs] scratch; a call with more right-hand sides than before grows it
 * (allocation and a sync of the context's stream), so such a call is not capturable:
 * make the first call with the largest nrhs outside stream capture.
 */
DOGIP_API int dogip_apply(dogip_ctx* ctx, const void* u, void* y, int nrhs, int prec,
                int scatter, void* cuda_stream);

/*
 * y += K u: the same operator as dogip_apply (Algorithm 1 with the Dirichlet rows
 * y_b += u_b), added into the caller's y instead of overwriting it, so y is not
 * cleared first.  With the staged, self-feeding or tensor-core kernel (atomic
 * scatter over the whole mesh) the call enqueues exactly one kernel.  Arguments,
 * layout, precisions and errors as dogip_apply; y must hold valid numbers.
 * Asynchronous on cuda_stream.
 */
DOGIP_API int dogip_apply_add(dogip_ctx* ctx, const void* u, void* y, int nrhs, int prec,
                              int scatter, void* cuda_stream);

/*
 * Comparator, not the DoGIP path: the conventional quadrature-point matrix-free
 * apply that the paper sets DoGIP against (§1 "alternative approaches", §3.3).
 * y = K u with, per cell, the geometry R_T, |det R_T|, R_T^-1 recomputed from the
 * vertex coordinates at every call, the cell's coefficient read from a per-cell
 * stream, and the integral evaluated at the points of the collapsed Gauss-Jacobi
 * rule with p + 1 (projection) or p (elliptic) points per direction, exact for
 * element-constant coefficients; the result equals dogip_apply's up to rounding.
 * Same arguments, layout and Dirichlet rows as dogip_apply; atomic scatter.
 * Errors: DOGIP_EINVAL (arguments), DOGIP_EUNSUPPORTED after
 * dogip_set_coef_inclusions (the per-cell coefficient no longer describes the
 * field; dogip_set_coef restores it).  Asynchronous on cuda_stream.
 */
DOGIP_API int dogip_apply_qp(dogip_ctx* ctx, const void* u, void* y, int nrhs, int prec,
                             void* cuda_stream);

/*
 * Load vector of an element-wise constant source: b_i = sum_T f_T int_T phi_i
 * (f = 1 when f_elem is NULL); boundary entries set to 0 when Dirichlet rows
 * are on.  f_elem: DEVICE [n_cells] caller order or NULL; b: DEVICE [n_dofs].
 * Asynchronous.
 */
DOGIP_API int dogip_load(dogip_ctx* ctx, const double* f_elem, double* b, void* cuda_stream);

/* ------------------------------------------------------------------- solve */
typedef struct {
  int mode;           /* DOGIP_SOLVE_FP64 or DOGIP_SOLVE_MIXED                */
  double tol;         /* target ||b - K u||_2 / ||b||_2 (FP64), per rhs        */
  int maxiter;        /* FP64 mode: PCG iterations; mixed: total inner ones    */
  double inner_tol;   /* mixed: relative residual reduction per inner solve;
                         a step asks for no more than the FP64 residual still
                         needs (0.2 tol / current residual, if that is larger) */
  int inner_maxiter;  /* mixed: iteration limit of one inner solve             */
  int max_outer;      /* mixed: refinement steps                               */
  int scatter;        /* -1 context default, else DOGIP_SCATTER_*              */
  int check_every;    /* iterations per device-resident chunk between host
                         convergence checks (>= 1)                             */
  int use_x0;         /* 1: u holds the initial guess; 0: start from u = 0     */
  double timeout_ms;  /* host wall-clock limit, <= 0 for none                  */
  double reliable_delta; /* MIXED_RELIABLE: FP64 correction when the FP32
                            residual has dropped by this factor (0.1)         */
  int inner_prec;     /* mixed modes: applies of the inner solves, DOGIP_FP32
                         (default, CUDA cores) or DOGIP_TF32 (tensor cores;
                         nrhs 1 or a multiple of 16, atomic scatter, else
                         DOGIP_EUNSUPPORTED)                                   */
  int inner_recurrence; /* MIXED inner FP32 PCG: 0 (default) the standard
                         Hestenes-Stiefel recurrence, 4 kernels an iteration
                         (apply, p.q, x/r update, p update); 1 the same with
                         (p, K p) reduced from the element energies
                         p_T . (K_T p_T) inside the apply (3 kernels); 2 the
                         single-reduction recurrence of Chronopoulos and Gear
                         (2 kernels: s = K p by recurrence; more FP32
                         iterations).  1 and 2 need nrhs 1, FP32, atomic
                         scatter and the staged apply kernel (else
                         EUNSUPPORTED); both measured slower than 0 on GB300  */
  int single_launch;  /* FP64 PCG and the MIXED inner FP32 PCG with the standard
                         recurrence can run the iterations of a solve inside
                         one cooperative kernel (two grid-wide barriers an
                         iteration, up to min(4096, 256 check_every)
                         iterations a launch, its grid sized to the problem;
                         nrhs 1, atomic scatter, 2D p <= 3 and 3D p <= 2,
                         element-wise storage).  -1 (default): the
                         FP32 inner solves at p <= 2 whose operator and
                         vectors fit in L2 take it (FP64 PCG and 2D P3
                         measured faster per step);
                         0 never (one kernel per step, graph-captured chunks
                         of check_every iterations); 1 whenever supported,
                         FP64 included (else as 0)                          */
} dogip_solve_opts;

typedef struct {
  int status;           /* same as the return value                          */
  int iterations;       /* FP64 PCG iterations, or total inner iterations    */
  int outer;            /* refinement steps (mixed)                          */
  double rel_residual;  /* max over rhs of the final FP64 true relative residual */
  double seconds;       /* host wall time of the call                        */
} dogip_solve_info;

DOGIP_API int dogip_solve_opts_default(dogip_solve_opts* o);

/*
 * Solve K u = b (K with Dirichlet rows when on; Jacobi preconditioner from
 * A_T).  b, u: DEVICE double [n_dofs x nrhs]; nrhs in {1, 2, 4, 8, 16, 32}.
 * FP64 mode: PCG until the recursive residual reaches tol, then the true
 * residual is evaluated in FP64 (restarting from it if the recursion drifted).
 * MIXED: r = b - K u, norms and u += s d in FP64 around restarted FP32 PCG
 * solves of K d = r / s (inner_tol, inner_maxiter, max_outer).
 * MIXED_RELIABLE: one PCG recursion in FP32; whenever its residual has dropped
 * by reliable_delta, the FP32 iterate is folded into the FP64 solution and
 * r = b - K u, recomputed in FP64, replaces the FP32 residual (the search
 * direction is kept); convergence is decided on that FP64 residual.
 * rel_residual_per_rhs: host [nrhs] or NULL.  Returns ENOTCONV (u written)
 * when the limits are reached first.  Synchronises cuda_stream.
 */
DOGIP_API int dogip_solve(dogip_ctx* ctx, const double* b, double* u, int nrhs,
                const dogip_solve_opts* o, dogip_solve_info* info,
                double* rel_residual_per_rhs, void* cuda_stream);

/*
 * dogip_solve with HOST b and u (pageable or pinned): copies b in, solves,
 * copies u out, all on cuda_stream.  Same arguments and errors otherwise.
 */
DOGIP_API int dogip_solve_host(dogip_ctx* ctx, const double* b_host, double* u_host,
                     int nrhs, const dogip_solve_opts* o,
                     dogip_solve_info* info, double* rel_residual_per_rhs,
                     void* cuda_stream);

/* --------------------------------------------------------------- autotuner */
typedef struct {
  int variant[2]; /* per precision (index DOGIP_FP64 / DOGIP_FP32): 3 tensor
                     cores (FP32 only), 2 self-feeding warps, 1 staged
                     producer/consumer kernel, 0 one thread per cell           */
  int block[2];   /* cells per CTA of the one-thread-per-cell kernel          */
} dogip_tune_info;

/*
 * Choose the apply kernel of this context per precision by timing the candidates
 * on its own data: the tensor-core kernel (FP32, where an instance exists), the
 * self-feeding-warps kernel, the bulk-async staged kernel, and the
 * one-thread-per-cell kernel with 64, 128 or 256 cells per CTA (orders above the
 * compiled tables: the run-time-table kernel against the tensor cores, FP32 only):
 * the kernel alone, best of 3 CUDA-event samples of 8 back-to-back launches after 3
 * warm-up launches, atomic scatter, one right-hand side.  In FP32 the staged kernel
 * is kept unless another is faster by more than 3 % (it also carries the (p, K p)
 * reduction of the mixed solve, one kernel less per inner iteration).
 * Applies with several right-hand sides use the staged kernel where it exists
 * (FP32 with nrhs a multiple of 4 and V_T <= 10 always), and the choice otherwise;
 * prec DOGIP_TF32 selects the tensor cores whatever the choice.  Choices are cached for the process
 * per (dim, p, form, precision, log2 cells) and reused without timing unless
 * force != 0; the environment variable DOGIP_TUNE_CACHE names a text file the cache
 * is read from and appended to.  Allocates two temporary vectors (stream-ordered)
 * and synchronises cuda_stream.  info: host or NULL.  Not part of the paper.
 */
DOGIP_API int dogip_autotune(dogip_ctx* ctx, int force, dogip_tune_info* info,
                             void* cuda_stream);

/* ---------------------------------------------------------- batched solves */
/*
 * Solve nprob independent problems K_i u_i = b_i together (one right-hand side
 * each; the contexts may differ in mesh, p and form, and must share a device and
 * be distinct).  Modes DOGIP_SOLVE_FP64 and DOGIP_SOLVE_MIXED; u_i start at 0.
 * The environment variable DOGIP_BATCH_MODE picks how:
 *   concurrent (default): every problem is an ordinary dogip_solve on its own
 *     context stream, run by a pool of host threads (16, or DOGIP_BATCH_THREADS),
 *     the problems with the least estimated work first (DOGIP_BATCH_ORDER =
 *     smallest, largest or given); problems refine independently and run side
 *     by side on the GPU, with the per-step PCG kernels unless o->single_launch
 *     is 1.  Call it from one host thread at a time per set of contexts.
 *   grouped: lockstep rounds; each phase (FP64 residual, chunk of CG iterations,
 *     correction) is one CUDA graph launch for the whole batch, the inner FP32
 *     iterations one launch per kernel over (problem, block) work items; every
 *     round of inner iterations lasts until all inner solves are done.
 *   branches: as grouped, with one graph branch per problem in every phase.
 * Converged problems skip their work on the device in the lockstep modes.
 *   ctxs : host array [nprob] of contexts;  b, u : host arrays [nprob] of DEVICE
 *   double [n_i] vectors;  infos : host [nprob] or NULL -- per problem status,
 *   iterations, refinement steps, final FP64 relative residual, and `seconds` =
 *   host time from the start of the call until that problem met the tolerance.
 * Returns DOGIP_OK when every problem converged, else the first failure code.
 * Synchronises cuda_stream.  Not part of the paper (a batching service).
 */
DOGIP_API int dogip_batch_solve(dogip_ctx* const* ctxs, int nprob, const double* const* b,
                                double* const* u, const dogip_solve_opts* o,
                                dogip_solve_info* infos, void* cuda_stream);

/* ---------------------------------------------------------------- gradient */
/*
 * Gradient of the compliance-type functional J = lambda^T K(A) u with respect
 * to the element coefficients: for J = b^T u with K u = b, the adjoint gives
 * dJ/dA = -(dK/dA)[u, lambda] with lambda = u.  Per cell (caller order):
 *   elliptic, tensor : dA[T,p,q] = -sum_j om_j (grad lambda)(x_j)_p (grad u)(x_j)_q
 *   elliptic, scalar : dA[T]     = -sum_j om_j  grad lambda(x_j) . grad u(x_j)
 *   projection       : dA[T]     = -sum_j om_j  lambda(x_j) u(x_j)
 * om_j = |det R_T| w_j, x_j the W nodes (eqs. wp_dogip_mul / ep_dogip_mul with
 * the coefficient factored out).  Boundary dofs are masked as in dogip_apply.
 * u, lam: DEVICE double [n_dofs]; dA: DEVICE double [n_cells (x dim x dim)].
 * Asynchronous.
 */
DOGIP_API int dogip_grad_coef(dogip_ctx* ctx, const double* u, const double* lam,
                    double* dA, void* cuda_stream);

/*
 * Synchronise cuda_stream and report device-side failures of earlier asynchronous
 * calls on this context: DOGIP_ETIMEOUT if a bounded wait inside a kernel (the
 * copy pipelines of the staged and self-feeding applies, the copy and MMA waits of
 * the tensor-core apply) gave up; the flag is then cleared.
 */
DOGIP_API int dogip_check(dogip_ctx* ctx, void* cuda_stream);

/* ----------------------------------------------------- allocation-free norms */
/*
 * FP64 residual norms that allocate nothing.  The paper has no counterpart: this
 * is a service of the library for callers that cannot allocate device memory --
 * a framework whose allocator owns all device memory and forbids raw cudaMalloc,
 * a latency-critical loop that cannot afford cudaMalloc/cudaFree (cudaFree
 * synchronises the device), a process held to a fixed device-memory budget.
 * It computes, in FP64 with a fused grid reduction in a fixed order (the result
 * does not change from run to run),
 *     r = b - Ky,   rel[k] = ||r_k||_2 / ||b_k||_2   (0 where b_k = 0),
 * for Ky = dogip_apply(u): rel equals the relative residual dogip_solve reports to
 * within FP64 rounding (the two reductions add in different orders).
 *   b, Ky : DEVICE double [n x nrhs] (dof-major); r: DEVICE [n x nrhs] or NULL;
 *   rel   : DEVICE double [nrhs];  1 <= nrhs <= 32 (else DOGIP_EINVAL); n >= 0
 *           (b and Ky may be NULL when n = 0).
 * The arrays must be on the current device and hold the stated sizes: without a
 * context the call cannot check them.
 * No context is needed.  The reduction scratch is a fixed 128 KiB + 256 B array in
 * the library's device memory, present on every GPU that loads the library until
 * the process exits; no cudaMalloc, cudaFree or allocating library routine is
 * called.  Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress); the first lookup on a device may load the library's
 * device code there, so make the first call on each device before any stream
 * capture.  Every call shares the array and leaves it holding its last contents
 * (the ticket counter is cleared at the start of each call), so calls whose work
 * overlaps on the GPU -- on different streams, or from different host threads --
 * race with each other and must be serialised by the caller.
 * Asynchronous on cuda_stream.
 */
DOGIP_API int dogip_residual_norms_noalloc(const double* b, const double* Ky, double* r,
                                           int64_t n, int nrhs, double* rel,
                                           void* cuda_stream);

/* ------------------------------------------------------------------ errors */
DOGIP_API const char* dogip_last_error(void); /* thread-local, never NULL */
DOGIP_API int dogip_version(void);            /* major * 10000 + minor * 100 + patch */

#ifdef __cplusplus
}
#endif
#endif /* DOGIP_H */
