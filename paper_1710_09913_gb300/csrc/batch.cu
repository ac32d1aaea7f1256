// Grouped kernels of the batched mixed solve (dogip_batch_solve): one launch works on
// every problem of the batch.  A launch walks a device table of work items -- (problem,
// block of cells) for the apply, (problem, block of dofs) for the vector kernels and
// the Dirichlet rows -- so an inner CG iteration of the whole batch is seven kernels
// (the apply once per order present, the Dirichlet rows, p.q, the x/r update and the
// p update) instead of four per problem.  Reductions stay per problem: the blocks of a
// problem write their partial sums into that problem's buffer and the last of them
// (a ticket per problem) adds them in block order and updates the problem's CG
// scalars, as the single-problem kernels do.  Problems whose inner solve has stopped
// skip their blocks.
#include "kernels.cuh"

namespace dogip {

namespace {

constexpr int kBThreads = 256;
constexpr int kBDofs = kBThreads * 8;  // dofs per vector work item

// Sum of v over the block in a fixed order (warp xor-shuffles, then warps in order);
// the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
  return t;
}

// Per-problem grid reduction of NV values: every block of the problem stores its sums
// in partial[block * NV + k]; the last block (ticket) returns true with the totals in
// tot[k] (block order, deterministic).
template <int NV>
__device__ bool problem_reduce(const BProb& pr, int lb, const double (&acc)[NV], double* tot) {
  __shared__ double ws[32];
  __shared__ bool last;
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = block_sum(acc[k], ws);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) pr.partial[(size_t)lb * NV + k] = s[k];
    __threadfence();
    last = atomicAdd(pr.counter, 1u) == (unsigned)pr.nvblocks - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < pr.nvblocks; b += blockDim.x) v += __ldcg(pr.partial + (size_t)b * NV + k);
    v = block_sum(v, ws);
    if (threadIdx.x == 0) tot[k] = v;
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ void problem_flags(const BProb& pr) {
  const CGScal& s = *pr.scal;
  pr.flags[0] = s.done | s.upd;
  pr.flags[1] = s.brk;
  pr.flags[2] = s.done;
  pr.flags[3] = s.upd;
  *pr.counter = 0u;
}

// q = K p for the problems of one (dimension, order, form): one thread per cell.
template <int D, int P, int FORM>
__global__ void __launch_bounds__(kBThreads) k_batch_apply(const BProb* probs, const int2* items) {
  const int2 it = items[blockIdx.x];  // (problem, block of cells)
  const BProb& pr = probs[it.x];
  if (*pr.flags) return;
  const int64_t e = (int64_t)it.y * kBThreads + threadIdx.x;
  if (e >= pr.E) return;
  ApplyArgs<float> a{pr.A, pr.conn, pr.p, pr.q, 0, pr.E, 1, nullptr};
  apply_cell<D, P, FORM, float, true, false>(a, e, 0);
}

// Dirichlet rows q_b = p_b.
__global__ void __launch_bounds__(kBThreads) k_batch_dirichlet(const BProb* probs, const int2* items) {
  const int2 it = items[blockIdx.x];
  const BProb& pr = probs[it.x];
  if (*pr.flags) return;
  const int64_t i = (int64_t)it.y * kBThreads + threadIdx.x;
  if (i >= pr.nbnd) return;
  const int64_t d = pr.bnd[i];
  pr.q[d] = pr.p[d];
}

// alpha = rho / p.q
__global__ void __launch_bounds__(kBThreads) k_batch_pq(const BProb* probs, const int2* items) {
  const int2 it = items[blockIdx.x];
  const BProb& pr = probs[it.x];
  if (*pr.flags) return;
  const int64_t i0 = (int64_t)it.y * kBDofs, i1 = min(pr.n, i0 + kBDofs);
  float a = 0.0f;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kBThreads) a += pr.p[i] * pr.q[i];
  const double acc[1] = {(double)a};
  __shared__ double tot[1];
  if (!problem_reduce<1>(pr, it.y, acc, tot)) return;
  if (threadIdx.x == 0) {
    CGScal& s = *pr.scal;
    const double v = tot[0];
    if (s.done) {
      s.alpha = 0.0;
    } else if (!(v > 0.0) || !isfinite(v)) {
      s.brk = 1;
      s.done = 1;
      s.alpha = 0.0;
    } else {
      s.pq = v;
      s.alpha = s.rho / v;
    }
    problem_flags(pr);
  }
}

// x += alpha p, r -= alpha q, rho' = r.(Dinv r), rr = r.r; beta, convergence test
__global__ void __launch_bounds__(kBThreads) k_batch_update(const BProb* probs, const int2* items) {
  const int2 it = items[blockIdx.x];
  const BProb& pr = probs[it.x];
  if (*pr.flags) return;
  const float al = (float)pr.scal->alpha;
  const int64_t i0 = (int64_t)it.y * kBDofs, i1 = min(pr.n, i0 + kBDofs);
  float a0 = 0.0f, a1 = 0.0f;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kBThreads) {
    pr.x[i] += al * pr.p[i];
    const float ri = pr.r[i] - al * pr.q[i];
    pr.r[i] = ri;
    a0 += ri * (pr.dinv[i] * ri);
    a1 += ri * ri;
  }
  const double acc[2] = {(double)a0, (double)a1};
  __shared__ double tot[2];
  if (!problem_reduce<2>(pr, it.y, acc, tot)) return;
  if (threadIdx.x == 0) {
    CGScal& s = *pr.scal;
    if (!s.done) {
      s.beta = tot[0] / s.rho;
      s.rho_prev = s.rho;
      s.rho = tot[0];
      s.rr = tot[1];
      s.iters += 1;
      if (sqrt(tot[1]) <= s.tol * s.r0) s.done = 1;
    } else {
      s.beta = 0.0;
    }
    problem_flags(pr);
  }
}

// p = Dinv r + beta p; q = 0 for the next scatter-add apply
__global__ void __launch_bounds__(kBThreads) k_batch_pupdate(const BProb* probs, const int2* items) {
  const int2 it = items[blockIdx.x];
  const BProb& pr = probs[it.x];
  if (*pr.flags) return;
  const bool upd = !pr.scal->done;
  const float be = (float)pr.scal->beta;
  const int64_t i0 = (int64_t)it.y * kBDofs, i1 = min(pr.n, i0 + kBDofs);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kBThreads) {
    pr.q[i] = 0.0f;
    if (upd) pr.p[i] = pr.dinv[i] * pr.r[i] + be * pr.p[i];
  }
}

// The CG scalars and flags of every problem into one array (one copy to the host).
__global__ void k_batch_status(const BProb* probs, int np, CGScal* scal_out, int* flags_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  scal_out[i] = *probs[i].scal;
  for (int k = 0; k < 4; ++k) flags_out[4 * i + k] = probs[i].flags[k];
}

template <int D, int P, int FORM>
void launch_group(const BProb* probs, const int2* items, int nitems, cudaStream_t s) {
  if (nitems > 0) k_batch_apply<D, P, FORM><<<nitems, kBThreads, 0, s>>>(probs, items);
}

}  // namespace

bool batch_apply_compiled(int d, int p, int form) {
  return !(d == 3 && p > 3) && !(d == 2 && p > 4) && p >= 1 && (d == 2 || d == 3) &&
         (form == DOGIP_PROJECTION || form == DOGIP_ELLIPTIC);
}

void batch_apply_group(int d, int p, int form, const BProb* probs, const int2* items, int nitems,
                       cudaStream_t s) {
  const int key = d * 100 + p * 2 + form;
  switch (key) {
#define DOGIP_BG(D, P)                                         \
  case D * 100 + P * 2 + 0: launch_group<D, P, 0>(probs, items, nitems, s); break; \
  case D * 100 + P * 2 + 1: launch_group<D, P, 1>(probs, items, nitems, s); break;
    DOGIP_BG(2, 1) DOGIP_BG(2, 2) DOGIP_BG(2, 3) DOGIP_BG(2, 4)
    DOGIP_BG(3, 1) DOGIP_BG(3, 2) DOGIP_BG(3, 3)
#undef DOGIP_BG
    default:
      fail(DOGIP_EUNSUPPORTED, "no grouped apply for this (dim, p, form)");
  }
  cuda_check(cudaGetLastError(), "grouped apply launch");
}

void batch_vec_step(const BProb* probs, const int2* bitems, int nbitems, const int2* vitems,
                    int nvitems, cudaStream_t s) {
  if (nbitems > 0) k_batch_dirichlet<<<nbitems, kBThreads, 0, s>>>(probs, bitems);
  k_batch_pq<<<nvitems, kBThreads, 0, s>>>(probs, vitems);
  k_batch_update<<<nvitems, kBThreads, 0, s>>>(probs, vitems);
  k_batch_pupdate<<<nvitems, kBThreads, 0, s>>>(probs, vitems);
  cuda_check(cudaGetLastError(), "grouped vector kernels");
}

void batch_status(const BProb* probs, int np, CGScal* scal_out, int* flags_out, cudaStream_t s) {
  k_batch_status<<<(np + 127) / 128, 128, 0, s>>>(probs, np, scal_out, flags_out);
  cuda_check(cudaGetLastError(), "batch status kernel");
}

int64_t batch_dofs_per_item() { return kBDofs; }
int64_t batch_cells_per_item() { return kBThreads; }

}  // namespace dogip
