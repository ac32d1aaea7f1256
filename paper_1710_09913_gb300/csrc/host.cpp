// Host side of the DoGIP library: mesh topology (dof map l_T, boundary set,
// colouring), context construction, queries, the solve driver and the C ABI.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "internal.h"
#include "quad.h"

namespace dogip {

namespace {
thread_local std::string g_last_error;
}

void fail(int code, const std::string& msg) { throw Failure{code, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? DOGIP_ENOMEM : DOGIP_ECUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}

namespace {

// ---------------------------------------------------------------- hashing
// Open-addressing table from a key of up to four 64-bit words to an int32.
struct KeyTable {
  static constexpr uint64_t kEmpty = ~0ull;
  std::vector<uint64_t> keys;  // 4 words per slot
  std::vector<int32_t> vals;
  size_t mask = 0, count = 0;

  explicit KeyTable(size_t expect) { init(expect); }
  void init(size_t expect) {
    size_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    keys.assign(cap * 4, kEmpty);
    vals.assign(cap, -1);
    mask = cap - 1;
    count = 0;
  }
  static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  static uint64_t hash(const uint64_t* k) {
    return mix(k[0] ^ mix(k[1] ^ mix(k[2] ^ mix(k[3] + 0x9E3779B97F4A7C15ull))));
  }
  // Returns the value for k, inserting `fresh` if absent (then *inserted = true).
  int32_t find_or_insert(const uint64_t* k, int32_t fresh, bool* inserted) {
    if (2 * (count + 1) > mask + 1) grow();
    size_t h = hash(k) & mask;
    while (true) {
      uint64_t* s = &keys[h * 4];
      if (s[0] == kEmpty) {
        std::memcpy(s, k, 32);
        vals[h] = fresh;
        ++count;
        *inserted = true;
        return fresh;
      }
      if (s[0] == k[0] && s[1] == k[1] && s[2] == k[2] && s[3] == k[3]) {
        *inserted = false;
        return vals[h];
      }
      h = (h + 1) & mask;
    }
  }
  void grow() {
    std::vector<uint64_t> ok;
    std::vector<int32_t> ov;
    ok.swap(keys);
    ov.swap(vals);
    const size_t oldcap = ov.size();
    keys.assign(oldcap * 2 * 4, kEmpty);
    vals.assign(oldcap * 2, -1);
    mask = oldcap * 2 - 1;
    for (size_t i = 0; i < oldcap; ++i) {
      if (ok[i * 4] == kEmpty) continue;
      size_t h = hash(&ok[i * 4]) & mask;
      while (keys[h * 4] != kEmpty) h = (h + 1) & mask;
      std::memcpy(&keys[h * 4], &ok[i * 4], 32);
      vals[h] = ov[i];
    }
  }
};

// Multi-indices |alpha| <= q in product order (last coordinate fastest).
std::vector<std::vector<int>> multi_indices(int d, int q) {
  std::vector<std::vector<int>> out;
  std::vector<int> a(d, 0);
  int lim = q + 1, tot = 1;
  for (int i = 0; i < d; ++i) tot *= lim;
  for (int c = 0; c < tot; ++c) {
    int t = c, s = 0;
    for (int i = d - 1; i >= 0; --i) {
      a[i] = t % lim;
      t /= lim;
      s += a[i];
    }
    if (s <= q) out.push_back(a);
  }
  return out;
}

// Barycentric multi-indices (p - |alpha|, alpha) of the local P_p nodes.
std::vector<std::vector<int>> local_betas(int d, int p) {
  std::vector<std::vector<int>> out;
  for (auto& a : multi_indices(d, p)) {
    std::vector<int> b(d + 1);
    int s = 0;
    for (int i = 0; i < d; ++i) {
      b[i + 1] = a[i];
      s += a[i];
    }
    b[0] = p - s;
    out.push_back(b);
  }
  return out;
}

// Node numbering by first appearance: node identity = multiset {(v_i, beta_i): beta_i > 0}
// of the order-q nodes; ids[e * V_q + l]; first[...] = 1 where the cell introduces the node.
int64_t number_nodes(int d, int q, int64_t E, const int32_t* cells, std::vector<int32_t>& ids,
                     std::vector<uint8_t>* first) {
  auto betas = local_betas(d, q);
  const int V = (int)betas.size();
  ids.assign((size_t)E * V, 0);
  if (first) first->assign((size_t)E * V, 0);
  KeyTable tab((size_t)E * V / 2 + 64);
  int32_t next = 0;
  uint64_t key[4];
  std::pair<uint64_t, int> pr[4];
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* cv = cells + e * (d + 1);
    for (int l = 0; l < V; ++l) {
      int m = 0;
      for (int i = 0; i <= d; ++i)
        if (betas[l][i] > 0) pr[m++] = {(uint64_t)(uint32_t)cv[i], betas[l][i]};
      std::sort(pr, pr + m);
      for (int k = 0; k < 4; ++k) key[k] = k < m ? ((pr[k].first << 8) | (uint64_t)pr[k].second) : KeyTable::kEmpty - 1;
      bool ins = false;
      const int32_t id = tab.find_or_insert(key, next, &ins);
      if (ins) {
        if (next == (int32_t)kIdMask) fail(DOGIP_EINVAL, "too many nodes (>= 2^30)");
        ++next;
        if (first) (*first)[(size_t)e * V + l] = 1;
      }
      ids[(size_t)e * V + l] = id;
    }
  }
  return next;
}

void build_dofmap(Ctx& c, const int32_t* cells) {
  c.n = number_nodes(c.d, c.p, c.E, cells, c.dofmap, nullptr);
}

// Boundary dofs: nodes with beta_i = 0 for a local facet i (opposite vertex i)
// that belongs to exactly one cell.
void build_boundary(Ctx& c, const int32_t* cells) {
  const int d = c.d, V = c.VT;
  auto betas = local_betas(d, c.p);
  c.bmask.assign(c.n, 0);
  if (!c.dirichlet) return;
  KeyTable tab((size_t)c.E * (d + 1) / 2 + 64);
  std::vector<int32_t> fid((size_t)c.E * (d + 1));
  std::vector<int32_t> cnt;
  uint64_t key[4];
  for (int64_t e = 0; e < c.E; ++e) {
    const int32_t* cv = cells + e * (d + 1);
    for (int i = 0; i <= d; ++i) {
      uint64_t f[3];
      int m = 0;
      for (int k = 0; k <= d; ++k)
        if (k != i) f[m++] = (uint64_t)(uint32_t)cv[k];
      std::sort(f, f + m);
      for (int k = 0; k < 4; ++k) key[k] = k < m ? f[k] : KeyTable::kEmpty - 1;
      bool ins = false;
      const int32_t id = tab.find_or_insert(key, (int32_t)cnt.size(), &ins);
      if (ins) cnt.push_back(0);
      cnt[id] += 1;
      fid[(size_t)e * (d + 1) + i] = id;
    }
  }
  for (int64_t e = 0; e < c.E; ++e)
    for (int i = 0; i <= d; ++i)
      if (cnt[fid[(size_t)e * (d + 1) + i]] == 1)
        for (int l = 0; l < V; ++l)
          if (betas[l][i] == 0) c.bmask[c.dofmap[(size_t)e * V + l]] = 1;
}

// Greedy colouring: cells in order take the smallest colour not used by an
// earlier cell sharing a vertex.
void build_colouring(Ctx& c, const int32_t* cells) {
  const int d = c.d;
  std::vector<int64_t> start(c.nv + 1, 0);
  for (int64_t k = 0; k < c.E * (d + 1); ++k) start[cells[k] + 1]++;
  for (int64_t v = 0; v < c.nv; ++v) start[v + 1] += start[v];
  std::vector<int32_t> inc(c.E * (d + 1));
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t e = 0; e < c.E; ++e)
    for (int i = 0; i <= d; ++i) inc[fill[cells[e * (d + 1) + i]]++] = (int32_t)e;
  c.colour.assign(c.E, -1);
  std::vector<int64_t> stamp(64, -1);
  int ncol = 0;
  for (int64_t e = 0; e < c.E; ++e) {
    for (int i = 0; i <= d; ++i) {
      const int32_t v = cells[e * (d + 1) + i];
      for (int64_t k = start[v]; k < start[v + 1]; ++k) {
        const int32_t f = inc[k];
        if (f >= e) break;  // incidence lists are in increasing cell order
        const int cf = c.colour[f];
        if (cf >= (int)stamp.size()) stamp.resize(cf * 2 + 1, -1);
        stamp[cf] = e;
      }
    }
    int col = 0;
    while (col < (int)stamp.size() && stamp[col] == e) ++col;
    if (col >= (int)stamp.size()) stamp.resize(col * 2 + 1, -1);
    c.colour[e] = col;
    ncol = std::max(ncol, col + 1);
  }
  c.ncolours = ncol;
}

template <typename T>
T* dev_alloc(size_t count) {
  if (count == 0) count = 1;
  T* p = nullptr;
  if (cudaMalloc((void**)&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "device allocation failed");
  }
  return p;
}

void free_ctx(Ctx* c) {
  if (!c) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  vec_free(c->work);
  for (void* p : {(void*)c->d_coords, (void*)c->d_cells, (void*)c->d_perm, (void*)c->d_conn,
                  (void*)c->d_A64, (void*)c->d_A32, (void*)c->d_geo, (void*)c->d_diag,
                  (void*)c->d_dinv64, (void*)c->d_dinv32, (void*)c->d_bnd, (void*)c->d_coef,
                  (void*)c->d_qp64, (void*)c->d_qp32, (void*)c->d_err, (void*)c->d_kerr,
                  (void*)c->d_connW, (void*)c->d_Aw64, (void*)c->d_Aw32, (void*)c->d_w64,
                  (void*)c->d_w32, (void*)c->d_hiB64, (void*)c->d_hiB32, (void*)c->d_hiW,
                  (void*)c->d_hiIV})
    if (p) cudaFree(p);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  cudaSetDevice(cur);
  delete c;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cuda_check(cudaSetDevice(dev), "cudaSetDevice");
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace
void ensure_w_scratch(Ctx& c, int R) {
  if (!c.global_w || R <= c.w_cap) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cuda_check(cudaStreamIsCapturing(c.stream, &cs), "capture status");
  if (cs != cudaStreamCaptureStatusNone) fail(DOGIP_EINVAL, "global double-grid scratch grows during capture");
  cuda_check(cudaStreamSynchronize(c.stream), "scratch sync");
  if (c.d_w64) cudaFree(c.d_w64);
  if (c.d_w32) cudaFree(c.d_w32);
  c.d_w64 = nullptr;
  c.d_w32 = nullptr;
  c.d_w64 = dev_alloc<double>((size_t)c.nW * R);
  c.d_w32 = dev_alloc<float>((size_t)c.nW * R);
  c.w_cap = R;
}
namespace {

void check_coef_status(Ctx& c, cudaStream_t s) {
  int err = 0;
  cuda_check(cudaMemcpyAsync(&err, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "read flags");
  cuda_check(cudaStreamSynchronize(s), "setup kernels");
  if (err) {
    std::string m = "invalid input:";
    if (err & kErrGeometry) m += " degenerate or non-finite cell;";
    if (err & kErrNonFinite) m += " non-finite coefficient;";
    if (err & kErrSymmetry) m += " non-symmetric coefficient tensor;";
    if (err & kErrNotPos) m += " coefficient not positive (definite);";
    fail(DOGIP_EINVAL, m);
  }
}

Ctx* setup(const dogip_mesh* m, int p, int form, int coef_kind, const double* coef,
           const dogip_opts* opts) {
  if (!m || !coef) fail(DOGIP_EINVAL, "mesh and coefficients are required");
  if (m->dim != 2 && m->dim != 3) fail(DOGIP_EINVAL, "dim must be 2 or 3");
  if (form != DOGIP_PROJECTION && form != DOGIP_ELLIPTIC) fail(DOGIP_EINVAL, "unknown form");
  if (coef_kind != DOGIP_COEF_ELEM_SCALAR && coef_kind != DOGIP_COEF_ELEM_TENSOR)
    fail(DOGIP_EINVAL, "unknown coefficient kind");
  if (form == DOGIP_PROJECTION && coef_kind != DOGIP_COEF_ELEM_SCALAR)
    fail(DOGIP_EINVAL, "the weighted projection takes a scalar coefficient");
  if (m->n_vertices <= 0 || m->n_cells <= 0 || !m->coords || !m->cells)
    fail(DOGIP_EINVAL, "empty mesh");
  if (m->n_vertices >= (int64_t)1 << 31) fail(DOGIP_EINVAL, "too many vertices");
  if (p < 1) fail(DOGIP_EINVAL, "p must be >= 1");
  dogip_opts o;
  dogip_opts_default(&o);
  if (opts) o = *opts;
  int NB, W, V;
  long long nnz, nnz1;
  if (!table_info(m->dim, p, form, &NB, &W, &V, &nnz, &nnz1))
    fail(DOGIP_EUNSUPPORTED, "p outside the built range (2D 1..8, 3D 1..4)");
  const int d = m->dim;
  for (int64_t k = 0; k < m->n_cells * (d + 1); ++k)
    if (m->cells[k] < 0 || m->cells[k] >= m->n_vertices)
      fail(DOGIP_EINVAL, "cell vertex id out of range");
  for (int64_t k = 0; k < m->n_vertices * d; ++k)
    if (!std::isfinite(m->coords[k])) fail(DOGIP_EINVAL, "non-finite vertex coordinate");

  int dev = o.device;
  if (dev < 0) cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  DeviceGuard guard(dev);

  Ctx* c = new Ctx();  // Ctx is the ABI's dogip_ctx
  try {
    c->device = dev;
    c->d = d;
    c->p = p;
    c->form = form;
    c->coef_kind = coef_kind;
    c->NB = NB;
    c->WT = W;
    c->VT = V;
    c->NS = form == DOGIP_ELLIPTIC ? d * (d + 1) / 2 : 1;
    c->nnzb = nnz;
    c->nnzb1 = nnz1;
    c->dirichlet = o.dirichlet < 0 ? form == DOGIP_ELLIPTIC : o.dirichlet != 0;
    c->scatter = o.scatter == DOGIP_SCATTER_COLOUR ? DOGIP_SCATTER_COLOUR : DOGIP_SCATTER_ATOMIC;
    c->keep32 = o.keep_fp32 != 0;
    c->factorized = o.factorized != 0;
    if (c->factorized && c->scatter == DOGIP_SCATTER_COLOUR)
      fail(DOGIP_EINVAL, "factorized storage needs atomic scatter");
    c->hi = !table_is_compiled(d, p, form);
    if (c->hi && c->factorized) fail(DOGIP_EUNSUPPORTED, "factorized storage is built for p <= 4 (3D: 3)");
    c->global_w = o.global_w != 0;
    if (c->hi && c->global_w) fail(DOGIP_EUNSUPPORTED, "the global double grid is built for p <= 4 (3D: 3)");
    if (c->global_w) {
      if (form != DOGIP_PROJECTION) fail(DOGIP_EINVAL, "the global double grid is for the projection");
      if (c->factorized || c->scatter == DOGIP_SCATTER_COLOUR || c->dirichlet)
        fail(DOGIP_EINVAL, "the global double grid needs factorized = 0, atomic scatter, no Dirichlet rows");
    }
    c->E = m->n_cells;
    c->Epad = (c->E + kTile - 1) / kTile * kTile;
    c->nv = m->n_vertices;

    build_dofmap(*c, m->cells);
    if (c->global_w) c->nW = number_nodes(d, 2 * p, c->E, m->cells, c->wdofmap, &c->wowner);
    build_boundary(*c, m->cells);
    build_colouring(*c, m->cells);

    // processing order: colour-sorted (stable) for colour scatter, else identity
    c->perm.resize(c->E);
    std::iota(c->perm.begin(), c->perm.end(), 0);
    if (c->scatter == DOGIP_SCATTER_COLOUR) {
      std::stable_sort(c->perm.begin(), c->perm.end(),
                       [&](int64_t a, int64_t b) { return c->colour[a] < c->colour[b]; });
      c->colour_start.assign(c->ncolours + 1, 0);
      for (int64_t e = 0; e < c->E; ++e) c->colour_start[c->colour[e] + 1]++;
      for (int k = 0; k < c->ncolours; ++k) c->colour_start[k + 1] += c->colour_start[k];
    } else {
      c->colour_start = {0, c->E};
    }

    std::vector<int32_t> bnd;
    for (int64_t i = 0; i < c->n; ++i)
      if (c->bmask[i]) bnd.push_back((int32_t)i);
    c->nbnd = (int64_t)bnd.size();

    std::vector<uint32_t> conn((size_t)c->Epad * V, 0u);
    std::vector<int32_t> pcells((size_t)c->E * (d + 1));
    for (int64_t pos = 0; pos < c->E; ++pos) {
      const int64_t e = c->perm[pos];
      for (int l = 0; l < V; ++l) {
        const int32_t id = c->dofmap[(size_t)e * V + l];
        conn[(size_t)(pos / kTile) * V * kTile + (size_t)l * kTile + pos % kTile] =
            (uint32_t)id | (c->bmask[id] ? kBndBit : 0u);
      }
      for (int i = 0; i <= d; ++i) pcells[(size_t)pos * (d + 1) + i] = m->cells[e * (d + 1) + i];
    }

    cuda_check(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
    cuda_check(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "event");
    cuda_check(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming), "event");
    const size_t ncoef = (size_t)c->E * (coef_kind == DOGIP_COEF_ELEM_TENSOR ? d * d : 1);
    c->d_coords = dev_alloc<double>((size_t)c->nv * d);
    c->d_cells = dev_alloc<int32_t>(pcells.size());
    c->d_perm = dev_alloc<int64_t>(c->E);
    c->d_conn = dev_alloc<uint32_t>(conn.size());
    const size_t nA = c->global_w ? 0 : (size_t)c->Epad * (c->factorized ? 1 : W) * c->NS;
    if (nA) c->d_A64 = dev_alloc<double>(nA);
    if (nA && c->keep32) c->d_A32 = dev_alloc<float>(nA);
    std::vector<uint32_t> connW;
    if (c->global_w) {
      connW.assign((size_t)c->Epad * W, 0u);
      for (int64_t e = 0; e < c->E; ++e)  // processing order = caller order (atomic scatter)
        for (int j = 0; j < W; ++j)
          connW[(size_t)(e / kTile) * W * kTile + (size_t)j * kTile + e % kTile] =
              (uint32_t)c->wdofmap[(size_t)e * W + j] | (c->wowner[(size_t)e * W + j] ? kBndBit : 0u);
      c->d_connW = dev_alloc<uint32_t>(connW.size());
      c->d_Aw64 = dev_alloc<double>(c->nW);
      if (c->keep32) c->d_Aw32 = dev_alloc<float>(c->nW);
      ensure_w_scratch(*c, 1);
    }
    c->d_geo = dev_alloc<double>((size_t)c->E * (d * d + 1));
    c->d_diag = dev_alloc<double>(c->n);
    c->d_dinv64 = dev_alloc<double>(c->n);
    c->d_dinv32 = dev_alloc<float>(c->n);
    c->d_bnd = dev_alloc<int32_t>(bnd.size());
    c->d_coef = dev_alloc<double>(ncoef);
    c->d_qp64 = dev_alloc<double>((size_t)c->E * c->NS);
    if (c->keep32) c->d_qp32 = dev_alloc<float>((size_t)c->E * c->NS);
    c->d_err = dev_alloc<int>(1);
    c->d_kerr = dev_alloc<int>(1);
    {
      int l2 = 0;
      cuda_check(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device), "L2 size");
      c->l2_bytes = l2;
    }
    if (const char* v = std::getenv("DOGIP_APPLY_VARIANT")) c->apply_variant = std::atoi(v);
    if (const char* v = std::getenv("DOGIP_GRAPH_PDL")) c->graph_pdl = std::atoi(v) != 0;
    // Test hooks for the device-side failure path: a shorter wait budget, and one
    // chunk of the staged apply whose copy is never issued, so that its bounded
    // wait expires (nothing faults or hangs; the kernel reports and returns).
    if (const char* v = std::getenv("DOGIP_TEST_WAIT_CYCLES")) c->wait_budget = std::atoll(v);
    if (const char* v = std::getenv("DOGIP_TEST_SKIP_CHUNK")) c->test_skip_chunk = std::atoll(v);
    cudaStream_t s = c->stream;
    cuda_check(cudaMemcpyAsync(c->d_coords, m->coords, sizeof(double) * c->nv * d,
                               cudaMemcpyHostToDevice, s), "upload coords");
    cuda_check(cudaMemcpyAsync(c->d_cells, pcells.data(), sizeof(int32_t) * pcells.size(),
                               cudaMemcpyHostToDevice, s), "upload cells");
    cuda_check(cudaMemcpyAsync(c->d_perm, c->perm.data(), sizeof(int64_t) * c->E,
                               cudaMemcpyHostToDevice, s), "upload perm");
    cuda_check(cudaMemcpyAsync(c->d_conn, conn.data(), sizeof(uint32_t) * conn.size(),
                               cudaMemcpyHostToDevice, s), "upload conn");
    if (!bnd.empty())
      cuda_check(cudaMemcpyAsync(c->d_bnd, bnd.data(), sizeof(int32_t) * bnd.size(),
                                 cudaMemcpyHostToDevice, s), "upload boundary");
    cuda_check(cudaMemcpyAsync(c->d_coef, coef, sizeof(double) * ncoef, cudaMemcpyHostToDevice, s),
               "upload coefficients");
    // padding of A_T stays zero
    if (nA) cuda_check(cudaMemsetAsync(c->d_A64, 0, sizeof(double) * nA, s), "memset A");
    if (nA && c->keep32) cuda_check(cudaMemsetAsync(c->d_A32, 0, sizeof(float) * nA, s), "memset A32");
    if (c->global_w)
      cuda_check(cudaMemcpyAsync(c->d_connW, connW.data(), sizeof(uint32_t) * connW.size(),
                                 cudaMemcpyHostToDevice, s), "upload W nodes");
    std::vector<float> hiB32;
    if (c->hi) {  // run-time reference tables of the higher orders
      const double *hB, *hw, *hiv;
      hi_table(d, p, form, nullptr, nullptr, nullptr, nullptr, nullptr, &hB, &hw, &hiv);
      const size_t nb = (size_t)NB * W * V;
      c->d_hiB64 = dev_alloc<double>(nb);
      c->d_hiB32 = dev_alloc<float>(nb);
      c->d_hiW = dev_alloc<double>(W);
      c->d_hiIV = dev_alloc<double>(V);
      hiB32.assign(hB, hB + nb);
      cuda_check(cudaMemcpyAsync(c->d_hiB64, hB, sizeof(double) * nb, cudaMemcpyHostToDevice, s),
                 "upload tables");
      cuda_check(cudaMemcpyAsync(c->d_hiB32, hiB32.data(), sizeof(float) * nb,
                                 cudaMemcpyHostToDevice, s), "upload tables");
      cuda_check(cudaMemcpyAsync(c->d_hiW, hw, sizeof(double) * W, cudaMemcpyHostToDevice, s),
                 "upload tables");
      cuda_check(cudaMemcpyAsync(c->d_hiIV, hiv, sizeof(double) * V, cudaMemcpyHostToDevice, s),
                 "upload tables");
    }
    cuda_check(cudaMemsetAsync(c->d_err, 0, sizeof(int), s), "memset err");
    cuda_check(cudaMemsetAsync(c->d_kerr, 0, sizeof(int), s), "memset kernel err");
    launch_ahat(*c, c->d_coef, coef_kind, s);
    check_coef_status(*c, s);
    c->qp_ok = !c->hi;
    prepare_apply(*c);
  } catch (...) {
    free_ctx(c);
    throw;
  }
  return c;
}

void set_coef(Ctx& c, int coef_kind, const double* coef, cudaStream_t s) {
  if (!coef) fail(DOGIP_EINVAL, "coefficients are required");
  if (c.form == DOGIP_PROJECTION && coef_kind != DOGIP_COEF_ELEM_SCALAR)
    fail(DOGIP_EINVAL, "the weighted projection takes a scalar coefficient");
  if (coef_kind != DOGIP_COEF_ELEM_SCALAR && coef_kind != DOGIP_COEF_ELEM_TENSOR)
    fail(DOGIP_EINVAL, "unknown coefficient kind");
  DeviceGuard guard(c.device);
  c.coef_kind = coef_kind;
  cuda_check(cudaMemsetAsync(c.d_err, 0, sizeof(int), s), "memset err");
  launch_ahat(c, coef, coef_kind, s);
  check_coef_status(c, s);
  c.qp_ok = !c.hi;
}


// Equispaced Lagrange basis of degree q (Silvester's product form) at a reference
// point, in double precision: phi_beta = prod_i prod_{m < beta_i} (q lambda_i - m)/(m+1).
void w_basis_at(int d, int q, const double* x, std::vector<double>& out) {
  out.clear();
  if (q == 0) {
    out.push_back(1.0);
    return;
  }
  double lam[4];
  lam[0] = 1.0;
  for (int i = 0; i < d; ++i) {
    lam[i + 1] = x[i];
    lam[0] -= x[i];
  }
  for (auto& beta : local_betas(d, q)) {
    double v = 1.0;
    for (int i = 0; i <= d; ++i)
      for (int m = 0; m < beta[i]; ++m) v *= (q * lam[i] - m) / (m + 1);
    out.push_back(v);
  }
}

void set_coef_inclusions(Ctx& c, int nb, const double* centres, const double* radii, double inside,
                         double outside, int nq, cudaStream_t s) {
  if (c.factorized) fail(DOGIP_EINVAL, "sub-element integration needs per-node storage (factorized = 0)");
  if (c.global_w) fail(DOGIP_EUNSUPPORTED, "sub-element integration is not built for the global double grid");
  if (c.hi) fail(DOGIP_EUNSUPPORTED, "sub-element integration is built for p <= 4 (3D: 3)");
  if (nb < 0 || (nb > 0 && (!centres || !radii))) fail(DOGIP_EINVAL, "inclusion arrays required");
  if (nq < 1 || nq > 16) fail(DOGIP_EINVAL, "points per direction must be in 1..16");
  if (!(inside > 0.0) || !(outside > 0.0) || !std::isfinite(inside) || !std::isfinite(outside))
    fail(DOGIP_EINVAL, "coefficient values must be positive and finite");
  for (int b = 0; b < nb; ++b) {
    if (!(radii[b] > 0.0) || !std::isfinite(radii[b])) fail(DOGIP_EINVAL, "radii must be positive");
    for (int k = 0; k < c.d; ++k)
      if (!std::isfinite(centres[b * c.d + k])) fail(DOGIP_EINVAL, "non-finite inclusion centre");
  }
  DeviceGuard guard(c.device);
  c.qp_ok = false;  // the comparator's per-cell coefficient no longer describes the field
  std::vector<double> pts, wts;
  simplex_rule(c.d, nq, pts, wts);
  const int q = c.form == DOGIP_PROJECTION ? 2 * c.p : 2 * c.p - 2;
  const int NQ = (int)wts.size();
  std::vector<double> phi((size_t)NQ * c.WT), row;
  for (int i = 0; i < NQ; ++i) {
    w_basis_at(c.d, q, &pts[(size_t)i * c.d], row);
    for (int j = 0; j < c.WT; ++j) phi[(size_t)i * c.WT + j] = row[j];
  }
  // one staging buffer (stream-ordered) for points, weights, table, balls
  const size_t n_total = pts.size() + wts.size() + phi.size() + (size_t)nb * c.d + nb;
  double* buf = nullptr;
  cuda_check(cudaMallocAsync((void**)&buf, sizeof(double) * std::max<size_t>(n_total, 1), s),
             "quadrature staging");
  std::vector<double> host;
  host.reserve(n_total);
  host.insert(host.end(), pts.begin(), pts.end());
  host.insert(host.end(), wts.begin(), wts.end());
  host.insert(host.end(), phi.begin(), phi.end());
  host.insert(host.end(), centres, centres + (size_t)nb * c.d);
  host.insert(host.end(), radii, radii + nb);
  QuadCoef qc;
  qc.pts = buf;
  qc.wts = buf + pts.size();
  qc.phi = qc.wts + wts.size();
  qc.nq = NQ;
  qc.centres = qc.phi + phi.size();
  qc.radii = qc.centres + (size_t)nb * c.d;
  qc.nb = nb;
  qc.inside = inside;
  qc.outside = outside;
  try {
    cuda_check(cudaMemcpyAsync(buf, host.data(), sizeof(double) * n_total, cudaMemcpyHostToDevice, s),
               "quadrature upload");
    cuda_check(cudaMemsetAsync(c.d_err, 0, sizeof(int), s), "memset err");
    launch_ahat_quad(c, qc, s);
    cuda_check(cudaFreeAsync(buf, s), "quadrature staging free");
  } catch (...) {
    cudaFreeAsync(buf, s);
    throw;
  }
  check_coef_status(c, s);
  c.coef_kind = DOGIP_COEF_INCLUSIONS;
}

// ------------------------------------------------------------------- solve

bool r_ok(int R) { return R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32; }

// Turn every edge of g between two marked kernel nodes into a programmatic dependency
// (the downstream kernel is launched once all blocks of the upstream one have started,
// and waits inside for its completion); returns the number of edges changed.
int make_programmatic_edges(cudaGraph_t g) {
  size_t ne = 0;
  cuda_check(cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne), "graph edges");
  if (ne == 0) return 0;
  std::vector<cudaGraphNode_t> from(ne), to(ne);
  std::vector<cudaGraphEdgeData> ed(ne);
  cuda_check(cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &ne), "graph edges");
  auto marked_kernel = [](cudaGraphNode_t nd) {
    cudaGraphNodeType ty;
    cuda_check(cudaGraphNodeGetType(nd, &ty), "graph node type");
    if (ty != cudaGraphNodeTypeKernel) return false;
    cudaKernelNodeParams kp{};
    cuda_check(cudaGraphKernelNodeGetParams(nd, &kp), "kernel node params");
    return pdl_marked(kp.func);
  };
  int changed = 0;
  for (size_t i = 0; i < ne; ++i) {
    if (ed[i].type != cudaGraphDependencyTypeDefault || ed[i].from_port != 0) continue;
    if (!marked_kernel(from[i]) || !marked_kernel(to[i])) continue;
    cuda_check(cudaGraphRemoveDependencies(g, &from[i], &to[i], &ed[i], 1), "remove edge");
    cudaGraphEdgeData pe{};
    pe.from_port = cudaGraphKernelNodePortProgrammatic;
    pe.type = cudaGraphDependencyTypeProgrammatic;
    cuda_check(cudaGraphAddDependencies(g, &from[i], &to[i], &pe, 1), "programmatic edge");
    ++changed;
  }
  return changed;
}

// One chunk of `k` CG iterations on the solver stream, captured once as a CUDA
// graph and replayed; ends with a copy of the flags and scalars to pinned host.
// rec (FP32, one right-hand side): 0 the standard recurrence in four kernels (apply,
// p.q, x/r update, p update); 1 the same with p.Kp reduced from the element energies
// inside the apply (three kernels); 2 the single-reduction recurrence of Chronopoulos
// and Gear (two kernels: vec_cgcg_step, then the apply with the energy reduction).
void run_chunk(Ctx& c, int prec, int scatter, double* x64, int k, double delta, int rec = 0) {
  SolveWork& w = c.work;
  cudaStream_t s = c.stream;
  const void* key0 = prec == DOGIP_FP64 ? (const void*)x64 : (const void*)w.x32;
  const bool hit = w.graph && w.graph_prec == prec && w.graph_scatter == scatter &&
                   w.graph_chunk == k && w.graph_key[0] == key0 && w.graph_key[1] == (void*)w.p64 &&
                   w.graph_delta == delta && w.graph_fused == rec;
  if (!hit) {
    if (w.graph) cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
    const int64_t launches_before = c.launches;  // captured launches run only on replay
    cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    try {
      const void* dinv = prec == DOGIP_FP64 ? (const void*)c.d_dinv64 : (const void*)c.d_dinv32;
      for (int it = 0; it < k && rec == 2; ++it) {
        c.launches += vec_cgcg_step(w, c.d_dinv32, s);
        launch_apply_energy(c, w.p32, w.q32, s, w, 1);
      }
      for (int it = 0; it < k && rec == 1; ++it) {
        launch_apply_energy(c, w.p32, w.q32, s, w, 0);  // q = K p, alpha = rho / (p, K p)
        c.launches += vec_cg_step(w, DOGIP_FP32, x64, dinv, delta, s, true, false);
      }
      for (int it = 0; it < k && rec == 0; ++it) {
        if (prec == DOGIP_FP64) launch_apply_cg(c, w.p64, w.q64, w.R, DOGIP_FP64, scatter, s, w);
        else launch_apply_cg(c, w.p32, w.q32, w.R, prec, scatter, s, w);  // FP32 or TF32 apply
        c.launches += vec_cg_step(w, prec == DOGIP_FP64 ? DOGIP_FP64 : DOGIP_FP32, x64, dinv, delta,
                                  s, scatter == DOGIP_SCATTER_ATOMIC);
      }
      cuda_check(cudaMemcpyAsync(w.h_flags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s),
                 "flags copy");
      cuda_check(cudaMemcpyAsync(w.h_flags + 4, c.d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s),
                 "kernel flag copy");
      cuda_check(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(CGScal) * w.R, cudaMemcpyDeviceToHost, s),
                 "scal copy");
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    c.launches = launches_before;
    cudaGraph_t g = nullptr;
    cuda_check(cudaStreamEndCapture(s, &g), "end capture");
    try {
      if (c.graph_pdl) make_programmatic_edges(g);
    } catch (...) {
      cudaGraphDestroy(g);
      throw;
    }
    size_t nn = 0;
    cuda_check(cudaGraphGetNodes(g, nullptr, &nn), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(nn);
    cuda_check(cudaGraphGetNodes(g, nodes.data(), &nn), "graph nodes");
    w.graph_kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cuda_check(cudaGraphNodeGetType(nd, &ty), "graph node type");
      if (ty == cudaGraphNodeTypeKernel) ++w.graph_kernels;
    }
    cudaError_t e = cudaGraphInstantiate(&w.graph, g, 0);
    cudaGraphDestroy(g);
    cuda_check(e, "graph instantiate");
    w.graph_prec = prec;
    w.graph_scatter = scatter;
    w.graph_chunk = k;
    w.graph_delta = delta;
    w.graph_fused = rec;
    w.graph_key[0] = key0;
    w.graph_key[1] = w.p64;
  }
  cuda_check(cudaGraphLaunch(w.graph, s), "graph launch");
  c.launches += w.graph_kernels;
  cuda_check(cudaStreamSynchronize(s), "cg chunk");
  if (w.h_flags[4]) fail(DOGIP_ETIMEOUT, "a bounded wait inside a kernel expired");
}

void read_scal(Ctx& c) {
  SolveWork& w = c.work;
  cuda_check(cudaMemcpyAsync(w.h_scal, w.scal, sizeof(CGScal) * w.R, cudaMemcpyDeviceToHost, c.stream),
             "scal copy");
  cuda_check(cudaMemcpyAsync(w.h_flags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, c.stream),
             "flags copy");
  cuda_check(cudaStreamSynchronize(c.stream), "scal sync");
}

int solve(Ctx& c, const double* b, double* u, int R, const dogip_solve_opts* opts,
          dogip_solve_info* info, double* rel_out, cudaStream_t user) {
  const auto t0 = std::chrono::steady_clock::now();
  dogip_solve_opts o;
  dogip_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!b || !u) fail(DOGIP_EINVAL, "b and u are required");
  if (!r_ok(R)) fail(DOGIP_EINVAL, "nrhs must be 1, 2, 4, 8, 16 or 32 for solves");
  if (o.mode != DOGIP_SOLVE_FP64 && o.mode != DOGIP_SOLVE_MIXED && o.mode != DOGIP_SOLVE_MIXED_RELIABLE)
    fail(DOGIP_EINVAL, "unknown mode");
  if (o.mode != DOGIP_SOLVE_FP64 && !c.keep32) fail(DOGIP_EINVAL, "mixed modes need keep_fp32");
  if (o.mode == DOGIP_SOLVE_MIXED_RELIABLE && !(o.reliable_delta > 0.0 && o.reliable_delta < 1.0))
    fail(DOGIP_EINVAL, "reliable_delta must lie in (0, 1)");
  if (!(o.tol > 0.0)) fail(DOGIP_EINVAL, "tol must be positive");
  int scatter = o.scatter < 0 ? c.scatter : o.scatter;
  if (scatter == DOGIP_SCATTER_COLOUR && c.scatter != DOGIP_SCATTER_COLOUR)
    fail(DOGIP_EINVAL, "colour scatter needs a context set up with scatter = COLOUR");
  if (o.inner_prec != DOGIP_FP32 && o.inner_prec != DOGIP_TF32)
    fail(DOGIP_EINVAL, "inner_prec must be DOGIP_FP32 or DOGIP_TF32");
  const int ip = o.mode == DOGIP_SOLVE_FP64 ? DOGIP_FP64 : o.inner_prec;  // inner apply
  if (o.inner_recurrence < 0 || o.inner_recurrence > 2)
    fail(DOGIP_EINVAL, "inner_recurrence must be 0, 1 or 2");
  // inner FP32 recurrence of the mixed mode (run_chunk's rec)
  const bool fusable = o.mode == DOGIP_SOLVE_MIXED && cgcg_eligible(c, R, ip, scatter);
  const int rec = o.mode == DOGIP_SOLVE_MIXED ? o.inner_recurrence : 0;
  if (rec != 0 && !fusable)
    fail(DOGIP_EUNSUPPORTED,
         "the fused (p, K p) and single-reduction inner recurrences need one right-hand side, "
         "FP32 inner applies, atomic scatter and the staged apply kernel");
  if (ip == DOGIP_TF32 && ((R != 1 && R % 16 != 0) || scatter != DOGIP_SCATTER_ATOMIC ||
                           c.global_w || c.factorized || !apply_tc_available(c.d, c.p, c.form)))
    fail(DOGIP_EUNSUPPORTED,
         "TF32 inner applies need 1 or a multiple of 16 right-hand sides, atomic scatter and a "
         "tensor-core instance");
  const int chunk = std::max(1, o.check_every);
  DeviceGuard guard(c.device);
  ensure_w_scratch(c, R);
  vec_alloc(c.work, c.n, R);
  SolveWork& w = c.work;
  cudaStream_t s = c.stream;
  // The PCG iterations (FP64 mode, or the standard FP32 inner recurrence of MIXED) in
  // one cooperative launch when the problem stays in L2: its iteration cost is then
  // latency, which the kernel boundaries of the graph-captured chunks would dominate.
  // By default only the FP32 inner solves at p <= 2 take it: measured on GB300 (2D P1
  // and P2 on 512 x 512 squares, 3D P1 and P2 on 32^3 cubes) it is faster there; at
  // 2D P3 (128 x 128 squares) it was 4 % slower, and FP64 PCG, whose one-thread-per-
  // cell apply is bound by the FP64 rate, is faster with the per-step kernels.
  const int cg_prec = o.mode == DOGIP_SOLVE_FP64 ? DOGIP_FP64 : DOGIP_FP32;
  bool single = false;
  if (o.single_launch != 0 && R == 1 && scatter == DOGIP_SCATTER_ATOMIC && rec == 0 &&
      o.mode != DOGIP_SOLVE_MIXED_RELIABLE && (o.mode == DOGIP_SOLVE_FP64 || ip == DOGIP_FP32) &&
      pcg_small_supported(c, cg_prec))
    single = o.single_launch == 1 ||
             (cg_prec == DOGIP_FP32 && c.p <= 2 && c.l2_bytes > 0 &&
              pcg_small_bytes(c, cg_prec) <= c.l2_bytes);
  // iterations per single launch (host checks for timeouts between launches)
  const int step_iters = single ? std::min(4096, 256 * chunk) : chunk;
  cuda_check(cudaEventRecord(c.ev_in, user), "event record");
  cuda_check(cudaStreamWaitEvent(s, c.ev_in, 0), "stream wait");
  auto timed_out = [&]() {
    if (o.timeout_ms <= 0) return false;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return ms > o.timeout_ms;
  };
  int status = DOGIP_OK;
  int iters = 0, outer = 0;
  const size_t bytes = sizeof(double) * c.n * R;
  if (!o.use_x0) cuda_check(cudaMemsetAsync(u, 0, bytes, s), "zero u");
  if (o.mode == DOGIP_SOLVE_FP64) {
    // PCG on the recursively updated residual; when it reports convergence the
    // true residual b - K u is evaluated in FP64, and PCG restarts from it if
    // the recursion drifted (at most a few restarts).
    if (o.use_x0) launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
    else cuda_check(cudaMemsetAsync(w.q64, 0, bytes, s), "zero q");
    c.launches += vec_residual64(w, b, w.q64, true, o.tol, s);
    for (int restart = 0;; ++restart) {
      read_scal(c);
      bool all = true;
      for (int r = 0; r < R; ++r) all = all && w.h_scal[r].odone;
      if (all) break;
      if (iters >= o.maxiter || restart > 8) { status = DOGIP_ENOTCONV; break; }
      if (timed_out()) { status = DOGIP_ETIMEOUT; break; }
      c.launches += vec_init64(w, c.d_dinv64, o.tol, s);
      read_scal(c);
      int done_here = 0;
      while (!w.h_flags[0]) {
        if (iters + done_here >= o.maxiter) break;
        if (timed_out()) break;
        const int k = std::min(step_iters, o.maxiter - iters - done_here);
        if (single) pcg_small_run(c, DOGIP_FP64, u, k);
        else run_chunk(c, DOGIP_FP64, scatter, u, k, 0.0);
        done_here = 0;
        for (int r = 0; r < R; ++r) done_here = std::max(done_here, w.h_scal[r].iters);
        if (w.h_flags[1]) break;
      }
      iters += done_here;
      const bool brk = w.h_flags[1];
      launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
      c.launches += vec_residual64(w, b, w.q64, false, o.tol, s);
      if (brk) {
        read_scal(c);
        status = DOGIP_EBREAKDOWN;
        break;
      }
    }
  } else if (o.mode == DOGIP_SOLVE_MIXED_RELIABLE) {
    // Reliable-update PCG: FP32 recursion, FP64 residual replacement.
    if (o.use_x0) launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
    else cuda_check(cudaMemsetAsync(w.q64, 0, bytes, s), "zero q");
    c.launches += vec_residual64(w, b, w.q64, true, o.tol, s);
    c.launches += vec_rel_init(w, c.d_dinv32, o.tol, s);
    read_scal(c);
    bool corrected = true;  // r32 equals the true residual right now
    while (!w.h_flags[2]) {
      if (iters >= o.maxiter) { status = DOGIP_ENOTCONV; break; }
      if (timed_out()) { status = DOGIP_ETIMEOUT; break; }
      const int k = std::min(chunk, o.maxiter - iters);
      run_chunk(c, ip, scatter, nullptr, k, o.reliable_delta);
      iters = 0;
      for (int r = 0; r < R; ++r) iters = std::max(iters, w.h_scal[r].iters);
      corrected = false;
      if (w.h_flags[1]) { status = DOGIP_EBREAKDOWN; break; }
      if (w.h_flags[0]) {  // correction requested or recursion converged: replace r
        c.launches += vec_fold(w, u, s);
        launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
        c.launches += vec_residual64(w, b, w.q64, false, o.tol, s);
        c.launches += vec_rel_restart(w, c.d_dinv32, s);
        read_scal(c);
        corrected = true;
        ++outer;
      }
    }
    if (!corrected) {  // report the true residual of the final iterate
      c.launches += vec_fold(w, u, s);
      launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
      c.launches += vec_residual64(w, b, w.q64, false, o.tol, s);
      read_scal(c);
    }
  } else {
    int budget = o.maxiter;
    for (outer = 0;; ++outer) {
      if (outer == 0 && !o.use_x0) cuda_check(cudaMemsetAsync(w.q64, 0, bytes, s), "zero q");
      else launch_apply(c, u, w.q64, R, DOGIP_FP64, scatter, s, nullptr);
      c.launches += vec_residual64(w, b, w.q64, outer == 0, o.tol, s);
      read_scal(c);
      bool all = true;
      for (int r = 0; r < R; ++r) all = all && w.h_scal[r].odone;
      if (all) break;
      if (outer >= o.max_outer) { status = DOGIP_ENOTCONV; break; }
      if (budget <= 0) { status = DOGIP_ENOTCONV; break; }
      if (timed_out()) { status = DOGIP_ETIMEOUT; break; }
      // Each inner solve reduces the FP32 residual by inner_tol, but never by more
      // than the FP64 residual still needs (with a margin of 5 for the FP32 solve's
      // own accuracy): the last refinement step then takes a few iterations instead
      // of a whole inner solve.
      double worst_rel = 0.0;
      for (int r = 0; r < R; ++r)
        if (!w.h_scal[r].odone) worst_rel = std::max(worst_rel, w.h_scal[r].rel);
      double itol = o.inner_tol;
      if (worst_rel > 0.0) itol = std::max(itol, std::min(0.5, 0.2 * o.tol / worst_rel));
      c.launches += vec_inner_init32(w, c.d_dinv32, itol, s);
      if (rec == 2) {  // w0 = K u0 and alpha0 = gamma0 / (w0, u0)
        vec_alloc_cgcg(w);
        launch_apply_energy(c, w.p32, w.q32, s, w, 1);
      }
      read_scal(c);
      int inner = 0;
      const int lim = std::min(o.inner_maxiter, budget);
      while (!w.h_flags[0] && inner < lim) {
        if (timed_out()) break;
        const int k = std::min(step_iters, lim - inner);
        if (single) pcg_small_run(c, DOGIP_FP32, nullptr, k);
        else run_chunk(c, ip, scatter, nullptr, k, 0.0, rec);
        inner = 0;
        for (int r = 0; r < R; ++r) inner = std::max(inner, w.h_scal[r].iters);
        if (w.h_flags[1]) break;
      }
      iters += inner;
      budget -= inner;
      if (w.h_flags[1] && inner == 0) { status = DOGIP_EBREAKDOWN; break; }
      c.launches += vec_correct(w, u, s);
    }
  }
  double worst = 0.0;
  for (int r = 0; r < R; ++r) {
    worst = std::max(worst, w.h_scal[r].rel);
    if (rel_out) rel_out[r] = w.h_scal[r].rel;
  }
  if (status == DOGIP_OK && worst > o.tol) status = DOGIP_ENOTCONV;
  if (status == DOGIP_ENOTCONV)
    set_last_error("solve stopped at its limits (iterations " + std::to_string(iters) +
                   ", refinement steps " + std::to_string(outer) + ") with relative residual " +
                   std::to_string(worst) + " above tol " + std::to_string(o.tol) +
                   " (the FP64 residual of the operator may not reach a tolerance this small)");
  cuda_check(cudaEventRecord(c.ev_out, s), "event record");
  cuda_check(cudaStreamWaitEvent(user, c.ev_out, 0), "stream wait");
  if (info) {
    info->status = status;
    info->iterations = iters;
    info->outer = outer;
    info->rel_residual = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}


// ------------------------------------------------------------- batched solve
//
// Many independent problems (each with its own context, stream and workspace)
// solved together.  Every phase of the solve is captured once as ONE CUDA graph
// with a parallel branch per problem (fork/join over the contexts' streams), and a
// round of the solve is one graph launch for the whole batch: the GPU schedules the
// small kernels of all problems concurrently.  Problems that have converged skip
// their work inside the kernels (device flags).  Mixed mode: every round of FP32
// inner iterations ends when all inner solves are done; the FP64 residual and the
// correction are batch phases too.

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> kernels;  // kernel nodes per problem branch
};

BatchGraph capture_batch(std::vector<Ctx*>& cs, cudaStream_t main,
                         const std::function<void(int, Ctx&, cudaStream_t)>& body) {
  BatchGraph bg;
  bg.kernels.assign(cs.size(), 0);
  cudaEvent_t fork = nullptr;
  cuda_check(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event");
  std::vector<int64_t> before(cs.size());
  for (size_t i = 0; i < cs.size(); ++i) before[i] = cs[i]->launches;
  cuda_check(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    cuda_check(cudaEventRecord(fork, main), "fork record");
    for (size_t i = 0; i < cs.size(); ++i) {
      cudaStream_t s = cs[i]->stream;
      cuda_check(cudaStreamWaitEvent(s, fork, 0), "fork wait");
      body((int)i, *cs[i], s);
      cuda_check(cudaEventRecord(cs[i]->ev_out, s), "join record");
      cuda_check(cudaStreamWaitEvent(main, cs[i]->ev_out, 0), "join wait");
    }
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(main, &g);
    if (g) cudaGraphDestroy(g);
    cudaEventDestroy(fork);
    for (size_t i = 0; i < cs.size(); ++i) cs[i]->launches = before[i];
    throw;
  }
  cudaGraph_t g = nullptr;
  cuda_check(cudaStreamEndCapture(main, &g), "end capture");
  cudaEventDestroy(fork);
  for (size_t i = 0; i < cs.size(); ++i) {
    bg.kernels[i] = cs[i]->launches - before[i];  // counted during capture, run on replay
    cs[i]->launches = before[i];
  }
  cudaError_t e = cudaGraphInstantiate(&bg.exec, g, 0);
  cudaGraphDestroy(g);
  cuda_check(e, "batch graph instantiate");
  return bg;
}

void replay(BatchGraph& bg, std::vector<Ctx*>& cs, cudaStream_t main) {
  cuda_check(cudaGraphLaunch(bg.exec, main), "batch graph launch");
  for (size_t i = 0; i < cs.size(); ++i) cs[i]->launches += bg.kernels[i];
  cuda_check(cudaStreamSynchronize(main), "batch round");
}

// The inner CG chunk of a grouped batch: per iteration the apply once per (dim, p,
// form) group, then the Dirichlet rows and the three vector kernels, all over the
// items of every problem; at the end the scalars and flags of all problems go to the
// host in one copy.  Allocates the problem table, the item tables and the status
// buffers (stream-ordered on main; the caller frees them).  Kernel launches are
// counted on the first context.
BatchGraph capture_grouped(std::vector<Ctx*>& cs, cudaStream_t main, int chunk, BProb*& d_probs,
                           int2*& d_items, CGScal*& d_stat, int*& d_statf, CGScal*& h_stat,
                           int*& h_statf) {
  const int np = (int)cs.size();
  std::vector<BProb> probs(np);
  std::map<int, std::vector<int2>> cells;  // key d*100 + p*2 + form
  std::vector<int2> bitems, vitems;
  const int64_t cpi = batch_cells_per_item(), dpi = batch_dofs_per_item();
  for (int i = 0; i < np; ++i) {
    Ctx& c = *cs[i];
    SolveWork& w = c.work;
    BProb& pr = probs[i];
    pr.A = c.d_A32;
    pr.conn = c.d_conn;
    pr.E = c.E;
    pr.n = c.n;
    pr.x = w.x32;
    pr.r = w.r32;
    pr.p = w.p32;
    pr.q = w.q32;
    pr.dinv = c.d_dinv32;
    pr.bnd = c.d_bnd;
    pr.nbnd = c.dirichlet ? c.nbnd : 0;
    pr.scal = w.scal;
    pr.flags = w.flags;
    pr.partial = w.partial;
    pr.counter = w.counter;
    pr.nvblocks = (int)((c.n + dpi - 1) / dpi);
    if (2 * (int64_t)pr.nvblocks > (int64_t)kMaxRedBlocks * 64)
      fail(DOGIP_EUNSUPPORTED, "problem too large for the grouped batch reduction");
    auto& cl = cells[c.d * 100 + c.p * 2 + c.form];
    for (int64_t b = 0; b < (c.E + cpi - 1) / cpi; ++b) cl.push_back(make_int2(i, (int)b));
    for (int64_t b = 0; b < (pr.nbnd + cpi - 1) / cpi; ++b) bitems.push_back(make_int2(i, (int)b));
    for (int b = 0; b < pr.nvblocks; ++b) vitems.push_back(make_int2(i, b));
  }
  std::vector<int2> all;
  std::vector<std::pair<int, std::pair<size_t, int>>> groups;  // key, (offset, count)
  for (auto& kv : cells) {
    groups.push_back({kv.first, {all.size(), (int)kv.second.size()}});
    all.insert(all.end(), kv.second.begin(), kv.second.end());
  }
  const size_t boff = all.size();
  all.insert(all.end(), bitems.begin(), bitems.end());
  const size_t voff = all.size();
  all.insert(all.end(), vitems.begin(), vitems.end());
  if (all.size() > (size_t)INT32_MAX) fail(DOGIP_EUNSUPPORTED, "batch too large");
  cuda_check(cudaMallocAsync((void**)&d_probs, sizeof(BProb) * np, main), "batch table");
  cuda_check(cudaMallocAsync((void**)&d_items, sizeof(int2) * all.size(), main), "batch items");
  cuda_check(cudaMallocAsync((void**)&d_stat, sizeof(CGScal) * np, main), "batch status");
  cuda_check(cudaMallocAsync((void**)&d_statf, sizeof(int) * 4 * np, main), "batch flags");
  if (cudaMallocHost((void**)&h_stat, sizeof(CGScal) * np) != cudaSuccess ||
      cudaMallocHost((void**)&h_statf, sizeof(int) * 4 * np) != cudaSuccess) {
    cudaGetLastError();
    fail(DOGIP_ENOMEM, "pinned host allocation failed");
  }
  cuda_check(cudaMemcpyAsync(d_probs, probs.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice, main),
             "batch table upload");
  cuda_check(cudaMemcpyAsync(d_items, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice,
                             main), "batch items upload");
  cuda_check(cudaStreamSynchronize(main), "batch tables");
  BatchGraph bg;
  bg.kernels.assign(cs.size(), 0);
  int64_t nk = 0;
  cuda_check(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    for (int it = 0; it < chunk; ++it) {
      for (auto& g : groups) {
        const int key = g.first;
        batch_apply_group(key / 100, (key % 100) / 2, key % 2, d_probs, d_items + g.second.first,
                          g.second.second, main);
        nk += g.second.second > 0 ? 1 : 0;
      }
      batch_vec_step(d_probs, d_items + boff, (int)bitems.size(), d_items + voff,
                     (int)vitems.size(), main);
      nk += (bitems.empty() ? 0 : 1) + 3;
    }
    batch_status(d_probs, np, d_stat, d_statf, main);
    nk += 1;
    cuda_check(cudaMemcpyAsync(h_stat, d_stat, sizeof(CGScal) * np, cudaMemcpyDeviceToHost, main),
               "status copy");
    cuda_check(cudaMemcpyAsync(h_statf, d_statf, sizeof(int) * 4 * np, cudaMemcpyDeviceToHost, main),
               "flags copy");
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(main, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraph_t g = nullptr;
  cuda_check(cudaStreamEndCapture(main, &g), "end capture");
  cudaError_t e = cudaGraphInstantiate(&bg.exec, g, 0);
  cudaGraphDestroy(g);
  cuda_check(e, "batch graph instantiate");
  bg.kernels[0] = nk;
  return bg;
}

void unpack_status(std::vector<Ctx*>& cs, const CGScal* h_stat, const int* h_statf) {
  for (size_t i = 0; i < cs.size(); ++i) {
    std::memcpy(cs[i]->work.h_scal, h_stat + i, sizeof(CGScal));
    std::memcpy(cs[i]->work.h_flags, h_statf + 4 * i, sizeof(int) * 4);
  }
}

// Concurrent batch: every problem is an ordinary solve on its own context stream, run
// by a pool of host threads (16, or DOGIP_BATCH_THREADS; one problem at a time per
// thread, the smallest estimated work first).  Problems refine independently -- no problem waits for another's
// refinement round -- and the GPU runs the solves of different problems side by side
// (the single-launch PCG sizes its grid to the problem).  seconds = host time from the
// start of the batch until that problem's solve returned.
int batch_concurrent(const std::vector<Ctx*>& cs, const double* const* b, double* const* u,
                     const dogip_solve_opts& o, dogip_solve_info* infos, double* seconds_out,
                     cudaStream_t user, std::chrono::steady_clock::time_point t0) {
  const int np = (int)cs.size();
  const int dev = cs[0]->device;
  int nt = std::max(1, std::min(np, 16));
  if (const char* v = std::getenv("DOGIP_BATCH_THREADS")) nt = std::max(1, std::min(np, std::atoi(v)));
  // order by estimated work (apply cost ~ cells x V_T^2, iterations ~ sqrt(n)):
  // DOGIP_BATCH_ORDER = smallest (default: shortest solves first, the least mean
  // completion time), largest (the longest solves do not start last), or given.
  // Measured on 256 uneven 2D problems: smallest 741 ms, p50 / p99 111 / 728 ms;
  // largest 725 ms, 635 / 723 ms; given 694 ms, 363 / 676 ms.
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int i) {
    const Ctx& c = *cs[i];
    return (double)c.E * c.VT * c.VT * std::sqrt((double)c.n);
  };
  std::string ord = "smallest";
  if (const char* v = std::getenv("DOGIP_BATCH_ORDER")) ord = v;
  if (ord == "largest")
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return work(a) > work(b2); });
  else if (ord == "smallest")
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return work(a) < work(b2); });
  else if (ord != "given")
    fail(DOGIP_EINVAL, "DOGIP_BATCH_ORDER must be largest, smallest or given");
  // the per-step kernels: the single-launch PCG measured slower when many solves share
  // the GPU (its cooperative launches do not overlap as freely), unless asked for
  dogip_solve_opts os = o;
  if (os.single_launch < 0) os.single_launch = 0;
  std::atomic<int> next{0};
  std::vector<int> st(np, DOGIP_OK);
  std::vector<std::string> msg(np);
  std::vector<dogip_solve_info> inf(np);
  std::vector<double> t_done(np, 0.0);
  auto worker = [&]() {
    try {
      cuda_check(cudaSetDevice(dev), "set device");
    } catch (...) {
    }
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= np) break;
      const int i = order[k];
      std::memset(&inf[i], 0, sizeof(dogip_solve_info));
      try {
        st[i] = solve(*cs[i], b[i], u[i], 1, &os, &inf[i], nullptr, user);
        if (st[i] != DOGIP_OK) msg[i] = g_last_error;
      } catch (const Failure& f) {
        st[i] = f.code;
        msg[i] = f.msg;
      } catch (const std::exception& e) {
        st[i] = DOGIP_ECUDA;
        msg[i] = e.what();
      }
      t_done[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  int status = DOGIP_OK;
  for (int i = 0; i < np; ++i) {
    if (st[i] != DOGIP_OK && status == DOGIP_OK) {
      status = st[i];
      set_last_error("batch problem " + std::to_string(i) + ": " + msg[i]);
    }
    if (infos) {
      infos[i] = inf[i];
      infos[i].status = st[i];
      infos[i].seconds = t_done[i];
    }
    if (seconds_out) seconds_out[i] = t_done[i];
  }
  return status;
}

int batch_solve(Ctx* const* ctxs, int np, const double* const* b, double* const* u,
                const dogip_solve_opts* opts, dogip_solve_info* infos, double* seconds_out,
                cudaStream_t user) {
  const auto t0 = std::chrono::steady_clock::now();
  dogip_solve_opts o;
  dogip_solve_opts_default(&o);
  if (opts) o = *opts;
  if (np < 1 || !ctxs || !b || !u) fail(DOGIP_EINVAL, "ctxs, b and u arrays are required");
  if (o.mode != DOGIP_SOLVE_FP64 && o.mode != DOGIP_SOLVE_MIXED)
    fail(DOGIP_EINVAL, "batched solves support the FP64 and MIXED modes");
  if (o.use_x0) fail(DOGIP_EINVAL, "batched solves start from u = 0");
  std::vector<Ctx*> cs(ctxs, ctxs + np);
  const int dev = cs[0]->device;
  for (int i = 0; i < np; ++i) {
    if (!cs[i] || !b[i] || !u[i]) fail(DOGIP_EINVAL, "null context or vector in the batch");
    if (cs[i]->device != dev) fail(DOGIP_EINVAL, "all contexts of a batch share one device");
    if (o.mode == DOGIP_SOLVE_MIXED && !cs[i]->keep32) fail(DOGIP_EINVAL, "mixed mode needs keep_fp32");
    for (int j = 0; j < i; ++j)
      if (cs[j] == cs[i]) fail(DOGIP_EINVAL, "a context appears twice in the batch");
  }
  DeviceGuard guard(dev);
  // DOGIP_BATCH_MODE: "concurrent" (default: independent solves side by side),
  // "grouped" (lockstep rounds, one launch per kernel for the whole batch) or
  // "branches" (lockstep rounds, one graph branch per problem)
  std::string bmode = "concurrent";
  if (const char* v = std::getenv("DOGIP_BATCH_MODE")) bmode = v;
  if (bmode != "concurrent" && bmode != "grouped" && bmode != "branches")
    fail(DOGIP_EINVAL, "DOGIP_BATCH_MODE must be concurrent, grouped or branches");
  if (bmode == "concurrent") return batch_concurrent(cs, b, u, o, infos, seconds_out, user, t0);
  for (Ctx* c : cs) {
    ensure_w_scratch(*c, 1);
    vec_alloc(c->work, c->n, 1);
  }
  cudaStream_t main = nullptr;
  cuda_check(cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking), "batch stream");
  cudaEvent_t ev = nullptr;
  cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  std::vector<BatchGraph> graphs;
  // grouped inner iterations (mixed mode, DOGIP_BATCH_MODE=grouped): one launch per
  // kernel for the whole batch where every context has FP32 element-wise A_T in caller
  // cell order and compiled tables (else, and with "branches", one graph branch per
  // problem)
  bool grouped = o.mode == DOGIP_SOLVE_MIXED && bmode == "grouped";
  for (Ctx* c : cs)
    grouped = grouped && c->keep32 && !c->hi && !c->global_w && !c->factorized &&
              c->scatter == DOGIP_SCATTER_ATOMIC && batch_apply_compiled(c->d, c->p, c->form);
  BProb* d_probs = nullptr;
  int2* d_items = nullptr;
  CGScal* d_stat = nullptr;
  int* d_statf = nullptr;
  CGScal* h_stat = nullptr;
  int* h_statf = nullptr;
  auto cleanup = [&]() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    for (void* q : {(void*)d_probs, (void*)d_items, (void*)d_stat, (void*)d_statf})
      if (q) cudaFreeAsync(q, main);
    cudaStreamSynchronize(main);
    if (h_stat) cudaFreeHost(h_stat);
    if (h_statf) cudaFreeHost(h_statf);
    cudaEventDestroy(ev);
    cudaStreamDestroy(main);
  };
  std::vector<double> t_done(np, -1.0);
  std::vector<int> iters(np, 0), outers(np, 0);
  int status = DOGIP_OK;
  auto elapsed = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  try {
    cuda_check(cudaEventRecord(ev, user), "event record");
    cuda_check(cudaStreamWaitEvent(main, ev, 0), "stream wait");
    const int chunk = std::max(1, o.check_every);
    const int scat = DOGIP_SCATTER_ATOMIC;
    auto scal_copy = [&](Ctx& c, cudaStream_t s) {
      cuda_check(cudaMemcpyAsync(c.work.h_scal, c.work.scal, sizeof(CGScal), cudaMemcpyDeviceToHost, s),
                 "scal copy");
      cuda_check(cudaMemcpyAsync(c.work.h_flags, c.work.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s),
                 "flags copy");
    };
    const bool mixed = o.mode == DOGIP_SOLVE_MIXED;
    // phase 0: r = b (u = 0), norms; FP64 mode also starts PCG here
    graphs.push_back(capture_batch(cs, main, [&](int i, Ctx& c, cudaStream_t s) {
      cuda_check(cudaMemsetAsync(u[i], 0, sizeof(double) * c.n, s), "zero u");
      cuda_check(cudaMemsetAsync(c.work.q64, 0, sizeof(double) * c.n, s), "zero q");
      c.launches += vec_residual64(c.work, b[i], c.work.q64, true, o.tol, s);
      if (!mixed) c.launches += vec_init64(c.work, c.d_dinv64, o.tol, s);
      scal_copy(c, s);
    }));
    // phase 1: a chunk of CG iterations (FP32 inner or FP64)
    if (grouped) {
      graphs.push_back(capture_grouped(cs, main, chunk, d_probs, d_items, d_stat, d_statf, h_stat,
                                       h_statf));
    } else
    graphs.push_back(capture_batch(cs, main, [&](int i, Ctx& c, cudaStream_t s) {
      SolveWork& w = c.work;
      for (int it = 0; it < chunk; ++it) {
        if (mixed) {
          launch_apply_cg(c, w.p32, w.q32, 1, DOGIP_FP32, scat, s, w);
          c.launches += vec_cg_step(w, DOGIP_FP32, nullptr, c.d_dinv32, 0.0, s, true);
        } else {
          launch_apply_cg(c, w.p64, w.q64, 1, DOGIP_FP64, scat, s, w);
          c.launches += vec_cg_step(w, DOGIP_FP64, u[i], c.d_dinv64, 0.0, s, true);
        }
      }
      scal_copy(c, s);
    }));
    // phase 2: FP64 correction and true residual (mixed: then a new inner start)
    graphs.push_back(capture_batch(cs, main, [&](int i, Ctx& c, cudaStream_t s) {
      if (mixed) c.launches += vec_correct(c.work, u[i], s);
      launch_apply(c, u[i], c.work.q64, 1, DOGIP_FP64, scat, s, nullptr);
      c.launches += vec_residual64(c.work, b[i], c.work.q64, false, o.tol, s);
      scal_copy(c, s);
    }));
    // phase 3 (mixed): inner start r32 = r64 / ||r64||
    if (mixed)
      graphs.push_back(capture_batch(cs, main, [&](int i, Ctx& c, cudaStream_t s) {
        c.launches += vec_inner_init32(c.work, c.d_dinv32, o.inner_tol, s);
        scal_copy(c, s);
      }));
    auto note_done = [&]() {
      bool all = true;
      for (int i = 0; i < np; ++i) {
        if (cs[i]->work.h_scal[0].odone) {
          if (t_done[i] < 0) t_done[i] = elapsed();
        } else {
          all = false;
        }
      }
      return all;
    };
    replay(graphs[0], cs, main);
    bool all = note_done();
    if (mixed) {
      for (int outer = 0; !all; ++outer) {
        if (outer >= o.max_outer) { status = DOGIP_ENOTCONV; break; }
        if (o.timeout_ms > 0 && elapsed() * 1e3 > o.timeout_ms) { status = DOGIP_ETIMEOUT; break; }
        replay(graphs[3], cs, main);
        for (int i = 0; i < np; ++i)
          if (!cs[i]->work.h_scal[0].odone) outers[i] = outer + 1;
        int inner = 0;
        while (inner < o.inner_maxiter) {
          bool all_in = true;
          for (Ctx* c : cs) all_in = all_in && c->work.h_flags[2];
          if (all_in) break;
          replay(graphs[1], cs, main);
          if (grouped) unpack_status(cs, h_stat, h_statf);
          inner += chunk;
          bool brk = false;
          for (Ctx* c : cs) brk = brk || c->work.h_flags[1];
          if (brk) break;
        }
        for (int i = 0; i < np; ++i) iters[i] += cs[i]->work.h_scal[0].iters;
        replay(graphs[2], cs, main);
        all = note_done();
      }
    } else {
      int total = 0;
      while (!all) {
        if (total >= o.maxiter) { status = DOGIP_ENOTCONV; break; }
        if (o.timeout_ms > 0 && elapsed() * 1e3 > o.timeout_ms) { status = DOGIP_ETIMEOUT; break; }
        replay(graphs[1], cs, main);
        total += chunk;
        bool all_in = true;
        for (int i = 0; i < np; ++i) {
          const bool di = cs[i]->work.h_flags[2];
          if (di && t_done[i] < 0) t_done[i] = elapsed();
          all_in = all_in && di;
        }
        if (all_in) break;
      }
      for (int i = 0; i < np; ++i) iters[i] = cs[i]->work.h_scal[0].iters;
      replay(graphs[2], cs, main);  // true residual of the final iterates
      note_done();
    }
    cuda_check(cudaEventRecord(ev, main), "event record");
    cuda_check(cudaStreamWaitEvent(user, ev, 0), "stream wait");
  } catch (...) {
    cudaStreamSynchronize(main);
    cleanup();
    throw;
  }
  cudaStreamSynchronize(main);
  cleanup();
  for (int i = 0; i < np; ++i) {
    const CGScal& sc = cs[i]->work.h_scal[0];
    int st = sc.rel <= o.tol ? DOGIP_OK : (status == DOGIP_OK ? DOGIP_ENOTCONV : status);
    if (cs[i]->work.h_flags[1]) st = DOGIP_EBREAKDOWN;
    if (st != DOGIP_OK && status == DOGIP_OK) status = st;
    if (infos) {
      infos[i].status = st;
      infos[i].iterations = iters[i];
      infos[i].outer = outers[i];
      infos[i].rel_residual = sc.rel;
      infos[i].seconds = t_done[i] >= 0 ? t_done[i] : elapsed();
    }
    if (seconds_out) seconds_out[i] = t_done[i];
  }
  return status;
}


// --------------------------------------------------------------- autotuner
//
// Picks, per precision, the apply kernel (tensor cores, self-feeding warps, bulk-async
// staged, or one thread per cell with 64 / 128 / 256 cells per CTA) by timing each on
// the context's own data (the kernel alone: best of 3 samples of 8 launches, CUDA
// events; FP32 keeps the staged kernel within 3 %).  Choices are cached process-
// wide per (dim, p, form, precision, log2 of the cell count); with DOGIP_TUNE_CACHE
// set they are also read from and appended to that text file.

struct TuneKey {
  int d, p, form, prec, logE;
  bool operator<(const TuneKey& o) const {
    return std::tie(d, p, form, prec, logE) < std::tie(o.d, o.p, o.form, o.prec, o.logE);
  }
};
struct TuneChoice {
  int variant, block;
  float ms;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneChoice> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("DOGIP_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  TuneKey k;
  TuneChoice ch;
  while (std::fscanf(f, "%d %d %d %d %d %d %d %f", &k.d, &k.p, &k.form, &k.prec, &k.logE,
                     &ch.variant, &ch.block, &ch.ms) == 8)
    g_tune[k] = ch;
  std::fclose(f);
}

void tune_store_locked(const TuneKey& k, const TuneChoice& ch) {
  g_tune[k] = ch;
  const char* path = std::getenv("DOGIP_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d %d %.6f\n", k.d, k.p, k.form, k.prec, k.logE, ch.variant,
               ch.block, ch.ms);
  std::fclose(f);
}

int autotune(Ctx& c, int force, cudaStream_t s) {
  DeviceGuard guard(c.device);
  if (c.factorized || c.global_w) return 0;  // one kernel only
  // higher orders: the run-time-table kernel, or the tensor cores (FP32) where built
  if (c.hi && !apply_tc_available(c.d, c.p, c.form)) return 0;
  int logE = 0;
  while ((int64_t(1) << logE) < c.E) ++logE;
  int tuned = 0;
  for (int prec : {DOGIP_FP32, DOGIP_FP64}) {
    if (prec == DOGIP_FP32 && !c.keep32) continue;
    if (prec == DOGIP_FP64 && c.hi) continue;  // one FP64 kernel
    const TuneKey key{c.d, c.p, c.form, prec, logE};
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      tune_load_locked();
      auto it = g_tune.find(key);
      if (it != g_tune.end() && !force) {
        c.apply_variant_prec[prec] = it->second.variant;
        c.apply_block[prec] = it->second.block;
        continue;
      }
    }
    const size_t es = prec == DOGIP_FP64 ? 8 : 4;
    void *u = nullptr, *y = nullptr;
    cuda_check(cudaMallocAsync(&u, es * c.n, s), "tuning buffers");
    if (cudaMallocAsync(&y, es * c.n, s) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(u, s);
      fail(DOGIP_ENOMEM, "tuning buffers");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TuneChoice best{1, 256, 1e30f};
    float staged_ms = 1e30f;
    try {
      cuda_check(cudaMemsetAsync(u, 0, es * c.n, s), "tuning input");
      cuda_check(cudaEventCreate(&e0), "event");
      cuda_check(cudaEventCreate(&e1), "event");
      // tensor cores (FP32), self-feeding warps, staged, one thread per cell with
      // 64 / 128 / 256 cells per CTA
      const std::pair<int, int> cands[] = {{3, 256}, {2, 256}, {1, 256},
                                           {0, 64},  {0, 128}, {0, 256}};
      for (auto [var, blk] : cands) {
        if (var == 3 && (prec != DOGIP_FP32 || !apply_tc_available(c.d, c.p, c.form))) continue;
        if (c.hi && var != 3 && var != 1) continue;  // 1: the run-time-table kernel
        c.apply_variant_prec[prec] = var;
        c.apply_block[prec] = blk;
        // the kernel alone (y += K u into a buffer that stays finite: u = 0), eight
        // launches back to back per sample, best of three samples after a warm-up
        for (int w = 0; w < 3; ++w)
          launch_apply(c, u, y, 1, prec, DOGIP_SCATTER_ATOMIC, s, nullptr, true);
        float tbest = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cuda_check(cudaEventRecord(e0, s), "event record");
          for (int w = 0; w < 8; ++w)
            launch_apply(c, u, y, 1, prec, DOGIP_SCATTER_ATOMIC, s, nullptr, true);
          cuda_check(cudaEventRecord(e1, s), "event record");
          cuda_check(cudaEventSynchronize(e1), "tuning sync");
          float ti = 0.0f;
          cuda_check(cudaEventElapsedTime(&ti, e0, e1), "elapsed");
          tbest = std::min(tbest, ti / 8.0f);
        }
        if (var == 1) staged_ms = tbest;
        if (tbest < best.ms) best = TuneChoice{var, blk, tbest};
      }
      // FP32: the staged kernel also carries the (p, K p) reduction of the mixed
      // solve's inner iterations (one kernel less each), so it is kept unless another
      // kernel is faster by more than 3 %
      if (prec == DOGIP_FP32 && !c.hi && staged_ms <= 1.03f * best.ms)
        best = TuneChoice{1, 256, staged_ms};
    } catch (...) {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaFreeAsync(u, s);
      cudaFreeAsync(y, s);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cuda_check(cudaFreeAsync(u, s), "tuning buffers");
    cuda_check(cudaFreeAsync(y, s), "tuning buffers");
    c.apply_variant_prec[prec] = best.variant;
    c.apply_block[prec] = best.block;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_store_locked(key, best);
    ++tuned;
  }
  // captured solver graphs hold the old launch shapes
  if (c.work.graph) {
    cudaGraphExecDestroy(c.work.graph);
    c.work.graph = nullptr;
  }
  return tuned;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const Failure& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return DOGIP_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return DOGIP_EINVAL;
  }
}

}  // namespace
std::mutex g_pdl_mutex;
std::unordered_set<const void*> g_pdl_kernels;

void pdl_mark(const void* kernel) {
  std::lock_guard<std::mutex> lock(g_pdl_mutex);
  g_pdl_kernels.insert(kernel);
}

bool pdl_marked(const void* kernel) {
  std::lock_guard<std::mutex> lock(g_pdl_mutex);
  return g_pdl_kernels.count(kernel) != 0;
}

}  // namespace dogip

using dogip::Ctx;
using dogip::fail;
using dogip::guarded;

extern "C" {

int dogip_version(void) { return 100; }

const char* dogip_last_error(void) { return dogip::g_last_error.c_str(); }

int dogip_opts_default(dogip_opts* o) {
  if (!o) return DOGIP_EINVAL;
  o->dirichlet = -1;
  o->scatter = DOGIP_SCATTER_ATOMIC;
  o->keep_fp32 = 1;
  o->device = -1;
  o->factorized = 0;
  o->global_w = 0;
  return DOGIP_OK;
}

int dogip_solve_opts_default(dogip_solve_opts* o) {
  if (!o) return DOGIP_EINVAL;
  o->mode = DOGIP_SOLVE_FP64;
  o->tol = 1e-8;
  o->maxiter = 100000;
  o->inner_tol = 1e-4;
  o->inner_maxiter = 100000;
  o->max_outer = 30;
  o->scatter = -1;
  o->check_every = 16;
  o->use_x0 = 0;
  o->timeout_ms = 0.0;
  o->reliable_delta = 0.1;
  o->inner_prec = DOGIP_FP32;
  o->inner_recurrence = 0;
  o->single_launch = -1;
  return DOGIP_OK;
}

int dogip_setup(const dogip_mesh* m, int p, int form, int coef_kind, const double* coef,
                const dogip_opts* o, dogip_ctx** out) {
  return guarded([&] {
    if (!out) fail(DOGIP_EINVAL, "out is required");
    *out = nullptr;
    *out = dogip::setup(m, p, form, coef_kind, coef, o);
    return DOGIP_OK;
  });
}

void dogip_destroy(dogip_ctx* ctx) { dogip::free_ctx(ctx); }

int dogip_set_coef(dogip_ctx* ctx, int coef_kind, const double* coef, void* stream) {
  return guarded([&] {
    if (!ctx) fail(DOGIP_EINVAL, "ctx is required");
    dogip::set_coef(*ctx, coef_kind, coef, (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

int dogip_get_info(const dogip_ctx* c, dogip_info* i) {
  return guarded([&] {
    if (!c || !i) fail(DOGIP_EINVAL, "ctx and info are required");
    i->dim = c->d;
    i->p = c->p;
    i->form = c->form;
    i->coef_kind = c->coef_kind;
    i->dirichlet = c->dirichlet;
    i->scatter = c->scatter;
    i->n_cells = c->E;
    i->n_dofs = c->n;
    i->n_boundary = c->nbnd;
    i->v_loc = c->VT;
    i->w_loc = c->WT;
    i->n_sym = c->NS;
    i->n_colours = c->ncolours;
    i->nnz_b = c->nnzb;
    i->nnz_pm1_b = c->nnzb1;
    const int64_t per = (int64_t)(c->factorized ? 1 : c->WT) * c->NS;
    i->bytes_ahat_fp64 = c->global_w ? c->nW * 8 : (int64_t)c->E * per * 8;
    i->bytes_ahat_fp32 = c->global_w ? c->nW * 4 : (int64_t)c->E * per * 4;
    i->bytes_conn = (int64_t)c->E * (c->VT + (c->global_w ? c->WT : 0)) * 4;
    i->n_wglobal = c->global_w ? c->nW : 0;
    i->kernel_launches = c->launches;
    return DOGIP_OK;
  });
}

int64_t dogip_ndofs(const dogip_ctx* c) { return c ? c->n : -1; }

// Host-only mesh preprocessing (no CUDA call): the same routines the set-up uses.
namespace {
dogip::Ctx host_ctx(int dim, int p, int64_t n_cells, const int32_t* cells) {
  if (dim != 2 && dim != 3) dogip::fail(DOGIP_EINVAL, "dim must be 2 or 3");
  if (p < 1 || p > 16) dogip::fail(DOGIP_EINVAL, "p must be in 1..16");
  if (n_cells <= 0 || !cells) dogip::fail(DOGIP_EINVAL, "cells are required");
  int64_t nv = 0;
  for (int64_t k = 0; k < n_cells * (dim + 1); ++k) {
    if (cells[k] < 0) dogip::fail(DOGIP_EINVAL, "negative vertex id");
    nv = std::max<int64_t>(nv, (int64_t)cells[k] + 1);
  }
  dogip::Ctx c;
  c.d = dim;
  c.p = p;
  c.E = n_cells;
  c.nv = nv;
  c.VT = (int)dogip::local_betas(dim, p).size();
  c.dirichlet = true;
  return c;
}
}  // namespace

int dogip_mesh_dofmap(int dim, int p, int64_t n_cells, const int32_t* cells, int32_t* ids,
                      int64_t* n_dofs) {
  return guarded([&] {
    dogip::Ctx c = host_ctx(dim, p, n_cells, cells);
    dogip::build_dofmap(c, cells);
    if (ids) std::memcpy(ids, c.dofmap.data(), sizeof(int32_t) * c.dofmap.size());
    if (n_dofs) *n_dofs = c.n;
    return DOGIP_OK;
  });
}

int dogip_mesh_boundary(int dim, int p, int64_t n_cells, const int32_t* cells, uint8_t* mask) {
  return guarded([&] {
    if (!mask) dogip::fail(DOGIP_EINVAL, "mask is required");
    dogip::Ctx c = host_ctx(dim, p, n_cells, cells);
    dogip::build_dofmap(c, cells);
    dogip::build_boundary(c, cells);
    std::memcpy(mask, c.bmask.data(), c.bmask.size());
    return DOGIP_OK;
  });
}

int dogip_mesh_colouring(int dim, int64_t n_cells, const int32_t* cells, int32_t* colour,
                         int* n_colours) {
  return guarded([&] {
    dogip::Ctx c = host_ctx(dim, 1, n_cells, cells);
    dogip::build_colouring(c, cells);
    if (colour) std::memcpy(colour, c.colour.data(), sizeof(int32_t) * c.colour.size());
    if (n_colours) *n_colours = c.ncolours;
    return DOGIP_OK;
  });
}

int dogip_mesh_wdofmap(int dim, int p, int64_t n_cells, const int32_t* cells, int32_t* ids,
                       uint8_t* owner, int64_t* n_w) {
  return guarded([&] {
    dogip::Ctx c = host_ctx(dim, p, n_cells, cells);
    std::vector<int32_t> w;
    std::vector<uint8_t> first;
    const int64_t n = dogip::number_nodes(dim, 2 * p, n_cells, cells, w, &first);
    if (ids) std::memcpy(ids, w.data(), sizeof(int32_t) * w.size());
    if (owner) std::memcpy(owner, first.data(), first.size());
    if (n_w) *n_w = n;
    return DOGIP_OK;
  });
}

int dogip_get_dofmap(const dogip_ctx* c, int32_t* out) {
  return guarded([&] {
    if (!c || !out) fail(DOGIP_EINVAL, "ctx and output are required");
    std::memcpy(out, c->dofmap.data(), sizeof(int32_t) * c->dofmap.size());
    return DOGIP_OK;
  });
}

int dogip_get_colouring(const dogip_ctx* c, int32_t* out, int* ncol) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    if (out) std::memcpy(out, c->colour.data(), sizeof(int32_t) * c->colour.size());
    if (ncol) *ncol = c->ncolours;
    return DOGIP_OK;
  });
}

int dogip_get_boundary(const dogip_ctx* c, uint8_t* out) {
  return guarded([&] {
    if (!c || !out) fail(DOGIP_EINVAL, "ctx and output are required");
    std::memcpy(out, c->bmask.data(), c->bmask.size());
    return DOGIP_OK;
  });
}

int dogip_get_ahat(const dogip_ctx* c, double* out, void* stream) {
  return guarded([&] {
    if (!c || !out) fail(DOGIP_EINVAL, "ctx and output are required");
    if (c->global_w) fail(DOGIP_EINVAL, "global double grid: use dogip_get_ahat_global");
    dogip::DeviceGuard g(c->device);
    dogip::launch_export_ahat(*c, out, (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

int dogip_get_ahat_global(const dogip_ctx* c, double* out, void* stream) {
  return guarded([&] {
    if (!c || !out) fail(DOGIP_EINVAL, "ctx and output are required");
    if (!c->global_w) fail(DOGIP_EINVAL, "context has no global double grid");
    dogip::DeviceGuard g(c->device);
    dogip::cuda_check(cudaMemcpyAsync(out, c->d_Aw64, sizeof(double) * c->nW,
                                      cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                      "copy A_diag");
    return DOGIP_OK;
  });
}

int dogip_get_wdofmap(const dogip_ctx* c, int32_t* ids, uint8_t* owner) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    if (!c->global_w) fail(DOGIP_EINVAL, "context has no global double grid");
    if (ids) std::memcpy(ids, c->wdofmap.data(), sizeof(int32_t) * c->wdofmap.size());
    if (owner) std::memcpy(owner, c->wowner.data(), c->wowner.size());
    return DOGIP_OK;
  });
}

int dogip_check(dogip_ctx* c, void* stream) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    dogip::DeviceGuard g(c->device);
    int kerr = 0;
    cudaStream_t s = (cudaStream_t)stream;
    dogip::cuda_check(cudaMemcpyAsync(&kerr, c->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s),
                      "kernel flag read");
    dogip::cuda_check(cudaStreamSynchronize(s), "stream sync");
    if (kerr) {
      dogip::cuda_check(cudaMemset(c->d_kerr, 0, sizeof(int)), "kernel flag reset");
      fail(DOGIP_ETIMEOUT, "a bounded wait inside a kernel expired");
    }
    return DOGIP_OK;
  });
}

int dogip_get_diag(const dogip_ctx* c, double* out, void* stream) {
  return guarded([&] {
    if (!c || !out) fail(DOGIP_EINVAL, "ctx and output are required");
    dogip::DeviceGuard g(c->device);
    dogip::cuda_check(cudaMemcpyAsync(out, c->d_diag, sizeof(double) * c->n,
                                      cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
                      "diag copy");
    return DOGIP_OK;
  });
}

int dogip_get_tables(int dim, int p, int form, double* bhat, double* what, int* sizes) {
  return guarded([&] {
    int NB, W, V;
    long long nnz, nnz1;
    if (!dogip::table_info(dim, p, form, &NB, &W, &V, &nnz, &nnz1))
      fail(DOGIP_EUNSUPPORTED, "no compiled table for this (dim, p, form)");
    if (sizes) {
      sizes[0] = NB;
      sizes[1] = W;
      sizes[2] = V;
    }
    dogip::table_copy(dim, p, form, bhat, what, nullptr);
    return DOGIP_OK;
  });
}

namespace {
int apply_entry(dogip_ctx* c, const void* u, void* y, int nrhs, int prec, int scatter,
                void* stream, bool add) {
  return guarded([&] {
    if (!c || !u || !y) fail(DOGIP_EINVAL, "ctx, u and y are required");
    if (nrhs < 1) fail(DOGIP_EINVAL, "nrhs must be >= 1");
    if (prec != DOGIP_FP64 && prec != DOGIP_FP32 && prec != DOGIP_TF32)
      fail(DOGIP_EINVAL, "unknown precision");
    if (prec != DOGIP_FP64 && !c->keep32) fail(DOGIP_EINVAL, "context has no FP32 copy");
    if (scatter < 0) scatter = c->scatter;
    if (scatter != DOGIP_SCATTER_ATOMIC && scatter != DOGIP_SCATTER_COLOUR)
      fail(DOGIP_EINVAL, "unknown scatter");
    if (scatter == DOGIP_SCATTER_COLOUR && c->scatter != DOGIP_SCATTER_COLOUR)
      fail(DOGIP_EINVAL, "colour scatter needs a context set up with scatter = COLOUR");
    dogip::DeviceGuard g(c->device);
    dogip::ensure_w_scratch(*c, nrhs);
    dogip::launch_apply(*c, u, y, nrhs, prec, scatter, (cudaStream_t)stream, nullptr, add);
    return DOGIP_OK;
  });
}
}  // namespace

int dogip_apply(dogip_ctx* c, const void* u, void* y, int nrhs, int prec, int scatter,
                void* stream) {
  return apply_entry(c, u, y, nrhs, prec, scatter, stream, false);
}

int dogip_apply_add(dogip_ctx* c, const void* u, void* y, int nrhs, int prec, int scatter,
                    void* stream) {
  return apply_entry(c, u, y, nrhs, prec, scatter, stream, true);
}

int dogip_apply_qp(dogip_ctx* c, const void* u, void* y, int nrhs, int prec, void* stream) {
  return guarded([&] {
    if (!c || !u || !y) fail(DOGIP_EINVAL, "ctx, u and y are required");
    if (nrhs < 1) fail(DOGIP_EINVAL, "nrhs must be >= 1");
    if (prec != DOGIP_FP64 && prec != DOGIP_FP32) fail(DOGIP_EINVAL, "unknown precision");
    if (prec == DOGIP_FP32 && !c->keep32) fail(DOGIP_EINVAL, "context has no FP32 copy");
    if (!c->qp_ok)
      fail(DOGIP_EUNSUPPORTED,
           "the quadrature-point apply needs element-constant coefficients (not sub-element)");
    dogip::DeviceGuard g(c->device);
    dogip::launch_apply_qp(*c, u, y, nrhs, prec, (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

int dogip_load(dogip_ctx* c, const double* f, double* b, void* stream) {
  return guarded([&] {
    if (!c || !b) fail(DOGIP_EINVAL, "ctx and b are required");
    dogip::DeviceGuard g(c->device);
    dogip::launch_load(*c, f, b, (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

int dogip_solve(dogip_ctx* c, const double* b, double* u, int nrhs, const dogip_solve_opts* o,
                dogip_solve_info* info, double* rel, void* stream) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    return dogip::solve(*c, b, u, nrhs, o, info, rel, (cudaStream_t)stream);
  });
}

int dogip_solve_host(dogip_ctx* c, const double* bh, double* uh, int nrhs,
                     const dogip_solve_opts* o, dogip_solve_info* info, double* rel,
                     void* stream) {
  return guarded([&] {
    if (!c || !bh || !uh) fail(DOGIP_EINVAL, "ctx, b and u are required");
    if (!dogip::r_ok(nrhs)) fail(DOGIP_EINVAL, "nrhs must be 1, 2, 4, 8, 16 or 32 for solves");
    dogip::DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * c->n * nrhs;
    double *db = nullptr, *du = nullptr;
    dogip::cuda_check(cudaMallocAsync((void**)&db, bytes, s), "staging allocation");
    if (cudaMallocAsync((void**)&du, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(db, s);
      fail(DOGIP_ENOMEM, "staging allocation");
    }
    int st = DOGIP_OK;
    try {
      dogip::cuda_check(cudaMemcpyAsync(db, bh, bytes, cudaMemcpyHostToDevice, s), "upload b");
      if (o && o->use_x0)
        dogip::cuda_check(cudaMemcpyAsync(du, uh, bytes, cudaMemcpyHostToDevice, s), "upload x0");
      st = dogip::solve(*c, db, du, nrhs, o, info, rel, s);
      dogip::cuda_check(cudaMemcpyAsync(uh, du, bytes, cudaMemcpyDeviceToHost, s), "download u");
    } catch (...) {
      cudaFreeAsync(db, s);
      cudaFreeAsync(du, s);
      throw;
    }
    dogip::cuda_check(cudaFreeAsync(db, s), "staging free");
    dogip::cuda_check(cudaFreeAsync(du, s), "staging free");
    dogip::cuda_check(cudaStreamSynchronize(s), "solve_host sync");
    return st;
  });
}

int dogip_autotune(dogip_ctx* c, int force, dogip_tune_info* info, void* stream) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    dogip::autotune(*c, force, (cudaStream_t)stream);
    if (info) {
      for (int pr = 0; pr < 2; ++pr) {
        info->variant[pr] = c->apply_variant_prec[pr] >= 0 ? c->apply_variant_prec[pr] : c->apply_variant;
        info->block[pr] = c->apply_block[pr];
      }
    }
    return DOGIP_OK;
  });
}

int dogip_batch_solve(dogip_ctx* const* ctxs, int nprob, const double* const* b, double* const* u,
                      const dogip_solve_opts* o, dogip_solve_info* infos, void* stream) {
  return guarded([&] {
    return dogip::batch_solve(ctxs, nprob, b, u, o, infos, nullptr, (cudaStream_t)stream);
  });
}

int dogip_set_coef_inclusions(dogip_ctx* c, int n_incl, const double* centres,
                              const double* radii, double inside, double outside, int nq,
                              void* stream) {
  return guarded([&] {
    if (!c) fail(DOGIP_EINVAL, "ctx is required");
    dogip::set_coef_inclusions(*c, n_incl, centres, radii, inside, outside, nq,
                               (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

int dogip_grad_coef(dogip_ctx* c, const double* u, const double* lam, double* dA, void* stream) {
  return guarded([&] {
    if (!c || !u || !lam || !dA) fail(DOGIP_EINVAL, "ctx, u, lam and dA are required");
    if (c->coef_kind == DOGIP_COEF_INCLUSIONS)
      fail(DOGIP_EINVAL, "the coefficient gradient needs element-wise coefficients");
    dogip::DeviceGuard g(c->device);
    dogip::launch_grad(*c, u, lam, dA, (cudaStream_t)stream);
    return DOGIP_OK;
  });
}

}  // extern "C"
