// fd_capi.cu -- the C ABI of include/fd_layout.h: handle set-up, CSR
// validation, distance construction, and the launches of the cooperative
// layout kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "fd_internal.cuh"
#include "fd_layout.h"

namespace fdl {
cudaError_t launch_bfs(int code, int n, int nb, const int* rp, const int* ci, const int* tile_base,
                       const int* strip_len, void* D, unsigned long long* scratch, size_t stride, int grid,
                       int* maxlevel, int* overflow, int* sweeps, cudaStream_t st);
cudaError_t launch_bfs_wide(int code, int n, int nb, const int* rp, const int* ci, const int* tile_base,
                            const int* strip_len, void* D, void* words, int lcap, const int4* tasks, int ntasks,
                            void* hubacc, int* hubcnt, const int* hubparts, int nhub, unsigned long long* bar3,
                            Ctrl* ctrl, long long timeout_ns, int sm_count, int* maxlevel, int* overflow, int* sweeps,
                            cudaStream_t st);
cudaError_t launch_sssp(int n, int nb, const int* rp, const int* ci, const float* len, const int* tile_base,
                        const int* strip_len, float* D, int* scratch, int grid, int* maxbits, int* err,
                        cudaStream_t st);
cudaError_t launch_fill(int code, int n, int nb, int ntiles, const int2* tile_ik, void* D, float fill, int write,
                        unsigned long long* count, int grid, cudaStream_t st);
cudaError_t launch_rowsum(int code, int n, int nb, const int* tile_base, const int* strip_len, const void* D,
                          float* s, float* inv_s, cudaStream_t st);
cudaError_t launch_distance_rows(int code, int n, int nb, const int* tile_base, const int* strip_len,
                                 const void* D, int row0, int nrows, int hop_counts, double* out, cudaStream_t st);
cudaError_t main_config_d1(int code, size_t lut_bytes, int nbuf, int tps, int* blocks_per_sm, size_t* smem);
cudaError_t main_config_d2(int code, size_t lut_bytes, int nbuf, int tps, int* blocks_per_sm, size_t* smem);
cudaError_t main_config_d3(int code, size_t lut_bytes, int nbuf, int tps, int* blocks_per_sm, size_t* smem);
cudaError_t launch_main_d1(int code, const KParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_main_d2(int code, const KParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_main_d3(int code, const KParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t measure_fp32_peak(int packed, int sm_count, int reps, double* tflops, double* best_ms);
cudaError_t launch_direct_factor(int n, int n_pad, int nb, int code, const void* D, const int2* tile_ik, int ntiles,
                                 const float* s, float shift, float* M, float* P, float* QT, float* AT, int* err,
                                 int sm_count, cudaStream_t st);
cudaError_t launch_bfs_multi(const BGraph* graphs, const int2* items, int nitems, const int* rp, const int* ci,
                             unsigned char* D, int n_max, int* maxlevel, int* overflow, int grid, cudaStream_t st);
cudaError_t launch_fill_multi(const BGraph* graphs, const int* tile_graph, const int2* tile_ik, long long ntiles,
                              unsigned char* D, const int* maxlevel, int write, int* unreached, int* overflow, int grid,
                              cudaStream_t st);
cudaError_t launch_rowsum_multi(const BGraph* graphs, const int2* items, int nitems, const unsigned char* D, float* s,
                                float* inv_s, int grid, cudaStream_t st);
cudaError_t launch_distance_graph(const unsigned char* Dg, int n, int nb, double* out, cudaStream_t st);
cudaError_t launch_adjoint_prep(int n, int dim, const float* Xk, const float* Xk1, const float* Xb1, int accepted,
                                float omega, const float* oms, float* Y, float* Yb, float* Xb, cudaStream_t st);
cudaError_t launch_pair_adjoint(int code, int n, int nb, int dim, const int2* tile_ik, int ntiles, const void* D,
                                const float* X, const float* lam, const float* Y, float* Xb, float* Db, int sm_count,
                                cudaStream_t st);
cudaError_t launch_sp_backprop(int n, int nb, const float* Gt, const int* rp, const int* ci, const float* len,
                               const int* rev, int nnz, float* gacc, float* out, int sm_count, int global_path,
                               int* scratch, int* err, cudaStream_t st);
cudaError_t launch_length_grad(int n, int nb, int dim, const int2* tile_ik, int ntiles, const float* D,
                               const float* X, float* Gt, const int* rp, const int* ci, const float* len,
                               const int* rev, int nnz, float* gacc, float* out, int sm_count, int global_path,
                               int* scratch, int* err, cudaStream_t st);
size_t sp_backprop_scratch_ints(int n, int sm_count);
constexpr int SP_SMEM_MAX_N = 4096;  // shared-memory back-propagation up to this size (fd_grad.cu)
cudaError_t batch_config_d1(int W, int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem);
cudaError_t batch_config_d2(int W, int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem);
cudaError_t batch_config_d3(int W, int lut_bytes, int n_pad_max, int nbuf, int* blocks_per_sm, size_t* smem);
cudaError_t launch_batch_d1(int W, int cls, const BParams* p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_batch_d2(int W, int cls, const BParams* p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_batch_d3(int W, int cls, const BParams* p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_retile_multi(const BGraph* graphs, const int* list, int count, const unsigned char* D,
                                unsigned char* DT, int grid, cudaStream_t st);
}  // namespace fdl

using namespace fdl;

struct fd_layout {
  int n = 0, dim = 0, dimp = 0, n_pad = 0, nb = 0, ntiles = 0, ntasks = 0;
  int code = CODE_U8, diameter = 0, disconnected = 0;
  int device = 0, sm_count = 0, grid = 0;
  size_t smem = 0;
  cudaStream_t stream = nullptr;
  // device memory
  void* D = nullptr;
  size_t D_bytes = 0;
  int* d_tile_base = nullptr;
  int* d_strip_len = nullptr;
  TaskDesc* d_tasks = nullptr;
  int* d_cta_task_ptr = nullptr;
  unsigned char* d_lut = nullptr;
  int lut_rows = 0;
  float* d_s = nullptr;
  float* d_inv_s = nullptr;
  float* d_vec = nullptr;  // pool of the per-vertex vectors
  double* d_acc = nullptr;     // [3][n_pad][dimp] per-vertex accumulators (FP64)
  int weighted = 0;             // 1 if the graph was given edge lengths
  int nbuf = 2;                 // stages of the kernel's tile pipeline
  int tps = 1;                  // tiles per stage
  Ctrl* d_ctrl = nullptr;
  float* d_stage_in = nullptr;
  float* d_stage_out = nullptr;
  double* d_omega = nullptr;
  double* d_trace_f = nullptr;
  double* d_trace_om = nullptr;
  double* d_trace_crit = nullptr;
  double* d_trace_fh = nullptr;
  double* d_trace_ft = nullptr;
  double* d_trace_t = nullptr;
  int* d_trace_acc = nullptr;
  int* d_trace_cg = nullptr;
  int trace_cap = 0;
  int last_iters = 0;
  // host
  std::vector<int> tile_base, strip_len, cta_task_ptr;
  std::vector<TaskDesc> tasks;
  fd_status last_error = FD_OK;
  fd_stats stats;
  long long timeout_ns = 30000000000LL;      // copy (mbarrier) waits
  long long bar_timeout_ns = 30000000000LL;  // grid-barrier waits
  double apsp_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double* d_timeline = nullptr;  // tracing: [timeline_cap][2]
  int timeline_cap = 0;
  int timeline_n = 0;
  // weighted graphs: the CSR kept for the derivative in the edge lengths
  int* d_wrp = nullptr;
  int* d_wci = nullptr;
  float* d_wlen = nullptr;
  int* d_wrev = nullptr;  // index of the reverse entry of every CSR entry
  int wnnz = 0;
  int wsimple = 0;        // no self loops, no repeated entries
  int bfs_sweeps = 0;     // passes over the edge list of all multi-source searches
  int bfs_sources = 0;    // sources per search: 64 (one CTA each) or 256 (all CTAs, level-synchronous)
  // unrolled differentiation: pair sensitivities summed over the adjoint steps (tile layout)
  float* d_dbar = nullptr;
  float* d_adj = nullptr;  // [4][n][dim]: Y, Yb, lam, Xb staging
  // per-vertex relaxation factors m_i (omega_i = omega m_i, Sec. 6); NULL: none
  float* d_om_scale = nullptr;  // [n_pad], padding 0
  // direct solver: (L^W + sigma/n 1 1^T)^-1, [n_pad][n_pad] (fd_factor)
  float* d_ainv = nullptr;
  double factor_ms = 0.0;
};

namespace {

fd_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FD_OK;
  if (e == cudaErrorMemoryAllocation) return FD_ERR_OOM;
  return FD_ERR_CUDA;
}

#define FD_CK(expr)                          \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) {                 \
      cudaGetLastError();                    \
      return cuda_status(e_);                \
    }                                        \
  } while (0)

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
fd_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return cuda_status(e);
  }
  return FD_OK;
}

template <class T>
void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Copies count elements of a caller array (host or device) to a host vector.
template <class T>
fd_status fetch_host(std::vector<T>& out, const T* src, size_t count) {
  out.resize(count);
  if (count == 0) return FD_OK;
  if (is_device_ptr(src)) {
    FD_CK(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), src, count * sizeof(T));
  }
  return FD_OK;
}

// CSR checks: shape, ranges, symmetry (with equal lengths when given).
fd_status validate_csr(int n, const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<float>* len) {
  if ((int)rp.size() != n + 1 || rp[0] != 0) return FD_ERR_CSR;
  for (int v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return FD_ERR_CSR;
  const size_t nnz = (size_t)rp[n];
  if (ci.size() != nnz) return FD_ERR_CSR;
  for (size_t e = 0; e < nnz; ++e)
    if (ci[e] < 0 || ci[e] >= n) return FD_ERR_CSR;
  if (len) {
    for (size_t e = 0; e < nnz; ++e)
      if (!(std::isfinite((*len)[e]) && (*len)[e] > 0.f)) return FD_ERR_CSR;
  }
  // per-row sorted (neighbour, shortest length) lists
  std::vector<std::pair<int, float>> adj(nnz);
  for (int v = 0; v < n; ++v) {
    for (int e = rp[v]; e < rp[v + 1]; ++e) adj[e] = {ci[e], len ? (*len)[e] : 1.f};
    std::sort(adj.begin() + rp[v], adj.begin() + rp[v + 1]);
  }
  for (int u = 0; u < n; ++u) {
    for (int e = rp[u]; e < rp[u + 1]; ++e) {
      const int v = adj[e].first;
      if (e > rp[u] && adj[e - 1].first == v) continue;  // first (shortest) entry of a repeated edge
      if (v == u) continue;
      auto b = adj.begin() + rp[v], en = adj.begin() + rp[v + 1];
      auto it = std::lower_bound(b, en, std::make_pair(u, -INFINITY));
      if (it == en || it->first != u) return FD_ERR_CSR;
      if (len && it->second != adj[e].second) return FD_ERR_CSR;
    }
  }
  return FD_OK;
}

// Hop eccentricity of vertex 0 within its component (host BFS).
int host_ecc0(int n, const std::vector<int>& rp, const std::vector<int>& ci) {
  std::vector<int> dist(n, -1), q;
  q.reserve(n);
  dist[0] = 0;
  q.push_back(0);
  int ecc = 0;
  for (size_t h = 0; h < q.size(); ++h) {
    const int u = q[h];
    for (int e = rp[u]; e < rp[u + 1]; ++e) {
      const int v = ci[e];
      if (dist[v] < 0) {
        dist[v] = dist[u] + 1;
        ecc = std::max(ecc, dist[v]);
        q.push_back(v);
      }
    }
  }
  return ecc;
}

uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Probabilistic strategy of Sec. 5.2.3 (prior 0.3, 0.3, 0.2, 0.2 over 0.5, 1, 1.5, 2).
double omega_prob(uint64_t seed, uint64_t k) {
  const double u = (double)(splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
  if (u < 0.3) return 0.5;
  if (u < 0.6) return 1.0;
  if (u < 0.8) return 1.5;
  return 2.0;
}

void build_geometry(fd_layout* h) {
  h->n_pad = ((h->n + TILE - 1) / TILE) * TILE;
  h->nb = h->n_pad / TILE;
  const int nb = h->nb;
  h->strip_len.assign(nb, 0);
  h->tile_base.assign(nb + 1, 0);
  for (int I = 0; I < nb; ++I) {
    int L;
    if (nb % 2 == 1) L = (nb + 1) / 2;
    else L = (I < nb / 2) ? nb / 2 + 1 : nb / 2;
    h->strip_len[I] = L;
    h->tile_base[I + 1] = h->tile_base[I] + L;
  }
  h->ntiles = h->tile_base[nb];
}

void build_tasks(fd_layout* h) {
  // CTA b owns tiles [T b / G, T (b+1) / G) of the strip-major order: equal
  // work per CTA and few, long tasks (one per strip the range touches)
  const long long T = h->ntiles, G = h->grid;
  h->tasks.clear();
  h->cta_task_ptr.assign(h->grid + 1, 0);
  int I = 0;
  for (long long b = 0; b < G; ++b) {
    const long long t0 = T * b / G, t1 = T * (b + 1) / G;
    long long t = t0;
    while (t < t1) {
      while (h->tile_base[I + 1] <= t) ++I;
      const long long e = std::min<long long>(t1, h->tile_base[I + 1]);
      TaskDesc d;
      d.I = I;
      d.k0 = (int)(t - h->tile_base[I]);
      d.k1 = (int)(e - h->tile_base[I]);
      d.tile0 = (int)t;
      h->tasks.push_back(d);
      t = e;
    }
    h->cta_task_ptr[b + 1] = (int)h->tasks.size();
  }
  h->ntasks = (int)h->tasks.size();
}

cudaError_t main_config(int dim, int code, size_t lut_bytes, int nbuf, int tps, int* bps, size_t* smem) {
  if (dim == 1) return main_config_d1(code, lut_bytes, nbuf, tps, bps, smem);
  if (dim == 2) return main_config_d2(code, lut_bytes, nbuf, tps, bps, smem);
  return main_config_d3(code, lut_bytes, nbuf, tps, bps, smem);
}

cudaError_t launch_main(int dim, int code, const KParams& p, int grid, size_t smem, cudaStream_t st) {
  if (dim == 1) return launch_main_d1(code, p, grid, smem, st);
  if (dim == 2) return launch_main_d2(code, p, grid, smem, st);
  return launch_main_d3(code, p, grid, smem, st);
}

void release(fd_layout* h) {
  dev_free(h->D);
  dev_free(h->d_tile_base);
  dev_free(h->d_strip_len);
  dev_free(h->d_tasks);
  dev_free(h->d_cta_task_ptr);
  dev_free(h->d_lut);
  dev_free(h->d_s);
  dev_free(h->d_inv_s);
  dev_free(h->d_vec);
  dev_free(h->d_acc);
  dev_free(h->d_ctrl);
  dev_free(h->d_stage_in);
  dev_free(h->d_stage_out);
  dev_free(h->d_omega);
  dev_free(h->d_trace_f);
  dev_free(h->d_trace_om);
  dev_free(h->d_trace_crit);
  dev_free(h->d_trace_fh);
  dev_free(h->d_trace_ft);
  dev_free(h->d_trace_t);
  dev_free(h->d_trace_acc);
  dev_free(h->d_trace_cg);
  dev_free(h->d_timeline);
  dev_free(h->d_wrp);
  dev_free(h->d_wci);
  dev_free(h->d_wlen);
  dev_free(h->d_wrev);
  dev_free(h->d_dbar);
  dev_free(h->d_adj);
  dev_free(h->d_om_scale);
  dev_free(h->d_ainv);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  h->ev0 = h->ev1 = nullptr;
}

fd_status fail(fd_layout* h, fd_status s) {
  if (h) h->last_error = s;
  return s;
}

// Distances for unit edges (BFS) or lengths (relaxation); returns the code
// kind actually used (u8 may fall back to f32 on a large diameter).
fd_status build_distances(fd_layout* h, const std::vector<int>& rp, const std::vector<int>& ci,
                          const std::vector<float>* len, int policy) {
  const int n = h->n, nb = h->nb;
  cudaStream_t st = h->stream;
  int *d_rp = nullptr, *d_ci = nullptr, *d_flags = nullptr;
  float* d_len = nullptr;
  int2* d_tile_ik = nullptr;
  unsigned long long* d_count = nullptr;
  void* scratch = nullptr;
  fd_status s = FD_OK;
  const size_t nnz = rp[n];
  auto cleanup = [&]() {
    dev_free(d_rp);
    dev_free(d_ci);
    dev_free(d_len);
    dev_free(d_flags);
    dev_free(d_tile_ik);
    dev_free(d_count);
    if (scratch) cudaFree(scratch);
    scratch = nullptr;
  };
#define FD_TRY(expr)            \
  do {                          \
    s = (expr);                 \
    if (s != FD_OK) {           \
      cleanup();                \
      return s;                 \
    }                           \
  } while (0)
#define FD_TRYC(expr) FD_TRY(cuda_status(expr))

  FD_TRY(dev_alloc(&d_rp, n + 1));
  FD_TRY(dev_alloc(&d_ci, nnz));
  FD_TRY(dev_alloc(&d_flags, 5));
  FD_TRY(dev_alloc(&d_count, 1));
  FD_TRYC(cudaMemcpyAsync(d_rp, rp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  if (nnz) FD_TRYC(cudaMemcpyAsync(d_ci, ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<int2> tile_ik(h->ntiles);
  for (int I = 0; I < nb; ++I)
    for (int k = 0; k < h->strip_len[I]; ++k) tile_ik[h->tile_base[I] + k] = make_int2(I, k);
  FD_TRY(dev_alloc(&d_tile_ik, h->ntiles));
  FD_TRYC(cudaMemcpyAsync(d_tile_ik, tile_ik.data(), h->ntiles * sizeof(int2), cudaMemcpyHostToDevice, st));

  int code = len ? CODE_F32 : CODE_U8;
  const int ecc0 = n ? host_ecc0(n, rp, ci) : 0;
  if (code == CODE_U8 && ecc0 >= 254) code = CODE_F32;
  float fill = 0.f;
  for (int attempt = 0; attempt < 2; ++attempt) {
    h->code = code;
    const size_t cb = (code == CODE_U8) ? 1 : 4;
    h->D_bytes = (size_t)h->ntiles * TILE * TILE * cb;
    dev_free(h->D);
    FD_TRY(dev_alloc((unsigned char**)&h->D, h->D_bytes));
    FD_TRYC(cudaMemsetAsync(h->D, 0, h->D_bytes, st));
    FD_TRYC(cudaMemsetAsync(d_flags, 0, 5 * sizeof(int), st));
    int diameter = 0;
    if (!len) {
      if (scratch) cudaFree(scratch);
      scratch = nullptr;
      // Level-synchronous 256-source searches over all CTAs for large graphs
      // of few levels (a grid barrier per level); one 64-source search per
      // CTA otherwise.  FDLAYOUT_BFS_WIDE=0/1 forces either (testing).
      bool wide = n >= 65536 && ecc0 <= 32;
      if (const char* e = std::getenv("FDLAYOUT_BFS_WIDE")) wide = (e[0] == '1');
      Ctrl* d_bctrl = nullptr;
      int4* d_tasks = nullptr;
      int *d_hubcnt = nullptr, *d_hubparts = nullptr;
      void* d_hubacc = nullptr;
      std::vector<int4> tasks;
      std::vector<int> hubparts;
      // frontiers kept for the end-of-batch 1-byte codes: the levels of
      // vertex 0's component are <= 2 ecc0, other components' may be more
      // (deeper levels write their codes as reached)
      const int lcap = (code == CODE_U8) ? std::min(255, std::max(16, 2 * ecc0 + 1)) : 0;
      const size_t wbytes = (size_t)(lcap + 4) * n * 32, cbytes = (sizeof(Ctrl) + 255) / 256 * 256;
      if (wide) {
        // warp tasks: vertices of degree > 16 (WIDE_BIG_DEG), largest first;
        // a hub of degree > 256 (WIDE_HUB_CHUNK) as tasks of 256 edges
        std::vector<int> big;
        for (int v = 0; v < n; ++v)
          if (rp[v + 1] - rp[v] > 16) big.push_back(v);
        std::stable_sort(big.begin(), big.end(),
                         [&](int a, int b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
        for (int v : big) {
          const int deg = rp[v + 1] - rp[v];
          if (deg > 256) {
            const int hid = (int)hubparts.size(), parts = (deg + 255) / 256;
            hubparts.push_back(parts);
            for (int q = 0; q < parts; ++q)
              tasks.push_back(make_int4(v, rp[v] + 256 * q, std::min(rp[v] + 256 * (q + 1), rp[v + 1]),
                                        2 * hid + (q == 0 ? 1 : 0)));
          } else {
            tasks.push_back(make_int4(v, rp[v], rp[v + 1], -1));
          }
        }
        const size_t nh = hubparts.size();
        const size_t tbytes = (tasks.size() * sizeof(int4) + 255) / 256 * 256;
        const size_t hbytes = nh * 32 + nh * sizeof(int);  // hub words, hub counters (zeroed)
        // [lcap + 4][n] 32-byte words, the 3 barrier slots, the error state,
        // tasks, hub words and counters, hub task counts
        char* base = nullptr;
        FD_TRYC(cudaMalloc(&scratch, wbytes + 256 + cbytes + tbytes + hbytes + nh * sizeof(int) + 16));
        base = (char*)scratch + wbytes;
        FD_TRYC(cudaMemsetAsync(base, 0, 256 + cbytes, st));
        d_bctrl = reinterpret_cast<Ctrl*>(base + 256);
        d_tasks = reinterpret_cast<int4*>(base + 256 + cbytes);
        d_hubacc = base + 256 + cbytes + tbytes;
        d_hubcnt = reinterpret_cast<int*>(base + 256 + cbytes + tbytes + nh * 32);
        d_hubparts = d_hubcnt + nh;
        if (!tasks.empty())
          FD_TRYC(cudaMemcpyAsync(d_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        if (nh) {
          FD_TRYC(cudaMemsetAsync(d_hubacc, 0, hbytes, st));
          FD_TRYC(cudaMemcpyAsync(d_hubparts, hubparts.data(), nh * sizeof(int), cudaMemcpyHostToDevice, st));
        }
      } else {
        const int nbatches = (n + 63) / 64;
        const int grid = std::max(1, std::min(nbatches, 2 * h->sm_count));
        const size_t stride = (size_t)3 * n;
        FD_TRYC(cudaMalloc(&scratch, (size_t)grid * stride * sizeof(unsigned long long)));
      }
      FD_TRYC(cudaEventRecord(h->ev0, st));
      if (wide) {
        FD_TRYC(launch_bfs_wide(code, n, nb, d_rp, d_ci, h->d_tile_base, h->d_strip_len, h->D, scratch, lcap, d_tasks,
                                (int)tasks.size(), d_hubacc, d_hubcnt, d_hubparts, (int)hubparts.size(),
                                (unsigned long long*)((char*)scratch + wbytes), d_bctrl, h->bar_timeout_ns,
                                h->sm_count, d_flags, d_flags + 1, d_flags + 3, st));
      } else {
        const int nbatches = (n + 63) / 64;
        const int grid = std::max(1, std::min(nbatches, 2 * h->sm_count));
        FD_TRYC(launch_bfs(code, n, nb, d_rp, d_ci, h->d_tile_base, h->d_strip_len, h->D,
                           (unsigned long long*)scratch, (size_t)3 * n, grid, d_flags, d_flags + 1, d_flags + 3, st));
      }
      FD_TRYC(cudaEventRecord(h->ev1, st));
      int flags[4];
      FD_TRYC(cudaMemcpyAsync(flags, d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
      int berr = 0;
      if (wide) FD_TRYC(cudaMemcpyAsync(&berr, &d_bctrl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
      FD_TRYC(cudaStreamSynchronize(st));
      if (berr) {  // a grid-barrier wait ran out
        cleanup();
        return FD_ERR_TIMEOUT;
      }
      h->bfs_sources = wide ? 256 : 64;
      float ms = 0.f;
      FD_TRYC(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
      h->apsp_ms = ms;
      h->bfs_sweeps = flags[3];
      diameter = flags[0];
      if (flags[1] && code == CODE_U8) {  // a level above 255: store float codes
        code = CODE_F32;
        continue;
      }
      fill = (float)(diameter + 1);
    } else {
      FD_TRY(dev_alloc(&d_len, nnz));
      FD_TRYC(cudaMemcpyAsync(d_len, len->data(), nnz * sizeof(float), cudaMemcpyHostToDevice, st));
      const int grid = std::max(1, std::min(n, 2 * h->sm_count));
      if (scratch) cudaFree(scratch);
      scratch = nullptr;
      FD_TRYC(cudaMalloc(&scratch, (size_t)grid * 4 * n * sizeof(int)));  // per CTA: distances, stamps, 2 frontiers
      FD_TRYC(cudaEventRecord(h->ev0, st));
      FD_TRYC(launch_sssp(n, nb, d_rp, d_ci, d_len, h->d_tile_base, h->d_strip_len, (float*)h->D, (int*)scratch,
                          grid, d_flags + 2, d_flags + 4, st));
      FD_TRYC(cudaEventRecord(h->ev1, st));
      int bits, serr = 0;
      FD_TRYC(cudaMemcpyAsync(&bits, d_flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
      FD_TRYC(cudaMemcpyAsync(&serr, d_flags + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
      FD_TRYC(cudaStreamSynchronize(st));
      if (serr) {  // a search ran out of rounds
        cleanup();
        return FD_ERR_TIMEOUT;
      }
      float ms = 0.f;
      FD_TRYC(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
      h->apsp_ms = ms;
      float dmax;
      std::memcpy(&dmax, &bits, sizeof(float));
      diameter = (int)std::ceil(dmax);
      fill = dmax + 1.f;
    }
    // unreachable pairs
    unsigned long long count = 0;
    FD_TRYC(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    const int fgrid = 4 * h->sm_count;
    if (code == CODE_U8 && policy == 1 && fill > 255.f) {
      code = CODE_F32;  // fill value does not fit a byte
      continue;
    }
    FD_TRYC(launch_fill(code, n, nb, h->ntiles, d_tile_ik, h->D, fill, policy == 1 ? 1 : 0, d_count, fgrid, st));
    FD_TRYC(cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, st));
    FD_TRYC(cudaStreamSynchronize(st));
    if (count > 0 && policy != 1) {
      cleanup();
      return FD_ERR_DISCONNECTED;
    }
    h->disconnected = count > 0 ? 1 : 0;
    h->diameter = diameter;
    break;
  }
  cleanup();
  return FD_OK;
#undef FD_TRY
#undef FD_TRYC
}

fd_status ensure_traces(fd_layout* h, int max_iter) {
  if (h->trace_cap >= max_iter + 1) return FD_OK;
  dev_free(h->d_omega);
  dev_free(h->d_trace_f);
  dev_free(h->d_trace_om);
  dev_free(h->d_trace_crit);
  dev_free(h->d_trace_fh);
  dev_free(h->d_trace_ft);
  dev_free(h->d_trace_t);
  dev_free(h->d_trace_acc);
  dev_free(h->d_trace_cg);
  h->trace_cap = 0;
  const int cap = max_iter + 1;
  fd_status s;
  if ((s = dev_alloc(&h->d_omega, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_f, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_om, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_crit, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_fh, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_ft, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_t, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_acc, cap)) != FD_OK) return s;
  if ((s = dev_alloc(&h->d_trace_cg, cap)) != FD_OK) return s;
  h->trace_cap = cap;
  return FD_OK;
}

KParams base_params(fd_layout* h, int mode) {
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.g.n = h->n;
  p.g.n_pad = h->n_pad;
  p.g.nb = h->nb;
  p.g.dim = h->dim;
  p.g.ntiles = h->ntiles;
  p.g.ntasks = h->ntasks;
  p.g.tile_base = h->d_tile_base;
  p.g.strip_len = h->d_strip_len;
  p.g.tasks = h->d_tasks;
  p.g.cta_task_ptr = h->d_cta_task_ptr;
  p.mode = mode;
  p.D = h->D;
  p.lut = h->d_lut;
  p.lut_rows = h->lut_rows;
  p.nbuf = h->nbuf;
  p.tps = h->tps;
  p.s = h->d_s;
  p.inv_s = h->d_inv_s;
  const size_t vs = (size_t)h->n_pad * h->dimp;
  float* v = h->d_vec;
  float** slots[] = {&p.X, &p.R0, &p.Xt, &p.B, &p.Bz, &p.Bt, &p.Zw, &p.R, &p.U, &p.W, &p.P, &p.S};
  for (int k = 0; k < 12; ++k) *slots[k] = v + k * vs;
  p.acc = h->d_acc;
  p.ctrl = h->d_ctrl;
  p.timeout_ns = h->timeout_ns;
  p.bar_timeout_ns = h->bar_timeout_ns;
  p.max_iter = 0;
  p.timeline = h->timeline_cap > 0 ? h->d_timeline : nullptr;
  p.timeline_cap = h->timeline_cap;
  return p;
}

// Runs one cooperative launch; returns the device status and the control block.
fd_status run_kernel(fd_layout* h, KParams& p, Ctrl* ctrl_out, double* kernel_ms) {
  cudaStream_t st = h->stream;
  FD_CK(cudaMemsetAsync(h->d_ctrl, 0, sizeof(Ctrl), st));
  FD_CK(cudaEventRecord(h->ev0, st));
  FD_CK(launch_main(h->dim, h->code, p, h->grid, h->smem, st));
  FD_CK(cudaEventRecord(h->ev1, st));
  FD_CK(cudaMemcpyAsync(ctrl_out, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  FD_CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  FD_CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  *kernel_ms = ms;
  h->timeline_n = std::min(ctrl_out->timeline_n, h->timeline_cap);
  if (ctrl_out->err != 0) return (fd_status)ctrl_out->err;
  return FD_OK;
}

void fill_stats(fd_layout* h, const Ctrl& c, double kms) {
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->stats.iterations = c.iters;
  h->stats.cg_steps = c.cg_steps;
  h->stats.cg_maxed = c.cg_maxed;
  h->stats.accepted = c.accepted;
  h->stats.pair_passes = c.pair_passes;
  h->stats.pairs = 0.5 * (double)h->n * (double)(h->n - 1);
  h->stats.final_stress = c.f_final;
  h->stats.final_crit = c.crit_final;
  h->stats.matvec_passes = c.matvec_passes;
  h->stats.stress_passes = c.stress_passes;
  h->stats.kernel_ms = kms;
  h->stats.cg_stalled = c.cg_stalled;
  h->stats.enum_candidate_passes = c.enum_passes;
  h->stats.rhs_skipped = c.rhs_skipped;
}

// Positions in: device pointers are used in place, host arrays are staged.
fd_status stage_input(fd_layout* h, const float* X, const float** dev_x) {
  if (is_device_ptr(X)) {
    *dev_x = X;
    return FD_OK;
  }
  FD_CK(cudaMemcpyAsync(h->d_stage_in, X, (size_t)h->n * h->dim * sizeof(float), cudaMemcpyHostToDevice,
                        h->stream));
  *dev_x = h->d_stage_in;
  return FD_OK;
}

}  // namespace

extern "C" {

void fd_options_default(fd_options* opt) {
  if (!opt) return;
  opt->omega = 0.5;
  opt->strategy = FD_OMEGA_FIXED;
  opt->stop = FD_STOP_REL_DISP;
  opt->seed = 0;
  opt->tol = 1e-4;
  opt->max_iter = 1000;
  opt->cg_max = 200;
  opt->cg_tol = 1e-6;
  opt->solver = FD_SOLVER_CG;
  opt->first_iter = 0;
}

const char* fd_status_string(fd_status s) {
  switch (s) {
    case FD_OK: return "FD_OK";
    case FD_ERR_ARG: return "FD_ERR_ARG";
    case FD_ERR_CSR: return "FD_ERR_CSR";
    case FD_ERR_DISCONNECTED: return "FD_ERR_DISCONNECTED";
    case FD_ERR_NONFINITE: return "FD_ERR_NONFINITE";
    case FD_ERR_CG_BREAKDOWN: return "FD_ERR_CG_BREAKDOWN";
    case FD_ERR_CG_MAXITER: return "FD_ERR_CG_MAXITER";
    case FD_ERR_TIMEOUT: return "FD_ERR_TIMEOUT";
    case FD_ERR_OOM: return "FD_ERR_OOM";
    case FD_ERR_CUDA: return "FD_ERR_CUDA";
    case FD_ERR_UNIMPLEMENTED: return "FD_ERR_UNIMPLEMENTED";
  }
  return "FD_ERR_UNKNOWN";
}

fd_status fd_layout_create(fd_layout** out, int32_t n, int32_t dim, const int32_t* row_ptr, const int32_t* col_idx,
                           const float* edge_len, int32_t disconnected_policy, void* cuda_stream) {
  if (!out) return FD_ERR_ARG;
  *out = nullptr;
  if (n < 1 || dim < 1 || dim > 3 || !row_ptr || (disconnected_policy != 0 && disconnected_policy != 1))
    return FD_ERR_ARG;
  std::vector<int> rp, ci;
  std::vector<float> len;
  fd_status s = fetch_host(rp, row_ptr, (size_t)n + 1);
  if (s != FD_OK) return s;
  if (rp[0] != 0 || rp[n] < 0) return FD_ERR_CSR;
  if (rp[n] > 0 && !col_idx) return FD_ERR_ARG;
  if ((s = fetch_host(ci, col_idx, (size_t)rp[n])) != FD_OK) return s;
  if (edge_len) {
    if ((s = fetch_host(len, edge_len, (size_t)rp[n])) != FD_OK) return s;
  }
  if ((s = validate_csr(n, rp, ci, edge_len ? &len : nullptr)) != FD_OK) return s;

  fd_layout* h = new (std::nothrow) fd_layout();
  if (!h) return FD_ERR_OOM;
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->n = n;
  h->dim = dim;
  h->dimp = (dim == 3) ? 4 : dim;
  h->stream = (cudaStream_t)cuda_stream;
  auto bail = [&](fd_status e) {
    release(h);
    delete h;
    return e;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  build_geometry(h);
  if ((s = dev_alloc(&h->d_tile_base, h->nb + 1)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_strip_len, h->nb)) != FD_OK) return bail(s);
  if (cudaMemcpy(h->d_tile_base, h->tile_base.data(), (h->nb + 1) * sizeof(int), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(h->d_strip_len, h->strip_len.data(), h->nb * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  h->weighted = edge_len ? 1 : 0;
  if ((s = build_distances(h, rp, ci, edge_len ? &len : nullptr, disconnected_policy)) != FD_OK) return bail(s);
  if (edge_len) {
    // keep the CSR on the device for fd_energy_length_grad, with the reverse of every entry
    const int nnz = rp[n];
    std::vector<int> rev(nnz, -1);
    bool simple = true;
    for (int u = 0; u < n && simple; ++u) {
      for (int e = rp[u]; e < rp[u + 1]; ++e) {
        const int v = ci[e];
        if (v == u || (e > rp[u] && std::find(ci.begin() + rp[u], ci.begin() + e, v) != ci.begin() + e)) {
          simple = false;
          break;
        }
        for (int f = rp[v]; f < rp[v + 1]; ++f)
          if (ci[f] == u) {
            rev[e] = f;
            break;
          }
      }
    }
    h->wsimple = simple ? 1 : 0;
    h->wnnz = nnz;
    if (simple && nnz > 0) {
      if ((s = dev_alloc(&h->d_wrp, (size_t)n + 1)) != FD_OK || (s = dev_alloc(&h->d_wci, (size_t)nnz)) != FD_OK ||
          (s = dev_alloc(&h->d_wlen, (size_t)nnz)) != FD_OK || (s = dev_alloc(&h->d_wrev, (size_t)nnz)) != FD_OK)
        return bail(s);
      if (cudaMemcpy(h->d_wrp, rp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_wci, ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_wlen, len.data(), nnz * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->d_wrev, rev.data(), nnz * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return bail(FD_ERR_CUDA);
      }
    }
  }

  // replicated lookup table for uint8 codes 0 .. lut_rows-1 (shared memory):
  // row c = 32 x float 1/c, then 32 x float 1/c^2 (one copy per lane); row 0 (no pair) is zero
  h->lut_rows = (h->code == CODE_U8) ? std::min(LUT_N, h->diameter + 2) : 0;
  std::vector<unsigned char> lut((size_t)std::max(h->lut_rows, 1) * LUT_ROW, 0);
  for (int c = 1; c < h->lut_rows; ++c) {
    float* row = reinterpret_cast<float*>(lut.data() + (size_t)c * LUT_ROW);
    const float w = (float)(1.0 / ((double)c * c)), inv = (float)(1.0 / c);
    for (int k = 0; k < 32; ++k) {
      row[k] = inv;
      row[32 + k] = w;
    }
  }
  // launch configuration of the cooperative kernel: the most resident CTAs,
  // then two tiles per stage (uint8 codes: half the per-tile copy issue,
  // barrier and vector formation) when two such stages keep that residency,
  // then the most stages
  const size_t lut_bytes = (size_t)h->lut_rows * LUT_ROW;
  int bps = 0, best_bps = 0, best_nbuf = 0, best_tps = 1;
  int nbuf_only = 0, tps_only = 0;
  if (const char* e = std::getenv("FDLAYOUT_NBUF")) nbuf_only = std::atoi(e);  // testing: force the stage count
  if (const char* e = std::getenv("FDLAYOUT_TPS")) tps_only = std::atoi(e);    // testing: force tiles per stage
  for (int tps = 2; tps >= 1; --tps) {
    // Two-tile stages measured faster only for uint8 codes with a small lookup
    // table (there two of them fit beside it at two CTAs per SM; 8 KB = hop
    // diameters up to 30): L^W passes 10 % faster in 2-D, 5-7 % in 3-D (two
    // stages there); 64 KB float tiles take one per stage, and beside a large
    // table one-tile stages (more of them) win.
    const bool tps2_ok = h->code == CODE_U8 && lut_bytes <= 8192;
    if (tps == 2 && !tps2_ok && tps_only != 2) continue;
    if (tps == 2 && h->code != CODE_U8) continue;  // not instantiated
    if (tps_only && tps != tps_only) continue;
    for (int nbuf = MAX_NBUF; nbuf >= 2; --nbuf) {
      if (nbuf_only && nbuf != nbuf_only) continue;
      size_t smem = 0;
      if (main_config(dim, h->code, lut_bytes, nbuf, tps, &bps, &smem) != cudaSuccess) {
        cudaGetLastError();
        bps = 0;
      }
      if (bps > best_bps) {
        best_bps = bps;
        best_nbuf = nbuf;
        best_tps = tps;
      }
    }
  }
  if (best_bps < 1 || main_config(dim, h->code, lut_bytes, best_nbuf, best_tps, &bps, &h->smem) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  h->nbuf = best_nbuf;
  h->tps = best_tps;
  h->grid = bps * h->sm_count;
  if (const char* t = std::getenv("FDLAYOUT_BARRIER_TIMEOUT_NS")) {  // testing: make grid-barrier waits run out
    const long long v = std::atoll(t);
    if (v > 0) h->bar_timeout_ns = v;
  }
  if (const char* cap = std::getenv("FDLAYOUT_MAX_CTAS")) {  // testing: force many tasks per CTA
    const int c = std::atoi(cap);
    if (c > 0 && c < h->grid) h->grid = c;
  }
  build_tasks(h);
  const size_t vs = (size_t)h->n_pad * h->dimp;
  if ((s = dev_alloc(&h->d_lut, lut.size())) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_s, h->n_pad)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_inv_s, h->n_pad)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_vec, 12 * vs)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_acc, 3 * vs)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_ctrl, 1)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_stage_in, (size_t)n * dim)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_stage_out, (size_t)n * dim)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_tasks, h->ntasks)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&h->d_cta_task_ptr, h->grid + 1)) != FD_OK) return bail(s);
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(h->d_lut, lut.data(), lut.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(h->d_acc, 0, 3 * vs * sizeof(double), st) != cudaSuccess ||
      cudaMemcpyAsync(h->d_tasks, h->tasks.data(), h->ntasks * sizeof(TaskDesc), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->d_cta_task_ptr, h->cta_task_ptr.data(), (h->grid + 1) * sizeof(int),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(h->d_vec, 0, 12 * vs * sizeof(float), st) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  if (launch_rowsum(h->code, n, h->nb, h->d_tile_base, h->d_strip_len, h->D, h->d_s, h->d_inv_s, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  *out = h;
  return FD_OK;
}

void fd_layout_destroy(fd_layout* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  release(h);
  delete h;
}

fd_status fd_energy(fd_layout* h, const float* X, double* f_out) {
  if (!h) return FD_ERR_ARG;
  if (!X || !f_out) return fail(h, FD_ERR_ARG);
  const float* dx = nullptr;
  fd_status s = stage_input(h, X, &dx);
  if (s != FD_OK) return fail(h, s);
  KParams p = base_params(h, KM_ENERGY);
  p.x_in = dx;
  Ctrl c;
  double kms = 0.0;
  std::memset(&c, 0, sizeof(c));
  s = run_kernel(h, p, &c, &kms);
  fill_stats(h, c, kms);
  if (s != FD_OK) return fail(h, s);
  *f_out = c.f_final;
  return FD_OK;
}

fd_status fd_forces(fd_layout* h, const float* X, float* F_out) {
  if (!h) return FD_ERR_ARG;
  if (!X || !F_out) return fail(h, FD_ERR_ARG);
  const float* dx = nullptr;
  fd_status s = stage_input(h, X, &dx);
  if (s != FD_OK) return fail(h, s);
  KParams p = base_params(h, KM_FORCES);
  p.x_in = dx;
  const bool dev_out = is_device_ptr(F_out);
  p.x_out = dev_out ? F_out : h->d_stage_out;
  Ctrl c;
  double kms = 0.0;
  std::memset(&c, 0, sizeof(c));
  s = run_kernel(h, p, &c, &kms);
  fill_stats(h, c, kms);
  if (s != FD_OK) return fail(h, s);
  if (!dev_out) {
    if (cudaMemcpyAsync(F_out, h->d_stage_out, (size_t)h->n * h->dim * sizeof(float), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, FD_ERR_CUDA);
    }
  }
  return FD_OK;
}

// Scratch of the shortest-path back-propagation: none for the shared-memory
// kernel; 7 n ints per CTA plus an error flag for the global one (larger
// graphs, or FDLAYOUT_SP_GLOBAL=1 to test it on small ones).
struct SpScratch {
  int global_path = 0;
  int* ints = nullptr;  // [sp_backprop_scratch_ints]; the last int is the error flag
  int* err = nullptr;
  ~SpScratch() { dev_free(ints); }
  fd_status init(const fd_layout* h, cudaStream_t st) {
    const char* g = std::getenv("FDLAYOUT_SP_GLOBAL");
    global_path = (h->n > SP_SMEM_MAX_N || (g && std::atoi(g) != 0)) ? 1 : 0;
    if (!global_path) return FD_OK;
    const size_t cnt = sp_backprop_scratch_ints(h->n, h->sm_count) + 1;
    fd_status s = dev_alloc(&ints, cnt);
    if (s != FD_OK) return s;
    err = ints + cnt - 1;
    FD_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    return FD_OK;
  }
  // after the stream is synchronised: FD_ERR_TIMEOUT if a search ran out of rounds
  fd_status check() const {
    if (!err) return FD_OK;
    int v = 0;
    if (cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return FD_ERR_CUDA;
    }
    return v ? FD_ERR_TIMEOUT : FD_OK;
  }
};

fd_status fd_energy_length_grad(fd_layout* h, const float* X, float* grad_len, double* f_out) {
  if (!h) return FD_ERR_ARG;
  if (!X || !grad_len) return fail(h, FD_ERR_ARG);
  if (h->code != CODE_F32 || !h->d_wrp || h->wnnz == 0) return fail(h, FD_ERR_ARG);  // not a weighted graph
  if (h->n > FD_GRAD_MAX_N || h->disconnected || !h->wsimple) return fail(h, FD_ERR_UNIMPLEMENTED);
  const float* dx = nullptr;
  fd_status s = stage_input(h, X, &dx);
  if (s != FD_OK) return fail(h, s);
  // the stress itself (one stress pass of the layout kernel)
  KParams p = base_params(h, KM_ENERGY);
  p.x_in = dx;
  Ctrl c;
  double kms = 0.0;
  std::memset(&c, 0, sizeof(c));
  s = run_kernel(h, p, &c, &kms);
  fill_stats(h, c, kms);
  if (s != FD_OK) return fail(h, s);
  std::vector<int2> tile_ik(h->ntiles);
  for (int I = 0; I < h->nb; ++I)
    for (int k = 0; k < h->strip_len[I]; ++k) tile_ik[h->tile_base[I] + k] = make_int2(I, k);
  int2* d_tik = nullptr;
  float *d_G = nullptr, *d_acc = nullptr, *d_out = nullptr;
  const bool dev_out = is_device_ptr(grad_len);
  auto cleanup = [&]() {
    dev_free(d_tik);
    dev_free(d_G);
    dev_free(d_acc);
    dev_free(d_out);
  };
  if ((s = dev_alloc(&d_tik, (size_t)h->ntiles)) != FD_OK || (s = dev_alloc(&d_G, (size_t)h->ntiles * TILE * TILE)) != FD_OK ||
      (s = dev_alloc(&d_acc, (size_t)h->wnnz)) != FD_OK || (!dev_out && (s = dev_alloc(&d_out, (size_t)h->wnnz)) != FD_OK)) {
    cleanup();
    return fail(h, s);
  }
  cudaStream_t st = h->stream;
  SpScratch sp;
  if ((s = sp.init(h, st)) != FD_OK) {
    cleanup();
    return fail(h, s);
  }
  cudaError_t e = cudaMemcpyAsync(d_tik, tile_ik.data(), h->ntiles * sizeof(int2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_length_grad(h->n, h->nb, h->dim, d_tik, h->ntiles, (const float*)h->D, dx, d_G, h->d_wrp, h->d_wci,
                           h->d_wlen, h->d_wrev, h->wnnz, d_acc, dev_out ? grad_len : d_out, h->sm_count,
                           sp.global_path, sp.ints, sp.err, st);
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(grad_len, d_out, (size_t)h->wnnz * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, cuda_status(e));
  }
  if ((s = sp.check()) != FD_OK) return fail(h, s);
  if (f_out) *f_out = c.f_final;
  return FD_OK;
}

// Tile coordinates (block row, strip offset) of every stored tile, on the device.
// The H-step solver of a launch: CG, or refinement with the factored inverse.
static fd_status set_solver(fd_layout* h, int32_t solver, KParams* p) {
  if (solver == FD_SOLVER_CG) {
    p->solver = SOLVER_CG;
    return FD_OK;
  }
  if (solver != FD_SOLVER_DIRECT || !h->d_ainv) return FD_ERR_ARG;
  p->solver = SOLVER_DIRECT;
  p->ainv = h->d_ainv;
  return FD_OK;
}

static fd_status upload_tile_ik(fd_layout* h, int2** out) {
  std::vector<int2> tile_ik(h->ntiles);
  for (int I = 0; I < h->nb; ++I)
    for (int k = 0; k < h->strip_len[I]; ++k) tile_ik[h->tile_base[I] + k] = make_int2(I, k);
  fd_status s = dev_alloc(out, (size_t)h->ntiles);
  if (s != FD_OK) return s;
  FD_CK(cudaMemcpyAsync(*out, tile_ik.data(), h->ntiles * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
  return FD_OK;
}

fd_status fd_adjoint_reset(fd_layout* h) {
  if (!h) return FD_ERR_ARG;
  if (h->code != CODE_F32 || !h->d_wrp || h->wnnz == 0) return fail(h, FD_ERR_ARG);
  if (h->n > FD_GRAD_MAX_N || h->disconnected || !h->wsimple) return fail(h, FD_ERR_UNIMPLEMENTED);
  const size_t cnt = (size_t)h->ntiles * TILE * TILE;
  if (!h->d_dbar) {
    fd_status s = dev_alloc(&h->d_dbar, cnt);
    if (s != FD_OK) return fail(h, s);
  }
  if (cudaMemsetAsync(h->d_dbar, 0, cnt * sizeof(float), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  return FD_OK;
}

fd_status fd_sor_step_adjoint(fd_layout* h, const float* X_k, const float* X_k1, int32_t accepted, double omega,
                              const float* Xbar_k1, float* Xbar_k, const fd_options* opt, int32_t* cg_steps) {
  if (!h) return FD_ERR_ARG;
  if (!X_k || !X_k1 || !Xbar_k1 || !Xbar_k || !(omega >= 0.0) || !std::isfinite(omega)) return fail(h, FD_ERR_ARG);
  fd_options o;
  fd_options_default(&o);
  if (opt) o = *opt;
  if (o.cg_max < 0 || !(o.cg_tol >= 0.0)) return fail(h, FD_ERR_ARG);
  const size_t nd = (size_t)h->n * h->dim;
  fd_status s = FD_OK;
  if (!h->d_adj && (s = dev_alloc(&h->d_adj, 7 * nd)) != FD_OK) return fail(h, s);
  float* Y = h->d_adj;
  float* Yb = Y + nd;
  float* lam = Y + 2 * nd;
  float* Xb = Y + 3 * nd;
  float* in0 = Y + 4 * nd;  // staging of host inputs
  float* in1 = Y + 5 * nd;
  float* in2 = Y + 6 * nd;
  cudaStream_t st = h->stream;
  auto stage = [&](const float* src, float* dst) -> const float* {
    if (is_device_ptr(src)) return src;
    if (cudaMemcpyAsync(dst, src, nd * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    return dst;
  };
  const float* xk = stage(X_k, in0);
  const float* xk1 = stage(X_k1, in1);
  const float* xb1 = stage(Xbar_k1, in2);
  if (!xk || !xk1 || !xb1) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  const bool dev_out = is_device_ptr(Xbar_k);
  float* xb = dev_out ? Xbar_k : Xb;
  if (launch_adjoint_prep(h->n, h->dim, xk, xk1, xb1, accepted ? 1 : 0, (float)omega, h->d_om_scale, Y, Yb, xb, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  // lam: L^W lam = Yb (one H-step solve of the layout kernel)
  KParams p = base_params(h, KM_SOLVE);
  p.x_in = Yb;
  p.x_out = lam;
  p.max_iter = 1;
  p.cg_max = o.cg_max;
  p.cg_tol = o.cg_tol;
  p.tol = 0.0;
  if ((s = set_solver(h, o.solver, &p)) != FD_OK) return fail(h, s);
  Ctrl c;
  double kms = 0.0;
  std::memset(&c, 0, sizeof(c));
  s = run_kernel(h, p, &c, &kms);
  fill_stats(h, c, kms);
  if (s != FD_OK) return fail(h, s);
  int2* d_tik = nullptr;
  if ((s = upload_tile_ik(h, &d_tik)) != FD_OK) return fail(h, s);
  cudaError_t e = launch_pair_adjoint(h->code, h->n, h->nb, h->dim, d_tik, h->ntiles, h->D, xk, lam, Y, xb, h->d_dbar,
                                      h->sm_count, st);
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(Xbar_k, xb, nd * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(d_tik);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, cuda_status(e));
  }
  if (cg_steps) *cg_steps = c.cg_steps;
  return FD_OK;
}

fd_status fd_adjoint_length_grad(fd_layout* h, float* grad_len) {
  if (!h || !grad_len) return FD_ERR_ARG;
  if (!h->d_dbar) return fail(h, FD_ERR_ARG);  // fd_adjoint_reset first
  float *d_acc = nullptr, *d_out = nullptr;
  const bool dev_out = is_device_ptr(grad_len);
  fd_status s = dev_alloc(&d_acc, (size_t)h->wnnz);
  if (s == FD_OK && !dev_out) s = dev_alloc(&d_out, (size_t)h->wnnz);
  if (s != FD_OK) {
    dev_free(d_acc);
    return fail(h, s);
  }
  cudaStream_t st = h->stream;
  SpScratch sp;
  if ((s = sp.init(h, st)) != FD_OK) {
    dev_free(d_acc);
    dev_free(d_out);
    return fail(h, s);
  }
  cudaError_t e = launch_sp_backprop(h->n, h->nb, h->d_dbar, h->d_wrp, h->d_wci, h->d_wlen, h->d_wrev, h->wnnz, d_acc,
                                     dev_out ? grad_len : d_out, h->sm_count, sp.global_path, sp.ints, sp.err, st);
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(grad_len, d_out, (size_t)h->wnnz * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(d_acc);
  dev_free(d_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, cuda_status(e));
  }
  if ((s = sp.check()) != FD_OK) return fail(h, s);
  return FD_OK;
}

fd_status fd_fp32_peak(int32_t packed, double* tflops, double* ms) {
  if (!tflops || !ms) return FD_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FD_ERR_CUDA;
  }
  cudaError_t e = measure_fp32_peak(packed ? 1 : 0, sms, 5, tflops, ms);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return FD_OK;
}

fd_status fd_factor(fd_layout* h) {
  if (!h) return FD_ERR_ARG;
  if (h->n > FD_DIRECT_MAX_N) return fail(h, FD_ERR_ARG);
  cudaStream_t st = h->stream;
  const size_t np = (size_t)h->n_pad;
  fd_status s = FD_OK;
  if (!h->d_ainv && (s = dev_alloc(&h->d_ainv, np * np)) != FD_OK) return fail(h, s);
  float *P = nullptr, *QT = nullptr, *AT = nullptr;
  int* err = nullptr;
  int2* tik = nullptr;
  auto cleanup = [&] {
    dev_free(P);
    dev_free(QT);
    dev_free(AT);
    dev_free(err);
    dev_free(tik);
  };
  const size_t panel = (size_t)h->nb * TILE * TILE;
  if ((s = dev_alloc(&P, (size_t)TILE * TILE)) != FD_OK || (s = dev_alloc(&QT, panel)) != FD_OK ||
      (s = dev_alloc(&AT, panel)) != FD_OK || (s = dev_alloc(&err, 1)) != FD_OK ||
      (s = upload_tile_ik(h, &tik)) != FD_OK) {
    cleanup();
    dev_free(h->d_ainv);
    return fail(h, s);
  }
  // shift sigma / n with sigma = mean_i s_i (the eigenvalue the null vector 1 of L^W gets)
  std::vector<float> hs((size_t)h->n);
  cudaError_t e = cudaMemcpy(hs.data(), h->d_s, (size_t)h->n * sizeof(float), cudaMemcpyDeviceToHost);
  double sigma = 0.0;
  for (float v : hs) sigma += v;
  sigma /= h->n;
  if (!(sigma > 0.0)) sigma = 1.0;  // n = 1: L^W = 0
  int herr = 0;
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev0, st);
  if (e == cudaSuccess)
    e = launch_direct_factor(h->n, h->n_pad, h->nb, h->code, h->D, tik, h->ntiles, h->d_s, (float)(sigma / h->n),
                             h->d_ainv, P, QT, AT, err, h->sm_count, st);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  cleanup();
  if (e != cudaSuccess) {
    cudaGetLastError();
    dev_free(h->d_ainv);
    return fail(h, cuda_status(e));
  }
  if (herr) {
    dev_free(h->d_ainv);
    return fail(h, FD_ERR_CG_BREAKDOWN);
  }
  h->factor_ms = ms;
  return FD_OK;
}

fd_status fd_factor_rows(fd_layout* h, int32_t row0, int32_t nrows, double* out) {
  if (!h) return FD_ERR_ARG;
  if (!h->d_ainv || !out || row0 < 0 || nrows < 0 || row0 + nrows > h->n) return fail(h, FD_ERR_ARG);
  if (nrows == 0) return FD_OK;
  std::vector<float> buf((size_t)nrows * h->n);
  if (cudaMemcpy2D(buf.data(), (size_t)h->n * sizeof(float), h->d_ainv + (size_t)row0 * h->n_pad,
                   (size_t)h->n_pad * sizeof(float), (size_t)h->n * sizeof(float), (size_t)nrows,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  for (size_t k = 0; k < buf.size(); ++k) out[k] = buf[k];
  return FD_OK;
}

fd_status fd_factor_release(fd_layout* h) {
  if (!h) return FD_ERR_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  dev_free(h->d_ainv);
  h->factor_ms = 0.0;
  return FD_OK;
}

static fd_status run_impl(fd_layout* h, float* X, const fd_options* opt, int k0, int max_iter, Ctrl* c_out) {
  if (!X || !opt) return FD_ERR_ARG;
  if (!(opt->omega >= 0.0) || !std::isfinite(opt->omega) || max_iter < 1 || opt->cg_max < 0 ||
      !(opt->tol >= 0.0) || !(opt->cg_tol >= 0.0) || (opt->stop != FD_STOP_REL_DISP && opt->stop != FD_STOP_REL_STRESS))
    return FD_ERR_ARG;
  if (opt->strategy != FD_OMEGA_FIXED && opt->strategy != FD_OMEGA_PROB && opt->strategy != FD_OMEGA_ENUM)
    return FD_ERR_ARG;
  fd_status s = ensure_traces(h, max_iter);
  if (s != FD_OK) return s;
  std::vector<double> om(max_iter);
  for (int k = 0; k < max_iter; ++k)
    om[k] = (opt->strategy == FD_OMEGA_PROB)   ? omega_prob(opt->seed, (uint64_t)(k0 + k))
            : (opt->strategy == FD_OMEGA_ENUM) ? 0.0
                                               : opt->omega;
  FD_CK(cudaMemcpyAsync(h->d_omega, om.data(), max_iter * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  const float* dx = nullptr;
  if ((s = stage_input(h, X, &dx)) != FD_OK) return s;
  KParams p = base_params(h, KM_RUN);
  p.x_in = dx;
  const bool dev_out = is_device_ptr(X);
  p.x_out = dev_out ? X : h->d_stage_out;
  p.omega_seq = h->d_omega;
  p.trace_f = h->d_trace_f;
  p.trace_acc = h->d_trace_acc;
  p.trace_om = h->d_trace_om;
  p.trace_cg = h->d_trace_cg;
  p.trace_crit = h->d_trace_crit;
  p.trace_fh = h->d_trace_fh;
  p.trace_ft = h->d_trace_ft;
  p.trace_t = h->d_trace_t;
  p.max_iter = max_iter;
  p.enum_omega = (opt->strategy == FD_OMEGA_ENUM) ? 1 : 0;
  p.om_scale = h->d_om_scale;
  if ((s = set_solver(h, opt->solver, &p)) != FD_OK) return s;
  p.stop = opt->stop;
  p.cg_max = opt->cg_max;
  p.tol = opt->tol;
  p.cg_tol = opt->cg_tol;
  double kms = 0.0;
  std::memset(c_out, 0, sizeof(*c_out));
  s = run_kernel(h, p, c_out, &kms);
  fill_stats(h, *c_out, kms);
  h->last_iters = c_out->iters;
  if (s != FD_OK) return s;
  if (!dev_out) {
    FD_CK(cudaMemcpyAsync(X, h->d_stage_out, (size_t)h->n * h->dim * sizeof(float), cudaMemcpyDeviceToHost,
                          h->stream));
    FD_CK(cudaStreamSynchronize(h->stream));
  }
  return FD_OK;
}

fd_status fd_set_vertex_omega(fd_layout* h, const float* m) {
  if (!h) return FD_ERR_ARG;
  if (!m) {
    dev_free(h->d_om_scale);
    return FD_OK;
  }
  std::vector<float> hm((size_t)h->n_pad, 0.f);
  if (is_device_ptr(m)) {
    if (cudaMemcpy(hm.data(), m, (size_t)h->n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, FD_ERR_CUDA);
    }
  } else {
    std::memcpy(hm.data(), m, (size_t)h->n * sizeof(float));
  }
  for (int i = 0; i < h->n; ++i)
    if (!std::isfinite(hm[i]) || hm[i] < 0.f) return fail(h, FD_ERR_ARG);
  if (!h->d_om_scale) {
    fd_status s = dev_alloc(&h->d_om_scale, (size_t)h->n_pad);
    if (s != FD_OK) return fail(h, s);
  }
  if (cudaMemcpy(h->d_om_scale, hm.data(), (size_t)h->n_pad * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  return FD_OK;
}

fd_status fd_sor_step(fd_layout* h, float* X, const fd_options* opt, int32_t k, double* f_out, int32_t* accepted,
                      double* crit_out) {
  if (!h) return FD_ERR_ARG;
  if (k < 0) return fail(h, FD_ERR_ARG);
  Ctrl c;
  fd_status s = run_impl(h, X, opt, k, 1, &c);
  if (s != FD_OK) return fail(h, s);
  int acc = 0;
  if (cudaMemcpy(&acc, h->d_trace_acc, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  if (f_out) *f_out = c.f_final;
  if (accepted) *accepted = acc;
  if (crit_out) *crit_out = c.crit_final;
  return FD_OK;
}

fd_status fd_run(fd_layout* h, float* X, const fd_options* opt, int32_t* iters_out, double* f_out, double* trace_f) {
  if (!h) return FD_ERR_ARG;
  if (!opt) return fail(h, FD_ERR_ARG);
  if (opt->first_iter < 0) return fail(h, FD_ERR_ARG);
  Ctrl c;
  fd_status s = run_impl(h, X, opt, opt->first_iter, opt->max_iter, &c);
  if (s != FD_OK) return fail(h, s);
  if (iters_out) *iters_out = c.iters;
  if (f_out) *f_out = c.f_final;
  if (trace_f) {
    if (cudaMemcpy(trace_f, h->d_trace_f, (size_t)(c.iters + 1) * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      cudaGetLastError();
      return fail(h, FD_ERR_CUDA);
    }
  }
  return FD_OK;
}

fd_status fd_run_trace(fd_layout* h, int32_t* accepted, double* omega, int32_t* cg_steps, double* crit) {
  if (!h) return FD_ERR_ARG;
  const int k = h->last_iters;
  if (k <= 0) return FD_OK;
  struct {
    void* dst;
    const void* src;
    size_t bytes;
  } cp[] = {{accepted, h->d_trace_acc, k * sizeof(int)},
            {omega, h->d_trace_om, k * sizeof(double)},
            {cg_steps, h->d_trace_cg, k * sizeof(int)},
            {crit, h->d_trace_crit, k * sizeof(double)}};
  for (auto& c : cp) {
    if (!c.dst) continue;
    if (cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, FD_ERR_CUDA);
    }
  }
  return FD_OK;
}

fd_status fd_run_trace_ext(fd_layout* h, double* f_h, double* f_extrapolated, double* t_ms) {
  if (!h) return FD_ERR_ARG;
  const int k = h->last_iters;
  if (k <= 0) return FD_OK;
  struct {
    void* dst;
    const void* src;
  } cp[] = {{f_h, h->d_trace_fh}, {f_extrapolated, h->d_trace_ft}, {t_ms, h->d_trace_t}};
  for (auto& c : cp) {
    if (!c.dst) continue;
    if (cudaMemcpy(c.dst, c.src, k * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, FD_ERR_CUDA);
    }
  }
  return FD_OK;
}

fd_status fd_distance_rows(fd_layout* h, int32_t row0, int32_t nrows, double* out) {
  if (!h) return FD_ERR_ARG;
  if (!out || row0 < 0 || nrows < 0 || row0 + nrows > h->n) return fail(h, FD_ERR_ARG);
  if (nrows == 0) return FD_OK;
  double* d = nullptr;
  fd_status s = dev_alloc(&d, (size_t)nrows * h->n);
  if (s != FD_OK) return fail(h, s);
  cudaError_t e = launch_distance_rows(h->code, h->n, h->nb, h->d_tile_base, h->d_strip_len, h->D, row0, nrows,
                                       h->weighted ? 0 : 1, d, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d, (size_t)nrows * h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, cuda_status(e));
  }
  return FD_OK;
}

fd_status fd_layout_info(const fd_layout* h, fd_info* info) {
  if (!h || !info) return FD_ERR_ARG;
  info->n = h->n;
  info->dim = h->dim;
  info->diameter = h->diameter;
  info->code_bytes = (h->code == CODE_U8) ? 1 : 4;
  info->tile = TILE;
  info->num_tiles = h->ntiles;
  info->distance_bytes = (int64_t)h->D_bytes;
  info->disconnected = h->disconnected;
  info->sm_count = h->sm_count;
  info->grid = h->grid;
  info->tasks = h->ntasks;
  info->apsp_ms = h->apsp_ms;
  info->stages = h->nbuf;
  info->tiles_per_stage = h->tps;
  info->bfs_sweeps = h->bfs_sweeps;
  info->bfs_sources = h->bfs_sources;
  info->factored = h->d_ainv ? 1 : 0;
  info->factor_ms = h->factor_ms;
  return FD_OK;
}

fd_status fd_last_stats(const fd_layout* h, fd_stats* stats) {
  if (!h || !stats) return FD_ERR_ARG;
  *stats = h->stats;
  return FD_OK;
}

fd_status fd_last_error(const fd_layout* h) { return h ? h->last_error : FD_ERR_ARG; }

fd_status fd_timeline_enable(fd_layout* h, int32_t cap) {
  if (!h || cap < 0) return FD_ERR_ARG;
  dev_free(h->d_timeline);
  h->timeline_cap = 0;
  h->timeline_n = 0;
  if (cap == 0) return FD_OK;
  fd_status s = dev_alloc(&h->d_timeline, (size_t)2 * cap);
  if (s != FD_OK) return fail(h, s);
  h->timeline_cap = cap;
  return FD_OK;
}

fd_status fd_timeline_read(fd_layout* h, double* out, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return FD_ERR_ARG;
  const int k = std::min(cap, h->timeline_n);
  *count = h->timeline_n;
  if (k > 0 && cudaMemcpy(out, h->d_timeline, (size_t)2 * k * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, FD_ERR_CUDA);
  }
  return FD_OK;
}

}  // extern "C"

// ==========================================================================
// Batched form
// ==========================================================================

struct fd_batch {
  int G = 0, dim = 0, dimp = 0, N = 0, P = 0, max_n = 0, n_pad_max = 0;
  long long ntiles = 0;
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  std::vector<BGraph> graphs;
  std::vector<int> order;    // by size, largest first
  std::vector<int> run_order;  // the graphs of tile class 0, 1, 2, each largest first
  int cls_off[4] = {0, 0, 0, 0};
  int tiles[FD_BATCH_BUCKETS];  // tile edge per size bucket
  BGraph* d_graphs = nullptr;
  int* d_order = nullptr;
  int* d_order_sub = nullptr;  // [G] order of a run over a subset (the tuner's probes)
  unsigned char* D = nullptr;
  size_t D_bytes = 0;
  unsigned char* DT = nullptr;  // T x T tiles of the graphs with T < TILE
  size_t DT_bytes = 0, DT_cap = 0;
  unsigned char* d_lut = nullptr;
  int lut_rows = 0, max_diam = 0, disconnected = 0;
  float* d_s = nullptr;
  float* d_inv_s = nullptr;
  float* d_pool = nullptr;   // X, Z, R, P, B, R0: [6][P][dimp]
  float* d_xin = nullptr;    // [N][dim] staging of host layouts
  double* d_omega = nullptr; // [G]
  double* d_omega_seq = nullptr;
  int omega_seq_cap = 0;
  int* d_queue = nullptr;    // [0..2] queue position per tile class, [3] launch error
  int* d_iout = nullptr;     // [4][G] iterations, CG steps, accepted, status
  double* d_dout = nullptr;  // [5][G] final stress, criterion, L^W passes, stress passes, device ms
  BParams* d_params = nullptr;
  int W = 2, nbuf = 2, grid = 0;
  size_t smem = 0;
  cudaGraphExec_t gexec = nullptr;
  int g_W = 0, g_nbuf = 0, g_grid = 0;
  size_t g_smem = 0;
  int captured = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // the three tile classes run concurrently (fork / join on events), so that
  // the SMs a class leaves at its end take up the next class's graphs
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  double apsp_ms = 0.0;
  long long timeout_ns = 30000000000LL;
  std::vector<int> h_iout;
  std::vector<double> h_dout;
  fd_stats stats;
};

namespace {

void batch_release(fd_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  dev_free(b->d_graphs);
  dev_free(b->d_order);
  dev_free(b->d_order_sub);
  dev_free(b->D);
  dev_free(b->DT);
  dev_free(b->d_lut);
  dev_free(b->d_s);
  dev_free(b->d_inv_s);
  dev_free(b->d_pool);
  dev_free(b->d_xin);
  dev_free(b->d_omega);
  dev_free(b->d_omega_seq);
  dev_free(b->d_queue);
  dev_free(b->d_iout);
  dev_free(b->d_dout);
  dev_free(b->d_params);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  b->ev0 = b->ev1 = nullptr;
  for (int c = 0; c < 3; ++c) {
    if (b->aux[c]) cudaStreamDestroy(b->aux[c]);
    if (b->ev_join[c]) cudaEventDestroy(b->ev_join[c]);
    b->aux[c] = nullptr;
    b->ev_join[c] = nullptr;
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  b->ev_fork = nullptr;
}

cudaError_t batch_config(int dim, int W, int lut_bytes, int n_pad_max, int nbuf, int* bps, size_t* smem) {
  if (dim == 1) return batch_config_d1(W, lut_bytes, n_pad_max, nbuf, bps, smem);
  if (dim == 2) return batch_config_d2(W, lut_bytes, n_pad_max, nbuf, bps, smem);
  return batch_config_d3(W, lut_bytes, n_pad_max, nbuf, bps, smem);
}

cudaError_t launch_batch(int dim, int W, int cls, const BParams* p, int grid, size_t smem, cudaStream_t st) {
  if (dim == 1) return launch_batch_d1(W, cls, p, grid, smem, st);
  if (dim == 2) return launch_batch_d2(W, cls, p, grid, smem, st);
  return launch_batch_d3(W, cls, p, grid, smem, st);
}

// The three persistent launches of a run (tile classes T = 128, 64, 32; a
// class without graphs ends at its first queue read), after the queues and
// the error flag are cleared.  They run concurrently on the batch's own
// streams (class 0, the largest graphs, first and at the highest priority),
// forked from and joined back into st: a CTA of the next class starts on an
// SM as soon as a CTA of an earlier class has run out of graphs.
cudaError_t launch_batch_all(fd_batch* b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, st);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    e = cudaStreamWaitEvent(b->aux[c], b->ev_fork, 0);
    if (e == cudaSuccess) e = launch_batch(b->dim, b->W, c, b->d_params, b->grid, b->smem, b->aux[c]);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[c], b->aux[c]);
  }
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(st, b->ev_join[c], 0);
  return e;
}

// Size bucket of an n-vertex graph: n <= 32, 64, 128, 256, 512, 1024, 2048.
int batch_bucket(int n) {
  int k = 0;
  while (k < FD_BATCH_BUCKETS - 1 && n > (32 << k)) ++k;
  return k;
}

int tile_class(int T) { return (T == TILE) ? 0 : (T == 64) ? 1 : 2; }

// Tile edges chosen by fd_batch_tune, per (size bucket, dimension), for this
// process: a later batch of the same dimension starts from them.
std::mutex g_tile_mu;
int g_tile_cache[4][FD_BATCH_BUCKETS] = {};  // 0 = not tuned

// The order of a run over the graphs `ids` (ascending positions in the
// size order): grouped by tile class, largest first inside each class.
void class_order(const std::vector<BGraph>& gs, const std::vector<int>& ids, std::vector<int>& out, int* off) {
  out.clear();
  for (int c = 0; c < 3; ++c) {
    off[c] = (int)out.size();
    for (int g : ids)
      if (tile_class(gs[g].T) == c) out.push_back(g);
  }
  off[3] = (int)out.size();
}

// Gives every graph the tile edge of its size bucket and builds the small-
// tile pool (the graphs with T < TILE, re-tiled from the TILE x TILE pool).
fd_status batch_set_tiles(fd_batch* b, const int* tiles) {
  for (int k = 0; k < FD_BATCH_BUCKETS; ++k)
    if (tiles[k] != 32 && tiles[k] != 64 && tiles[k] != TILE) return FD_ERR_ARG;
  std::vector<BGraph> gs = b->graphs;
  std::vector<int> small;
  long long dt = 0;
  for (int g = 0; g < b->G; ++g) {
    BGraph& gr = gs[g];
    gr.T = tiles[batch_bucket(gr.n)];
    gr.nbt = (gr.n + gr.T - 1) / gr.T;
    gr.dt = 0;
    if (gr.T < TILE) {
      gr.dt = dt;
      dt += (long long)hr_tiles(gr.nbt) * gr.T * gr.T;
      small.push_back(g);
    }
  }
  cudaStream_t st = b->stream;
  if ((size_t)dt > b->DT_cap) {
    dev_free(b->DT);
    b->DT_cap = 0;
    fd_status s = dev_alloc(&b->DT, (size_t)dt);
    if (s != FD_OK) return s;
    b->DT_cap = (size_t)dt;
  }
  std::vector<int> ord;
  int off[4];
  class_order(gs, b->order, ord, off);
  int* d_list = nullptr;
  fd_status s = FD_OK;
  if (!small.empty() && (s = dev_alloc(&d_list, small.size())) != FD_OK) return s;
  cudaError_t e = cudaMemcpyAsync(b->d_graphs, gs.data(), gs.size() * sizeof(BGraph), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !small.empty()) {
    e = cudaMemcpyAsync(d_list, small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_retile_multi(b->d_graphs, d_list, (int)small.size(), b->D, b->DT,
                              std::max(1, std::min((int)small.size(), 8 * b->sm_count)), st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(d_list);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  b->graphs = gs;
  b->run_order = ord;
  std::memcpy(b->cls_off, off, sizeof(off));
  std::memcpy(b->tiles, tiles, sizeof(b->tiles));
  b->DT_bytes = (size_t)dt;
  return FD_OK;
}

// Sets the launch shape if it is feasible (at least one resident CTA per SM).
fd_status batch_shape(fd_batch* b, int W, int nbuf) {
  if ((W != 1 && W != 2) || nbuf < 2 || nbuf > 3) return FD_ERR_ARG;
  int bps = 0;
  size_t smem = 0;
  if (batch_config(b->dim, W, b->lut_rows * LUT_ROW, b->n_pad_max, nbuf, &bps, &smem) != cudaSuccess) {
    cudaGetLastError();
    return FD_ERR_ARG;
  }
  if (bps < 1) return FD_ERR_ARG;
  b->W = W;
  b->nbuf = nbuf;
  b->smem = smem;
  b->grid = bps * b->sm_count;
  return FD_OK;
}

// One launch of the persistent batched kernel (from a captured CUDA graph
// when the stream can be captured); returns the launch-level error flag.
fd_status batch_launch(fd_batch* b, double* kernel_ms) {
  cudaStream_t st = b->stream;
  const bool same = b->gexec && b->g_W == b->W && b->g_nbuf == b->nbuf && b->g_grid == b->grid && b->g_smem == b->smem;
  if (!same && b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (!b->gexec && st != nullptr) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e2 = launch_batch_all(b, st);
      cudaError_t e3 = cudaStreamEndCapture(st, &graph);
      if (e2 == cudaSuccess && e3 == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&b->gexec, graph, 0) != cudaSuccess) b->gexec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    if (b->gexec) {
      b->g_W = b->W;
      b->g_nbuf = b->nbuf;
      b->g_grid = b->grid;
      b->g_smem = b->smem;
    }
  }
  FD_CK(cudaEventRecord(b->ev0, st));
  if (b->gexec) {
    FD_CK(cudaGraphLaunch(b->gexec, st));
    b->captured = 1;
  } else {
    FD_CK(launch_batch_all(b, st));
    b->captured = 0;
  }
  FD_CK(cudaEventRecord(b->ev1, st));
  int q[4] = {0, 0, 0, 0};
  b->h_iout.resize((size_t)4 * b->G);
  b->h_dout.resize((size_t)5 * b->G);
  FD_CK(cudaMemcpyAsync(q, b->d_queue, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  FD_CK(cudaMemcpyAsync(b->h_iout.data(), b->d_iout, (size_t)4 * b->G * sizeof(int), cudaMemcpyDeviceToHost, st));
  FD_CK(cudaMemcpyAsync(b->h_dout.data(), b->d_dout, (size_t)5 * b->G * sizeof(double), cudaMemcpyDeviceToHost, st));
  FD_CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  FD_CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  *kernel_ms = ms;
  if (q[3] != 0) return (fd_status)q[3];
  return FD_OK;
}

// Runs Algorithm 2 on every graph (or on the graphs `subset`, positions in
// the size order) from the layouts at x_in, writing x_out.
fd_status batch_run_dev(fd_batch* b, const float* x_in, float* x_out, const fd_options* opt, const double* omega,
                        int max_iter, double* kernel_ms, const std::vector<int>* subset = nullptr) {
  if (!opt || !(opt->omega >= 0.0) || !std::isfinite(opt->omega) || max_iter < 1 || opt->cg_max < 0 ||
      !(opt->tol >= 0.0) || !(opt->cg_tol >= 0.0) || (opt->stop != FD_STOP_REL_DISP && opt->stop != FD_STOP_REL_STRESS))
    return FD_ERR_ARG;
  if (opt->strategy == FD_OMEGA_ENUM || opt->solver == FD_SOLVER_DIRECT) return FD_ERR_UNIMPLEMENTED;
  if (opt->first_iter < 0) return FD_ERR_ARG;
  if (opt->strategy != FD_OMEGA_FIXED && opt->strategy != FD_OMEGA_PROB) return FD_ERR_ARG;
  if (opt->solver != FD_SOLVER_CG) return FD_ERR_ARG;
  cudaStream_t st = b->stream;
  std::vector<double> om((size_t)b->G, opt->omega);
  if (omega && opt->strategy == FD_OMEGA_FIXED) {
    fd_status s = fetch_host(om, omega, (size_t)b->G);
    if (s != FD_OK) return s;
    for (double v : om)
      if (!(v >= 0.0) || !std::isfinite(v)) return FD_ERR_ARG;
  }
  FD_CK(cudaMemcpyAsync(b->d_omega, om.data(), (size_t)b->G * sizeof(double), cudaMemcpyHostToDevice, st));
  const double* seq = nullptr;
  std::vector<double> omk;
  if (opt->strategy == FD_OMEGA_PROB) {
    if (b->omega_seq_cap < max_iter) {
      dev_free(b->d_omega_seq);
      b->omega_seq_cap = 0;
      fd_status s = dev_alloc(&b->d_omega_seq, (size_t)max_iter);
      if (s != FD_OK) return s;
      b->omega_seq_cap = max_iter;
    }
    omk.resize(max_iter);
    for (int k = 0; k < max_iter; ++k) omk[k] = omega_prob(opt->seed, (uint64_t)(opt->first_iter + k));
    FD_CK(cudaMemcpyAsync(b->d_omega_seq, omk.data(), max_iter * sizeof(double), cudaMemcpyHostToDevice, st));
    seq = b->d_omega_seq;
  }
  BParams p;
  std::memset(&p, 0, sizeof(p));
  p.graphs = b->d_graphs;
  p.order = b->d_order;
  std::memcpy(p.cls_off, b->cls_off, sizeof(p.cls_off));
  if (subset) {
    std::vector<int> ord;
    class_order(b->graphs, *subset, ord, p.cls_off);
    if (!ord.empty())
      FD_CK(cudaMemcpyAsync(b->d_order_sub, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    p.order = b->d_order_sub;
  }
  p.G = b->G;
  p.dim = b->dim;
  p.D = b->D;
  p.DT = b->DT;
  p.lut = b->d_lut;
  p.lut_rows = b->lut_rows;
  p.s = b->d_s;
  p.inv_s = b->d_inv_s;
  p.x_in = x_in;
  p.x_out = x_out;
  const size_t ps = (size_t)b->P * b->dimp;
  p.X = b->d_pool;
  p.Z = b->d_pool + ps;
  p.R = b->d_pool + 2 * ps;
  p.Pd = b->d_pool + 3 * ps;
  p.B = b->d_pool + 4 * ps;
  p.R0 = b->d_pool + 5 * ps;
  p.omega = b->d_omega;
  p.omega_seq = seq;
  p.max_iter = max_iter;
  p.cg_max = opt->cg_max;
  p.stop = opt->stop;
  p.tol = opt->tol;
  p.cg_tol = opt->cg_tol;
  p.queue = b->d_queue;
  p.err = b->d_queue + 3;
  const size_t G = (size_t)b->G;
  p.iters = b->d_iout;
  p.cg_steps = b->d_iout + G;
  p.accepted = b->d_iout + 2 * G;
  p.status = b->d_iout + 3 * G;
  p.f_final = b->d_dout;
  p.crit_final = b->d_dout + G;
  p.passes_mv = b->d_dout + 2 * G;
  p.passes_st = b->d_dout + 3 * G;
  p.graph_ms = b->d_dout + 4 * G;
  p.nbuf = b->nbuf;
  p.n_pad_max = b->n_pad_max;
  p.timeout_ns = b->timeout_ns;
  FD_CK(cudaMemcpyAsync(b->d_params, &p, sizeof(p), cudaMemcpyHostToDevice, st));
  FD_CK(cudaMemsetAsync(b->d_iout, 0, 4 * G * sizeof(int), st));
  fd_status s = batch_launch(b, kernel_ms);
  // statistics (sums over graphs)
  fd_stats& S = b->stats;
  std::memset(&S, 0, sizeof(S));
  double pairs_w = 0.0, mv = 0.0, sp = 0.0, f = 0.0;
  for (int g = 0; g < b->G; ++g) {
    const double pg = 0.5 * (double)b->graphs[g].n * (double)(b->graphs[g].n - 1);
    S.iterations += b->h_iout[g];
    S.cg_steps += b->h_iout[G + g];
    S.accepted += b->h_iout[2 * G + g];
    const double m = b->h_dout[2 * G + g], t = b->h_dout[3 * G + g];
    mv += m;
    sp += t;
    pairs_w += (m + t) * pg;
    f += b->h_dout[g];
  }
  S.pair_passes = mv + sp;
  S.pairs = pairs_w;
  S.matvec_passes = mv;
  S.stress_passes = sp;
  S.final_stress = f;
  S.kernel_ms = *kernel_ms;
  if (s != FD_OK) return s;
  for (int g = 0; g < b->G; ++g)
    if (b->h_iout[3 * G + g] != 0) return (fd_status)b->h_iout[3 * G + g];
  return FD_OK;
}

}  // namespace

extern "C" {

fd_status fd_batch_create(fd_batch** out, int32_t num_graphs, int32_t dim, const int32_t* graph_ptr,
                          const int32_t* row_ptr, const int32_t* col_idx, int32_t disconnected_policy,
                          void* cuda_stream) {
  if (!out) return FD_ERR_ARG;
  *out = nullptr;
  if (num_graphs < 1 || dim < 1 || dim > 3 || !graph_ptr || !row_ptr ||
      (disconnected_policy != 0 && disconnected_policy != 1))
    return FD_ERR_ARG;
  const int G = num_graphs;
  std::vector<int> gp, rp, ci;
  fd_status s = fetch_host(gp, graph_ptr, (size_t)G + 1);
  if (s != FD_OK) return s;
  if (gp[0] != 0) return FD_ERR_ARG;
  for (int g = 0; g < G; ++g)
    if (gp[g + 1] - gp[g] < 1 || gp[g + 1] - gp[g] > BMAX_N) return FD_ERR_ARG;
  const int N = gp[G];
  if ((s = fetch_host(rp, row_ptr, (size_t)N + 1)) != FD_OK) return s;
  if (rp[0] != 0 || rp[N] < 0) return FD_ERR_CSR;
  if (rp[N] > 0 && !col_idx) return FD_ERR_ARG;
  if ((s = fetch_host(ci, col_idx, (size_t)rp[N])) != FD_OK) return s;
  if ((s = validate_csr(N, rp, ci, nullptr)) != FD_OK) return s;
  for (int g = 0; g < G; ++g)
    for (int e = rp[gp[g]]; e < rp[gp[g + 1]]; ++e)
      if (ci[e] < gp[g] || ci[e] >= gp[g + 1]) return FD_ERR_CSR;  // an edge between two graphs

  fd_batch* b = new (std::nothrow) fd_batch();
  if (!b) return FD_ERR_OOM;
  std::memset(&b->stats, 0, sizeof(b->stats));
  auto bail = [&](fd_status e) {
    batch_release(b);
    delete b;
    return e;
  };
  b->G = G;
  b->dim = dim;
  b->dimp = (dim == 3) ? 4 : dim;
  b->N = N;
  b->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      cudaGetLastError();
      return bail(FD_ERR_CUDA);
    }
    for (int c = 0; c < 3; ++c) {
      if (cudaStreamCreateWithPriority(&b->aux[c], cudaStreamNonBlocking, c == 0 ? greatest : least) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_join[c], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(FD_ERR_CUDA);
      }
    }
  }
  // geometry: padded vertex pools and tile pool, graph order (largest first)
  b->graphs.resize(G);
  long long p0 = 0, t0 = 0;
  for (int g = 0; g < G; ++g) {
    BGraph& gr = b->graphs[g];
    gr.n = gp[g + 1] - gp[g];
    gr.nb = (gr.n + TILE - 1) / TILE;
    gr.v0 = gp[g];
    gr.p0 = (int)p0;
    gr.t0 = t0;
    gr.T = TILE;
    gr.nbt = gr.nb;
    gr.dt = 0;
    p0 += (long long)gr.nb * TILE;
    t0 += hr_tiles(gr.nb);
    b->max_n = std::max(b->max_n, gr.n);
  }
  if (p0 > INT32_MAX) return bail(FD_ERR_ARG);
  b->P = (int)p0;
  b->ntiles = t0;
  b->n_pad_max = ((b->max_n + TILE - 1) / TILE) * TILE;
  b->order.resize(G);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return b->graphs[a].n > b->graphs[c].n; });
  cudaStream_t st = b->stream;
  b->D_bytes = (size_t)b->ntiles * TILE * TILE;
  if ((s = dev_alloc(&b->d_graphs, G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_order, G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_order_sub, G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->D, b->D_bytes)) != FD_OK) return bail(s);
  if (cudaMemcpyAsync(b->d_graphs, b->graphs.data(), G * sizeof(BGraph), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->d_order, b->order.data(), G * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(b->D, 0, b->D_bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  // distances: batched BFS, then the unreached pairs
  {
    std::vector<int2> items, rows;
    for (int g = 0; g < G; ++g) {
      for (int s0 = 0; s0 < b->graphs[g].n; s0 += 64) items.push_back(make_int2(g, s0));
      for (int R = 0; R < b->graphs[g].nb; ++R) rows.push_back(make_int2(g, R));
    }
    std::vector<int> tile_graph((size_t)b->ntiles);
    std::vector<int2> tile_ik((size_t)b->ntiles);
    for (int g = 0; g < G; ++g) {
      const BGraph& gr = b->graphs[g];
      for (int I = 0; I < gr.nb; ++I)
        for (int k = 0; k < hr_len(gr.nb, I); ++k) {
          const size_t t = (size_t)gr.t0 + hr_base(gr.nb, I) + k;
          tile_graph[t] = g;
          tile_ik[t] = make_int2(I, k);
        }
    }
    int *d_rp = nullptr, *d_ci = nullptr, *d_flags = nullptr, *d_tg = nullptr;
    int2 *d_items = nullptr, *d_rows = nullptr, *d_tik = nullptr;
    auto cleanup = [&]() {
      dev_free(d_rp);
      dev_free(d_ci);
      dev_free(d_flags);
      dev_free(d_tg);
      dev_free(d_items);
      dev_free(d_rows);
      dev_free(d_tik);
    };
    const size_t nnz = (size_t)rp[N];
    fd_status e = FD_OK;
    if ((e = dev_alloc(&d_rp, (size_t)N + 1)) != FD_OK || (e = dev_alloc(&d_ci, nnz)) != FD_OK ||
        (e = dev_alloc(&d_flags, (size_t)2 * G + 1)) != FD_OK || (e = dev_alloc(&d_tg, (size_t)b->ntiles)) != FD_OK ||
        (e = dev_alloc(&d_items, items.size())) != FD_OK || (e = dev_alloc(&d_rows, rows.size())) != FD_OK ||
        (e = dev_alloc(&d_tik, (size_t)b->ntiles)) != FD_OK) {
      cleanup();
      return bail(e);
    }
    int* d_maxlevel = d_flags;
    int* d_unreached = d_flags + G;
    int* d_overflow = d_flags + 2 * G;
    std::vector<int> flags((size_t)2 * G + 1, 0);
    float ms = 0.f;
    cudaError_t ce = cudaMemcpyAsync(d_rp, rp.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess && nnz) ce = cudaMemcpyAsync(d_ci, ci.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_flags, 0, (2 * G + 1) * sizeof(int), st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_rows, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_tg, tile_graph.data(), tile_graph.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(d_tik, tile_ik.data(), tile_ik.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(b->ev0, st);
    if (ce == cudaSuccess) {
      const int grid = std::max(1, std::min((int)items.size(), 4 * b->sm_count));
      ce = launch_bfs_multi(b->d_graphs, d_items, (int)items.size(), d_rp, d_ci, b->D, b->max_n, d_maxlevel,
                            d_overflow, grid, st);
    }
    if (ce == cudaSuccess) {
      const int grid = (int)std::max(1LL, std::min(b->ntiles, 8LL * b->sm_count));
      ce = launch_fill_multi(b->d_graphs, d_tg, d_tik, b->ntiles, b->D, d_maxlevel, disconnected_policy == 1 ? 1 : 0,
                             d_unreached, d_overflow, grid, st);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(b->ev1, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(flags.data(), d_flags, (2 * G + 1) * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return bail(cuda_status(ce));
    }
    b->apsp_ms = ms;
    bool any_unreached = false;
    for (int g = 0; g < G; ++g) {
      const int unr = flags[G + g];
      b->max_diam = std::max(b->max_diam, flags[g] + (unr ? 1 : 0));
      if (unr) {
        any_unreached = true;
        ++b->disconnected;
      }
    }
    if (any_unreached && disconnected_policy != 1) {
      cleanup();
      return bail(FD_ERR_DISCONNECTED);
    }
    if (flags[2 * G] != 0 || b->max_diam > 253) {
      cleanup();
      return bail(FD_ERR_UNIMPLEMENTED);
    }
    // diagonal of every graph's L^W
    if ((e = dev_alloc(&b->d_s, (size_t)b->P)) != FD_OK || (e = dev_alloc(&b->d_inv_s, (size_t)b->P)) != FD_OK) {
      cleanup();
      return bail(e);
    }
    const int rgrid = std::max(1, std::min((int)rows.size(), 8 * b->sm_count));
    ce = launch_rowsum_multi(b->d_graphs, d_rows, (int)rows.size(), b->D, b->d_s, b->d_inv_s, rgrid, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cleanup();
    if (ce != cudaSuccess) {
      cudaGetLastError();
      return bail(cuda_status(ce));
    }
  }
  // lookup table of 1/d and 1/d^2 (replicated per lane), as for one graph
  b->lut_rows = std::min(LUT_N, b->max_diam + 2);
  std::vector<unsigned char> lut((size_t)b->lut_rows * LUT_ROW, 0);
  for (int c = 1; c < b->lut_rows; ++c) {
    float* row = reinterpret_cast<float*>(lut.data() + (size_t)c * LUT_ROW);
    const float w = (float)(1.0 / ((double)c * c)), inv = (float)(1.0 / c);
    for (int k = 0; k < 32; ++k) {
      row[k] = inv;
      row[32 + k] = w;
    }
  }
  const size_t ps = (size_t)b->P * b->dimp;
  if ((s = dev_alloc(&b->d_lut, lut.size())) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_pool, 6 * ps)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_xin, (size_t)N * dim)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_omega, (size_t)G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_queue, 4)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_iout, (size_t)4 * G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_dout, (size_t)5 * G)) != FD_OK) return bail(s);
  if ((s = dev_alloc(&b->d_params, 1)) != FD_OK) return bail(s);
  if (cudaMemcpyAsync(b->d_lut, lut.data(), lut.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(b->d_pool, 0, 6 * ps * sizeof(float), st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return bail(FD_ERR_CUDA);
  }
  // default launch shape: two tile groups, two stages, else the first that fits
  const int shapes[4][2] = {{2, 2}, {1, 2}, {2, 3}, {1, 3}};
  s = FD_ERR_ARG;
  for (auto& sh : shapes)
    if ((s = batch_shape(b, sh[0], sh[1])) == FD_OK) break;
  if (s != FD_OK) return bail(FD_ERR_CUDA);
  // tile edges: the ones tuned earlier in this process for this dimension, else TILE
  int tiles[FD_BATCH_BUCKETS];
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (int k = 0; k < FD_BATCH_BUCKETS; ++k) tiles[k] = g_tile_cache[dim][k] ? g_tile_cache[dim][k] : TILE;
  }
  if ((s = batch_set_tiles(b, tiles)) != FD_OK) return bail(s);
  *out = b;
  return FD_OK;
}

void fd_batch_destroy(fd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  batch_release(b);
  delete b;
}

fd_status fd_batch_run(fd_batch* b, float* X, const fd_options* opt, const double* omega, int32_t* iters,
                       double* f_out) {
  if (!b || !X || !opt) return FD_ERR_ARG;
  const bool dev = is_device_ptr(X);
  const size_t nx = (size_t)b->N * b->dim;
  if (!dev) {
    FD_CK(cudaMemcpyAsync(b->d_xin, X, nx * sizeof(float), cudaMemcpyHostToDevice, b->stream));
  }
  // a device layout is updated in place: each graph reads its rows before it writes them
  float* xo = dev ? X : b->d_xin;
  double kms = 0.0;
  fd_status s = batch_run_dev(b, dev ? X : b->d_xin, xo, opt, omega, opt->max_iter, &kms);
  if (s != FD_OK && s != FD_ERR_NONFINITE) return s;
  if (!dev) {
    FD_CK(cudaMemcpyAsync(X, b->d_xin, nx * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    FD_CK(cudaStreamSynchronize(b->stream));
  }
  const size_t G = (size_t)b->G;
  for (size_t g = 0; g < G; ++g) {
    if (iters) iters[g] = b->h_iout[g];
    if (f_out) f_out[g] = b->h_dout[g];
  }
  return s;
}

fd_status fd_batch_results(const fd_batch* b, int32_t* status, int32_t* cg_steps, int32_t* accepted, double* crit,
                           double* matvec_passes, double* stress_passes, double* graph_ms) {
  if (!b) return FD_ERR_ARG;
  const size_t G = (size_t)b->G;
  if (b->h_iout.size() < 4 * G) return FD_ERR_ARG;  // no run yet
  for (size_t g = 0; g < G; ++g) {
    if (status) status[g] = b->h_iout[3 * G + g];
    if (cg_steps) cg_steps[g] = b->h_iout[G + g];
    if (accepted) accepted[g] = b->h_iout[2 * G + g];
    if (crit) crit[g] = b->h_dout[G + g];
    if (matvec_passes) matvec_passes[g] = b->h_dout[2 * G + g];
    if (stress_passes) stress_passes[g] = b->h_dout[3 * G + g];
    if (graph_ms) graph_ms[g] = b->h_dout[4 * G + g];
  }
  return FD_OK;
}

fd_status fd_batch_set_shape(fd_batch* b, int32_t groups, int32_t stages) {
  if (!b) return FD_ERR_ARG;
  return batch_shape(b, groups, stages);
}

fd_status fd_batch_tune(fd_batch* b, const float* X, const fd_options* opt, int32_t probe_iter, int32_t repeats,
                        int32_t* groups, int32_t* stages) {
  if (!b || !X || !opt || probe_iter < 1 || repeats < 1) return FD_ERR_ARG;
  const size_t nx = (size_t)b->N * b->dim;
  float* d_out = nullptr;
  fd_status s = dev_alloc(&d_out, nx);
  if (s != FD_OK) return s;
  const cudaMemcpyKind kind = is_device_ptr(X) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // best of `repeats` probe runs (over `subset`, or every graph)
  auto probe = [&](const std::vector<int>* subset, double* t_best) -> fd_status {
    *t_best = 1e300;
    for (int r = 0; r < repeats; ++r) {
      if (cudaMemcpyAsync(b->d_xin, X, nx * sizeof(float), kind, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return FD_ERR_CUDA;
      }
      double kms = 0.0;
      fd_status e = batch_run_dev(b, b->d_xin, d_out, opt, nullptr, probe_iter, &kms, subset);
      if (e != FD_OK && e != FD_ERR_NONFINITE) return e;
      *t_best = std::min(*t_best, kms);
    }
    return FD_OK;
  };
  // 1. launch shape (tile groups x stages) at the current tile edges
  const int W0 = b->W, nbuf0 = b->nbuf;
  int bestW = W0, bestN = nbuf0;
  double best = 1e300;
  const int shapes[4][2] = {{1, 2}, {1, 3}, {2, 2}, {2, 3}};
  for (auto& sh : shapes) {
    if (batch_shape(b, sh[0], sh[1]) != FD_OK) continue;
    double t = 0.0;
    if ((s = probe(nullptr, &t)) != FD_OK) break;
    if (t < best) {
      best = t;
      bestW = sh[0];
      bestN = sh[1];
    }
  }
  if (s == FD_OK) s = batch_shape(b, bestW, bestN);
  // 2. tile edge per size bucket: each bucket's graphs alone at T = 32, 64, 128
  int tiles[FD_BATCH_BUCKETS];
  std::memcpy(tiles, b->tiles, sizeof(tiles));
  for (int k = 0; k < FD_BATCH_BUCKETS && s == FD_OK; ++k) {
    std::vector<int> ids;
    for (int g : b->order)
      if (batch_bucket(b->graphs[g].n) == k) ids.push_back(g);
    if (ids.empty()) continue;
    int bestT = tiles[k];
    double tb = 1e300;
    for (int T : {TILE, 64, 32}) {
      int trial[FD_BATCH_BUCKETS];
      std::memcpy(trial, tiles, sizeof(trial));
      trial[k] = T;
      if ((s = batch_set_tiles(b, trial)) != FD_OK) break;
      double t = 0.0;
      if ((s = probe(&ids, &t)) != FD_OK) break;
      if (t < tb) {
        tb = t;
        bestT = T;
      }
    }
    tiles[k] = bestT;
  }
  dev_free(d_out);
  if (s != FD_OK) {
    batch_shape(b, W0, nbuf0);
    return s;
  }
  if ((s = batch_set_tiles(b, tiles)) != FD_OK) return s;
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    for (int k = 0; k < FD_BATCH_BUCKETS; ++k) g_tile_cache[b->dim][k] = tiles[k];
  }
  if (groups) *groups = b->W;
  if (stages) *stages = b->nbuf;
  return FD_OK;
}

fd_status fd_batch_set_tiles(fd_batch* b, const int32_t* tiles) {
  if (!b || !tiles) return FD_ERR_ARG;
  int t[FD_BATCH_BUCKETS];
  for (int k = 0; k < FD_BATCH_BUCKETS; ++k) t[k] = tiles[k];
  return batch_set_tiles(b, t);
}

fd_status fd_batch_get_tiles(const fd_batch* b, int32_t* tiles) {
  if (!b || !tiles) return FD_ERR_ARG;
  for (int k = 0; k < FD_BATCH_BUCKETS; ++k) tiles[k] = b->tiles[k];
  return FD_OK;
}

fd_status fd_batch_cached_tiles(int32_t dim, int32_t* tiles) {
  if (dim < 1 || dim > 3 || !tiles) return FD_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_tile_mu);
  for (int k = 0; k < FD_BATCH_BUCKETS; ++k) tiles[k] = g_tile_cache[dim][k];
  return FD_OK;
}

void fd_batch_clear_tile_cache(void) {
  std::lock_guard<std::mutex> lk(g_tile_mu);
  std::memset(g_tile_cache, 0, sizeof(g_tile_cache));
}

fd_status fd_batch_distances(fd_batch* b, int32_t g, double* out) {
  if (!b || !out || g < 0 || g >= b->G) return FD_ERR_ARG;
  const BGraph& gr = b->graphs[g];
  const size_t nn = (size_t)gr.n * gr.n;
  double* d = nullptr;
  fd_status s = dev_alloc(&d, nn);
  if (s != FD_OK) return s;
  cudaError_t e = launch_distance_graph(b->D + (size_t)gr.t0 * TILE * TILE, gr.n, gr.nb, d, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, nn * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return FD_OK;
}

fd_status fd_batch_get_info(const fd_batch* b, fd_batch_info* info) {
  if (!b || !info) return FD_ERR_ARG;
  info->num_graphs = b->G;
  info->dim = b->dim;
  info->total_vertices = b->N;
  info->num_tiles = b->ntiles;
  info->distance_bytes = (int64_t)b->D_bytes;
  info->max_n = b->max_n;
  info->max_diameter = b->max_diam;
  info->disconnected = b->disconnected;
  info->sm_count = b->sm_count;
  info->grid = b->grid;
  info->groups = b->W;
  info->stages = b->nbuf;
  info->graph_captured = b->captured;
  info->apsp_ms = b->apsp_ms;
  info->small_tile_bytes = (int64_t)b->DT_bytes;
  int counts[3] = {0, 0, 0};
  for (const BGraph& gr : b->graphs) ++counts[tile_class(gr.T)];
  info->graphs_t128 = counts[0];
  info->graphs_t64 = counts[1];
  info->graphs_t32 = counts[2];
  return FD_OK;
}

fd_status fd_batch_last_stats(const fd_batch* b, fd_stats* stats) {
  if (!b || !stats) return FD_ERR_ARG;
  *stats = b->stats;
  return FD_OK;
}

}  // extern "C"
