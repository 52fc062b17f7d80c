// k_batch.cu -- many small graphs in one persistent launch (the batched workload).
//
// Each graph g (n_g <= RD_BATCH_MAX_N nodes, gain gamma_g) goes through the whole method
// (Sec. 2 eq. Y-defined and R-defined; Sec. 4.1 rounded distance): M = I - gamma A, Y = M^-1,
// D = ceil(log_gamma Y - tau), D_ii = 0.  The inverse is a blocked Gauss-Jordan elimination
// without pivoting in FP64 (M is a strictly column diagonally dominant M-matrix under the gain
// check, so every pivot block is invertible without row exchanges and the Schur complements stay
// dominant).  For each 64-wide block k:
//   D_kk = M_kk^-1;  M_kj <- D_kk M_kj (j != k);  M_ij <- M_ij - M_ik M_kj (i, j != k);
//   M_ik <- -M_ik D_kk (i != k);  M_kk <- D_kk
// which leaves M^-1 in place after the last block (2 n^3 flops, like LU + inverses + product).
//
// One CTA owns one graph at a time; CTAs take graphs from an atomic counter over an order sorted
// by decreasing n (longest first).  The graph's matrix lives in a workspace slice in HBM/L2; the
// diagonal block and the operand tiles of the rank-64 updates are staged in shared memory, and
// each thread keeps a 4 x 4 tile of the 64 x 64 output tile in registers (FP64 pipe bound).
#include <cstdio>
#include <vector>
#include <algorithm>
#include <numeric>

#include "rd_internal.cuh"

namespace {

constexpr int BB = 64;           // block width
constexpr int BT = 256;          // threads per CTA
constexpr int LDS = BB + 1;      // padded shared-memory row (conflict-free column reads)

struct BatchArgs {
  const uint8_t* A;      // packed adjacency matrices (graph g at off[g], n_g x n_g bytes)
  int32_t* D;            // packed distances (graph g at off[g], n_g x n_g int32)
  double* W;             // workspace (graph g at off[g], n_g x n_g doubles)
  const int64_t* off;
  const int32_t* n;
  const double* gamma;
  const int32_t* order;  // graphs by decreasing n
  int G;
  int* counter;          // work queue head (zeroed before the launch)
  int32_t* status;       // per graph: RD_OK, RD_ERR_GAMMA, RD_ERR_NUMERIC
  double tau;
  const int32_t* done;   // per graph: 1 = already computed (the split variant kept its result); may be null
};

// C (rows x cols tile at global (r0, c0) of an n x n matrix) -= A (rows x kb) B (kb x cols), with
// A and B staged in shared memory (LDS-padded), C read and written through global memory; each
// thread owns the 4 x 4 entries (4 (t / 16) + a, 4 (t % 16) + b).  sign = -1 computes C = -A B
// (C not read).
__device__ __forceinline__ void tile_update(double* __restrict__ M, int n, int r0, int c0, int rows, int cols,
                                            const double (*sa)[LDS], const double (*sb)[LDS], int kb, bool overwrite) {
  const int t = threadIdx.x, i0 = 4 * (t / 16), j0 = 4 * (t % 16);
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k = 0; k < kb; ++k) {
    double x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = sa[i0 + a][k];
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = sb[k][j0 + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + a;
    if (i >= rows) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + b;
      if (j >= cols) continue;
      double* c = M + (long long)(r0 + i) * n + (c0 + j);
      *c = overwrite ? -acc[a][b] : *c - acc[a][b];
    }
  }
}

// stage the rows x cols block at (r0, c0) of the n x n matrix into s (zero outside)
__device__ __forceinline__ void stage(const double* __restrict__ M, int n, int r0, int c0, int rows, int cols,
                                      double (*s)[LDS]) {
  for (int e = threadIdx.x; e < BB * BB; e += BT) {
    const int i = e / BB, j = e % BB;
    s[i][j] = (i < rows && j < cols) ? M[(long long)(r0 + i) * n + (c0 + j)] : 0.0;
  }
}

__global__ void __launch_bounds__(BT) batch_kernel(const BatchArgs p) {
  extern __shared__ double smem_b[];
  double(*dk)[LDS] = reinterpret_cast<double(*)[LDS]>(smem_b);                // D_kk
  double(*sa)[LDS] = reinterpret_cast<double(*)[LDS]>(smem_b + BB * LDS);     // A operand tile
  double(*sb)[LDS] = reinterpret_cast<double(*)[LDS]>(smem_b + 2 * BB * LDS); // B operand tile
  __shared__ int s_graph, s_bad;
  __shared__ double s_red[BT / 32];
  const int t = threadIdx.x;
  for (;;) {
    if (t == 0) {
      const int q = atomicAdd(p.counter, 1);
      s_graph = q < p.G ? p.order[q] : -1;
      s_bad = 0;
    }
    __syncthreads();
    const int g = s_graph;
    if (g < 0) return;
    if (p.done && p.done[g]) {  // (uniform: every thread reads the same flag)
      __syncthreads();            // every thread has read s_graph before thread 0 takes the next
      continue;
    }
    const int n = p.n[g];
    const double gamma = p.gamma[g];
    const uint8_t* A = p.A + p.off[g];
    double* M = p.W + p.off[g];
    int32_t* Dg = p.D + p.off[g];
    // ---- gain check (a1): the largest column sum of gamma A must stay below 1
    double mx = 0.0;
    for (int j = t; j < n; j += BT) {
      int deg = 0;
      for (int i = 0; i < n; ++i) deg += A[(long long)i * n + j] ? 1 : 0;
      mx = fmax(mx, gamma * deg);
    }
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((t & 31) == 0) s_red[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
      double m = 0.0;
      for (int w = 0; w < BT / 32; ++w) m = fmax(m, s_red[w]);
      if (!(m < 1.0) || !(gamma > 0.0 && gamma < 1.0)) s_bad = RD_ERR_GAMMA;
    }
    __syncthreads();
    if (s_bad) {
      if (t == 0) p.status[g] = s_bad;
      __syncthreads();
      continue;
    }
    // ---- M = I - gamma A (a2)
    for (long long e = t; e < (long long)n * n; e += BT) {
      const int i = (int)(e / n), j = (int)(e % n);
      M[e] = (i == j ? 1.0 : 0.0) - (A[e] ? gamma : 0.0);
    }
    __syncthreads();
    // ---- blocked Gauss-Jordan (a3-a5 in one sweep)
    const int nb = (n + BB - 1) / BB;
    for (int kbk = 0; kbk < nb; ++kbk) {
      const int k0 = kbk * BB, kb = min(BB, n - k0);
      // D_kk = M_kk^-1 by unblocked Gauss-Jordan in shared memory (identity padding past kb)
      for (int e = t; e < BB * BB; e += BT) {
        const int i = e / BB, j = e % BB;
        dk[i][j] = (i < kb && j < kb) ? M[(long long)(k0 + i) * n + (k0 + j)] : (i == j ? 1.0 : 0.0);
      }
      __syncthreads();
      for (int q = 0; q < kb; ++q) {
        const double piv = dk[q][q];
        if (!(piv > 0.0) || !isfinite(piv)) {
          if (t == 0) s_bad = RD_ERR_NUMERIC;
        }
        const double rp = 1.0 / piv;
        __syncthreads();
        // column q of the other rows (the multipliers), kept before row q changes
        double mult = 0.0;
        const int i_own = t / 4;            // 64 rows x 4 column groups of 16
        const int jg = (t % 4) * 16;
        if (i_own < BB) mult = dk[i_own][q];
        __syncthreads();
        if (t < BB) dk[q][t] *= rp;         // row q scaled; column q becomes 1/piv below
        __syncthreads();
        if (i_own != q) {
          for (int j = jg; j < jg + 16; ++j) {
            if (j == q) continue;
            dk[i_own][j] = fma(-mult, dk[q][j], dk[i_own][j]);
          }
        }
        __syncthreads();
        if (t < BB) {
          if (t == q)
            dk[q][q] = rp;
          else
            dk[t][q] = -dk[t][q] * rp;  // not yet touched in column q: -m_iq / piv
        }
        __syncthreads();
      }
      // row panel: M_kj <- D_kk M_kj for the other column tiles
      for (int jt = 0; jt < nb; ++jt) {
        if (jt == kbk) continue;
        const int c0 = jt * BB, cols = min(BB, n - c0);
        stage(M, n, k0, c0, kb, cols, sb);
        __syncthreads();
        // C = D_kk (kb x kb) * sb: written over M_kj (overwrite with sign flip twice = plain product)
        {
          const int i0 = 4 * (t / 16), j0 = 4 * (t % 16);
          double acc[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
          for (int k = 0; k < kb; ++k) {
            double x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = dk[i0 + a][k];
#pragma unroll
            for (int b = 0; b < 4; ++b) y[b] = sb[k][j0 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (i0 + a < kb && j0 + b < cols) M[(long long)(k0 + i0 + a) * n + (c0 + j0 + b)] = acc[a][b];
        }
        __syncthreads();
      }
      // trailing update and column panel, one row tile at a time
      for (int it = 0; it < nb; ++it) {
        if (it == kbk) continue;
        const int r0 = it * BB, rows = min(BB, n - r0);
        stage(M, n, r0, k0, rows, kb, sa);  // the old M_ik
        __syncthreads();
        for (int jt = 0; jt < nb; ++jt) {
          if (jt == kbk) continue;
          const int c0 = jt * BB, cols = min(BB, n - c0);
          stage(M, n, k0, c0, kb, cols, sb);  // the new M_kj
          __syncthreads();
          tile_update(M, n, r0, c0, rows, cols, sa, sb, kb, false);
          __syncthreads();
        }
        // M_ik <- -M_ik D_kk
        tile_update(M, n, r0, k0, rows, kb, sa, dk, kb, true);
        __syncthreads();
      }
      // M_kk <- D_kk
      for (int e = t; e < kb * kb; e += BT) {
        const int i = e / kb, j = e % kb;
        M[(long long)(k0 + i) * n + (k0 + j)] = dk[i][j];
      }
      __syncthreads();
    }
    // ---- decode (a5 epilogue)
    const double lg = log(gamma);
    const float ilg2 = (float)(1.0 / log2(gamma));
    bool nonfinite = false;
    for (long long e = t; e < (long long)n * n; e += BT) {
      const int i = (int)(e / n), j = (int)(e % n);
      const double y = M[e];
      int32_t d;
      if (!isfinite(y)) {
        nonfinite = true;
        d = RD_UNREACHABLE;
      } else {
        d = (i == j) ? 0 : rd_decode_entry_fast(y, ilg2, lg, p.tau);
      }
      Dg[e] = d;
    }
    if (nonfinite) s_bad = RD_ERR_NUMERIC;
    __syncthreads();
    if (t == 0) p.status[g] = s_bad ? s_bad : RD_OK;
    __syncthreads();
  }
}

}  // namespace

struct rd_batch {
  int device = 0;
  int G = 0;
  int64_t total = 0;        // sum of n_g^2
  int max_n = 0;
  double tau = 1e-9;
  std::vector<int64_t> off;
  int64_t* d_off = nullptr;
  int32_t* d_n = nullptr;
  double* d_gamma = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_status = nullptr;
  int* d_counter = nullptr;
  double* d_W = nullptr;
  int blocks = 0;
  std::string err;
  std::vector<int32_t> n;      // node counts (host)
  std::vector<double> gamma;   // gains (host)
  // split precision (rd_batch_set_precision): the split plan of the size classes that run on it
  int precision = RD_PREC_FP64;
  rd_batch_split* split = nullptr;
  int32_t* d_done = nullptr;    // per graph: 1 = the split variant kept its result
  int32_t* d_routes = nullptr;  // per graph: the route of its last run (rd_batch_routes)
  double tune_ms_fp64[RD_BATCH_CLASSES] = {}, tune_ms_split[RD_BATCH_CLASSES] = {};
  int32_t tune_split[RD_BATCH_CLASSES] = {};
  int32_t tune_graphs[RD_BATCH_CLASSES] = {};
  int64_t launches = 0;  // kernel launches of the last run
};

namespace {
constexpr size_t BATCH_SMEM = 3 * BB * LDS * sizeof(double);

void batch_free(rd_batch* b) {
  rd_bsplit_destroy(b->split);
  b->split = nullptr;
  void* ptrs[] = {b->d_off, b->d_n, b->d_gamma, b->d_order, b->d_status, b->d_counter, b->d_W, b->d_done, b->d_routes};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

// size class of a graph: n rounded up to a multiple of 128, as an index 0..RD_BATCH_CLASSES-1
int size_class(int n) { return (n + RD_PAD - 1) / RD_PAD - 1; }

// Seeded directed Erdos-Renyi graphs (p = 4/n, no self-loops) for the autotuner's probes: A packed
// as a batch (A_ij != 0 iff edge j -> i), gain 0.5 / (Delta + 1).  SplitMix64 per entry.
uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
void probe_graphs(const std::vector<int32_t>& n, std::vector<uint8_t>& A, std::vector<double>& gamma,
                  std::vector<int64_t>& off) {
  off.assign(n.size() + 1, 0);
  for (size_t g = 0; g < n.size(); ++g) off[g + 1] = off[g] + (int64_t)n[g] * n[g];
  A.assign((size_t)off.back(), 0);
  gamma.resize(n.size());
  for (size_t g = 0; g < n.size(); ++g) {
    const int m = n[g];
    const uint64_t thr = (uint64_t)((4.0 / m) * 18446744073709551615.0);
    std::vector<int> deg(m, 0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        if (i != j && splitmix(((uint64_t)g << 40) ^ ((uint64_t)i << 20) ^ (uint64_t)j) < thr) {
          A[off[g] + (int64_t)i * m + j] = 1;
          deg[j]++;
        }
    gamma[g] = 0.5 / (*std::max_element(deg.begin(), deg.end()) + 1);
  }
}

// Device time (ms) of the second of two runs of a batch on `st` (CUDA events).
double time_runs(rd_batch* b, const uint8_t* A, int32_t* D, cudaStream_t st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  rd_batch_apsp(b, A, D, st);
  cudaEventRecord(e0, st);
  rd_batch_apsp(b, A, D, st);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}
}  // namespace

extern "C" {

rd_status rd_batch_create(const int32_t* n, const double* gamma, int32_t G, rd_batch_handle* out) {
  if (!out) return RD_ERR_ARG;
  *out = nullptr;
  if (!n || !gamma || G < 1) {
    rd_record_error("rd_batch_create: n and gamma must be host arrays of G >= 1 entries");
    return RD_ERR_ARG;
  }
  rd_batch* b = new rd_batch();
  b->G = G;
  b->off.resize((size_t)G + 1);
  b->off[0] = 0;
  for (int g = 0; g < G; ++g) {
    if (n[g] < 1 || n[g] > RD_BATCH_MAX_N) {
      delete b;
      rd_record_error("rd_batch_create: every n must lie in [1, RD_BATCH_MAX_N]");
      return RD_ERR_ARG;
    }
    b->off[g + 1] = b->off[g] + (int64_t)n[g] * n[g];
    b->max_n = std::max(b->max_n, (int)n[g]);
  }
  b->total = b->off[G];
  b->n.assign(n, n + G);
  b->gamma.assign(gamma, gamma + G);
  std::vector<int32_t> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return n[a] > n[c]; });
  cudaError_t e = cudaGetDevice(&b->device);
  auto get = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  get((void**)&b->d_off, (G + 1) * sizeof(int64_t));
  get((void**)&b->d_n, G * sizeof(int32_t));
  get((void**)&b->d_gamma, G * sizeof(double));
  get((void**)&b->d_order, G * sizeof(int32_t));
  get((void**)&b->d_status, G * sizeof(int32_t));
  get((void**)&b->d_counter, sizeof(int));
  get((void**)&b->d_W, (size_t)b->total * sizeof(double));
  get((void**)&b->d_done, G * sizeof(int32_t));
  get((void**)&b->d_routes, G * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_off, b->off.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_n, n, G * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_gamma, gamma, G * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_order, order.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0xff, G * sizeof(int32_t));  // -1: not run yet
  if (e == cudaSuccess) e = cudaMemset(b->d_routes, 0, G * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_SMEM);
  int per_sm = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, BT, BATCH_SMEM);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    rd_record_error(std::string("rd_batch_create: ") + cudaGetErrorString(e));
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
  }
  b->blocks = std::max(1, std::min(G, per_sm * sms));
  *out = b;
  return RD_OK;
}

rd_status rd_batch_offsets(rd_batch_handle b, int64_t* off) {
  if (!b || !off) return RD_ERR_ARG;
  std::copy(b->off.begin(), b->off.end(), off);
  return RD_OK;
}

rd_status rd_batch_apsp(rd_batch_handle b, const uint8_t* A, int32_t* D, void* stream) {
  if (!b || !A || !D) return RD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
  b->launches = 1;
  if (e == cudaSuccess && b->split) {
    // the split variant first (its stacks decide on the device which graphs it keeps), then the
    // FP64 kernel for every other graph
    e = cudaMemsetAsync(b->d_done, 0, b->G * sizeof(int32_t), s);
    int64_t n_split = 0;
    if (e == cudaSuccess) e = rd_bsplit_run(b->split, A, D, b->d_status, b->d_done, b->d_routes, s, &n_split);
    b->launches += n_split;
  }
  if (e != cudaSuccess) {
    b->err = cudaGetErrorString(e);
    return RD_ERR_CUDA;
  }
  BatchArgs a{};
  a.A = A;
  a.D = D;
  a.W = b->d_W;
  a.off = b->d_off;
  a.n = b->d_n;
  a.gamma = b->d_gamma;
  a.order = b->d_order;
  a.G = b->G;
  a.counter = b->d_counter;
  a.status = b->d_status;
  a.tau = b->tau;
  a.done = b->split ? b->d_done : nullptr;
  batch_kernel<<<b->blocks, BT, BATCH_SMEM, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    b->err = cudaGetErrorString(e);
    return RD_ERR_CUDA;
  }
  return RD_OK;
}

rd_status rd_batch_status(rd_batch_handle b, int32_t* status) {
  if (!b || !status) return RD_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, b->d_status, b->G * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    b->err = cudaGetErrorString(e);
    return RD_ERR_CUDA;
  }
  return RD_OK;
}

void rd_batch_destroy(rd_batch_handle b) {
  if (!b) return;
  batch_free(b);
  delete b;
}

rd_status rd_batch_set_precision(rd_batch_handle b, int32_t mode, int32_t autotune) {
  if (!b) return RD_ERR_ARG;
  if (mode != RD_PREC_FP64 && mode != RD_PREC_SPLIT_BF16) {
    rd_record_error("rd_batch_set_precision: unknown precision mode");
    return RD_ERR_ARG;
  }
  cudaError_t e = cudaDeviceSynchronize();
  rd_bsplit_destroy(b->split);
  b->split = nullptr;
  b->precision = mode;
  for (int c = 0; c < RD_BATCH_CLASSES; ++c) {
    b->tune_ms_fp64[c] = b->tune_ms_split[c] = 0.0;
    b->tune_split[c] = 0;
    b->tune_graphs[c] = 0;
  }
  if (e == cudaSuccess) e = cudaMemset(b->d_routes, 0, b->G * sizeof(int32_t));
  if (e != cudaSuccess) {
    rd_record_error(std::string("rd_batch_set_precision: ") + cudaGetErrorString(e));
    return RD_ERR_CUDA;
  }
  if (mode == RD_PREC_FP64) return RD_OK;
  std::vector<std::vector<int32_t>> cls(RD_BATCH_CLASSES);
  for (int g = 0; g < b->G; ++g) cls[size_class(b->n[g])].push_back(g);
  std::string err;
  cudaStream_t st = nullptr;
  for (int c = 0; c < RD_BATCH_CLASSES; ++c) {
    b->tune_graphs[c] = (int32_t)cls[c].size();
    if (cls[c].empty()) continue;
    if (!autotune) {
      b->tune_split[c] = 1;
      continue;
    }
    // The autotuner: time both variants on up to 152 seeded random graphs of this class's sizes (a
    // full wave of the FP64 kernel) and keep the faster per graph
    const size_t P = std::min<size_t>(cls[c].size(), 152);
    std::vector<int32_t> pn(P), pid(P);
    for (size_t q = 0; q < P; ++q) {
      pn[q] = b->n[cls[c][q]];
      pid[q] = (int32_t)q;
    }
    std::vector<uint8_t> pA;
    std::vector<double> pg;
    std::vector<int64_t> poff;
    probe_graphs(pn, pA, pg, poff);
    rd_batch* pb = nullptr;
    rd_status rs = rd_batch_create(pn.data(), pg.data(), (int32_t)P, &pb);
    uint8_t* dA = nullptr;
    int32_t* dD = nullptr;
    if (rs == RD_OK) {
      e = cudaMalloc((void**)&dA, pA.size());
      if (e == cudaSuccess) e = cudaMalloc((void**)&dD, pA.size() * sizeof(int32_t));
      if (e == cudaSuccess) e = cudaMemcpy(dA, pA.data(), pA.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) b->tune_ms_fp64[c] = time_runs(pb, dA, dD, st) / P;
      if (e == cudaSuccess) rs = rd_bsplit_create(pn.data(), pg.data(), poff.data(), pid.data(), (int)P, b->tau,
                                                  &pb->split, &err);
      if (e == cudaSuccess && rs == RD_OK) b->tune_ms_split[c] = time_runs(pb, dA, dD, st) / P;
      if (e == cudaSuccess && rs == RD_OK) e = cudaDeviceSynchronize();
    }
    if (dA) cudaFree(dA);
    if (dD) cudaFree(dD);
    rd_batch_destroy(pb);
    if (rs != RD_OK || e != cudaSuccess) {
      rd_record_error("rd_batch_set_precision: autotuner: " + (e != cudaSuccess ? std::string(cudaGetErrorString(e)) : err));
      return rs != RD_OK ? rs : RD_ERR_CUDA;
    }
    b->tune_split[c] = b->tune_ms_split[c] < b->tune_ms_fp64[c] ? 1 : 0;
  }
  std::vector<int32_t> gids;
  for (int c = 0; c < RD_BATCH_CLASSES; ++c)
    if (b->tune_split[c]) gids.insert(gids.end(), cls[c].begin(), cls[c].end());
  if (gids.empty()) return RD_OK;
  const rd_status rs = rd_bsplit_create(b->n.data(), b->gamma.data(), b->off.data(), gids.data(), (int)gids.size(),
                                        b->tau, &b->split, &err);
  if (rs != RD_OK) rd_record_error("rd_batch_set_precision: " + err);
  return rs;
}

rd_status rd_batch_split_info(rd_batch_handle b, int32_t* digits, int32_t* passes, double* residual,
                              double* screen_bits) {
  if (!b || !digits || !passes || !residual || !screen_bits) return RD_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return RD_ERR_CUDA;
  return rd_bsplit_info(b->split, b->G, digits, passes, residual, screen_bits);
}

rd_status rd_batch_routes(rd_batch_handle b, int32_t* routes) {
  if (!b || !routes) return RD_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(routes, b->d_routes, b->G * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    b->err = cudaGetErrorString(e);
    return RD_ERR_CUDA;
  }
  return RD_OK;
}

rd_status rd_batch_tuning(rd_batch_handle b, int32_t* graphs, int32_t* split, double* ms_fp64, double* ms_split,
                          int64_t* launches) {
  if (!b || !graphs || !split || !ms_fp64 || !ms_split || !launches) return RD_ERR_ARG;
  *launches = b->launches;
  for (int c = 0; c < RD_BATCH_CLASSES; ++c) {
    graphs[c] = b->tune_graphs[c];
    split[c] = b->tune_split[c];
    ms_fp64[c] = b->tune_ms_fp64[c];
    ms_split[c] = b->tune_ms_split[c];
  }
  return RD_OK;
}

}  // extern "C"
