// k_batch_split.cu -- the split-precision variant of the batched graphs (rd_batch_* in
// RD_PREC_SPLIT_BF16): many small graphs through the split path's tensor-core digit products at
// once.
//
// Graphs of one padded size N (a multiple of 128) are stacked, at most BS_PART at a time, in a
// stacked handle (rd_ctx::nbatch): graph b's M, factors and inverses sit N * N doubles apart, and
// every launch of the split path's recursive factorisation (k_split.cu: 64 x 64 FP64 leaves, FP64
// products for nodes of at most 128 rows, tensor-core digit products above) and of the final
// product with the fused decode covers every graph of the stack.  A graph of a few hundred nodes
// is a handful of 128 x 128 tiles, too few for the tensor cores alone, but a stack of hundreds
// fills the GPU.  Every decision is taken on the device, so a run is a fixed sequence of launches
// that a CUDA graph can capture:
//   screen    per graph: the gain check (Theorem 4's condition, gamma times the largest out-degree
//             below 1), successor lists in shared memory, BFS from 16 sampled sources, and the
//             largest hop spread within a 256-node chunk times log2(1/gamma): the digit count is
//             the fewest (at least 8) whose 7 bits each cover that plus 40 bits of result (the
//             single-graph range screen, with twice its sources: a few hundred nodes make them
//             cheap); beyond 15 digits, or with too many edges to screen, the graph leaves the
//             split path
//   build     M = I - gamma A per graph on the split path (Sec. 2), the identity on the padding
//   factor    LU and both triangular inverses of every graph (rd_lu_split), then
//   product   Y = U^-1 L^-1 with D decoded in the epilogue into the caller's packed D; Y is kept
//             in the stack's LU matrices for the check
//   check     every entry of M Y - I against (|M| |Y|) entrywise (the componentwise backward
//             error), limit min(1e-9, tau |ln gamma| / 16), at least 1e-12 (the single-graph
//             self-check's)
//   finalize  a graph within the limit keeps its split D; one above it takes a second pass of
//             build / factor / product / check with the digits its residual r asks for (about
//             log2(r / 2^-40) / 7 more, as the single-graph escalation), and one that fails again,
//             or would need more than 15, is redone by the FP64 Gauss-Jordan kernel (k_batch.cu),
//             which runs after the stacks.  Every launch skips the graphs without work in its pass.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rd_internal.cuh"

namespace {

constexpr int BS_PART = 512;     // graphs per stacked handle
constexpr int BS_THREADS = 256;
constexpr int BS_MAX_N = RD_BATCH_MAX_N;
constexpr int BS_EDGES = 12288;  // successor entries a screen holds in shared memory
constexpr int BS_CHUNKS = (BS_MAX_N + RD_SCREEN_CHUNK - 1) / RD_SCREEN_CHUNK;
constexpr int BS_SRC = 2 * RD_SCREEN_SOURCES;  // BFS sources of the batch screen
static_assert(BS_MAX_N <= 512, "one screen thread per node");

// a run's per-graph outcome starts clean (n, gamma, off and the decode constants stay)
__global__ void bs_reset_kernel(rd_batch_graph* bg, int nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bg[b].s = 0;
  bg[b].status[0] = bg[b].status[1] = 0;
  bg[b].route = 0;
  bg[b].residual = 0.0;
  bg[b].screen_bits = -1.0;
  bg[b].digits = 0;
  bg[b].passes = 0;
}

// M = I - gamma A of graph blockIdx.y (n x n bytes at A + off, A_ij != 0 iff edge j -> i) into its
// N x N slot, identity on the padding; 8 rows per CTA, threads along the columns (coalesced).
__global__ void __launch_bounds__(BS_THREADS) bs_build_kernel(const uint8_t* __restrict__ A, double* __restrict__ LU,
                                                              int N, const rd_batch_graph* __restrict__ bg) {
  const int b = blockIdx.y;
  if (bg[b].s == 0) return;  // not on the split path in this pass
  const int n = bg[b].n;
  const double g = bg[b].gamma;
  const uint8_t* Ag = A + bg[b].off;
  double* M = LU + (long long)b * N * N;
  const int i1 = min(N, (int)blockIdx.x * 8 + 8);
  for (int i = blockIdx.x * 8; i < i1; ++i)
    for (int j = threadIdx.x; j < N; j += BS_THREADS) {
      double v = (i == j) ? 1.0 : 0.0;
      if (i < n && j < n && Ag[(long long)i * n + j]) v -= g;
      M[(long long)i * N + j] = v;
    }
}

// The gain check and the range screen of graph blockIdx.x (one thread per node; see the file
// comment).  Sources: nodes q n / 16 + n / 32.
__global__ void __launch_bounds__(BS_MAX_N) bs_screen_kernel(const uint8_t* __restrict__ A, rd_batch_graph* bg) {
  __shared__ int ptr_s[BS_MAX_N + 1];
  __shared__ int16_t succ_s[BS_EDGES];
  __shared__ int16_t dist_s[BS_SRC][BS_MAX_N];
  __shared__ int lo_s[BS_SRC][BS_CHUNKS], hi_s[BS_SRC][BS_CHUNKS];
  __shared__ int maxdeg_s, total_s, flag_s;
  const int b = blockIdx.x, v = threadIdx.x;
  const int n = bg[b].n;
  const uint8_t* Ag = A + bg[b].off;
  // out-degree of node v: column v of A (the edges v -> i); a warp reads consecutive bytes of a row
  int deg = 0;
  if (v < n)
    for (int i = 0; i < n; ++i) deg += Ag[(long long)i * n + v] != 0;
  if (v == 0) maxdeg_s = 0;
  __syncthreads();
  atomicMax(&maxdeg_s, deg);
  if (v < n) ptr_s[v + 1] = deg;
  __syncthreads();
  if (v == 0) {
    ptr_s[0] = 0;
    for (int u = 0; u < n; ++u) ptr_s[u + 1] += ptr_s[u];
    total_s = ptr_s[n];
  }
  __syncthreads();
  const double gamma = bg[b].gamma;
  if (!(gamma * maxdeg_s < 1.0)) {  // not strictly column diagonally dominant: the FP64 kernel reports it
    if (v == 0) bg[b].route = 2;
    return;
  }
  if (total_s > BS_EDGES) {  // successor lists beyond shared memory: not screened, FP64
    if (v == 0) bg[b].route = 3;
    return;
  }
  if (v < n) {
    int w = ptr_s[v];
    for (int i = 0; i < n; ++i)
      if (Ag[(long long)i * n + v]) succ_s[w++] = (int16_t)i;
  }
  for (int q = 0; q < BS_SRC; ++q) {
    const int src = q * n / BS_SRC + n / (2 * BS_SRC);
    if (v < n) dist_s[q][v] = (v == src) ? 0 : -1;
  }
  if (v < BS_SRC * BS_CHUNKS) {
    lo_s[v / BS_CHUNKS][v % BS_CHUNKS] = 1 << 30;
    hi_s[v / BS_CHUNKS][v % BS_CHUNKS] = -1;
  }
  __syncthreads();
  // level-synchronous BFS from every source at once (a node reached at level l + 1 is only
  // expanded in the next round; concurrent writers write the same level)
  for (int level = 0; level < n; ++level) {
    if (v == 0) flag_s = 0;
    __syncthreads();
    if (v < n)
      for (int q = 0; q < BS_SRC; ++q)
        if (dist_s[q][v] == level)
          for (int e = ptr_s[v]; e < ptr_s[v + 1]; ++e) {
            const int u = succ_s[e];
            if (dist_s[q][u] < 0) {
              dist_s[q][u] = (int16_t)(level + 1);
              flag_s = 1;
            }
          }
    __syncthreads();
    const int more = flag_s;
    __syncthreads();
    if (!more) break;
  }
  if (v < n) {
    const int c = v / RD_SCREEN_CHUNK;
    for (int q = 0; q < BS_SRC; ++q) {
      const int d = dist_s[q][v];
      if (d >= 0) {
        atomicMin(&lo_s[q][c], d);
        atomicMax(&hi_s[q][c], d);
      }
    }
  }
  __syncthreads();
  if (v == 0) {
    int spread = 0;
    for (int q = 0; q < BS_SRC; ++q)
      for (int c = 0; c < BS_CHUNKS; ++c)
        if (hi_s[q][c] >= 0) spread = max(spread, hi_s[q][c] - lo_s[q][c]);
    const double bits = spread * log2(1.0 / gamma);
    int s = (int)ceil((bits + RD_SCREEN_RESULT_BITS) / RD_SPLIT_DIGIT_BITS);
    if (s < RD_SPLIT_MIN) s = RD_SPLIT_MIN;
    bg[b].screen_bits = bits;
    if (s > RD_SPLIT_MAX) {
      bg[b].route = 3;
    } else {
      bg[b].s = s;
    }
  }
}

// Entrywise residual of graph blockIdx.y's Y (its N x N slot) in row i = blockIdx.x:
//   (M Y - I)_ij = Y_ij - [i == j] - gamma sum_{k : A_ik != 0} Y_kj
// relative to (|M| |Y|)_ij = |Y_ij| + gamma sum |Y_kj|; the largest goes to bg.residual (atomicMax of
// the bits of a non-negative double).  An entry whose scale is below FP64's normal range carries no
// digits to check.  The predecessors k of i are listed in order (a deterministic sum).
__global__ void __launch_bounds__(BS_THREADS) bs_residual_kernel(const uint8_t* __restrict__ A,
                                                                 const double* __restrict__ Y, int N,
                                                                 rd_batch_graph* bg) {
  __shared__ int16_t pred[BS_MAX_N];
  __shared__ int npred;
  __shared__ double worst_s[BS_THREADS / 32];
  const int b = blockIdx.y, i = blockIdx.x;
  const int n = bg[b].n;
  if (i >= n || bg[b].s == 0) return;
  const uint8_t* row = A + bg[b].off + (long long)i * n;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < n; ++k)
      if (row[k]) pred[c++] = (int16_t)k;
    npred = c;
  }
  __syncthreads();
  const double g = bg[b].gamma;
  const double* Yg = Y + (long long)b * N * N;
  double worst = 0.0;
  for (int j = threadIdx.x; j < n; j += BS_THREADS) {
    double acc = 0.0, mag = 0.0;
    for (int q = 0; q < npred; ++q) {
      const double y = Yg[(long long)pred[q] * N + j];
      acc += y;
      mag += fabs(y);
    }
    const double yij = Yg[(long long)i * N + j];
    const double r = yij - (i == j ? 1.0 : 0.0) - g * acc;
    const double sc = fabs(yij) + g * mag;
    double rel = sc >= 0x1p-1022 ? fabs(r) / sc : 0.0;
    if (!(rel <= 1.0)) rel = 1.0;  // (also NaN)
    worst = fmax(worst, rel);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) worst_s[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BS_THREADS / 32; ++w) worst = fmax(worst, worst_s[w]);
    if (worst > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(&bg[b].residual), (unsigned long long)__double_as_longlong(worst));
  }
}

// The outcome of each graph of a stack after split pass `pass` (1 or 2).  A graph on the split path
// whose Y is finite and whose residual is within the limit keeps its D (done, status RD_OK, no work
// in later passes).  One above it takes pass 2 with the digits its residual asks for (at most 15);
// after pass 2, or beyond 15 digits, it goes to the FP64 kernel (route 1), as do graphs that
// failed the gain check (2) or were screened out (3).  routes[gid] (what rd_batch_routes reports):
// 1 split, 2 split redone in FP64, 3 screened out to FP64, 4 gain check failed.
__global__ void bs_finalize_kernel(rd_batch_graph* bg, int nb, const int32_t* __restrict__ gids, double tau, int pass,
                                   int32_t* status, int32_t* done, int32_t* routes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  rd_batch_graph& G = bg[b];
  if (G.digits > 0) return;  // kept in pass 1
  const int gid = gids[b];
  if (G.route == 0 && G.s > 0) {
    const double lim = fmin(RD_SPLIT_RESIDUAL, fmax(tau * fabs(G.log_gamma) / 16.0, 1e-12));
    if (G.residual <= lim && G.status[0] == 0) {
      done[gid] = 1;
      status[gid] = RD_OK;
      routes[gid] = 1;
      G.digits = G.s;
      G.passes = pass;
      G.s = 0;
      return;
    }
    int add = (G.residual <= 1.0 && G.status[0] == 0)
                  ? (int)ceil((log2(fmax(G.residual, 1e-300)) + RD_SCREEN_RESULT_BITS) / RD_SPLIT_DIGIT_BITS)
                  : RD_SPLIT_MAX;  // entries lost altogether (or not finite): no digit count will do
    const int next = G.s + max(1, add);
    if (pass == 1 && next <= RD_SPLIT_MAX) {  // pass 2 with more digits
      G.s = next;
      G.residual = 0.0;
      G.status[0] = G.status[1] = 0;
      done[gid] = 0;
      return;
    }
    G.route = 1;
  }
  G.s = 0;
  done[gid] = 0;
  routes[gid] = G.route == 1 ? 2 : (G.route == 3 ? 3 : 4);
}

}  // namespace

struct rd_batch_split {
  struct Part {
    rd_ctx* h = nullptr;   // stacked handle: nbatch graphs of padded size N
    int32_t* d_gids = nullptr;
  };
  int device = 0;
  double tau = 1e-9;
  std::vector<Part> parts;
  void* digA = nullptr;  // digit planes and exponents shared by the parts (they run in turn)
  void* digB = nullptr;
  int* eA = nullptr;
  int* eB = nullptr;
};

namespace {

void free_part(rd_batch_split::Part& p) {
  if (p.h) {
    rd_split_release(p.h);
    void* ptrs[] = {p.h->dLU, p.h->dT, p.h->dS, p.h->dStatus, p.h->dBatch};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    delete p.h;
  }
  if (p.d_gids) cudaFree(p.d_gids);
  p.h = nullptr;
  p.d_gids = nullptr;
}

}  // namespace

void rd_bsplit_destroy(rd_batch_split* b) {
  if (!b) return;
  for (auto& p : b->parts) free_part(p);
  void* ptrs[] = {b->digA, b->digB, b->eA, b->eB};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete b;
}

rd_status rd_bsplit_create(const int32_t* n, const double* gamma, const int64_t* off, const int32_t* gid,
                           int count, double tau, rd_batch_split** out, std::string* err) {
  *out = nullptr;
  rd_batch_split* b = new rd_batch_split();
  b->tau = tau;
  cudaError_t e = cudaGetDevice(&b->device);
  // stacks: the graphs of each padded size, at most BS_PART per stack
  std::vector<std::vector<int32_t>> by_size(RD_BATCH_MAX_N / RD_PAD + 1);
  for (int q = 0; q < count; ++q) by_size[(n[gid[q]] + RD_PAD - 1) / RD_PAD].push_back(gid[q]);
  size_t dig_max = 0, exp_max = 0;
  for (size_t k = 1; k < by_size.size() && e == cudaSuccess; ++k) {
    const auto& ids = by_size[k];
    for (size_t i0 = 0; i0 < ids.size() && e == cudaSuccess; i0 += BS_PART) {
      const int nb = (int)std::min<size_t>(BS_PART, ids.size() - i0);
      const int N = (int)k * RD_PAD;
      rd_batch_split::Part p;
      p.h = new rd_ctx();
      rd_ctx* h = p.h;
      h->device = b->device;
      h->n = h->N = N;
      h->nbatch = nb;
      h->fp64_node = 128;  // stacked products have tiles enough from 256 rows up
      h->tau = tau;
      h->precision = h->used_precision = RD_PREC_SPLIT_BF16;
      const size_t NN = (size_t)N * N;
      auto get = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
      };
      get((void**)&h->dLU, nb * NN * sizeof(double));
      get((void**)&h->dT, nb * NN * sizeof(double));
      get((void**)&h->dS, nb * (NN / 2) * sizeof(double));
      get((void**)&h->dStatus, 4 * sizeof(int));
      get((void**)&h->dBatch, nb * sizeof(rd_batch_graph));
      get((void**)&p.d_gids, nb * sizeof(int32_t));
      std::vector<rd_batch_graph> hb(nb);
      for (int q = 0; q < nb; ++q) {
        const int g = ids[i0 + q];
        rd_batch_graph& G = hb[q];
        memset(&G, 0, sizeof(G));
        G.gamma = gamma[g];
        G.n = n[g];
        G.off = off[g];
        G.log_gamma = std::log(gamma[g]);
        G.inv_log2_gamma = (float)(1.0 / std::log2(gamma[g]));
        G.screen_bits = -1.0;
      }
      if (e == cudaSuccess) e = cudaMemcpy(h->dBatch, hb.data(), nb * sizeof(rd_batch_graph), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(p.d_gids, ids.data() + i0, nb * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemset(h->dStatus, 0, 4 * sizeof(int));
      size_t dig = 0, ex = 0;
      rd_split_workspace(N, nb, RD_SPLIT_MAX, &dig, &ex);
      dig_max = std::max(dig_max, dig);
      exp_max = std::max(exp_max, ex);
      b->parts.push_back(p);
    }
  }
  auto get = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMalloc(ptr, bytes);
  };
  get(&b->digA, dig_max);
  get(&b->digB, dig_max);
  get((void**)&b->eA, exp_max);
  get((void**)&b->eB, exp_max);
  rd_status st = RD_OK;
  for (auto& p : b->parts)
    if (e == cudaSuccess && st == RD_OK) st = rd_split_prepare_borrowed(p.h, RD_SPLIT_MAX, b->digA, b->digB, b->eA, b->eB);
  if (e != cudaSuccess || st != RD_OK) {
    *err = e != cudaSuccess ? std::string("batched split workspace: ") + cudaGetErrorString(e)
                            : std::string("batched split plan: ") + (b->parts.empty() ? "" : b->parts[0].h->err);
    rd_bsplit_destroy(b);
    return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : (st != RD_OK ? st : RD_ERR_CUDA);
  }
  *out = b;
  return RD_OK;
}

cudaError_t rd_bsplit_run(rd_batch_split* b, const uint8_t* A, int32_t* D, int32_t* status, int32_t* done,
                          int32_t* routes, cudaStream_t s, int64_t* launches) {
  cudaError_t e = cudaSuccess;
  *launches = 0;
  for (auto& p : b->parts) {
    rd_ctx* h = p.h;
    const int64_t l0 = h->launches;
    const int nb = h->nbatch, N = h->N;
    h->stream = s;
    bs_reset_kernel<<<(nb + 127) / 128, 128, 0, s>>>(h->dBatch, nb);
    if ((e = cudaMemsetAsync(h->dStatus, 0, 4 * sizeof(int), s)) != cudaSuccess) return e;
    bs_screen_kernel<<<nb, BS_MAX_N, 0, s>>>(A, h->dBatch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int pass = 1; pass <= 2; ++pass) {
      h->factor_gen++;  // fresh factors: no digits of an earlier pass are reused
      bs_build_kernel<<<dim3((unsigned)(N / 8), (unsigned)nb), BS_THREADS, 0, s>>>(A, h->dLU, N, h->dBatch);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = rd_lu_split(h, s)) != cudaSuccess) return e;
      // Y = U^-1 L^-1 with D decoded into the caller's packed D (graph b at its offset, leading
      // dimension n_b); Y itself into the stack's LU matrices (free after the factorisation)
      if ((e = rd_trmm_decode_split(h, D, h->dLU, s)) != cudaSuccess) return e;
      bs_residual_kernel<<<dim3((unsigned)N, (unsigned)nb), BS_THREADS, 0, s>>>(A, h->dLU, N, h->dBatch);
      bs_finalize_kernel<<<(nb + 127) / 128, 128, 0, s>>>(h->dBatch, nb, p.d_gids, b->tau, pass, status, done,
                                                          routes);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    *launches += (h->launches - l0) + 9;  // the recursion's and the products', and the nine above
  }
  return cudaSuccess;
}

rd_status rd_bsplit_info(rd_batch_split* b, int G, int32_t* digits, int32_t* passes, double* residual,
                         double* screen_bits) {
  for (int g = 0; g < G; ++g) {
    digits[g] = passes[g] = 0;
    residual[g] = 0.0;
    screen_bits[g] = -1.0;
  }
  if (!b) return RD_OK;
  for (auto& p : b->parts) {
    const int nb = p.h->nbatch;
    std::vector<rd_batch_graph> hb(nb);
    std::vector<int32_t> gid(nb);
    if (cudaMemcpy(hb.data(), p.h->dBatch, nb * sizeof(rd_batch_graph), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(gid.data(), p.d_gids, nb * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return RD_ERR_CUDA;
    for (int q = 0; q < nb; ++q) {
      digits[gid[q]] = hb[q].digits;
      passes[gid[q]] = hb[q].passes;
      residual[gid[q]] = hb[q].residual;
      screen_bits[gid[q]] = hb[q].screen_bits;
    }
  }
  return RD_OK;
}
