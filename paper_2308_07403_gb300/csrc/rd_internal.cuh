// rd_internal.cuh -- handle layout and kernel launchers shared by the library's .cu files.
//
// Data layout in HBM (N = n rounded up to RD_PAD):
//   dLU  N x N f64  M, then its packed no-pivot LU factors (strict lower = L, upper = U).
//                   Rows/columns n..N-1 hold an identity block, so every kernel works on
//                   whole tiles and the padding never changes the n x n result.
//   dT   N x N f64  the triangular inverses, packed the same way: strict lower = L^-1
//                   (unit diagonal implied), upper = U^-1.
//   dS   N*N/2 f64  scratch for the off-diagonal products of the blocked triangular inverse.
//   dR   64 x N f64 right-hand sides of the goal solves.
//   dA   n x n u8   the graph (kept for reloads and the successor lists).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rd.h"

#define RD_PAD 128          // padding granule of N (the largest tile edge used)
#define RD_BF 64            // block size of the FP64 factorisation
#define RD_MAX_GOALS 64

// device status codes (first error wins)
#define RD_DEV_OK 0
#define RD_DEV_PIVOT 1      // non-positive or non-finite pivot
#define RD_DEV_NONFINITE 2  // non-finite entry of Y
#define RD_DEV_TIMEOUT 3    // a bounded wait expired
#define RD_DEV_BADGOAL 4    // a goal index in device memory outside [0, n) (detail: its position)
#define RD_SPLIT_START 12   // digit count of an unscreened graph (weighted) when the caller leaves it open
#define RD_SPLIT_MIN 8      // fewest digits the range screen picks
#define RD_SPLIT_MAX 15     // largest digit count in the natural order (exact group sums, 256-wide chunks)
#define RD_SPLIT_MAX_ORDERED 22  // the same in the locality order (64-wide chunks)
#define RD_SPLIT_DIGIT_BITS 7  // bits per digit of the split operands
#define RD_SCREEN_SOURCES 8  // BFS sources of the split path's range screen
#define RD_SCREEN_CHUNK 256  // operand chunk along K that shares one scale (the split path's KAPPA)
#define RD_SCREEN_CHUNK_ORDERED 64  // the same with the locality order
// Bits the digits keep below a chunk's spread (2^-40 ~ 1e-12).  D is exact only while Y's relative
// error stays below tau |ln gamma| (entries gamma^d of single paths sit exactly on the decode's
// integer boundaries): 1.6e-10 at gamma = 0.85.  With 34 bits a directed path at gamma = 0.85
// decoded wrongly (errors up to the self-check's 1e-9) although the six bench graphs, whose gains
// are small, stayed exact at 6 % less step time.
#define RD_SCREEN_RESULT_BITS 40
// Weighted graphs: the operands of the inverse products are path sums restricted to the
// elimination order, and with unequal edge weights those restricted paths can cost more than the
// true shortest paths that the weighted spread samples.  The largest operand-chunk scale over a
// result entry, against the sampled spread, measured 1.05x on a dense random graph with
// log-uniform weights in [1, 100] at gamma = 1e-7 (natural order) and 0.91x on a king-move grid
// with weights in [1, 4] in the locality order.  The screen scales a weighted spread by
// RD_SCREEN_WEIGHTED; a shortfall shows in the self-check's residual, which then sets the next
// digit count.
#define RD_SCREEN_WEIGHTED 1.1

// the split recursion's overlap (rd_ctx::split_overlap): the least N, and the deepest node it serves
#define RD_SIDE_MIN_N 8192
#define RD_SIDE_DEPTH 16

struct rd_split_plan;       // defined by the split path

// One graph of a stacked batch (device array, see rd_ctx::nbatch): the batched split path's
// per-graph parameters and outcome.
struct rd_batch_graph {
  double gamma;          // its gain
  int32_t n;             // nodes (at most the batch's padded size N)
  int32_t s;             // digits of its split products; 0: not on the split path (launches skip it)
  int64_t off;           // element offset of its packed D (n x n, leading dimension n)
  double log_gamma;      // the decode's log(gamma) and 1 / log2(gamma)
  float inv_log2_gamma;
  int32_t status[2];     // RD_DEV_* of this graph and its detail
  int32_t route;         // 0: on the split path; 1: failed the residual check; 2: failed the gain
                         // check; 3: screened out (these three go to the FP64 kernel)
  double residual;       // largest entrywise relative residual of its split Y (the self-check)
  double screen_bits;    // its range screen: chunk spread x log2(1 / gamma)
  int32_t digits;        // the digit count of its kept split result (0: none)
  int32_t passes;        // split passes it took (2: redone with more digits after the check)
};

struct rd_ctx {
  int device = 0;
  // device memory: cudaMalloc / cudaFree, or, for handles of a server, its stream-ordered pool
  // (cudaMallocFromPoolAsync / cudaFreeAsync on the handle's stream: no device-wide synchronisation)
  cudaMemPool_t pool = nullptr;
  int32_t n = 0, N = 0;
  double gamma = 0.0, tau = 1e-9, max_colsum = 0.0;
  int weighted = 0;
  unsigned long long factor_gen = 0;  // counts factorisations: keys reuse of derived data (sliced L^-1)
  int order_ready = 0;  // h->dOrd / h->dPos hold a locality order of the resident graph: 1 landmark, 2 scored
  int precision = RD_PREC_FP64;
  int slices_req = 0, slices = 0;
  cudaStream_t stream = nullptr;

  uint8_t* dA = nullptr;
  float* dW = nullptr;
  double* dLU = nullptr;
  double* dT = nullptr;
  double* dS = nullptr;
  double* dR = nullptr;
  int* dStatus = nullptr;      // [0] code, [1] detail, [2..3] spare
  unsigned long long* dRed = nullptr;  // reductions: [0] max degree, [1] max column sum bits
  int32_t* dDeg = nullptr;     // n+1: out-degree, then exclusive prefix (successor CSR ptr)
  double* dColsum = nullptr;   // n: column sums of X (gain check)
  int32_t* dSucc = nullptr;    // successor CSR indices
  float* dSuccW = nullptr;     // weighted graphs: the weight of each successor edge (same layout)
  int64_t succ_cap = 0;
  int64_t n_edges = 0;         // edges of the current graph (A_ij != 0)
  int succ_ready = 0;
  int32_t* dGoals = nullptr;   // RD_MAX_GOALS
  int32_t* dCheckGoals = nullptr;  // RD_MAX_GOALS: rows of the split path's self-check
  int32_t* dOrd = nullptr;     // n: locality order of the split path, node at each position
  int32_t* dPos = nullptr;     // n: its inverse, position of each node
  int32_t* dNext = nullptr;    // staging for host next-hop output (k x n)
  double* dYrows = nullptr;    // staging for host goal rows (k x n)
  int32_t* dDout = nullptr;    // staging for host D output (n x n), lazy
  double* dYout = nullptr;     // staging for host Y output (n x n), lazy
  double* dYres = nullptr;     // resident Y for incremental edge updates (n x n), lazy
  int y_current = 0;           // dYres holds the current graph's Y
  int updated = 0;             // edges changed since the factorisation: goal rows come from dYres
  int64_t edge_updates = 0, update_refactors = 0;

  int factored = 0;            // dLU holds the factors of the current graph
  int inverted = 0;            // dT holds the triangular inverses
  int used_precision = RD_PREC_FP64;  // precision that produced the current factors
  int split_floor = 0;         // per graph: least digit count to use, -1 = FP64 (self-check history)
  int split_start = 0;         // per graph: digit count picked by the range screen (0: none)
  int screened = 0;            // the range screen ran for the current graph and mode
  double screen_bits = -1.0;   // its estimate of the bits a chunk's spread costs (-1: not screened)
  double screen_per_hop = 1.0; // weight factor of a hop in that estimate (largest W; 1 unweighted)
  int ordered = 0;             // the split path runs on P M P^T with the locality order (dOrd)
  int kappa = 256;             // chunk width of the split digits: 256, or 64 with the locality order
  int split_pairs = 1;         // split GEMM as CTA pairs (tcgen05 cta_group::2) where the rows allow;
                               // 0: one CTA per tile (environment RD_SPLIT_CTA_PAIRS=0 at rd_create)
  int fp64_node = 512;         // recursion nodes of at most this many rows run their products in FP64
  // A stacked batch of nbatch graphs of one padded size N (the batched split path): graph b's
  // matrices start b * N * N doubles into dLU and dT and b * N * N / 2 into dS, and every launch
  // of the factorisation covers all of them (the CTA index or blockIdx.y/z picks the graph).
  // Pointers handed to the launchers are graph 0's; rd_batch_stride maps them to a stride.
  int nbatch = 1;
  rd_batch_graph* dBatch = nullptr;  // device, nbatch entries (nbatch > 1)
  int fallbacks = 0;           // split results redone (more digits or FP64) after the self-check
  double last_residual = 0.0;  // largest sampled-row residual of the last split result

  rd_split_plan* split = nullptr;
  // Overlap in the split recursion (one graph, N >= RD_SIDE_MIN_N): the first product of a node's
  // L-side inverse block, S_L = L21 L11^-1, needs only the left half, so it runs on a side stream of
  // the lowest priority, with its own digit workspace, while the node's right half is factored (whose
  // leaf chain and small FP64 products leave most SMs idle); dSL holds S_L of every depth of the
  // recursion at once.  Environment RD_SPLIT_OVERLAP=0 at rd_create turns it off.
  int split_overlap = 1;
  rd_split_plan* split_side = nullptr;
  cudaStream_t prio = nullptr;  // the recursion's own stream (highest priority), forked from and joined to the caller's
  cudaStream_t side = nullptr;  // the S_L products (lowest priority)
  cudaEvent_t prio_ev[2] = {};
  cudaEvent_t side_ev[2 * RD_SIDE_DEPTH] = {};
  double* dSL = nullptr;

  cudaEvent_t ev[8] = {};
  int ev_used[4] = {0, 0, 0, 0};
  double ms_factor = 0, ms_inverse = 0, ms_goal = 0, ms_greedy = 0;
  int64_t bytes = 0;
  std::string err;

  // launch accounting: every kernel launch of the library bumps `launches`; with profiling on,
  // each launch of the dense-contraction kernels is bracketed by a pair of events and its
  // algorithmic flop count is accumulated.
  int64_t launches = 0;
  int prof_on = 0;
  double prof_split_busy_ms = 0.0;  // union of the split GEMM's profiled launch intervals
  static constexpr int kProfPairs = 4096;
  cudaEvent_t* prof_ev = nullptr;  // 2 * kProfPairs
  int prof_used = 0;
  double prof_ms = 0.0, prof_flops = 0.0;
  int64_t prof_launches = 0;
  double prof_split_ms = 0.0, prof_split_flops = 0.0;  // the split GEMM's share of the above
  int64_t prof_split_launches = 0;
  double prof_update_ms = 0.0, prof_update_bytes = 0.0;  // the rank-1 update passes (HBM bound)
  int64_t prof_update_launches = 0;
  int8_t prof_kind[kProfPairs] = {};           // RD_PROF_* of each pending event pair
  double prof_pair_flops[kProfPairs] = {};
};

// Per-graph element stride of a matrix pointer of graph 0 of a stacked batch (0 for one graph):
// N * N inside dLU or dT, N * N / 2 inside dS.
inline long long rd_batch_stride(const rd_ctx* h, const void* p) {
  if (h->nbatch <= 1 || !p) return 0;
  const long long NN = (long long)h->N * h->N;
  const double* q = static_cast<const double*>(p);
  if ((q >= h->dLU && q < h->dLU + NN) || (q >= h->dT && q < h->dT + NN)) return NN;
  if (q >= h->dS && q < h->dS + NN / 2) return NN / 2;
  return 0;
}

// Device memory of a handle (see rd_ctx::pool); frees are stream-ordered for pooled handles.
cudaError_t rd_dev_alloc(rd_ctx* h, void** p, size_t bytes);
void rd_dev_free(rd_ctx* h, void* p);
// factors and both triangular inverses of the handle's graph resident (dT complete); synchronises
rd_status rd_prepare_inverses(rd_ctx* h);
// rd_create with every allocation of the handle (now and later) from `pool` on `stream`
rd_status rd_create_pooled(const uint8_t* A, int32_t n, double gamma, cudaMemPool_t pool, cudaStream_t stream,
                           rd_handle* out);

// Launch accounting around one kernel launch (see rd_ctx).  `kind` marks the dense GEMM kernels
// whose time and algorithmic flops are profiled (RD_PROF_NONE for every other kernel).
enum { RD_PROF_NONE = 0, RD_PROF_F64 = 1, RD_PROF_SPLIT = 2, RD_PROF_UPDATE = 3 };
cudaError_t rd_prof_begin(rd_ctx* h, cudaStream_t s, int kind);
cudaError_t rd_prof_end(rd_ctx* h, cudaStream_t s, int kind, double flops);
cudaError_t rd_prof_collect(rd_ctx* h);  // fold finished event pairs into prof_ms

// ---- FP64 GEMM (k_gemm_f64.cu) ----------------------------------------------------------
// C = beta*C + alpha * opA(A) * opB(B), all row-major, M, N multiples of 64, K multiple of 16.
// tri modes describe how a diagonal block of the packed triangular storage is read.
enum { RD_TRI_FULL = 0, RD_TRI_LOWER_UNIT = 1, RD_TRI_UPPER = 2 };

struct rd_gemm_f64_args {
  const double* A;
  long long lda;
  int a_tri;
  const double* B;
  long long ldb;
  int b_tri;
  double* C;
  long long ldc;
  int M, N, K;
  double alpha, beta;
  int store_c;           // write C (rows < c_rows, cols < c_cols)
  int c_rows, c_cols;
  // fused R-distance decode of the result (trmm epilogue); D == nullptr disables it
  int32_t* D;
  long long ldd;
  int d_rows, d_cols;
  double log_gamma, tau;
  int* status;
  // C overwrites A's row strip or B's column strip of the same product (beta must be 0): every
  // CTA must then own the whole strip it reads, so the 64 x 64 tile is kept and the aliased
  // extent (N when C aliases A, M when C aliases B) must be 64
  int aliased;
  // stacked batches: per-graph element strides of A, B and C (blockIdx.y is the graph), and the
  // graphs (bg[b].s == 0: no split work in this pass, skipped)
  long long a_gs, b_gs, c_gs;
  const rd_batch_graph* bg;
};

// flops: algorithmic flop count of the launch (for the profile), computed by the caller
cudaError_t rd_gemm_f64(rd_ctx* h, const rd_gemm_f64_args* probs, int nprob, cudaStream_t s,
                        double flops);

// ---- kernels in k_build.cu ----------------------------------------------------------------
cudaError_t rd_build_m(rd_ctx* h, cudaStream_t s);       // M into dLU, degrees, column sums
cudaError_t rd_build_succ(rd_ctx* h, cudaStream_t s);    // successor CSR from dA
// largest spread of the distance from nsrc sampled sources within chunks of `chunk` consecutive
// positions (node at position q: ord[q], or q when ord is null): hop counts (BFS), or weighted
// distances (Bellman-Ford on dSuccW) for a weighted graph; needs the successor lists; dist: nsrc * n
// words of scratch.  atomicMax of the spread's float bits into *out
cudaError_t rd_chunk_spread(rd_ctx* h, int nsrc, int chunk, const int32_t* ord, int32_t* dist,
                            unsigned long long* out, cudaStream_t s);
// locality order for the split path (dOrd, dPos; uses dS as scratch; synchronises once): the
// landmark bisection (scored = 0) or the bisection that scores four keys per part (scored = 1)
cudaError_t rd_locality_order(rd_ctx* h, int scored, cudaStream_t s);
// Collatz-Wielandt bracket [lo, hi] of the spectral radius of X after iters power-iteration steps
cudaError_t rd_spectral(rd_ctx* h, int iters, double* x, double* y, unsigned long long* red, double* lo, double* hi,
                        cudaStream_t s);
// dLU <- P M P^T (the permuted M; dT is used as the staging buffer and swapped in)
cudaError_t rd_permute_m(rd_ctx* h, cudaStream_t s);
cudaError_t rd_copy_rows_out(rd_ctx* h, const double* R, long long ldr, int rows, int cols,
                             double* out, long long ldo, cudaStream_t s);

// ---- FP64 factorisation and inverse (k_lu_f64.cu) --------------------------------------------
cudaError_t rd_lu_f64(rd_ctx* h, cudaStream_t s);
cudaError_t rd_trtri_f64(rd_ctx* h, cudaStream_t s);
cudaError_t rd_lu_diag(rd_ctx* h, int k0, cudaStream_t s);   // diag LU + its inverses
cudaError_t rd_trmm_decode_f64(rd_ctx* h, int32_t* D, double* Y, cudaStream_t s);

// ---- incremental edge updates (k_update.cu) ----------------------------------------------------
// Y <- Y + alpha Y e_i e_j^T Y with D decoded in the same pass; *lost counts cancelled entries
cudaError_t rd_rank1_update(rd_ctx* h, int i, int j, double delta, int32_t* D, unsigned int* lost, cudaStream_t s);
// A_ij (and W_ij), column sum j += delta and out-degree j += ddeg, on the device
cudaError_t rd_set_edge(rd_ctx* h, int i, int j, uint8_t present, float w, double delta, int ddeg,
                        cudaStream_t s);
// rows goals[c] of the resident Y
cudaError_t rd_rows_from_y(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s);

// ---- goals (k_goal.cu) ---------------------------------------------------------------------
cudaError_t rd_goal_f64(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s);
cudaError_t rd_greedy(rd_ctx* h, const int32_t* dgoals, int k, const double* yrows,
                      int32_t* next, cudaStream_t s);
// greedy walks of up to max_len steps from start[c] along the next hops of goal c (k <= 64)
cudaError_t rd_walk(rd_ctx* h, const int32_t* dnext, int k, const int32_t* dstart, int max_len, int32_t* dpath,
                    int32_t* dlen, cudaStream_t s);

// ---- split path (k_split.cu) -----------------------------------------------------------------
rd_status rd_split_prepare(rd_ctx* h, int slices);
void rd_split_release(rd_ctx* h);
// digit-plane bytes (each operand) and exponent bytes of a split plan for nbatch graphs of size N
void rd_split_workspace(int N, int nbatch, int s, size_t* dig_bytes, size_t* exp_bytes);
// a plan whose digit planes and exponents are caller-owned buffers of rd_split_workspace's sizes
rd_status rd_split_prepare_borrowed(rd_ctx* h, int s, void* digA, void* digB, int* eA, int* eB);
cudaError_t rd_lu_split(rd_ctx* h, cudaStream_t s);
cudaError_t rd_trmm_decode_split(rd_ctx* h, int32_t* D, double* Y, cudaStream_t s);
cudaError_t rd_goal_split(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s);
cudaError_t rd_split_row_check(rd_ctx* h, double* worst, cudaStream_t s);
#define RD_SPLIT_RESIDUAL 1e-9  // largest accepted entrywise relative residual of the sampled rows

// ---- the batched split path (k_batch_split.cu) ------------------------------------------------
struct rd_batch_split;
// Plan the split path for the graphs gid[0..count) of a batch (node counts n[], gains gamma[],
// packed offsets off[] of every graph of the batch): stacks of at most 512 graphs of one padded
// size, their workspaces and one shared digit workspace, allocated on the current device.
rd_status rd_bsplit_create(const int32_t* n, const double* gamma, const int64_t* off, const int32_t* gid,
                           int count, double tau, rd_batch_split** out, std::string* err);
// Enqueue a run on stream s: every planned graph's screen, factorisation, product with the decode
// into D, and self-check; done[g] = 1 (device) for graphs whose split result is kept (their
// status[g] set), 0 for graphs the FP64 kernel must redo; routes[g] (device) records why.
cudaError_t rd_bsplit_run(rd_batch_split* b, const uint8_t* A, int32_t* D, int32_t* status, int32_t* done,
                          int32_t* routes, cudaStream_t s, int64_t* launches);
void rd_bsplit_destroy(rd_batch_split* b);
// per graph of the batch (host arrays of G): digits of its kept split result (0: none), split
// passes it took, its last residual and its screen estimate (-1: not screened); synchronous
rd_status rd_bsplit_info(rd_batch_split* b, int G, int32_t* digits, int32_t* passes, double* residual,
                         double* screen_bits);

// ---- the serving runtime's device-resident goal loop (rd_serve_loop.cu) ------------------------
#define RD_LOOP_MAX_N 4096  // the loop's staging rows hold graphs of at most this many nodes
#define RD_LOOP_DEFAULT_N 1024  // goal requests on graphs of at most this many nodes run on the loop
struct rd_serve_loop;
rd_status rd_loop_create(int device, rd_serve_loop** out, std::string* err);
void rd_loop_destroy(rd_serve_loop* L);
// rows of Y for goals[0..k) of a resident graph whose inverses are complete (rd_prepare_inverses),
// computed by the loop; Y: host, k x n.  Blocks until done, at most timeout_ms (RD_ERR_TIMEOUT).
rd_status rd_loop_goals(rd_serve_loop* L, rd_ctx* h, const int32_t* goals, int k, double* Y, double timeout_ms);
// post a request whose descriptor is never marked ready: the loop's bounded wait runs out and it
// reports RD_ERR_TIMEOUT (the loop's failure path)
rd_status rd_loop_unready(rd_serve_loop* L, double timeout_ms);
int64_t rd_loop_requests(rd_serve_loop* L);

// ---- errors of calls without a handle (read back through rd_last_error(NULL)) -----------------
void rd_record_error(const std::string& msg);

// ---- device decode shared by the epilogues -----------------------------------------------------
__device__ __forceinline__ int32_t rd_decode_entry(double y, double log_gamma, double tau) {
  if (!(y > 0.0)) return RD_UNREACHABLE;
  double r = log(y) / log_gamma - tau;
  double c = ceil(r);
  if (c >= 2147483646.0) return RD_UNREACHABLE - 1;
  if (c <= -2147483647.0) return -2147483647;
  return (int32_t)c;
}

// The same decode with an FP32 fast path.  For a normal y = 2^e m (m in [1, 2)),
// R = (e + log2 m) / log2(gamma) is formed in FP32; its error is at most 2e-4 |1/log2 gamma|
// (the FP32 sum e + log2 m, |e| <= 1074, carries 2^-13; log2f and the 23-bit mantissa add
// < 1e-6) plus 2e-6 |R| (the product and the rounded 1/log2 gamma).  When R lies farther than
// that from every integer, its ceiling is the exact one (tau = 1e-9 is far inside the bound);
// otherwise, and for R beyond 2^22 where FP32 holds no fraction, the FP64 formula decides.
__device__ __forceinline__ int32_t rd_decode_entry_fast(double y, float inv_log2_gamma, double log_gamma,
                                                        double tau) {
  const long long b = __double_as_longlong(y);
  if (b > 0) {  // y > 0 (NaN and infinity fail the exponent test below), without the FP64 pipe
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex != 0 && ex != 0x7FF) {
      const float m = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7FFFFF));
      const float r = ((float)(ex - 1023) + log2f(m)) * inv_log2_gamma;
      const float fr = r - floorf(r);
      const float tol = 2e-4f * fabsf(inv_log2_gamma) + 2e-6f * fabsf(r) + 1e-6f;
      if (fabsf(r) < 4194304.f && fr > tol && fr < 1.f - tol) return (int32_t)ceilf(r);
    }
  }
  return rd_decode_entry(y, log_gamma, tau);
}

__device__ __forceinline__ void rd_set_status(int* status, int code, int detail) {
  if (status && atomicCAS(status, 0, code) == 0) status[1] = detail;
}

// A goal read from the caller's device memory: valid when in [0, n); otherwise the status word
// records RD_DEV_BADGOAL with its position c, and the caller's kernel must not index with it.
__device__ __forceinline__ bool rd_goal_ok(int32_t g, int n, int c, int* status) {
  if (g >= 0 && g < n) return true;
  rd_set_status(status, RD_DEV_BADGOAL, c);
  return false;
}
