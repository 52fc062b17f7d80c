/*
 * rd.h -- C ABI of the GB300 R-distance library (librd.so).
 *
 * The library computes the R-distance of Jing & Meister, "A fast algorithm for
 * All-Pairs-Shortest-Paths suitable for neural networks":
 *
 *   Y = (I - gamma A)^-1                         (Sec. 2, eq. Y-defined)
 *   Y = (I - X)^-1, X_ij = gamma^W_ij on edges   (Sec. 3.2, weighted extension)
 *   D_ij = ceil(log_gamma Y_ij)                  (Sec. 2 eq. R-defined; Sec. 4.1 eq.
 *                                                 rounded-distance-function)
 *
 * on one GPU, with every step of the path in the library's own CUDA kernels (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Orientation (Sec. 2, adjacency definition and its footnote): A[i*n + j] != 0 iff there
 *    is a directed edge from node j to node i.  Column j of A lists the successors of j and
 *    the out-degree of j is a column sum.  D[i*n + j] is the distance FROM j TO i.
 *    All matrices are dense, row-major, with leading dimension n.
 *  - Pointers may be host memory (pageable or pinned) or device memory of the handle's
 *    device; the library inspects each pointer.  Device pointers are used in place and the
 *    call is asynchronous on the handle's stream.  Host inputs are copied in; when an output
 *    is host memory the call waits for the stream before returning so the data is valid.
 *    The caller owns every buffer it passes; the library never keeps a caller pointer after
 *    a call returns (rd_create copies A and W).
 *  - The handle owns its device workspace (the packed LU factors, the triangular inverses
 *    and scratch, about 2.5 * 8 * N^2 bytes with N = n rounded up to a multiple of 128).
 *  - Errors found on the host are returned at once and nothing is enqueued.  Errors found on
 *    the device (a non-positive pivot, a non-finite Y) are recorded in a device status word
 *    and returned by the next call that synchronises (rd_sync, or any call with a host
 *    output).
 *  - A handle is not thread-safe; distinct handles are independent.
 *
 * Decode details (readings of the paper, identical in the CPU oracle):
 *  - D_ij = ceil(log(Y_ij)/log(gamma) - tau), tau = 1e-9 unless changed by rd_set_tau.  When
 *    Y_ij is an exact power of gamma (one path and no longer walks) R_ij is an integer and the
 *    snap keeps FP64 rounding from moving the ceil.
 *  - D_ii = 0.  Y_ij <= 0 (unreachable, or below the smallest double: Sec. 5.1, eq.
 *    gamma-precision) gives RD_UNREACHABLE.  A value too large for int32 is clamped to
 *    RD_UNREACHABLE - 1.  Off-diagonal Y_ij >= 1 (near the critical gain, Example 4.1) keeps
 *    the literal ceil, which may be 0 or negative.
 */
#ifndef RD_H_
#define RD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_UNREACHABLE INT32_MAX

typedef struct rd_ctx* rd_handle;

typedef enum {
  RD_OK = 0,
  RD_ERR_ARG = 1,         /* null pointer, n < 1, k out of range, goal index out of range   */
  RD_ERR_GAMMA = 2,       /* gamma not in (0,1), or the largest column sum of X is >= 1      */
  RD_ERR_OOM = 3,         /* a device allocation failed                                     */
  RD_ERR_CUDA = 4,        /* a CUDA runtime call failed (text in rd_last_error)             */
  RD_ERR_NUMERIC = 5,     /* the device saw a non-positive pivot or a non-finite Y          */
  RD_ERR_STATE = 6,       /* call out of order                                              */
  RD_ERR_TIMEOUT = 7,     /* a bounded device-side wait expired                             */
  RD_ERR_UNSUPPORTED = 8  /* mode not available on this device                              */
} rd_status;

/* Precision of the dense inverse. */
enum {
  RD_PREC_FP64 = 0,       /* plain FP64 GEMMs throughout                                    */
  RD_PREC_SPLIT_BF16 = 1  /* big GEMMs as exact BF16 slice products on the tensor cores,    */
                          /* FP64 kept for diagonal blocks, slicing, recombination, decode  */
};

typedef struct {
  int32_t n;              /* graph size                                                      */
  int32_t n_padded;       /* N: n rounded up to the tile size                                */
  int32_t precision;      /* RD_PREC_*                                                       */
  int32_t slices;         /* slice count used by the split path (0 for FP64)                 */
  double gamma;
  double max_column_sum;  /* largest column sum of X (gamma * Delta when unweighted)         */
  double tau;
  double ms_factor;       /* device time of the last LU factorisation                        */
  double ms_inverse;      /* device time of the last triangular inverses + product + decode  */
  double ms_goal;         /* device time of the last goal solve                              */
  double ms_greedy;       /* device time of the last greedy next-hop pass                    */
  int64_t bytes_device;   /* device bytes owned by the handle                                */
  int64_t launches;       /* kernel launches issued by this handle since it was created      */
  int64_t prof_launches;  /* profiled dense-contraction launches (see rd_set_profiling)      */
  double prof_ms;         /* their summed device time (CUDA events on the handle's stream)   */
  double prof_flops;      /* their summed flop count (split path: the issued digit products)  */
  int32_t precision_used; /* precision that produced the current graph's result              */
  int32_t fallbacks;      /* split results this handle redid (more digits or FP64)           */
  double split_residual;  /* largest entrywise relative residual of the sampled rows of the  */
                          /* last split result against M (the self-check; 1e-9 accepted)     */
  double split_screen_bits; /* range screen of the split path (digit count left open,        */
                          /* unweighted graph): largest hop spread of Y within a 256-node   */
                          /* chunk, seen from 8 sampled sources, times log2(1/gamma): the   */
                          /* bits a chunk's common scale costs the digits; -1 if not run    */
  int64_t prof_split_launches; /* the split GEMM's share of the profile: its launches,     */
  double prof_split_ms;   /* device time and issued digit-product flops (the rest of prof_*  */
  double prof_split_flops;/* is the FP64 GEMM)                                               */
  int32_t split_order;    /* 0: the caller's node order; 1 / 2: the split path ran on P M P^T */
                          /* with the library's locality order (compact 64-node parts,      */
                          /* 64-wide chunks) from the landmark bisection (1) or from the     */
                          /* bisection that scores four keys per part (2); D, Y and goal     */
                          /* rows are returned in the caller's node order either way         */
  int64_t edge_updates;   /* edges changed by rd_update_edge since rd_create / rd_load        */
  int64_t update_refactors; /* of those, updates that refactored (cancellation in Y)          */
  int64_t prof_update_launches; /* profiled rank-1 update passes of rd_update_edge, their      */
  double prof_update_ms;  /* summed device time and algorithmic bytes (read and write Y,      */
  double prof_update_bytes; /* write D: 20 n^2 per pass)                                      */
  double prof_split_busy_ms; /* the split GEMM's busy time: the union of its profiled launches' */
                          /* intervals (prof_split_ms sums their durations, which counts twice */
                          /* the time two launches of the recursion's two streams overlap)    */
} rd_stats;

/* Create a handle for the unweighted graph A (n x n bytes) and gain gamma: validates gamma
 * (0 < gamma < 1 and gamma * Delta < 1, Delta the largest out-degree: strict column diagonal
 * dominance of M, which makes the no-pivot LU stable -- the condition of Theorem 4), allocates
 * the workspace on the current device and forms M = I - gamma A (Sec. 2).  Synchronises once
 * (to read Delta).  On success *out receives the handle; on failure *out is NULL. */
rd_status rd_create(const uint8_t* A, int32_t n, double gamma, rd_handle* out);

/* As rd_create for the weighted extension (Sec. 3.2): X_ij = gamma^W_ij where A_ij != 0,
 * W float32 n x n, positive and finite on edges (entries off the edges are ignored).
 * Requires the largest column sum of X to be < 1. */
rd_status rd_create_weighted(const uint8_t* A, const float* W, int32_t n, double gamma,
                             rd_handle* out);

/* Load a new graph of the same n into an existing handle (re-validates gamma, rebuilds M,
 * drops cached factors).  W may be NULL for an unweighted graph.  Synchronises once. */
rd_status rd_load(rd_handle h, const uint8_t* A, const float* W, double gamma);

/* Use the given cudaStream_t (passed as void*) for all later work of this handle. */
rd_status rd_set_stream(rd_handle h, void* stream);

/* Select RD_PREC_FP64 or RD_PREC_SPLIT_BF16.  slices in [2, 15] fixes the digit count (no
 * screen, no self-check, the caller's node order: the caller owns the precision); 0 lets the
 * library choose per graph.  It first screens the graph (a few synchronisations): the digits of
 * each 256-wide chunk of the node order share one scale, so a chunk spanning S hops costs about
 * S log2(1/gamma) bits (for a weighted graph S is a weighted distance, and the estimate is
 * raised by 10%), and the digit count is the fewest (at least 8) whose 7 bits each cover that
 * plus 40 bits of result.  When the node order needs more than 12, it also screens its locality
 * order (compact 64-node parts, 64-wide chunks: rd_stats.split_order) and takes it when it needs
 * fewer; beyond 15 digits (22 in the locality order) the graph runs in FP64
 * (rd_stats.split_screen_bits, rd_stats.slices).  It then checks every split factorisation,
 * before any product uses it: 64 sampled rows of Y must satisfy y^T M = e_g^T to a relative
 * min(1e-9, tau |ln gamma| / 16) per entry, at least 1e-12 (rd_stats.split_residual; D is exact
 * while Y's relative error stays below tau |ln gamma|).  When the check fails it recomputes the graph's inverse with
 * the digits the residual r asks for (about log2(r / 2^-40) / 7 more), or in FP64 beyond the
 * order's limit.  Drops cached factors when the mode changes.
 * For a handle with N >= 8192 (N: n rounded up to 128) the split factorisation overlaps two of
 * each recursion node's products (S_L = L21 L11^-1 and V = U11^-1 U12, the U side's inverse block
 * then formed as -V U22^-1) with the factorisation of the node's right half, on two streams the
 * handle creates (the highest and the lowest priority), forked from and joined back to the
 * handle's stream with events: the caller still sees one ordered stream.  It takes about
 * 2 s (N/2)^2 BF16 digits and 2 N^2 / 3 doubles more device memory (s digits); the environment
 * variable RD_SPLIT_OVERLAP=0 at rd_create turns it off (one stream; the U side's block then
 * -U11^-1 (U12 U22^-1)). */
rd_status rd_set_precision(rd_handle h, int32_t mode, int32_t slices);

/* Change the decode snap tau (>= 0, < 0.5).  The split path's self-check limit follows tau at
 * the time of the factorisation; factors made under a larger tau are not re-checked (a change
 * of precision mode, or rd_load, refactors). */
rd_status rd_set_tau(rd_handle h, double tau);

/* All-pairs R-distance: D (n*n int32, row-major, D[i*n+j] = distance j -> i).  If Y is not
 * NULL it also receives Y (n*n float64).  Factors M on first use and keeps the factors for
 * rd_goal_solve.  In RD_PREC_SPLIT_BF16 with the digit count left to the library, the call
 * reads the self-check flags (one synchronisation after the factorisation and one after the
 * product) and recomputes with more digits or in FP64 when they fire; rd_stats.slices,
 * precision_used and fallbacks report what was used. */
rd_status rd_apsp(rd_handle h, int32_t* D, double* Y);

/* Bracket of the spectral radius of X = gamma A (or gamma^W): after `iters` (1..1e6) steps of
 * power iteration on X^T + I over the graph's successor lists, *lo and *hi receive the
 * Collatz-Wielandt bounds min_j and max_j of (B x)_j / x_j - 1, B = X^T + I, x > 0, which
 * enclose rho(X) for every non-negative X and close in on it for a strongly connected graph.
 * Theorem 1: the walk series sum gamma^k A^k (Sec. 3.1) converges, and Y = M^-1 is its sum, iff
 * rho(X) < 1; the gain check of rd_create (largest column sum of X < 1, Theorem 4's condition) is
 * the sufficient bound the factorisation needs.  Synchronises once.  RD_ERR_UNSUPPORTED for
 * graphs of more than 2^31 edges. */
rd_status rd_spectral_radius(rd_handle h, int32_t iters, double* lo, double* hi);

/* Goal rows (the local mode of Sec. 4.2): for each goal g = goals[c], 0 <= c < k, writes row
 * g of Y, Y_out[c*n + j] = Y_{g j} (the signal from j at the goal), by solving M^T y = e_g on
 * the resident LU factors (factoring first if needed).  1 <= k <= 64; goals in [0, n).  Host goals
 * outside [0, n) return RD_ERR_ARG at once; device goals are checked by the kernels that read them:
 * a goal outside [0, n) is never used as an index (its row of Y_out is left zero) and the next
 * synchronising call (rd_sync, or any call with a host output) returns RD_ERR_ARG. */
rd_status rd_goal_solve(rd_handle h, const int32_t* goals, int32_t k, double* Y_out);

/* Greedy next hop (Sec. 4.2, eq. descent, as ascent on Y per Theorem 4's proof): for goal
 * g = goals[c] and node i, next[c*n + i] = g if i == g or g is a successor of i; otherwise
 * the successor j of i (edge i -> j) with the largest Yrows[c*n + j], smallest j among equal
 * values; -1 if i has no successor.  Yrows is the output of rd_goal_solve for the same goals
 * (k x n).  Goals are checked as in rd_goal_solve (a device goal outside [0, n) gets next hops -1
 * and RD_ERR_ARG from the next synchronising call). */
rd_status rd_greedy_next(rd_handle h, const int32_t* goals, int32_t k, const double* Yrows,
                         int32_t* next);

/* Greedy walks (Sec. 4.2, the local navigation): for c < k, from start[c] follow next (k x n,
 * the output of rd_greedy_next for the same goals) until a node is its own next hop (the goal), a
 * node has none, or max_len (0..n) steps.  path (k x (max_len + 1)) receives the nodes visited,
 * start first, -1 past the end; len[c] the steps to the goal, or -1 if the walk did not reach it.
 * Buffers on the device or the host (host outputs synchronise). */
rd_status rd_greedy_walk(rd_handle h, const int32_t* next, int32_t k, const int32_t* start, int32_t max_len,
                         int32_t* path, int32_t* len);

/* Incremental edge update (the paper's map update when an obstacle appears, Sec. 6): the edge
 * j -> i becomes present (weight w for a weighted handle; ignored otherwise) or absent, and D
 * (n x n) -- and Y when not NULL -- receive the R-distance of the changed graph.  X_ij changes by
 * delta, M by -delta e_i e_j^T, and the handle's resident Y (materialised once from the factors,
 * n x n FP64) by the Sherman-Morrison rank-1 term alpha (Y e_i)(e_j^T Y), alpha = delta /
 * (1 - delta Y_ji), in one O(n^2) pass that also decodes D.  Added or strengthened edges add terms
 * of one sign; when a removal cancels an entry (more than 20 bits of it lost) the library factors
 * the changed graph from scratch instead (rd_stats.update_refactors).  RD_ERR_GAMMA when the
 * change would make column j's sum of X reach 1 (nothing changes).  Later goal solves read the
 * resident Y.  Synchronises. */
rd_status rd_update_edge(rd_handle h, int32_t i, int32_t j, int32_t present, float w, int32_t* D, double* Y);

/* Turn the per-kernel profile on (1: every dense-contraction kernel; 2: the split GEMM alone) or
 * off (0); either way its counters restart at zero (another value: RD_ERR_ARG).  With the profile
 * on, every launch of the profiled kernels is bracketed by a pair of CUDA events on the handle's
 * stream and its algorithmic flop count is accumulated; rd_get_stats reports the totals
 * (prof_launches, prof_ms, prof_flops, and the split GEMM's prof_split_*).  Mode 2 leaves the
 * small FP64 products of the split path's recursion without events. */
rd_status rd_set_profiling(rd_handle h, int32_t on);

/* Wait for the handle's stream and return the device status (RD_OK or RD_ERR_NUMERIC). */
rd_status rd_sync(rd_handle h);

/* Copy the handle's statistics (synchronises). */
rd_status rd_get_stats(rd_handle h, rd_stats* s);

/* Text of the last error on this handle (or, when h is NULL, of the last failed call made
 * without a handle: rd_create, rd_create_weighted, rd_apsp_noalloc).  Valid until the next
 * call on the handle. */
const char* rd_last_error(rd_handle h);

/* Name of a status code. */
const char* rd_status_string(rd_status s);

/* Free the handle and its device memory (synchronises its stream).  NULL is ignored. */
void rd_destroy(rd_handle h);

/* The tensor-core rate of the split path's digit products on the current device, with nothing else
 * in the loop (the ceiling the split GEMM is held against; no counterpart in the paper): one CTA
 * per SM issues 128 x 128 x 16 tcgen05 MMAs (kind 0: BF16 inputs, FP32 accumulation) from shared
 * memory back to back, `batches` x 64 per SM; *tera_ops receives the rate (10^12 flop/s) and
 * *seconds the device time.  Kind 1 (signed 8-bit digits, tcgen05.mma.kind::i8) returns
 * RD_ERR_UNSUPPORTED: the instruction does not exist for sm_103a.  Every wait is bounded
 * (RD_ERR_TIMEOUT).  Synchronises the device. */
rd_status rd_probe_mma(int32_t kind, int32_t batches, double* tera_ops, double* seconds);

/* Number of counters rd_split_stats can return. */
#define RD_SPLIT_STATS_N 13

/* Where the split GEMM's time goes (a diagnostic; no counterpart in the paper).  A library built with
 * the RD_SPLIT_STATS option (build(stats=True)) sums clock cycles of the kernel's roles over every
 * launch that carries the fused decode (the inverse product Y = U^-1 L^-1); the first n (1..13)
 * counters are copied to out (host memory) and, if reset is non-zero, set to zero:
 *   0 MMA-warp cycles, of which 1 waiting for a free accumulator buffer, 2 waiting for a full
 *   operand stage, 3 issuing (from a stage's arrival to its commit);
 *   4 producer-warp cycles, of which 5 waiting for a free stage;
 *   6 epilogue cycles (one warp per CTA), of which 7 waiting for a group sum, 8 in the per-chunk
 *   renormalisation;
 *   9 MMA warps counted, 10 epilogue warps counted, 11 digit groups, 12 MMA instructions issued
 *   (for a CTA pair, its leader's MMA and producer warps only).
 * The counters cost the kernel registers and a few percent of its speed, so the default build has
 * none: there the call returns RD_ERR_UNSUPPORTED.  Synchronises the device. */
rd_status rd_split_stats(uint64_t* out, int32_t n, int32_t reset);

/* Largest n accepted by rd_apsp_noalloc. */
#define RD_NOALLOC_MAX_N 512

/* All-pairs R-distance (the same FP64 kernels and result as rd_create + rd_apsp) for callers
 * that must not allocate device memory: for example a host program whose device memory is
 * handed out up front by another runtime or framework, or code that runs inside another
 * system's time-critical loop, where cudaMalloc is not allowed or its implicit device
 * synchronisation is not acceptable.  The paper has no counterpart; this is a deployment
 * variant of the library.
 *
 * No handle and no allocation: the workspace is a fixed array in device memory that the
 * library declares at file scope (about 5.3 MB, sized for n <= RD_NOALLOC_MAX_N); every GPU
 * that loads the library holds it until the process exits.  A (n x n bytes) and D (n x n
 * int32) must be device memory of the current device, owned by the caller; the work runs on
 * `stream` (a cudaStream_t, NULL for the default stream) and the call waits for it.
 * n > RD_NOALLOC_MAX_N returns RD_ERR_ARG without touching the GPU.  Every call looks up the
 * array's device address on the current device (cudaGetSymbolAddress, which allocates nothing,
 * so a context that was reset and made again is followed); the first call on a device also loads
 * the library's module there, so make that first call before any stream capture.  All calls
 * share the one array: each call resets what must start at zero and overwrites the rest, and calls whose
 * GPU work overlaps (other threads, other streams) race on it and must be serialised by the
 * caller.  Errors are readable with rd_last_error(NULL). */
rd_status rd_apsp_noalloc(const uint8_t* A, int32_t n, double gamma, int32_t* D, void* stream);

/* ---- Batched graphs (many small independent problems in one launch) -------------------------
 * The whole method (M = I - gamma A, Y = M^-1, D = ceil(log_gamma Y - tau) with D_ii = 0, the
 * sentinel for Y <= 0; Sec. 2 and Sec. 4.1) for G independent graphs of at most RD_BATCH_MAX_N
 * nodes each, in FP64, in one persistent kernel launch: each CTA takes the next graph (largest
 * first) from a queue and inverts its M by blocked Gauss-Jordan elimination without pivoting.  The
 * paper treats one graph at a time; batching is a deployment variant of the same computation. */
#define RD_BATCH_MAX_N 512

typedef struct rd_batch* rd_batch_handle;

/* Plan a batch: n (G node counts, each in [1, RD_BATCH_MAX_N]) and gamma (G gains) are host
 * arrays; graph g's adjacency matrix (n_g x n_g bytes, A[i*n_g+j] != 0 iff edge j -> i) and its D
 * (n_g x n_g int32, D[i*n_g+j] = distance j -> i) are packed at element offset off[g] of the
 * caller's buffers, off[0] = 0, off[g+1] = off[g] + n_g^2 (rd_batch_offsets).  Allocates the FP64
 * workspace (8 sum n_g^2 bytes) on the current device.  Synchronises. */
rd_status rd_batch_create(const int32_t* n, const double* gamma, int32_t G, rd_batch_handle* out);

/* The G + 1 packing offsets (host array). */
rd_status rd_batch_offsets(rd_batch_handle b, int64_t* off);

/* Run the batch: A (packed uint8) and D (packed int32) are device memory of the batch's device; the
 * work is one memset and one kernel launch on `stream` (a cudaStream_t; NULL = default stream),
 * asynchronous and capturable in a CUDA graph.  Per-graph outcomes: rd_batch_status. */
rd_status rd_batch_apsp(rd_batch_handle b, const uint8_t* A, int32_t* D, void* stream);

/* Per-graph status of the last run (host array of G): RD_OK, RD_ERR_GAMMA (gamma outside (0,1) or
 * a column sum of gamma A >= 1: not computed, D untouched), RD_ERR_NUMERIC (non-positive pivot or
 * non-finite Y).  Synchronises the device. */
rd_status rd_batch_status(rd_batch_handle b, int32_t* status);

/* Free a batch (NULL is ignored). */
void rd_batch_destroy(rd_batch_handle b);

/* Size classes of a batch: n in (128 c, 128 (c + 1)], c = 0..RD_BATCH_CLASSES-1. */
#define RD_BATCH_CLASSES 4

/* Precision of a batch's inverses.  RD_PREC_FP64 (the default): every graph by the FP64
 * Gauss-Jordan kernel above.  RD_PREC_SPLIT_BF16: the graphs of chosen size classes run the split
 * path (the single-graph method's recursive LU and triangular inverses with exact BF16 digit
 * products on the tensor cores, FP64 leaves and decode) with graphs of one class stacked, so that
 * every launch covers all of them; per graph, on the device, a range screen (BFS from 8 sources,
 * as rd_set_precision's) picks the digit count and a residual check of every entry of M Y - I
 * (the single-graph self-check's limit) keeps the result, and graphs that fail either (or fail the
 * gain check) are redone by the FP64 kernel in the same run.  A run stays one fixed sequence of
 * launches on the stream (no host synchronisation: capturable in a CUDA graph).  With autotune = 1
 * each size class runs on the split path only when it measured faster there, by timing both
 * variants on up to 152 seeded random graphs of the class's sizes (directed ER, p = 4/n); with 0
 * every class with graphs runs on the split path.  Allocates the split workspace (for up to 512
 * graphs of one class per stack, about 2 * 15 * 2 * N (N + 256) bytes of digit planes per graph of
 * the largest stack, shared by the stacks) and synchronises.  Extends the paper's method to many
 * graphs at once (no counterpart in the paper). */
rd_status rd_batch_set_precision(rd_batch_handle b, int32_t mode, int32_t autotune);

/* Per-graph route of the last run (host array of G): 0 FP64 kernel (its class is not on the split
 * path), 1 split path, 2 split path failed the residual check and was redone in FP64, 3 screened
 * off the split path (more than 15 digits, or too many edges to screen) and computed in FP64,
 * 4 failed the gain check (status RD_ERR_GAMMA).  Synchronises the device. */
rd_status rd_batch_routes(rd_batch_handle b, int32_t* routes);

/* Per graph of the split variant's last run (host arrays of G): the digit count of its kept split
 * result (0: not kept), the split passes it took (2: redone with more digits after the residual
 * check), its last residual, and its range-screen estimate in bits (-1: not screened).
 * Synchronises the device. */
rd_status rd_batch_split_info(rd_batch_handle b, int32_t* digits, int32_t* passes, double* residual,
                              double* screen_bits);

/* The autotuner's record per size class (host arrays of RD_BATCH_CLASSES): graphs of the batch in
 * the class, 1 if the class runs on the split path, and the measured device ms per graph of the
 * FP64 and split variants on the probe graphs (0 when not measured); *launches receives the kernel
 * launches of the last rd_batch_apsp. */
rd_status rd_batch_tuning(rd_batch_handle b, int32_t* graphs, int32_t* split, double* ms_fp64, double* ms_split,
                          int64_t* launches);

/* ---- Serving (continuous batching of requests over resident graphs) --------------------------
 * A server runs requests -- the full R-distance of a graph, or goal rows (the local mode of
 * Sec. 4.2) -- on `workers` threads, each with its own CUDA stream, one request per worker at a
 * time, so requests that arrive while others run start as soon as a worker and device memory are
 * free and their work overlaps on the device.  Goal requests on graphs of at most 1024 nodes run on
 * a device-resident loop: a persistent kernel (38 CTAs, while requests flow; every wait bounded)
 * takes request descriptors from a ring in mapped host memory and computes the rows of Y from the
 * graph's resident triangular inverses (row g of U^-1 times L^-1, FP64), so no kernel is launched
 * per request; larger goal requests run on the tensor-core path through the worker's stream.  Each graph's handle (its LU factors and inverses)
 * stays resident under the caller's graph id, so later goal solves on the same graph skip the
 * factorisation; when a new handle does not fit the device-memory budget, the least recently used
 * idle graphs are evicted.  Requests for one graph run one after another (a handle is not
 * thread-safe).  Latency is measured from submit to completion.  The paper has no counterpart;
 * this is a deployment layer over rd_create / rd_apsp / rd_goal_solve. */
enum { RD_REQ_APSP = 0, RD_REQ_GOALS = 1 };

typedef struct {
  int32_t kind;          /* RD_REQ_APSP or RD_REQ_GOALS                                        */
  int32_t graph_id;      /* caller's graph id: requests with one id share the resident factors */
                         /* (and must carry the same graph); < 0: not kept                     */
  const uint8_t* A;      /* host, n x n (copied at submit)                                      */
  int32_t n;
  double gamma;
  const int32_t* goals;  /* RD_REQ_GOALS: host, k goals (copied at submit)                      */
  int32_t k;             /* 1..64                                                               */
  int32_t precision;     /* RD_PREC_FP64 or RD_PREC_SPLIT_BF16 (digits chosen by the library)  */
  int32_t* D_out;        /* RD_REQ_APSP: host n x n, valid when the request completes           */
  double* Y_out;         /* RD_REQ_GOALS: host k x n, valid when the request completes          */
} rd_request;

typedef struct {
  int64_t completed, failed, queued;
  int32_t resident_graphs, max_inflight;
  int64_t bytes_used, evictions, reused;
  double p50_ms, p99_ms;  /* submit-to-completion latency over all completed requests           */
  double seconds;         /* since rd_serve_create                                              */
  int64_t launches;       /* kernel launches of all requests so far (not counting the loop)      */
  int64_t loop_requests;  /* goal requests served by the device-resident loop                    */
} rd_serve_report;

typedef struct rd_server* rd_server_handle;

/* Start a server on the current device with a device-memory budget (bytes) and 1..64 workers.
 * The server's handles allocate from one stream-ordered memory pool of the device (created here,
 * keeping up to the budget mapped between requests), so admitting a graph or evicting one never
 * synchronises the device. */
rd_status rd_serve_create(int64_t hbm_budget_bytes, int32_t workers, rd_server_handle* out);
/* Queue a request (its inputs are copied); *id identifies it for poll and wait.  RD_ERR_OOM when
 * the request's estimated device footprint (its handle's workspace, the split digit planes in
 * split precision, and staging for host outputs) exceeds the whole budget: such a request could
 * never be admitted.  Requests that fit wait for memory while other requests run. */
rd_status rd_serve_submit(rd_server_handle s, const rd_request* r, int64_t* id);
/* *done = 1 once the request completed (its outputs are valid). */
rd_status rd_serve_poll(rd_server_handle s, int64_t id, int32_t* done);
/* Block until the request completed; its status and latency (ms) are returned and the id is
 * released. */
rd_status rd_serve_wait(rd_server_handle s, int64_t id, rd_status* result, double* latency_ms);
/* As rd_serve_wait, but wait at most timeout_ms (host wall clock; < 0: no limit).  Returns
 * RD_ERR_TIMEOUT, with the request still running and its id still valid, when the time runs out. */
rd_status rd_serve_wait_for(rd_server_handle s, int64_t id, double timeout_ms, rd_status* result,
                            double* latency_ms);
rd_status rd_serve_stats(rd_server_handle s, rd_serve_report* out);
/* The failure path of the device-resident goal loop: posts a request to the loop whose descriptor is
 * never marked ready, so that the loop's bounded wait for it (0.2 s per work unit) runs out;
 * *result receives what the loop reported: RD_ERR_TIMEOUT when the wait ran out and the loop
 * recovered (it goes on serving), RD_ERR_STATE if it never reported.  A check for tests; it holds
 * one ring slot for about half a second. */
rd_status rd_serve_loop_check(rd_server_handle s, rd_status* result);
/* Finish the queued requests, then free every resident graph and the server. */
void rd_serve_destroy(rd_server_handle s);

#ifdef __cplusplus
}
#endif

#endif /* RD_H_ */
