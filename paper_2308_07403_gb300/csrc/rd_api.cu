// rd_api.cu -- the C ABI declared in include/rd.h: handles, argument checks, host/device
// pointer handling, and the order of the kernels of the path.
//
// Path of rd_apsp (all on the handle's stream, no host synchronisation unless an output is
// host memory):
//   rd_load:  copy A (and W) -> build M = I - X, degrees and column sums -> gain check (one
//             synchronisation to read the largest column sum)
//   factor:   blocked no-pivot LU of M (FP64, or split BF16 products on the tensor cores)
//   inverse:  blocked triangular inverses L^-1, U^-1
//   product:  Y = U^-1 L^-1 with D = ceil(log_gamma Y - tau) fused into the epilogue
#include <algorithm>
#include <utility>
#include <vector>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "rd_internal.cuh"

namespace {

thread_local std::string g_create_err;

}  // namespace

cudaError_t rd_dev_alloc(rd_ctx* h, void** p, size_t bytes) {
  if (h->pool) return cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream);
  return cudaMalloc(p, bytes);
}

void rd_dev_free(rd_ctx* h, void* p) {
  if (h->pool)
    cudaFreeAsync(p, h->stream);  // after the handle's work enqueued so far
  else
    cudaFree(p);
}

namespace {

rd_status fail(rd_ctx* h, rd_status st, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_err = msg;
  return st;
}

rd_status fail_cuda(rd_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA, m);
}

#define RD_CK(h, call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return fail_cuda((h), _e, #call); \
  } while (0)

// true when p is device (or managed) memory usable by the handle's device
bool is_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

bool is_foreign_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device != device;
}

template <class T>
cudaError_t dalloc(rd_ctx* h, T** p, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  cudaError_t e = rd_dev_alloc(h, (void**)p, bytes);
  if (e == cudaSuccess) h->bytes += (int64_t)bytes;
  return e;
}

void free_all(rd_ctx* h) {
  rd_split_release(h);
  if (h->prof_ev) {
    for (int i = 0; i < 2 * rd_ctx::kProfPairs; ++i)
      if (h->prof_ev[i]) cudaEventDestroy(h->prof_ev[i]);
    delete[] h->prof_ev;
    h->prof_ev = nullptr;
  }
  void* ptrs[] = {h->dA, h->dW, h->dLU, h->dT, h->dS, h->dR, h->dStatus, h->dRed, h->dDeg, h->dColsum,
                  h->dSucc, h->dGoals, h->dNext, h->dYrows, h->dDout, h->dYout, h->dOrd, h->dPos, h->dCheckGoals, h->dYres, h->dSuccW};
  for (void* p : ptrs)
    if (p) rd_dev_free(h, p);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
}

rd_status check_device_status(rd_ctx* h) {
  int st[2] = {0, 0};
  RD_CK(h, cudaMemcpyAsync(st, h->dStatus, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  RD_CK(h, cudaStreamSynchronize(h->stream));
  if (st[0] == RD_DEV_OK) return RD_OK;
  char buf[160];
  if (st[0] == RD_DEV_PIVOT) {
    snprintf(buf, sizeof buf, "non-positive pivot at row %d (gain too large for a no-pivot LU)", st[1]);
    return fail(h, RD_ERR_NUMERIC, buf);
  }
  if (st[0] == RD_DEV_NONFINITE) {
    snprintf(buf, sizeof buf, "non-finite entry of Y in row %d", st[1]);
    return fail(h, RD_ERR_NUMERIC, buf);
  }
  if (st[0] == RD_DEV_TIMEOUT) return fail(h, RD_ERR_TIMEOUT, "a bounded device wait expired");
  if (st[0] == RD_DEV_BADGOAL) {
    // reported once: the factors are intact and the handle stays usable
    snprintf(buf, sizeof buf, "goal index out of range at position %d of the device goal array", st[1]);
    RD_CK(h, cudaMemsetAsync(h->dStatus, 0, 2 * sizeof(int), h->stream));
    return fail(h, RD_ERR_ARG, buf);
  }
  snprintf(buf, sizeof buf, "device status %d (detail %d)", st[0], st[1]);
  return fail(h, RD_ERR_ARG, buf);
}

// successor lists (and, for a weighted graph, their edge weights) for `edges` edges
rd_status ensure_succ_capacity(rd_ctx* h, int64_t edges) {
  const bool need_w = h->weighted && !h->dSuccW;
  if (h->dSucc && edges <= h->succ_cap && !need_w) return RD_OK;  // (a graph without edges still gets lists)
  const int64_t cap = edges > h->succ_cap ? edges + edges / 8 + 1024 : h->succ_cap;
  if (h->dSucc) rd_dev_free(h, h->dSucc);
  if (h->dSuccW) rd_dev_free(h, h->dSuccW);
  h->bytes -= h->succ_cap * (int64_t)(sizeof(int32_t) + sizeof(float));
  h->dSucc = nullptr;
  h->dSuccW = nullptr;
  h->succ_cap = 0;
  h->succ_ready = 0;
  if (cap > 2147483647ll) return RD_OK;  // no successor lists: the screen and the self-check step aside
  RD_CK(h, dalloc(h, &h->dSucc, (size_t)cap));
  RD_CK(h, dalloc(h, &h->dSuccW, (size_t)cap));
  h->succ_cap = cap;
  return RD_OK;
}

rd_status load_impl(rd_ctx* h, const uint8_t* A, const float* W, double gamma) {
  if (!A) return fail(h, RD_ERR_ARG, "A is NULL");
  if (!(gamma > 0.0 && gamma < 1.0) || !std::isfinite(gamma))
    return fail(h, RD_ERR_GAMMA, "gamma must lie in (0, 1)");
  if (is_foreign_device_ptr(A, h->device) || (W && is_foreign_device_ptr(W, h->device)))
    return fail(h, RD_ERR_ARG, "input lives on another device");
  const size_t nn = (size_t)h->n * (size_t)h->n;
  RD_CK(h, cudaSetDevice(h->device));
  RD_CK(h, cudaMemcpyAsync(h->dA, A, nn, cudaMemcpyDefault, h->stream));
  h->weighted = W != nullptr;
  if (W) {
    if (!h->dW) RD_CK(h, dalloc(h, &h->dW, nn));
    RD_CK(h, cudaMemcpyAsync(h->dW, W, nn * sizeof(float), cudaMemcpyDefault, h->stream));
  }
  h->gamma = gamma;
  h->factored = h->inverted = 0;
  h->split_floor = 0;
  h->split_start = 0;
  h->screened = 0;
  h->order_ready = 0;
  h->screen_bits = -1.0;
  h->ordered = 0;
  h->kappa = RD_SCREEN_CHUNK;
  h->succ_ready = 0;
  h->y_current = h->updated = 0;
  RD_CK(h, cudaMemsetAsync(h->dStatus, 0, 4 * sizeof(int), h->stream));
  RD_CK(h, rd_build_m(h, h->stream));
  unsigned long long red[3];
  RD_CK(h, cudaMemcpyAsync(red, h->dRed, sizeof(red), cudaMemcpyDeviceToHost, h->stream));
  RD_CK(h, cudaStreamSynchronize(h->stream));
  h->n_edges = (int64_t)red[2];
  const rd_status st = ensure_succ_capacity(h, h->n_edges);
  if (st != RD_OK) return st;
  const double delta = (double)red[0];
  double colsum;
  memcpy(&colsum, &red[1], sizeof(double));
  if (!h->weighted) colsum = gamma * delta;
  h->max_colsum = colsum;
  if (!(colsum < 1.0) || !std::isfinite(colsum)) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "largest column sum of X is %.17g >= 1 (gamma * Delta with Delta = %.0f): M is not "
             "strictly column diagonally dominant",
             colsum, delta);
    return fail(h, RD_ERR_GAMMA, buf);
  }
  return RD_OK;
}

rd_status create_impl(const uint8_t* A, const float* W, int32_t n, double gamma, rd_handle* out,
                      cudaMemPool_t pool = nullptr, cudaStream_t stream = nullptr) {
  if (!out) return fail(nullptr, RD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!A) return fail(nullptr, RD_ERR_ARG, "A is NULL");
  if (n < 1) return fail(nullptr, RD_ERR_ARG, "n must be >= 1");
  if (n > 65536) return fail(nullptr, RD_ERR_ARG, "n must be <= 65536");
  if (!(gamma > 0.0 && gamma < 1.0) || !std::isfinite(gamma))
    return fail(nullptr, RD_ERR_GAMMA, "gamma must lie in (0, 1)");
  rd_ctx* h = new rd_ctx();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    delete h;
    return fail_cuda(nullptr, e, "cudaGetDevice");
  }
  h->device = dev;
  {
    const char* pairs = getenv("RD_SPLIT_CTA_PAIRS");
    h->split_pairs = (pairs && pairs[0] == '0') ? 0 : 1;
    const char* overlap = getenv("RD_SPLIT_OVERLAP");
    h->split_overlap = (overlap && overlap[0] == '0') ? 0 : 1;
  }
  h->pool = pool;
  h->stream = stream;
  h->n = n;
  h->N = (n + RD_PAD - 1) / RD_PAD * RD_PAD;
  const size_t N = (size_t)h->N;
  const size_t nn = (size_t)n * (size_t)n;
  rd_status st = RD_OK;
#define RD_ALLOC(ptr, cnt)                                  \
  if (st == RD_OK) {                                        \
    cudaError_t _e = dalloc(h, &(ptr), (cnt));              \
    if (_e != cudaSuccess) st = fail_cuda(h, _e, "cudaMalloc " #ptr); \
  }
  RD_ALLOC(h->dA, nn);
  RD_ALLOC(h->dLU, N * N);
  RD_ALLOC(h->dT, N * N);
  RD_ALLOC(h->dS, N * N / 2);
  RD_ALLOC(h->dR, (size_t)RD_MAX_GOALS * N);
  RD_ALLOC(h->dStatus, 4);
  RD_ALLOC(h->dRed, 3);
  RD_ALLOC(h->dDeg, 2 * (size_t)n + 2);
  RD_ALLOC(h->dColsum, (size_t)n);
  RD_ALLOC(h->dGoals, RD_MAX_GOALS);
  RD_ALLOC(h->dCheckGoals, RD_MAX_GOALS);
  RD_ALLOC(h->dOrd, (size_t)n);
  RD_ALLOC(h->dPos, (size_t)n);
#undef RD_ALLOC
  for (auto& ev : h->ev)
    if (st == RD_OK) {
      cudaError_t e2 = cudaEventCreate(&ev);
      if (e2 != cudaSuccess) st = fail_cuda(h, e2, "cudaEventCreate");
    }
  if (st == RD_OK) st = load_impl(h, A, W, gamma);
  if (st != RD_OK) {
    g_create_err = h->err;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return RD_OK;
}

// Split mode with the self-check: after the factorisation, 64 sampled rows of Y (computed with
// the same digit products) must satisfy y^T M = e_g^T to residual_limit(h) per entry.  When the
// caller leaves the digit count open, the library starts where the range screen says; a failed
// check sets the next count from the residual (escalate) or moves the graph to FP64, and the
// inverse is recomputed from M.
bool split_auto(const rd_ctx* h) { return h->precision == RD_PREC_SPLIT_BF16 && h->slices_req == 0; }

// The sampled-row residual a split result must meet.  D is exact while Y's relative error stays
// below tau |ln gamma| (the decode snaps within tau of an integer, and single-path entries gamma^d
// sit exactly on integers): the limit is that over 16, at most RD_SPLIT_RESIDUAL and at least
// 1e-12 (tau = 0 asks for no snap at all).
double residual_limit(const rd_ctx* h) {
  const double lim = h->tau * std::fabs(std::log(h->gamma)) / 16.0;
  return std::min(RD_SPLIT_RESIDUAL, std::max(lim, 1e-12));
}

double choose_locality_order(rd_ctx* h, double wf, rd_status* st);

// Each added digit carries 7 more bits of every operand chunk, so a residual r at s digits asks
// for about log2(r / 2^-40) / 7 more digits to reach the 2^-40 of result the screen aims at (a
// residual near 1, entries lost below the digits altogether, reads as at least RD_SCREEN_RESULT_BITS missing bits).
// Beyond RD_SPLIT_MAX digits the natural order moves to the locality order (RD_SPLIT_MAX_ORDERED
// at most); beyond that the graph runs in FP64.  The count grows by at least one digit per failure, so
// the loop ends.
rd_status escalate(rd_ctx* h, double worst) {
  h->fallbacks++;
  const int smax = h->ordered ? RD_SPLIT_MAX_ORDERED : RD_SPLIT_MAX;
  const double missing = std::log2(worst > 0.0 ? worst : 1.0) + RD_SCREEN_RESULT_BITS;
  int next = h->slices + (int)std::ceil(missing / RD_SPLIT_DIGIT_BITS);
  if (next <= h->slices) next = h->slices + 1;
  if (next > smax && !h->ordered && next <= RD_SPLIT_MAX_ORDERED && h->dSucc) {
    // the natural order ran out of digits: the locality order's 64-wide chunks carry up to 22
    if (!h->order_ready) {
      rd_status st;
      choose_locality_order(h, h->weighted ? RD_SCREEN_WEIGHTED : 1.0, &st);
      if (st != RD_OK) return st;
    }
    h->ordered = 1;
    h->kappa = RD_SCREEN_CHUNK_ORDERED;
    h->split_floor = next;
  } else {
    h->split_floor = next <= smax ? next : -1;
  }
  RD_CK(h, rd_build_m(h, h->stream));  // M again (the factorisation overwrote it)
  h->factored = h->inverted = 0;
  return RD_OK;
}

// Range screen of the split path, run once per graph when the caller leaves the digit count
// open.  The digits of a KAPPA-wide chunk of an operand row are scaled to the chunk's largest entry, and the entries of Y fall by log2(1/gamma) bits per hop (Y_ij ~ gamma^d
// for distance d), so a chunk whose nodes lie S hops apart as seen from one node costs about
// S log2(1/gamma) of the 7 s bits the digits carry.  The largest S over the chunks, seen from 8
// sampled sources, sets the digit count: the fewest (at least RD_SPLIT_MIN) whose 7 s bits cover
// the spread plus RD_SCREEN_RESULT_BITS bits of result.  When the natural node order (256-wide
// chunks) needs more than RD_SPLIT_START digits, the locality order (compact 64-node parts, see
// rcb_kernel, 64-wide chunks) is screened too and taken when it needs fewer digits; beyond
// RD_SPLIT_MAX (natural) or RD_SPLIT_MAX_ORDERED (locality order) digits the graph runs in FP64.
// On weighted graphs the spread is a weighted distance (Bellman-Ford on gamma^W's exponents),
// scaled by RD_SCREEN_WEIGHTED.  Large-diameter graphs (grids, meshes) are the ones
// that need the locality order: a 256-node run of their natural order spans a whole row of the
// mesh.  The screen only steers: the residual self-check still judges every split result.
double spread_bits(rd_ctx* h, const int32_t* ord, int chunk, rd_status* st) {
  *st = RD_OK;
  cudaError_t e = cudaMemsetAsync(h->dRed, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess)
    e = rd_chunk_spread(h, RD_SCREEN_SOURCES, chunk, ord, reinterpret_cast<int32_t*>(h->dS), h->dRed, h->stream);
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, h->dRed, sizeof(bits), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    *st = fail_cuda(h, e, "range screen");
    return 0.0;
  }
  const unsigned int fb = (unsigned int)bits;
  float spread;
  memcpy(&spread, &fb, sizeof(spread));
  return (double)spread * std::log2(1.0 / h->gamma);
}

// the fewest digits (at least RD_SPLIT_MIN) whose 7 bits each cover `bits` plus the result bits
int digits_for(double bits) {
  const int s = (int)std::ceil((bits + RD_SCREEN_RESULT_BITS) / RD_SPLIT_DIGIT_BITS);
  return s < RD_SPLIT_MIN ? RD_SPLIT_MIN : s;
}

// The locality order with the smaller screened spread: the landmark bisection, and, when its
// 64-node parts still need more than RD_SPLIT_MAX digits (parts that are not compact: on a
// king-move mesh the landmark axes cut strips), the scored bisection too.  Leaves the chosen
// order in dOrd / dPos (h->order_ready = 1 or 2) and returns its spread bits times wf.
double choose_locality_order(rd_ctx* h, double wf, rd_status* st) {
  *st = RD_OK;
  auto fail_order = [&](cudaError_t e) {
    *st = fail_cuda(h, e, "locality order");
    return 0.0;
  };
  cudaError_t e = rd_locality_order(h, 0, h->stream);
  if (e != cudaSuccess) return fail_order(e);
  h->order_ready = 1;
  const double landmark = wf * spread_bits(h, h->dOrd, RD_SCREEN_CHUNK_ORDERED, st);
  if (*st != RD_OK || digits_for(landmark) <= RD_SPLIT_MAX) return landmark;
  if ((e = rd_locality_order(h, 1, h->stream)) != cudaSuccess) return fail_order(e);
  h->order_ready = 2;
  const double scored = wf * spread_bits(h, h->dOrd, RD_SCREEN_CHUNK_ORDERED, st);
  if (*st != RD_OK || scored < landmark) return scored;
  if ((e = rd_locality_order(h, 0, h->stream)) != cudaSuccess) return fail_order(e);  // back to the landmark order
  h->order_ready = 1;
  return landmark;
}

rd_status screen_split(rd_ctx* h) {
  h->screened = 1;
  h->screen_bits = -1.0;
  h->ordered = 0;
  h->kappa = RD_SCREEN_CHUNK;
  if (!h->dSucc) return RD_OK;
  if (!h->succ_ready) {
    RD_CK(h, rd_build_succ(h, h->stream));
    h->succ_ready = 1;
  }
  rd_status st;
  const double wf = h->weighted ? RD_SCREEN_WEIGHTED : 1.0;
  const double nat = wf * spread_bits(h, nullptr, RD_SCREEN_CHUNK, &st);
  if (st != RD_OK) return st;
  h->screen_bits = nat;
  const int s_nat = digits_for(nat);
  if (s_nat <= RD_SPLIT_START) {
    h->split_start = s_nat;
    return RD_OK;
  }
  const double ord = choose_locality_order(h, wf, &st);
  if (st != RD_OK) return st;
  const int s_ord = digits_for(ord);
  // the locality order when it needs fewer digits, or when only it can carry more than 15
  if (s_ord <= RD_SPLIT_MAX_ORDERED && (s_ord < s_nat || s_nat > RD_SPLIT_MAX)) {
    h->ordered = 1;
    h->kappa = RD_SCREEN_CHUNK_ORDERED;
    h->screen_bits = ord;
    h->split_start = s_ord;
  } else if (s_nat <= RD_SPLIT_MAX) {
    h->split_start = s_nat;
  } else {
    h->split_floor = -1;
  }
  return RD_OK;
}

rd_status ensure_factored(rd_ctx* h) {
  if (h->factored) return RD_OK;
  if (split_auto(h) && !h->screened && h->split_floor == 0) {
    rd_status st = screen_split(h);
    if (st != RD_OK) return st;
  }
  RD_CK(h, cudaEventRecord(h->ev[0], h->stream));
  for (;;) {
    h->factor_gen++;  // new factors: digits sliced from the old ones are stale
    const bool split = h->precision == RD_PREC_SPLIT_BF16 && h->split_floor >= 0;
    if (!split) {
      h->ordered = 0;  // the FP64 path works in the caller's node order
      h->kappa = RD_SCREEN_CHUNK;
      RD_CK(h, rd_lu_f64(h, h->stream));
      h->used_precision = RD_PREC_FP64;
      h->factored = 1;
      h->inverted = 0;
      break;
    }
    int s = h->slices_req > 0 ? h->slices_req : (h->split_start > 0 ? h->split_start : RD_SPLIT_START);
    if (h->split_floor > s) s = h->split_floor;
    rd_status st = rd_split_prepare(h, s);
    if (st != RD_OK) return st;
    if (h->ordered) RD_CK(h, rd_permute_m(h, h->stream));  // factor P M P^T
    RD_CK(h, rd_lu_split(h, h->stream));  // LU and both triangular inverses
    h->used_precision = RD_PREC_SPLIT_BF16;
    h->factored = 1;
    h->inverted = 1;
    if (split_auto(h)) {
      // the self-check, before any product uses the inverses: sampled rows of Y against M
      double worst = 0.0;
      RD_CK(h, rd_split_row_check(h, &worst, h->stream));
      h->last_residual = worst;
      if (worst > residual_limit(h)) {
        // failed: more digits as the residual asks, or FP64; the loop factors M again
        if ((st = escalate(h, worst)) != RD_OK) return st;
        continue;
      }
    }
    break;
  }
  RD_CK(h, cudaEventRecord(h->ev[1], h->stream));
  h->ev_used[0] = 1;
  return RD_OK;
}

// Host goals are range-checked here; goals in device memory are checked by every kernel that reads
// them (a goal outside [0, n) leaves its row zero and its next hops -1, and records RD_DEV_BADGOAL,
// which the next synchronising call returns as RD_ERR_ARG).
rd_status ensure_goals(rd_ctx* h, const int32_t* goals, int32_t k) {
  if (!goals) return fail(h, RD_ERR_ARG, "goals is NULL");
  if (k < 1 || k > RD_MAX_GOALS) return fail(h, RD_ERR_ARG, "k must lie in [1, 64]");
  if (!is_device_ptr(goals, h->device)) {
    for (int c = 0; c < k; ++c)
      if (goals[c] < 0 || goals[c] >= h->n) return fail(h, RD_ERR_ARG, "goal index out of range");
  }
  RD_CK(h, cudaMemcpyAsync(h->dGoals, goals, k * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  return RD_OK;
}

double event_ms(rd_ctx* h, int slot) {
  float ms = 0.f;
  if (!h->ev_used[slot]) return 0.0;
  if (cudaEventElapsedTime(&ms, h->ev[2 * slot], h->ev[2 * slot + 1]) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return ms;
}

}  // namespace

void rd_record_error(const std::string& msg) { g_create_err = msg; }

// profile mode 1: every dense-contraction kernel; 2: the split GEMM alone
static bool prof_wanted(const rd_ctx* h, int kind) {
  return h->prof_on != 0 && kind != RD_PROF_NONE && (h->prof_on == 1 || kind == RD_PROF_SPLIT);
}

cudaError_t rd_prof_begin(rd_ctx* h, cudaStream_t s, int kind) {
  h->launches++;
  if (!prof_wanted(h, kind)) return cudaSuccess;
  if (h->prof_used == rd_ctx::kProfPairs) {
    cudaError_t e = rd_prof_collect(h);
    if (e != cudaSuccess) return e;
  }
  return cudaEventRecord(h->prof_ev[2 * h->prof_used], s);
}

cudaError_t rd_prof_end(rd_ctx* h, cudaStream_t s, int kind, double flops) {
  if (!prof_wanted(h, kind)) return cudaSuccess;
  cudaError_t e = cudaEventRecord(h->prof_ev[2 * h->prof_used + 1], s);
  if (e != cudaSuccess) return e;
  h->prof_kind[h->prof_used] = (int8_t)kind;
  h->prof_pair_flops[h->prof_used] = flops;
  h->prof_used++;
  return cudaSuccess;
}

cudaError_t rd_prof_collect(rd_ctx* h) {
  if (!h->prof_ev || h->prof_used == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  // every pair's end (the pairs of the split recursion's side stream may end after the last one
  // recorded on the handle's stream)
  for (int i = 0; i < h->prof_used && e == cudaSuccess; ++i) e = cudaEventSynchronize(h->prof_ev[2 * i + 1]);
  if (e != cudaSuccess) return e;
  // the split GEMM's busy time: the union of its launches' intervals (launches on the two streams of
  // the recursion overlap; their summed durations count the shared time twice)
  std::vector<std::pair<float, float>> iv;
  for (int i = 0; i < h->prof_used; ++i) {
    if (h->prof_kind[i] != RD_PROF_SPLIT) continue;
    float t0 = 0.f, t1 = 0.f;
    if ((e = cudaEventElapsedTime(&t0, h->prof_ev[0], h->prof_ev[2 * i])) != cudaSuccess) return e;
    if ((e = cudaEventElapsedTime(&t1, h->prof_ev[0], h->prof_ev[2 * i + 1])) != cudaSuccess) return e;
    iv.emplace_back(t0, t1);
  }
  std::sort(iv.begin(), iv.end());
  double busy = 0.0;
  for (size_t i = 0; i < iv.size();) {
    float a = iv[i].first, b = iv[i].second;
    for (++i; i < iv.size() && iv[i].first <= b; ++i) b = std::max(b, iv[i].second);
    busy += (double)(b - a);
  }
  h->prof_split_busy_ms += busy;
  for (int i = 0; i < h->prof_used; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    if (h->prof_kind[i] == RD_PROF_UPDATE) {  // bytes, not flops: kept apart
      h->prof_update_ms += ms;
      h->prof_update_bytes += h->prof_pair_flops[i];
      h->prof_update_launches++;
      continue;
    }
    h->prof_ms += ms;
    h->prof_flops += h->prof_pair_flops[i];
    h->prof_launches++;
    if (h->prof_kind[i] == RD_PROF_SPLIT) {
      h->prof_split_ms += ms;
      h->prof_split_flops += h->prof_pair_flops[i];
      h->prof_split_launches++;
    }
  }
  h->prof_used = 0;
  return cudaSuccess;
}

// The factors and both triangular inverses of the handle's graph resident in dT (the serving loop
// reads rows of U^-1 and columns of L^-1 there); waits for the handle's stream.
rd_status rd_prepare_inverses(rd_ctx* h) {
  RD_CK(h, cudaSetDevice(h->device));
  if (h->factored && h->inverted && !h->updated) return RD_OK;  // resident since an earlier request
  rd_status st = ensure_factored(h);
  if (st != RD_OK) return st;
  if (h->used_precision != RD_PREC_SPLIT_BF16 && !h->inverted) {
    RD_CK(h, rd_trtri_f64(h, h->stream));
    h->inverted = 1;
  }
  return check_device_status(h);
}

extern "C" {

rd_status rd_set_profiling(rd_handle h, int32_t on) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (on < 0 || on > 2) return fail(h, RD_ERR_ARG, "rd_set_profiling: on is 0, 1 or 2");
  RD_CK(h, cudaSetDevice(h->device));
  if (on && !h->prof_ev) {
    h->prof_ev = new cudaEvent_t[2 * rd_ctx::kProfPairs]();
    for (int i = 0; i < 2 * rd_ctx::kProfPairs; ++i) RD_CK(h, cudaEventCreate(&h->prof_ev[i]));
  }
  RD_CK(h, cudaStreamSynchronize(h->stream));
  h->prof_on = on;
  h->prof_used = 0;
  h->prof_ms = h->prof_flops = 0.0;
  h->prof_launches = 0;
  h->prof_split_ms = h->prof_split_flops = 0.0;
  h->prof_split_busy_ms = 0.0;
  h->prof_split_launches = 0;
  h->prof_update_ms = h->prof_update_bytes = 0.0;
  h->prof_update_launches = 0;
  return RD_OK;
}

rd_status rd_create(const uint8_t* A, int32_t n, double gamma, rd_handle* out) {
  return create_impl(A, nullptr, n, gamma, out);
}

}  // extern "C"

rd_status rd_create_pooled(const uint8_t* A, int32_t n, double gamma, cudaMemPool_t pool, cudaStream_t stream,
                           rd_handle* out) {
  return create_impl(A, nullptr, n, gamma, out, pool, stream);
}

extern "C" {

rd_status rd_create_weighted(const uint8_t* A, const float* W, int32_t n, double gamma, rd_handle* out) {
  if (!W) {
    if (out) *out = nullptr;
    return fail(nullptr, RD_ERR_ARG, "W is NULL");
  }
  return create_impl(A, W, n, gamma, out);
}

rd_status rd_load(rd_handle h, const uint8_t* A, const float* W, double gamma) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  return load_impl(h, A, W, gamma);
}

rd_status rd_set_stream(rd_handle h, void* stream) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  h->stream = (cudaStream_t)stream;
  return RD_OK;
}

rd_status rd_set_precision(rd_handle h, int32_t mode, int32_t slices) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (mode != RD_PREC_FP64 && mode != RD_PREC_SPLIT_BF16) return fail(h, RD_ERR_ARG, "unknown precision mode");
  if (slices < 0 || slices > 15 || slices == 1) return fail(h, RD_ERR_ARG, "slices must be 0 or lie in [2, 15]");
  if (mode != h->precision || slices != h->slices_req) {
    h->split_floor = 0;
    h->split_start = 0;
    h->screened = 0;
    h->order_ready = 0;
    h->screen_bits = -1.0;
    h->ordered = 0;
    h->kappa = RD_SCREEN_CHUNK;
    h->y_current = h->updated = 0;
    if (h->factored) {
      // the factors in dLU belong to the old mode: rebuild M from the resident graph
      RD_CK(h, cudaMemsetAsync(h->dStatus, 0, 2 * sizeof(int), h->stream));
      RD_CK(h, rd_build_m(h, h->stream));
    }
    h->factored = h->inverted = 0;
  }
  h->precision = mode;
  h->slices_req = slices;
  return RD_OK;
}

rd_status rd_set_tau(rd_handle h, double tau) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!(tau >= 0.0 && tau < 0.5)) return fail(h, RD_ERR_ARG, "tau must lie in [0, 0.5)");
  h->tau = tau;
  return RD_OK;
}

rd_status rd_apsp(rd_handle h, int32_t* D, double* Y) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!D) return fail(h, RD_ERR_ARG, "D is NULL");
  if (is_foreign_device_ptr(D, h->device) || (Y && is_foreign_device_ptr(Y, h->device)))
    return fail(h, RD_ERR_ARG, "output lives on another device");
  RD_CK(h, cudaSetDevice(h->device));
  rd_status st = ensure_factored(h);
  if (st != RD_OK) return st;
  const size_t nn = (size_t)h->n * (size_t)h->n;
  const bool d_host = !is_device_ptr(D, h->device);
  const bool y_host = Y && !is_device_ptr(Y, h->device);
  if (d_host && !h->dDout) RD_CK(h, dalloc(h, &h->dDout, nn));
  if (y_host && !h->dYout) RD_CK(h, dalloc(h, &h->dYout, nn));
  int32_t* dD = d_host ? h->dDout : D;
  double* dY = Y ? (y_host ? h->dYout : Y) : nullptr;
  RD_CK(h, cudaEventRecord(h->ev[2], h->stream));
  if (h->updated && h->y_current) {  // edges changed since the factorisation: Y is the resident one
    unsigned int* lost = reinterpret_cast<unsigned int*>(h->dRed);
    RD_CK(h, rd_rank1_update(h, 0, 0, 0.0, dD, lost, h->stream));  // alpha = 0: decode only
    if (dY) RD_CK(h, cudaMemcpyAsync(dY, h->dYres, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else if (h->used_precision == RD_PREC_SPLIT_BF16) {
    RD_CK(h, rd_trmm_decode_split(h, dD, dY, h->stream));
  } else {
    if (!h->inverted) RD_CK(h, rd_trtri_f64(h, h->stream));
    h->inverted = 1;
    RD_CK(h, rd_trmm_decode_f64(h, dD, dY, h->stream));
  }
  RD_CK(h, cudaEventRecord(h->ev[3], h->stream));
  h->ev_used[1] = 1;
  if (d_host) RD_CK(h, cudaMemcpyAsync(D, dD, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (y_host) RD_CK(h, cudaMemcpyAsync(Y, dY, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (d_host || y_host) return check_device_status(h);
  return RD_OK;
}

namespace {
// Y (resident) and D of the current factors: the inverse product into dYres
rd_status materialize_y(rd_ctx* h, int32_t* dD) {
  const size_t nn = (size_t)h->n * (size_t)h->n;
  if (!h->dYres) RD_CK(h, dalloc(h, &h->dYres, nn));
  rd_status st = ensure_factored(h);
  if (st != RD_OK) return st;
  if (h->used_precision == RD_PREC_SPLIT_BF16) {
    RD_CK(h, rd_trmm_decode_split(h, dD, h->dYres, h->stream));
  } else {
    if (!h->inverted) RD_CK(h, rd_trtri_f64(h, h->stream));
    h->inverted = 1;
    RD_CK(h, rd_trmm_decode_f64(h, dD, h->dYres, h->stream));
  }
  h->y_current = 1;
  h->updated = 0;
  return RD_OK;
}
}  // namespace

rd_status rd_update_edge(rd_handle h, int32_t i, int32_t j, int32_t present, float w, int32_t* D, double* Y) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!D) return fail(h, RD_ERR_ARG, "D is NULL");
  if (i < 0 || j < 0 || i >= h->n || j >= h->n) return fail(h, RD_ERR_ARG, "node index out of range");
  if (present && h->weighted && !(w > 0.f && std::isfinite(w)))
    return fail(h, RD_ERR_ARG, "an edge weight must be positive and finite");
  if (is_foreign_device_ptr(D, h->device) || (Y && is_foreign_device_ptr(Y, h->device)))
    return fail(h, RD_ERR_ARG, "output lives on another device");
  RD_CK(h, cudaSetDevice(h->device));
  const size_t nn = (size_t)h->n * (size_t)h->n;
  const bool d_host = !is_device_ptr(D, h->device);
  const bool y_host = Y && !is_device_ptr(Y, h->device);
  if (d_host && !h->dDout) RD_CK(h, dalloc(h, &h->dDout, nn));
  int32_t* dD = d_host ? h->dDout : D;
  // the entry now, the entry wanted, and column j's sum afterwards (the gain condition)
  const long long at = (long long)i * h->n + j;
  uint8_t a_old = 0;
  float w_old = 0.f;
  double colsum = 0.0;
  RD_CK(h, cudaMemcpyAsync(&a_old, h->dA + at, 1, cudaMemcpyDeviceToHost, h->stream));
  if (h->weighted) RD_CK(h, cudaMemcpyAsync(&w_old, h->dW + at, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  RD_CK(h, cudaMemcpyAsync(&colsum, h->dColsum + j, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  RD_CK(h, cudaStreamSynchronize(h->stream));
  // an edge of infinite weight is a missing edge (gamma^inf = 0): not counted in the degrees
  const bool old_on = a_old != 0 && (!h->weighted || std::isfinite(w_old));
  const double x_old = old_on ? (h->weighted ? std::pow(h->gamma, (double)w_old) : h->gamma) : 0.0;
  const double x_new = present ? (h->weighted ? std::pow(h->gamma, (double)w) : h->gamma) : 0.0;
  const double delta = x_new - x_old;
  if (!(colsum + delta < 1.0)) return fail(h, RD_ERR_GAMMA, "the update would make a column sum of X reach 1");
  rd_status st;
  if (!h->y_current && (st = materialize_y(h, dD)) != RD_OK) return st;
  unsigned int* lost = reinterpret_cast<unsigned int*>(h->dRed);
  if (delta != 0.0 || old_on != (present != 0) || (present && w != w_old)) {
    const int ddeg = (present ? 1 : 0) - (old_on ? 1 : 0);
    h->n_edges += ddeg;
    if ((st = ensure_succ_capacity(h, h->n_edges)) != RD_OK) return st;
    RD_CK(h, rd_set_edge(h, i, j, present ? 1 : 0, present ? w : 0.f, delta, ddeg, h->stream));
    h->succ_ready = 0;
    h->edge_updates++;
  }
  RD_CK(h, rd_rank1_update(h, i, j, delta, dD, lost, h->stream));
  unsigned int nlost = 0;
  RD_CK(h, cudaMemcpyAsync(&nlost, lost, sizeof(nlost), cudaMemcpyDeviceToHost, h->stream));
  RD_CK(h, cudaStreamSynchronize(h->stream));
  if (delta != 0.0) h->updated = 1;
  if (nlost) {
    // a removal cancelled some entries: factor the updated graph from scratch
    h->update_refactors++;
    RD_CK(h, cudaMemsetAsync(h->dStatus, 0, 2 * sizeof(int), h->stream));
    RD_CK(h, rd_build_m(h, h->stream));
    h->factored = h->inverted = 0;
    h->split_floor = h->split_start = 0;
    h->screened = 0;
    h->order_ready = 0;
    h->screen_bits = -1.0;
    h->ordered = 0;
    h->kappa = RD_SCREEN_CHUNK;
    if ((st = materialize_y(h, dD)) != RD_OK) return st;
  }
  if (Y) RD_CK(h, cudaMemcpyAsync(Y, h->dYres, nn * sizeof(double), cudaMemcpyDefault, h->stream));
  if (d_host) RD_CK(h, cudaMemcpyAsync(D, dD, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (d_host || y_host) return check_device_status(h);
  return RD_OK;
}

rd_status rd_goal_solve(rd_handle h, const int32_t* goals, int32_t k, double* Y_out) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!Y_out) return fail(h, RD_ERR_ARG, "Y_out is NULL");
  RD_CK(h, cudaSetDevice(h->device));
  rd_status st = ensure_goals(h, goals, k);
  if (st != RD_OK) return st;
  st = ensure_factored(h);
  if (st != RD_OK) return st;
  const bool host = !is_device_ptr(Y_out, h->device);
  if (host && !h->dYrows) RD_CK(h, dalloc(h, &h->dYrows, (size_t)RD_MAX_GOALS * h->n));
  double* dst = host ? h->dYrows : Y_out;
  RD_CK(h, cudaEventRecord(h->ev[4], h->stream));
  if (h->updated && h->y_current)
    RD_CK(h, rd_rows_from_y(h, h->dGoals, k, dst, h->stream));  // the factors predate the edge updates
  else if (h->used_precision == RD_PREC_SPLIT_BF16 && h->inverted)
    RD_CK(h, rd_goal_split(h, h->dGoals, k, dst, h->stream));  // rows of U^-1 times L^-1
  else
    RD_CK(h, rd_goal_f64(h, h->dGoals, k, dst, h->stream));
  RD_CK(h, cudaEventRecord(h->ev[5], h->stream));
  h->ev_used[2] = 1;
  if (host) {
    RD_CK(h, cudaMemcpyAsync(Y_out, dst, (size_t)k * h->n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    return check_device_status(h);
  }
  return RD_OK;
}

rd_status rd_greedy_walk(rd_handle h, const int32_t* next, int32_t k, const int32_t* start, int32_t max_len,
                         int32_t* path, int32_t* len) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!next || !start || !path || !len) return fail(h, RD_ERR_ARG, "NULL argument");
  if (k < 1 || k > RD_MAX_GOALS) return fail(h, RD_ERR_ARG, "k must lie in [1, 64]");
  if (max_len < 0 || max_len > h->n) return fail(h, RD_ERR_ARG, "max_len must lie in [0, n]");
  RD_CK(h, cudaSetDevice(h->device));
  const size_t kn = (size_t)k * h->n, kp = (size_t)k * ((size_t)max_len + 1);
  const bool next_host = !is_device_ptr(next, h->device), start_host = !is_device_ptr(start, h->device);
  const bool path_host = !is_device_ptr(path, h->device), len_host = !is_device_ptr(len, h->device);
  if (start_host)
    for (int c = 0; c < k; ++c)
      if (start[c] < 0 || start[c] >= h->n) return fail(h, RD_ERR_ARG, "start node out of range");
  // staging for host buffers: next in dNext, starts and lengths in dR, paths after them in dR
  // (64 N doubles hold 2 * 64 + 64 (n + 1) ints)
  if (next_host && !h->dNext) RD_CK(h, dalloc(h, &h->dNext, (size_t)RD_MAX_GOALS * h->n));
  int32_t* stage = reinterpret_cast<int32_t*>(h->dR);
  const int32_t* dnext = next;
  if (next_host) {
    RD_CK(h, cudaMemcpyAsync(h->dNext, next, kn * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    dnext = h->dNext;
  }
  const int32_t* dstart = start;
  if (start_host) {
    RD_CK(h, cudaMemcpyAsync(stage, start, k * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    dstart = stage;
  }
  int32_t* dlen = len_host ? stage + RD_MAX_GOALS : len;
  int32_t* dpath = path_host ? stage + 2 * RD_MAX_GOALS : path;
  RD_CK(h, rd_walk(h, dnext, k, dstart, max_len, dpath, dlen, h->stream));
  if (path_host) RD_CK(h, cudaMemcpyAsync(path, dpath, kp * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (len_host) RD_CK(h, cudaMemcpyAsync(len, dlen, k * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  if (path_host || len_host) RD_CK(h, cudaStreamSynchronize(h->stream));
  return RD_OK;
}

rd_status rd_spectral_radius(rd_handle h, int32_t iters, double* lo, double* hi) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!lo || !hi) return fail(h, RD_ERR_ARG, "lo and hi must not be NULL");
  if (iters < 1 || iters > 1000000) return fail(h, RD_ERR_ARG, "iters must lie in [1, 1000000]");
  if (!h->dSucc) return fail(h, RD_ERR_UNSUPPORTED, "no successor lists (more than 2^31 edges)");
  RD_CK(h, cudaSetDevice(h->device));
  if (!h->succ_ready) {
    RD_CK(h, rd_build_succ(h, h->stream));
    h->succ_ready = 1;
  }
  RD_CK(h, rd_spectral(h, iters, h->dR, h->dR + h->n, reinterpret_cast<unsigned long long*>(h->dRed), lo, hi,
                       h->stream));
  return RD_OK;
}

rd_status rd_greedy_next(rd_handle h, const int32_t* goals, int32_t k, const double* Yrows, int32_t* next) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  if (!Yrows || !next) return fail(h, RD_ERR_ARG, "Yrows and next must not be NULL");
  RD_CK(h, cudaSetDevice(h->device));
  rd_status st = ensure_goals(h, goals, k);
  if (st != RD_OK) return st;
  if (!h->dSucc) return fail(h, RD_ERR_UNSUPPORTED, "too many edges for int32 successor lists");
  if (!h->succ_ready) {
    // successor lists (CSR of the columns of A), sized at load from the edge count
    RD_CK(h, rd_build_succ(h, h->stream));
    h->succ_ready = 1;
  }
  const size_t kn = (size_t)k * h->n;
  const bool y_host = !is_device_ptr(Yrows, h->device);
  const bool n_host = !is_device_ptr(next, h->device);
  if (y_host) {
    if (!h->dYrows) RD_CK(h, dalloc(h, &h->dYrows, (size_t)RD_MAX_GOALS * h->n));
    RD_CK(h, cudaMemcpyAsync(h->dYrows, Yrows, kn * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  if (n_host && !h->dNext) RD_CK(h, dalloc(h, &h->dNext, (size_t)RD_MAX_GOALS * h->n));
  int32_t* dn = n_host ? h->dNext : next;
  RD_CK(h, cudaEventRecord(h->ev[6], h->stream));
  RD_CK(h, rd_greedy(h, h->dGoals, k, y_host ? h->dYrows : Yrows, dn, h->stream));
  RD_CK(h, cudaEventRecord(h->ev[7], h->stream));
  h->ev_used[3] = 1;
  if (n_host) {
    RD_CK(h, cudaMemcpyAsync(next, dn, kn * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    return check_device_status(h);
  }
  return RD_OK;
}

rd_status rd_sync(rd_handle h) {
  if (!h) return fail(nullptr, RD_ERR_ARG, "handle is NULL");
  return check_device_status(h);
}

rd_status rd_get_stats(rd_handle h, rd_stats* s) {
  if (!h || !s) return fail(h, RD_ERR_ARG, "NULL argument");
  rd_status st = check_device_status(h);
  s->n = h->n;
  s->n_padded = h->N;
  s->precision = h->precision;
  s->slices = h->precision == RD_PREC_SPLIT_BF16 ? h->slices : 0;
  s->precision_used = h->used_precision;
  s->fallbacks = h->fallbacks;
  s->split_residual = h->last_residual;
  s->split_screen_bits = h->screen_bits;
  s->split_order = h->ordered ? h->order_ready : 0;
  s->edge_updates = h->edge_updates;
  s->update_refactors = h->update_refactors;
  s->gamma = h->gamma;
  s->max_column_sum = h->max_colsum;
  s->tau = h->tau;
  s->ms_factor = event_ms(h, 0);
  s->ms_inverse = event_ms(h, 1);
  s->ms_goal = event_ms(h, 2);
  s->ms_greedy = event_ms(h, 3);
  s->bytes_device = h->bytes;
  cudaError_t e = rd_prof_collect(h);
  if (e != cudaSuccess) return fail_cuda(h, e, "rd_prof_collect");
  s->launches = h->launches;
  s->prof_launches = h->prof_launches;
  s->prof_ms = h->prof_ms;
  s->prof_flops = h->prof_flops;
  s->prof_split_launches = h->prof_split_launches;
  s->prof_split_ms = h->prof_split_ms;
  s->prof_split_flops = h->prof_split_flops;
  s->prof_update_launches = h->prof_update_launches;
  s->prof_update_ms = h->prof_update_ms;
  s->prof_update_bytes = h->prof_update_bytes;
  s->prof_split_busy_ms = h->prof_split_busy_ms;
  return st;
}

const char* rd_last_error(rd_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

const char* rd_status_string(rd_status s) {
  switch (s) {
    case RD_OK: return "RD_OK";
    case RD_ERR_ARG: return "RD_ERR_ARG";
    case RD_ERR_GAMMA: return "RD_ERR_GAMMA";
    case RD_ERR_OOM: return "RD_ERR_OOM";
    case RD_ERR_CUDA: return "RD_ERR_CUDA";
    case RD_ERR_NUMERIC: return "RD_ERR_NUMERIC";
    case RD_ERR_STATE: return "RD_ERR_STATE";
    case RD_ERR_TIMEOUT: return "RD_ERR_TIMEOUT";
    case RD_ERR_UNSUPPORTED: return "RD_ERR_UNSUPPORTED";
  }
  return "RD_ERR_UNKNOWN";
}

void rd_destroy(rd_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  // a pooled handle's memory returns to its pool in stream order (no wait); otherwise wait for the
  // handle's work before cudaFree
  if (!h->pool) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"
