// rd_serve_loop.cu -- the serving runtime's device-resident goal loop.
//
// Goal requests (rows of Y for up to 64 goals, the local mode of Sec. 4.2) on resident graphs run
// on a persistent kernel instead of launches from the host: the host writes a request descriptor
// into a ring in mapped pinned memory and advances a posted counter; the loop kernel's CTAs claim
// work units of posted requests from a device counter, compute them from the graph's resident
// triangular inverses, and the CTA that finishes a request's last unit marks it done in the ring,
// where the host's worker reads it.  No kernel is launched per request and no stream is
// synchronised: a request costs the host a descriptor, a fence and a poll.
//
//   row g of Y = (row g of U^-1) L^-1, entry q = sum_{k >= max(g, q)} U^-1[g][k] L^-1[k][q]
//
// (Y = M^-1 = U^-1 L^-1; L^-1 is unit lower triangular; both inverses are non-negative for the
// M-matrices of the method, so every sum adds terms of one sign.)  A work unit is a group of 16
// goals times a block of columns: 4 goal groups x 32 column blocks cover 64 goals and the padded
// size N.  FP64 is slow on this GPU (2 FMA per clock per SM), so a request is spread over many
// small units: a 256-node request with 32 goals is 16 units, one per SM.  A graph in the split
// path's locality order keeps its inverses in that order: goal g sits at position pos[g] and
// position q holds node ord[q], so the rows are written back in the caller's node order.
//
// Bounded waits.  Every wait of the kernel ends: a CTA without work polls the posted counter and
// leaves after LOOP_IDLE_NS idle (so the loop holds its SMs only while requests flow), and a CTA
// whose claimed request's descriptor is not ready gives up after LOOP_READY_NS and marks the
// request failed (RD_ERR_TIMEOUT to the host).  A CTA that leaves clears its alive word, fences,
// and re-reads the posted counter; the host posts, fences, and reads the alive words before it
// decides whether to launch the loop: one of the two sees the other's write, so a posted request
// never waits for a loop that has left.
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>

#include "rd_internal.cuh"

namespace {

constexpr int LOOP_RING = 32;          // request descriptors in flight
constexpr int LOOP_GG = 4;             // goal groups of 16 per request
constexpr int LOOP_CB = 32;            // column blocks per request
constexpr int LOOP_UNITS = LOOP_GG * LOOP_CB;  // work units per request
constexpr int LOOP_CTAS = 38;          // a quarter of the SMs, while requests flow
constexpr int LOOP_THREADS = 256;
constexpr int LOOP_KB = 32;            // K step of the staged tiles
constexpr int LOOP_COLS = 32;          // columns of a unit's sub-block
constexpr unsigned long long LOOP_IDLE_NS = 2000000ull;     // a CTA leaves after 2 ms without work (default)
constexpr unsigned long long LOOP_READY_NS = 200000000ull;  // wait for a posted descriptor: 0.2 s

struct LoopSlot {  // mapped pinned host memory; the host writes it before posting the request
  const double* T;            // the graph's resident inverses (device): strict lower L^-1, upper U^-1
  const int32_t* pos;         // node -> position (locality order) or null
  const int32_t* ord;         // position -> node (locality order) or null
  double* out;                // device address of the slot's staging rows (mapped), k x n
  int32_t n, N, k, cw;        // cw: columns per column block, a multiple of 32
  int32_t goals[RD_MAX_GOALS];
  volatile long long seq;     // the request's sequence number, written last
  volatile int32_t state;     // written by the device: 0 pending, 2 done, 3 a bounded wait expired
};

struct LoopCtl {  // mapped pinned host memory
  volatile long long posted;           // requests 0 .. posted - 1 are in the ring
  volatile int32_t stop;
  volatile int32_t alive[LOOP_CTAS];   // per CTA: 1 while it runs the loop
};

__device__ __forceinline__ unsigned long long loop_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One work unit: goals [16 gg, 16 gg + 16) of the request's k and columns [cb cw, (cb + 1) cw), unit
// = gg LOOP_CB + cb, in sub-blocks of 32 columns.  Thread t owns goal 16 gg + t / 16 and columns
// 2 (t % 16) and 2 (t % 16) + 1 of the sub-block; K advances LOOP_KB at a time through shared
// memory.  The descriptor (host memory that the host rewrites for every request of the slot) is
// read with volatile loads, never from a cached copy.
struct UnitDesc {
  const double* T;
  const int32_t* pos;
  const int32_t* ord;
  double* out;
  int n, N, k, cw;
};
__device__ void loop_unit(const LoopSlot* S_, int unit, double (*Us)[LOOP_KB + 1], double (*Ls)[LOOP_COLS + 1],
                          int* gpos, UnitDesc* d) {
  const volatile LoopSlot* S = S_;
  const int t = threadIdx.x;
  if (t == 0) {
    d->T = S->T;
    d->pos = S->pos;
    d->ord = S->ord;
    d->out = S->out;
    d->n = S->n;
    d->N = S->N;
    d->k = S->k;
    d->cw = S->cw;
  }
  __syncthreads();
  const int N = d->N, n = d->n, k = d->k, cw = d->cw;
  const int gg = unit / LOOP_CB, cb = unit % LOOP_CB;
  const int c0 = 16 * gg;
  if (c0 >= k || cb * cw >= n) return;  // (uniform) no goal or no column of this unit
  const double* __restrict__ T = d->T;
  const int32_t* pos = d->pos;
  const int32_t* ord = d->ord;
  double* out = d->out;
  if (t < 16) gpos[t] = (c0 + t < k) ? (pos ? pos[S->goals[c0 + t]] : S->goals[c0 + t]) : N;  // N: a zero row
  __syncthreads();
  const int ci = t / 16, cj = 2 * (t % 16);
  const int q1 = min(n, (cb + 1) * cw);
  for (int q0 = cb * cw; q0 < q1; q0 += LOOP_COLS) {
    double acc0 = 0.0, acc1 = 0.0;
    for (int k0 = q0; k0 < N; k0 += LOOP_KB) {  // L^-1[kk][q] = 0 for kk < q
      for (int e = t; e < 16 * LOOP_KB; e += LOOP_THREADS) {
        const int c = e / LOOP_KB, kk = k0 + e % LOOP_KB;
        const int g = gpos[c];
        Us[c][e % LOOP_KB] = (g < N && kk >= g && kk < N) ? T[(long long)g * N + kk] : 0.0;
      }
      for (int e = t; e < LOOP_KB * LOOP_COLS; e += LOOP_THREADS) {
        const int kk = k0 + e / LOOP_COLS, q = q0 + e % LOOP_COLS;
        double v = 0.0;
        if (kk < N && q < N) v = kk > q ? T[(long long)kk * N + q] : (kk == q ? 1.0 : 0.0);
        Ls[e / LOOP_COLS][e % LOOP_COLS] = v;
      }
      __syncthreads();
      if (c0 + ci < k) {  // (goal rows past k are zero: their warps skip the FMAs)
#pragma unroll 8
        for (int kk = 0; kk < LOOP_KB; ++kk) {
          const double x = Us[ci][kk];
          acc0 = fma(x, Ls[kk][cj], acc0);
          acc1 = fma(x, Ls[kk][cj + 1], acc1);
        }
      }
      __syncthreads();
    }
    const int c = c0 + ci;
    if (c < k) {  // positions n..N-1 are padding
      const int qa = q0 + cj, qb = qa + 1;
      if (qa < n) out[(long long)c * n + (ord ? ord[qa] : qa)] = acc0;
      if (qb < n) out[(long long)c * n + (ord ? ord[qb] : qb)] = acc1;
    }
  }
}

__global__ void __launch_bounds__(LOOP_THREADS) serve_loop_kernel(LoopSlot* ring, LoopCtl* ctl,
                                                                  unsigned long long* ctr, int* units_done,
                                                                  int* slot_err, unsigned long long idle_ns) {
  __shared__ double Us[16][LOOP_KB + 1];
  __shared__ double Ls[LOOP_KB][LOOP_COLS + 1];
  __shared__ int gpos[16];
  __shared__ long long s_unit;
  __shared__ int s_ready;
  __shared__ UnitDesc desc;
  const int t = threadIdx.x;
  unsigned long long idle_since = loop_time();  // (thread 0's)
  long long seen = -1;
  if (t == 0) {
    ctl->alive[blockIdx.x] = 1;
    __threadfence_system();
  }
  for (;;) {
    if (t == 0) {
      long long u = -2;  // -2: nothing claimed, keep polling; -3: leave
      const long long posted = ctl->posted;
      if (ctl->stop) {
        u = -3;
      } else {
        // claim the next unit of a posted request (never beyond the posted ones)
        const unsigned long long limit = (unsigned long long)posted * LOOP_UNITS;
        unsigned long long old = *(volatile unsigned long long*)ctr;
        while (old < limit) {
          const unsigned long long prev = atomicCAS(ctr, old, old + 1);
          if (prev == old) {
            u = (long long)old;
            break;
          }
          old = prev;
        }
        if (u < 0) {
          const unsigned long long now = loop_time();
          if (posted != seen) {
            seen = posted;
            idle_since = now;
          }
          if (now - idle_since > idle_ns) {
            ctl->alive[blockIdx.x] = 0;
            __threadfence_system();
            if (ctl->posted != posted && !ctl->stop) {  // work arrived meanwhile: stay
              ctl->alive[blockIdx.x] = 1;
              __threadfence_system();
              idle_since = now;
            } else {
              u = -3;
            }
          }
        }
      }
      if (u == -3) {
        ctl->alive[blockIdx.x] = 0;
        __threadfence_system();
      }
      s_unit = u;
    }
    __syncthreads();
    const long long u = s_unit;
    __syncthreads();  // (s_unit is rewritten in the next round)
    if (u == -3) break;
    if (u == -2) {
      __nanosleep(2000);
      continue;
    }
    const long long r = u / LOOP_UNITS;
    const int unit = (int)(u % LOOP_UNITS);
    const int sl = (int)(r % LOOP_RING);
    LoopSlot* S = ring + sl;
    if (t == 0) {  // request r's descriptor (written before it was posted; the wait is bounded)
      const unsigned long long t0 = loop_time();
      int ok = 1;
      while (((volatile LoopSlot*)S)->seq != r) {
        if (loop_time() - t0 > LOOP_READY_NS) {
          ok = 0;
          break;
        }
        __nanosleep(1000);
      }
      __threadfence_system();
      s_ready = ok;
    }
    __syncthreads();
    if (s_ready)
      loop_unit(S, unit, Us, Ls, gpos, &desc);
    else if (t == 0)
      atomicExch(&slot_err[sl], 1);
    __syncthreads();
    if (t == 0) {
      __threadfence_system();  // this unit's rows before its count
      if (atomicAdd(&units_done[sl], 1) == LOOP_UNITS - 1) {
        units_done[sl] = 0;
        const int err = atomicExch(&slot_err[sl], 0);
        __threadfence_system();
        S->state = err ? 3 : 2;
        __threadfence_system();
      }
      idle_since = loop_time();
    }
  }
}

}  // namespace

struct rd_serve_loop {
  int device = 0;
  cudaStream_t stream = nullptr;
  LoopSlot* ring_h = nullptr;
  LoopSlot* ring_d = nullptr;
  LoopCtl* ctl_h = nullptr;
  LoopCtl* ctl_d = nullptr;
  double* stage_h = nullptr;  // LOOP_RING x 64 x RD_LOOP_MAX_N doubles, mapped
  double* stage_d = nullptr;
  unsigned long long* ctr = nullptr;
  int* units_done = nullptr;
  int* slot_err = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  long long next_seq = 0;
  bool busy[LOOP_RING] = {};
  int64_t requests = 0;
  unsigned long long idle_ns = LOOP_IDLE_NS;  // RD_SERVE_LOOP_IDLE_US at creation
};

namespace {

int alive_count(const rd_serve_loop* L) {
  int a = 0;
  for (int c = 0; c < LOOP_CTAS; ++c) a += L->ctl_h->alive[c];
  return a;
}

// (caller holds L->mu, after posting) launch the loop unless CTAs of it still run
cudaError_t ensure_running(rd_serve_loop* L) {
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (alive_count(L) > 0) return cudaSuccess;
  serve_loop_kernel<<<LOOP_CTAS, LOOP_THREADS, 0, L->stream>>>(L->ring_d, L->ctl_d, L->ctr, L->units_done,
                                                               L->slot_err, L->idle_ns);
  return cudaGetLastError();
}

// take the next sequence number and its ring slot (bounded wait for the slot to free up)
bool take_slot(rd_serve_loop* L, std::unique_lock<std::mutex>& lk, long long* seq, int* sl, double timeout_ms) {
  const int want = (int)(L->next_seq % LOOP_RING);
  if (!L->cv.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), [&] { return !L->busy[want]; }))
    return false;
  *seq = L->next_seq++;
  *sl = want;
  L->busy[want] = true;
  return true;
}

// wait for the device to finish request slot sl (bounded); a loop that left without taking it is
// launched again (the handshake makes this a safety net only)
int wait_slot(rd_serve_loop* L, int sl, double timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  auto last_alive = t0;
  for (;;) {
    const int st = L->ring_h[sl].state;
    if (st != 0) {
      std::atomic_thread_fence(std::memory_order_acquire);
      return st;
    }
    const auto now = std::chrono::steady_clock::now();
    const double waited = std::chrono::duration<double, std::milli>(now - t0).count();
    if (waited > timeout_ms) return 0;
    {
      std::lock_guard<std::mutex> g(L->mu);
      if (alive_count(L) > 0)
        last_alive = now;
      else if (std::chrono::duration<double, std::milli>(now - last_alive).count() > 5.0)
        ensure_running(L), last_alive = now;
    }
    if (waited < 0.5)
      std::this_thread::yield();  // most requests finish within half a millisecond
    else
      std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void release_slot(rd_serve_loop* L, int sl) {
  std::lock_guard<std::mutex> g(L->mu);
  L->busy[sl] = false;
  L->cv.notify_all();
}

}  // namespace

rd_status rd_loop_create(int device, rd_serve_loop** out, std::string* err) {
  *out = nullptr;
  rd_serve_loop* L = new rd_serve_loop();
  L->device = device;
  if (const char* iu = getenv("RD_SERVE_LOOP_IDLE_US")) {  // how long idle CTAs keep polling (1 us .. 1 s)
    const long long us = atoll(iu);
    if (us >= 1 && us <= 1000000) L->idle_ns = (unsigned long long)us * 1000ull;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
  const size_t stage = (size_t)LOOP_RING * RD_MAX_GOALS * RD_LOOP_MAX_N * sizeof(double);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&L->ring_h, LOOP_RING * sizeof(LoopSlot), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&L->ctl_h, sizeof(LoopCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&L->stage_h, stage, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&L->ring_d, L->ring_h, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&L->ctl_d, L->ctl_h, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&L->stage_d, L->stage_h, 0);
  if (e == cudaSuccess) e = cudaMalloc((void**)&L->ctr, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&L->units_done, LOOP_RING * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&L->slot_err, LOOP_RING * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(L->ctr, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(L->units_done, 0, LOOP_RING * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(L->slot_err, 0, LOOP_RING * sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    *err = std::string("serving loop: ") + cudaGetErrorString(e);
    rd_loop_destroy(L);
    return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
  }
  memset((void*)L->ring_h, 0, LOOP_RING * sizeof(LoopSlot));
  for (int q = 0; q < LOOP_RING; ++q) L->ring_h[q].seq = -1;
  memset((void*)L->ctl_h, 0, sizeof(LoopCtl));
  *out = L;
  return RD_OK;
}

void rd_loop_destroy(rd_serve_loop* L) {
  if (!L) return;
  if (L->ctl_h) {
    L->ctl_h->stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
  if (L->stream) {
    cudaStreamSynchronize(L->stream);  // the loop's CTAs leave at their next poll
    cudaStreamDestroy(L->stream);
  }
  if (L->ring_h) cudaFreeHost(L->ring_h);
  if (L->ctl_h) cudaFreeHost(L->ctl_h);
  if (L->stage_h) cudaFreeHost(L->stage_h);
  void* ptrs[] = {L->ctr, L->units_done, L->slot_err};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete L;
}

rd_status rd_loop_goals(rd_serve_loop* L, rd_ctx* h, const int32_t* goals, int k, double* Y, double timeout_ms) {
  if (h->n > RD_LOOP_MAX_N || !h->inverted || k < 1 || k > RD_MAX_GOALS) return RD_ERR_UNSUPPORTED;
  long long seq;
  int sl;
  {
    std::unique_lock<std::mutex> lk(L->mu);
    if (!take_slot(L, lk, &seq, &sl, timeout_ms)) return RD_ERR_TIMEOUT;
    LoopSlot& S = L->ring_h[sl];
    S.T = h->dT;
    S.pos = h->ordered ? h->dPos : nullptr;
    S.ord = h->ordered ? h->dOrd : nullptr;
    S.out = L->stage_d + (size_t)sl * RD_MAX_GOALS * RD_LOOP_MAX_N;
    S.n = h->n;
    S.N = h->N;
    S.k = k;
    const int per_block = (h->N + LOOP_CB - 1) / LOOP_CB;
    S.cw = (per_block + LOOP_COLS - 1) / LOOP_COLS * LOOP_COLS;
    for (int c = 0; c < k; ++c) S.goals[c] = goals[c];
    S.state = 0;
    std::atomic_thread_fence(std::memory_order_release);
    S.seq = seq;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    L->ctl_h->posted = seq + 1;
    cudaError_t e = ensure_running(L);
    L->requests++;
    if (e != cudaSuccess) {
      L->busy[sl] = false;
      return RD_ERR_CUDA;
    }
  }
  const int st = wait_slot(L, sl, timeout_ms);
  if (st == 0) return RD_ERR_TIMEOUT;  // (the slot stays taken: the device may still write it)
  if (st == 2) memcpy(Y, L->stage_h + (size_t)sl * RD_MAX_GOALS * RD_LOOP_MAX_N, (size_t)k * h->n * sizeof(double));
  release_slot(L, sl);
  return st == 2 ? RD_OK : RD_ERR_TIMEOUT;
}

rd_status rd_loop_unready(rd_serve_loop* L, double timeout_ms) {
  long long seq;
  int sl;
  {
    std::unique_lock<std::mutex> lk(L->mu);
    if (!take_slot(L, lk, &seq, &sl, timeout_ms)) return RD_ERR_TIMEOUT;
    L->ring_h[sl].state = 0;
    L->ring_h[sl].seq = -1;  // never this request's: the loop's bounded wait for it runs out
    std::atomic_thread_fence(std::memory_order_seq_cst);
    L->ctl_h->posted = seq + 1;
    if (ensure_running(L) != cudaSuccess) {
      L->busy[sl] = false;
      return RD_ERR_CUDA;
    }
  }
  const int st = wait_slot(L, sl, timeout_ms);
  if (st == 0) return RD_ERR_STATE;  // the loop did not report at all
  release_slot(L, sl);
  return st == 2 ? RD_OK : RD_ERR_TIMEOUT;
}

int64_t rd_loop_requests(rd_serve_loop* L) {
  std::lock_guard<std::mutex> g(L->mu);
  return L->requests;
}
