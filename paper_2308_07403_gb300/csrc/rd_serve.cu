// rd_serve.cu -- the serving runtime: a request queue over handles, continuous batching on several
// CUDA streams, admission by device-memory footprint, resident factors per graph for repeated goal
// solves, latency accounting.  Host code only; every computation runs through rd_create / rd_apsp /
// rd_goal_solve on the workers' streams.
//
// Each worker thread runs on one non-blocking stream of the server's and runs one request at a time.  A request is
// runnable when its graph's handle is resident and idle (goal solves reuse the factors), or when a
// new handle fits the budget, after evicting least-recently-used idle handles if needed.  Requests
// that arrive while others are on the GPU start as soon as a worker and the memory are free, so
// the work of several requests overlaps on the device.  Requests for one graph never run at the
// same time (a handle is not thread-safe); a later request for a busy graph waits while the queue
// behind it moves on.
//
// Goal requests on graphs of at most RD_LOOP_DEFAULT_N nodes run on the device-resident loop
// (rd_serve_loop.cu): the worker makes the graph resident with its factors and both triangular
// inverses (the first request of a graph), then posts the request to the loop's ring and waits for
// it; no kernel is launched per request.  Full APSP requests, and goal requests on larger graphs,
// run through rd_apsp / rd_goal_solve on the worker's stream: the loop computes rows in FP64 on a
// few SMs, and a 4096-node request (4.5 ms there) queued behind the split kernels of concurrent
// APSP requests, which hold every SM, made the stream fall behind its arrivals, while the same
// request takes about half a millisecond on the tensor cores.  RD_SERVE_LOOP_MAX_N (0..4096) at
// rd_serve_create moves the limit (0: no loop requests).
//
// Device memory: every handle of the server allocates from one stream-ordered memory pool
// (cudaMallocFromPoolAsync on the worker's stream) and an evicted handle returns its memory with
// cudaFreeAsync, so admission and eviction never synchronise the device or stall the other
// workers' streams (cudaMalloc / cudaFree may).  The pool keeps up to the budget mapped for reuse.
// A request whose estimated footprint exceeds the whole budget is refused at submit (RD_ERR_OOM):
// every admitted request fits once the idle graphs are evicted.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rd_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  rd_request r{};
  std::vector<uint8_t> A;       // copied at submit
  std::vector<int32_t> goals;   // copied at submit
  clock_type::time_point t_submit, t_start, t_done;
  rd_status result = RD_OK;
  bool done = false;
  bool fresh = false;           // created a handle for this job
};

struct Resident {
  rd_handle h = nullptr;
  int32_t n = 0;
  int64_t bytes = 0;            // reserved or measured device bytes
  bool busy = false;
  bool ready = false;           // the handle exists (a reservation precedes it)
  uint64_t last_use = 0;
  int32_t precision = -1;
};

// device bytes of a handle of n nodes (the workspace rd_create allocates, the split digit planes
// when the precision asks for them, host-output staging), used to admit before creating
int64_t estimate_bytes(int32_t n, int32_t precision) {
  const int64_t N = ((int64_t)n + RD_PAD - 1) / RD_PAD * RD_PAD;
  int64_t b = (int64_t)n * n + 8 * N * N * 5 / 2 + 8 * 64 * N + 16 * (int64_t)n;
  b += 4 * (int64_t)n * n + 8 * (int64_t)n * n;  // staging of host D and Y outputs
  if (precision == RD_PREC_SPLIT_BF16) b += 2 * 2 * 15 * N * (N + 256) + 8 * (N + 256) * (N + 256) / 64;
  return b;
}

}  // namespace

struct rd_server {
  int device = 0;
  cudaMemPool_t pool = nullptr;  // the handles' device memory (see the file comment)
  rd_serve_loop* loop = nullptr;  // the device-resident goal loop
  int loop_max_n = RD_LOOP_DEFAULT_N;  // goal requests on graphs up to this size run on the loop
  int64_t budget = 0;
  int64_t used = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;
  std::unordered_map<int32_t, Resident> cache;  // graph id -> resident handle
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;  // one per worker; destroyed after the resident handles
  int64_t next_id = 1;
  uint64_t tick = 0;
  bool stop = false;
  int inflight = 0, max_inflight = 0;
  int64_t completed = 0, failed = 0, evictions = 0, reused = 0;
  int64_t launches = 0;  // kernel launches of the requests' handles (the handles' own counters)
  std::vector<double> lat_ms;
  clock_type::time_point t0;
};

namespace {

// drop an idle resident graph (caller holds the lock)
void release(rd_server* s, std::unordered_map<int32_t, Resident>::iterator e) {
  rd_destroy(e->second.h);
  s->used -= e->second.bytes;
  s->cache.erase(e);
}

// pick a runnable job (caller holds the lock); reserves memory / marks the graph busy
Job* take_runnable(rd_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    Job* j = *it;
    const int32_t gid = j->r.graph_id;
    auto c = (gid >= 0) ? s->cache.find(gid) : s->cache.end();
    if (c != s->cache.end() && c->second.n == j->r.n && c->second.precision == j->r.precision) {
      if (c->second.busy) continue;  // the graph is running: keep its order, let others pass
      c->second.busy = true;
      s->queue.erase(it);
      return j;
    }
    if (c != s->cache.end()) {  // same id but another size or precision: replace it
      if (c->second.busy) continue;  // (its running request keeps the handle until it ends)
      release(s, c);
      c = s->cache.end();
    }
    const int64_t need = estimate_bytes(j->r.n, j->r.precision);
    // evict least-recently-used idle handles until the job fits; a request never needs more than
    // the budget (refused at submit), so an idle server always makes room
    while (s->used + need > s->budget) {
      auto victim = s->cache.end();
      for (auto e = s->cache.begin(); e != s->cache.end(); ++e)
        if (!e->second.busy && e->second.ready && (victim == s->cache.end() || e->second.last_use < victim->second.last_use))
          victim = e;
      if (victim == s->cache.end()) break;
      release(s, victim);
      s->evictions++;
    }
    if (s->used + need > s->budget) continue;  // wait for running requests to free memory
    s->used += need;
    j->fresh = true;
    Resident rsd;
    rsd.n = j->r.n;
    rsd.bytes = need;
    rsd.busy = true;
    rsd.precision = j->r.precision;
    if (gid >= 0) s->cache[gid] = rsd;
    s->queue.erase(it);
    return j;
  }
  return nullptr;
}

void run_job(rd_server* s, Job* j, cudaStream_t st) {
  rd_handle h = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!j->fresh) h = s->cache[j->r.graph_id].h;
  }
  rd_status r = RD_OK;
  if (!h) {
    r = rd_create_pooled(j->A.data(), j->r.n, j->r.gamma, s->pool, st, &h);
    if (r == RD_OK) r = rd_set_precision(h, j->r.precision, 0);
  }
  if (r == RD_OK) r = rd_set_stream(h, (void*)st);  // this worker's stream, whoever ran it before
  // the handle is this worker's until the request ends; a handle made for it counts from its creation
  const int64_t launches0 = (h && !j->fresh) ? h->launches : 0;
  if (r == RD_OK) {
    if (j->r.kind == RD_REQ_APSP) {
      r = rd_apsp(h, j->r.D_out, nullptr);
    } else if (s->loop && j->r.n <= s->loop_max_n) {
      for (int c = 0; c < j->r.k && r == RD_OK; ++c)
        if (j->goals[c] < 0 || j->goals[c] >= j->r.n) r = RD_ERR_ARG;
      if (r == RD_OK) r = rd_prepare_inverses(h);
      if (r == RD_OK) r = rd_loop_goals(s->loop, h, j->goals.data(), j->r.k, j->r.Y_out, 60000.0);
    } else {
      r = rd_goal_solve(h, j->goals.data(), j->r.k, j->r.Y_out);
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (h) s->launches += h->launches - launches0;
  j->result = r;
  j->t_done = clock_type::now();
  j->done = true;
  const int32_t gid = j->r.graph_id;
  const bool cached = gid >= 0 && s->cache.count(gid) != 0;
  if (j->fresh) {
    const int64_t reserved = estimate_bytes(j->r.n, j->r.precision);
    if (r == RD_OK && h && cached) {
      Resident& e = s->cache[gid];
      rd_stats stt;
      const int64_t real = (rd_get_stats(h, &stt) == RD_OK) ? stt.bytes_device : reserved;
      s->used += real - reserved;
      e.h = h;
      e.bytes = real;
      e.ready = true;
      e.busy = false;
      e.last_use = ++s->tick;
    } else {  // failed, or a graph without an id: nothing stays resident
      if (h) rd_destroy(h);
      s->used -= reserved;
      if (cached) s->cache.erase(gid);
    }
  } else {
    s->reused++;
    if (cached) {
      Resident& e = s->cache[gid];
      e.busy = false;
      e.last_use = ++s->tick;
    }
  }
  s->inflight--;
  s->completed++;
  if (r != RD_OK) s->failed++;
  s->lat_ms.push_back(std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count());
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void worker_main(rd_server* s, cudaStream_t st) {
  cudaSetDevice(s->device);
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) break;
        j = take_runnable(s);
        if (j) break;
        s->cv_work.wait(lk);
      }
      if (!j) break;
      j->t_start = clock_type::now();
      s->inflight++;
      s->max_inflight = std::max(s->max_inflight, s->inflight);
    }
    run_job(s, j, st);
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace

extern "C" {

rd_status rd_serve_create(int64_t hbm_budget_bytes, int32_t workers, rd_server_handle* out) {
  if (!out) return RD_ERR_ARG;
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || workers < 1 || workers > 64) {
    rd_record_error("rd_serve_create: budget must be > 0 and workers in [1, 64]");
    return RD_ERR_ARG;
  }
  rd_server* s = new rd_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    rd_record_error("rd_serve_create: no CUDA device");
    return RD_ERR_CUDA;
  }
  s->budget = hbm_budget_bytes;
  s->t0 = clock_type::now();
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    rd_record_error("rd_serve_create: cudaMemPoolCreate failed");
    return RD_ERR_CUDA;
  }
  uint64_t keep = (uint64_t)hbm_budget_bytes;  // memory kept mapped in the pool between requests
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  std::string lerr;
  {
    // RD_SERVE_LOOP_MAX_N overrides the largest graph whose goal requests run on the loop (0: none)
    const char* lm = getenv("RD_SERVE_LOOP_MAX_N");
    if (lm) s->loop_max_n = std::max(0, std::min(RD_LOOP_MAX_N, atoi(lm)));
  }
  if (rd_loop_create(s->device, &s->loop, &lerr) != RD_OK) {
    cudaMemPoolDestroy(s->pool);
    delete s;
    rd_record_error("rd_serve_create: " + lerr);
    return RD_ERR_CUDA;
  }
  for (int w = 0; w < workers; ++w) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t q : s->streams) cudaStreamDestroy(q);
      rd_loop_destroy(s->loop);
      cudaMemPoolDestroy(s->pool);
      delete s;
      rd_record_error("rd_serve_create: cudaStreamCreate failed");
      return RD_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s, s->streams[w]);
  *out = s;
  return RD_OK;
}

rd_status rd_serve_submit(rd_server_handle s, const rd_request* r, int64_t* id) {
  if (!s || !r || !id || !r->A || r->n < 1 || !(r->gamma > 0.0 && r->gamma < 1.0)) return RD_ERR_ARG;
  if (r->kind != RD_REQ_APSP && r->kind != RD_REQ_GOALS) return RD_ERR_ARG;
  if (r->kind == RD_REQ_APSP && !r->D_out) return RD_ERR_ARG;
  if (r->kind == RD_REQ_GOALS && (!r->goals || !r->Y_out || r->k < 1 || r->k > RD_MAX_GOALS)) return RD_ERR_ARG;
  if (r->precision != RD_PREC_FP64 && r->precision != RD_PREC_SPLIT_BF16) return RD_ERR_ARG;
  if (r->n > 65536) return RD_ERR_ARG;
  if (estimate_bytes(r->n, r->precision) > s->budget) {
    rd_record_error("rd_serve_submit: the request's device footprint exceeds the server's budget");
    return RD_ERR_OOM;
  }
  Job* j = new Job();
  j->r = *r;
  j->A.assign(r->A, r->A + (size_t)r->n * r->n);
  if (r->kind == RD_REQ_GOALS) j->goals.assign(r->goals, r->goals + r->k);
  j->t_submit = clock_type::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete j;
      return RD_ERR_STATE;
    }
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
  *id = j->id;
  return RD_OK;
}

rd_status rd_serve_poll(rd_server_handle s, int64_t id, int32_t* done) {
  if (!s || !done) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RD_ERR_ARG;
  *done = it->second->done ? 1 : 0;
  return RD_OK;
}

rd_status rd_serve_wait(rd_server_handle s, int64_t id, rd_status* result, double* latency_ms) {
  return rd_serve_wait_for(s, id, -1.0, result, latency_ms);
}

rd_status rd_serve_wait_for(rd_server_handle s, int64_t id, double timeout_ms, rd_status* result,
                            double* latency_ms) {
  if (!s) return RD_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return RD_ERR_ARG;
  Job* j = it->second;
  if (timeout_ms < 0.0) {
    s->cv_done.wait(lk, [&] { return j->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                  [&] { return j->done; })) {
    return RD_ERR_TIMEOUT;  // still running: the id stays valid
  }
  if (result) *result = j->result;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
  s->jobs.erase(it);
  delete j;
  return RD_OK;
}

rd_status rd_serve_stats(rd_server_handle s, rd_serve_report* out) {
  if (!s || !out) return RD_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->resident_graphs = (int32_t)s->cache.size();
  out->max_inflight = s->max_inflight;
  out->bytes_used = s->used;
  out->evictions = s->evictions;
  out->reused = s->reused;
  out->launches = s->launches;
  out->loop_requests = s->loop ? rd_loop_requests(s->loop) : 0;
  out->p50_ms = percentile(s->lat_ms, 0.5);
  out->p99_ms = percentile(s->lat_ms, 0.99);
  out->seconds = std::chrono::duration<double>(clock_type::now() - s->t0).count();
  return RD_OK;
}

rd_status rd_serve_loop_check(rd_server_handle s, rd_status* result) {
  if (!s || !result || !s->loop) return RD_ERR_ARG;
  *result = rd_loop_unready(s->loop, 10000.0);
  return RD_OK;
}

void rd_serve_destroy(rd_server_handle s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  rd_loop_destroy(s->loop);  // every request is done: the loop reads no handle any more
  for (auto& e : s->cache)
    if (e.second.h) rd_destroy(e.second.h);
  for (auto& e : s->jobs) delete e.second;
  for (cudaStream_t q : s->streams) {
    cudaStreamSynchronize(q);  // the handles' stream-ordered frees
    cudaStreamDestroy(q);
  }
  cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
