// rd_noalloc.cu -- rd_apsp_noalloc: the FP64 R-distance for small graphs without any device
// allocation.
//
// Who needs this: callers that may not call cudaMalloc at all -- a host application whose
// device memory is carved out up front by another runtime, a plugin that runs inside someone
// else's time-critical loop (cudaMalloc can synchronise the device and stall other streams),
// or a process that must keep its device footprint fixed after start-up.  The handle-based
// entry points allocate their workspace in rd_create; this one takes its workspace from a
// fixed array in device memory instead, and the caller passes only its own input and output.
//
// The scratch is one file-scope array, sized for graphs of at most RD_NOALLOC_MAX_N nodes: it
// holds M / the LU factors (N x N doubles), the triangular inverses (N x N), the scratch of
// the blocked triangular inverse (N x N / 2) and a few words of status, degrees and
// reductions -- 2.5 * 512^2 * 8 bytes + 16 KiB, about 5.3 MB.  Every GPU that loads the
// library holds this array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device address, so every
// call asks the runtime for the array's device address on the current device with
// cudaGetSymbolAddress (it allocates nothing).  Asking on every call, rather than caching the
// address per device, keeps the address right when the device's context is destroyed and made
// again (cudaDeviceReset), which loads the module again, possibly at another address.  The first
// call on a device also loads the library's module there (lazy loading), so make it before any
// stream capture.  Every call shares the one array: each call clears what must start at zero (the
// status and reduction words) and overwrites everything else before reading it, and two calls
// whose work overlaps on the GPU race on the array.
#include "rd_internal.cuh"

namespace {

constexpr int kMaxN = RD_NOALLOC_MAX_N;                       // n and N (padded) limit
constexpr size_t kMatDoubles = (size_t)kMaxN * kMaxN;          // one N x N f64 matrix
constexpr size_t kIntWords = 4096;                             // status, reductions, degrees
constexpr size_t kScratchDoubles = 2 * kMatDoubles + kMatDoubles / 2 + kIntWords / 2;

static __device__ __align__(256) double g_rd_noalloc_scratch[kScratchDoubles];

// device address of the scratch array on the current device (asked for on every call)
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_rd_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

rd_status fail(rd_status st, const std::string& msg) {
  rd_record_error(msg);  // readable through rd_last_error(NULL)
  return st;
}

#define NA_CK(call)                                                             \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess)                                                      \
      return fail(_e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA,   \
                  std::string(#call) + ": " + cudaGetErrorString(_e));          \
  } while (0)

}  // namespace

extern "C" rd_status rd_apsp_noalloc(const uint8_t* A, int32_t n, double gamma, int32_t* D,
                                     void* stream) {
  if (!A || !D) return fail(RD_ERR_ARG, "A and D must not be NULL");
  if (n < 1) return fail(RD_ERR_ARG, "n must be >= 1");
  if (n > kMaxN)
    return fail(RD_ERR_ARG, "n exceeds the fixed scratch of rd_apsp_noalloc (at most " +
                                std::to_string(kMaxN) + " nodes); use rd_create/rd_apsp");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(RD_ERR_GAMMA, "gamma must lie in (0, 1)");
  int dev = 0;
  NA_CK(cudaGetDevice(&dev));
  if (!on_device(A, dev) || !on_device(D, dev))
    return fail(RD_ERR_ARG, "A and D must be device memory of the current device");
  double* base = nullptr;
  NA_CK(scratch_address(&base));

  rd_ctx h;  // a view of the scratch; owns nothing
  h.device = dev;
  h.n = n;
  h.N = (n + RD_PAD - 1) / RD_PAD * RD_PAD;
  h.gamma = gamma;
  h.stream = (cudaStream_t)stream;
  const size_t NN = (size_t)h.N * h.N;
  h.dA = const_cast<uint8_t*>(A);
  h.dLU = base;
  h.dT = base + NN;
  h.dS = base + 2 * NN;
  int* words = reinterpret_cast<int*>(base + 2 * kMatDoubles + kMatDoubles / 2);
  h.dStatus = words;                                                     // 4 ints
  h.dRed = reinterpret_cast<unsigned long long*>(words + 8);             // 3 words
  h.dDeg = words + 16;                                                   // 2n + 2 ints
  h.dColsum = reinterpret_cast<double*>(words + 1280);                   // n doubles
  static_assert(16 + 2 * kMaxN + 2 <= 1280, "integer words do not fit");
  static_assert(1280 + 2 * kMaxN <= kIntWords, "column sums do not fit");

  NA_CK(cudaMemsetAsync(h.dStatus, 0, 4 * sizeof(int), h.stream));
  NA_CK(rd_build_m(&h, h.stream));
  unsigned long long red[3];
  NA_CK(cudaMemcpyAsync(red, h.dRed, sizeof(red), cudaMemcpyDeviceToHost, h.stream));
  NA_CK(cudaStreamSynchronize(h.stream));
  if (!(gamma * (double)red[0] < 1.0))
    return fail(RD_ERR_GAMMA, "gamma * Delta >= 1: M is not strictly column diagonally dominant");
  NA_CK(rd_lu_f64(&h, h.stream));
  NA_CK(rd_trtri_f64(&h, h.stream));
  NA_CK(rd_trmm_decode_f64(&h, D, nullptr, h.stream));
  int st[2] = {0, 0};
  NA_CK(cudaMemcpyAsync(st, h.dStatus, sizeof(st), cudaMemcpyDeviceToHost, h.stream));
  NA_CK(cudaStreamSynchronize(h.stream));
  switch (st[0]) {
    case RD_DEV_OK: return RD_OK;
    case RD_DEV_PIVOT: return fail(RD_ERR_NUMERIC, "non-positive pivot at row " + std::to_string(st[1]));
    case RD_DEV_NONFINITE: return fail(RD_ERR_NUMERIC, "non-finite entry of Y in row " + std::to_string(st[1]));
    case RD_DEV_TIMEOUT: return fail(RD_ERR_TIMEOUT, "a bounded device wait expired");
    default: return fail(RD_ERR_CUDA, "unexpected device status " + std::to_string(st[0]));
  }
}
