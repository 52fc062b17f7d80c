// k_update.cu -- incremental edge updates of a resident Y (Sherman-Morrison).
//
// Changing X_ij (the edge j -> i) by delta changes M = I - X by -delta e_i e_j^T, so
//   Y' = (M - delta e_i e_j^T)^-1 = Y + alpha (Y e_i)(e_j^T Y),   alpha = delta / (1 - delta Y_ji)
// (Sherman-Morrison; 1 - delta Y_ji = det M' / det M > 0 while M' stays strictly column
// diagonally dominant).  One pass over Y (16 n^2 bytes: HBM bound) updates it in place and decodes
// D.  An added or strengthened edge (delta > 0) adds terms of one sign; a removed or weakened one
// subtracts, and an entry whose paths all used that edge cancels to a small difference: such
// entries (more than 20 bits lost) are counted, and the caller refactors instead.
#include "rd_internal.cuh"

namespace {

// u = Y[:, i], v = Y[j, :], and alpha = delta / (1 - delta Y_ji) at uv[2n]
__global__ void gather_uv_kernel(const double* __restrict__ Y, int n, int i, int j, double delta, double* uv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    uv[t] = Y[(long long)t * n + i];
    uv[n + t] = Y[(long long)j * n + t];
  }
  if (t == 0) uv[2 * n] = delta / (1.0 - delta * Y[(long long)j * n + i]);
}

// one entry: y = y0 + (alpha u_r) v_c as one FMA (the only FP64 instruction: GB300's FP64 pipe
// retires 2 per clock per SM, which would otherwise bound the pass), the cancellation count and
// the decode.  u, v >= 0, so the term's sign is the row's (neg); the tests on y compare the bit
// patterns of non-negative doubles as integers: y < y0 2^-20 when the exponent fell by more than
// 20 (y0 normal), y < 0 when the sign bit is set.
__device__ __forceinline__ void rank1_entry(double y0, double ar, double vc, bool neg, bool diag,
                                            float inv_log2_gamma, double log_gamma, double tau, double* y_out,
                                            int32_t* d_out, unsigned int* bad) {
  double y = fma(ar, vc, y0);
  if (neg) {
    const long long by = __double_as_longlong(y), b0 = __double_as_longlong(y0);
    if (by < b0 - (20ll << 52)) {  // cancellation: the entry kept fewer than ~33 bits
      ++*bad;
      if (by < 0) y = 0.0;
    }
  }
  *y_out = y;
  *d_out = diag ? 0 : rd_decode_entry_fast(y, inv_log2_gamma, log_gamma, tau);
}

// Y += alpha u v^T with the decode of D, row by row (a CTA per row in turn); with vec (n even and
// D 8-byte aligned; Y and u, v are the library's own, 256-byte aligned) two entries per access:
// 16-byte loads and stores of Y, 8-byte stores of D (rows start at 8 n and 4 n bytes).  HBM bound: 20 bytes per entry (read Y, write Y, write D); v stays in L2.
__global__ void __launch_bounds__(256) rank1_decode_kernel(double* __restrict__ Y, const double* __restrict__ uv,
                                                           int n, int32_t* __restrict__ D, float inv_log2_gamma,
                                                           double log_gamma, double tau, int vec,
                                                           unsigned int* lost) {
  const double alpha = uv[2 * n];
  const double* __restrict__ v = uv + n;
  unsigned int bad = 0;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const double ar = alpha * uv[r];
    const bool neg = __double_as_longlong(ar) < 0;
    double* yr = Y + (long long)r * n;
    int32_t* dr = D + (long long)r * n;
    if (vec) {
      for (int c = 2 * threadIdx.x; c < n; c += 2 * blockDim.x) {
        const double2 y0 = *reinterpret_cast<const double2*>(yr + c);
        const double2 vc = *reinterpret_cast<const double2*>(v + c);
        double2 y;
        int2 d;
        rank1_entry(y0.x, ar, vc.x, neg, r == c, inv_log2_gamma, log_gamma, tau, &y.x, &d.x, &bad);
        rank1_entry(y0.y, ar, vc.y, neg, r == c + 1, inv_log2_gamma, log_gamma, tau, &y.y, &d.y, &bad);
        *reinterpret_cast<double2*>(yr + c) = y;
        *reinterpret_cast<int2*>(dr + c) = d;
      }
    } else {
      for (int c = threadIdx.x; c < n; c += blockDim.x)
        rank1_entry(yr[c], ar, v[c], neg, r == c, inv_log2_gamma, log_gamma, tau, &yr[c], &dr[c], &bad);
    }
  }
  for (int o = 16; o; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(lost, bad);
}

__global__ void set_edge_kernel(uint8_t* A, float* W, double* colsum, int32_t* deg, int n, int i, int j,
                                uint8_t present, float w, double delta, int ddeg) {
  A[(long long)i * n + j] = present;
  if (W) W[(long long)i * n + j] = present ? w : 0.f;
  colsum[j] += delta;
  deg[j] += ddeg;  // out-degree of j: the successor lists are rebuilt from it
}

// Y rows goals[c] into out (k x n)
__global__ void rows_from_y_kernel(const double* __restrict__ Y, int n, const int32_t* __restrict__ goals, int k,
                                   double* __restrict__ out, int* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)k * n) return;
  const int c = (int)(t / n), col = (int)(t % n);
  const int32_t g = goals[c];
  if (!(g >= 0 && g < n)) {  // a goal outside [0, n): recorded, its row left zero
    if (col == 0) rd_goal_ok(g, n, c, status);
    out[t] = 0.0;
    return;
  }
  out[t] = Y[(long long)g * n + col];
}

}  // namespace

cudaError_t rd_rank1_update(rd_ctx* h, int i, int j, double delta, int32_t* D, unsigned int* lost, cudaStream_t s) {
  const int n = h->n;
  double* uv = h->dR;  // 64 x N doubles >= 2 n + 1
  cudaError_t e = cudaMemsetAsync(lost, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  gather_uv_kernel<<<(n + 255) / 256, 256, 0, s>>>(h->dYres, n, i, j, delta, uv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_UPDATE)) != cudaSuccess) return e;
  const int grid = n < 152 * 8 ? n : 152 * 8;  // 8 CTAs of 256 threads per SM, a row each in turn
  const int vec = (n % 2 == 0) && ((uintptr_t)D % 8 == 0);
  rank1_decode_kernel<<<grid, 256, 0, s>>>(h->dYres, uv, n, D, (float)(1.0 / log2(h->gamma)), log(h->gamma), h->tau,
                                           vec, lost);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_UPDATE, 20.0 * (double)n * (double)n);
}

cudaError_t rd_set_edge(rd_ctx* h, int i, int j, uint8_t present, float w, double delta, int ddeg,
                        cudaStream_t s) {
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  set_edge_kernel<<<1, 1, 0, s>>>(h->dA, h->weighted ? h->dW : nullptr, h->dColsum, h->dDeg, h->n, i, j, present, w,
                                  delta, ddeg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

cudaError_t rd_rows_from_y(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s) {
  const long long total = (long long)k * h->n;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  rows_from_y_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(h->dYres, h->n, dgoals, k, out, h->dStatus);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}
