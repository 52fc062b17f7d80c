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

__global__ void rank1_decode_kernel(double* __restrict__ Y, const double* __restrict__ uv, int n, int32_t* D,
                                    float inv_log2_gamma, double log_gamma, double tau, unsigned int* lost) {
  const double alpha = uv[2 * n];
  unsigned int bad = 0;
  const long long nn = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    const double y0 = Y[e];
    const double t = alpha * uv[r] * uv[n + c];
    double y = y0 + t;
    if (t < 0.0 && y < y0 * 0x1p-20) {  // cancellation: the entry kept fewer than ~33 bits
      bad++;
      if (y < 0.0) y = 0.0;
    }
    Y[e] = y;
    D[e] = (r == c) ? 0 : rd_decode_entry_fast(y, inv_log2_gamma, log_gamma, tau);
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
                                   double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)k * n) return;
  const int c = (int)(t / n), col = (int)(t % n);
  out[t] = Y[(long long)goals[c] * n + col];
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
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  rank1_decode_kernel<<<1216, 256, 0, s>>>(h->dYres, uv, n, D, (float)(1.0 / log2(h->gamma)), log(h->gamma), h->tau,
                                           lost);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
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
  rows_from_y_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(h->dYres, h->n, dgoals, k, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}
