// k_build.cu -- operator build (M = I - gamma A, or I - gamma^W), the gain check, and the
// successor lists used by the greedy next hop.
//
// Sec. 2 (eq. Y-defined) and Sec. 3.2 (X = gamma^W elementwise).  The gain check computes,
// for every column j, the out-degree Delta_j = sum_i [A_ij != 0] (Theorem 2's definition of
// Delta) and, for weighted graphs, the column sum of X; the host accepts the gain when the
// largest column sum of X is below one (strict column diagonal dominance of M).
//
// The kernels are HBM-bound streams over the n x n byte matrix (and the N x N FP64 M): one
// thread per column walks down a block of rows, so a warp reads 32 consecutive bytes of a row
// per step and writes consecutive doubles of M.
#include "rd_internal.cuh"

namespace {

// M for the rows of one row block; per-column edge counts and column sums are added with atomics
// (the column sums only feed the gain check, so their summation order does not matter).
__global__ void build_m_kernel(const uint8_t* __restrict__ A, const float* __restrict__ W, int n, int N,
                               int rows_per_block, double gamma, double* __restrict__ M,
                               int32_t* __restrict__ deg, double* __restrict__ colsum) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // column of M
  if (j >= N) return;
  const int r0 = blockIdx.y * rows_per_block;
  const int r1 = min(N, r0 + rows_per_block);
  int cnt = 0;
  double cs = 0.0;
  for (int i = r0; i < r1; ++i) {
    double x = 0.0;
    if (i < n && j < n && A[(long long)i * n + j]) {
      ++cnt;
      x = W ? pow(gamma, (double)W[(long long)i * n + j]) : gamma;
      cs += x;
    }
    M[(long long)i * N + j] = (i == j ? 1.0 : 0.0) - x;
  }
  if (j < n && cnt) {
    atomicAdd(&deg[j], cnt);
    atomicAdd(&colsum[j], cs);
  }
}

// largest degree, largest column sum (bits of a non-negative double) and the edge count
__global__ void build_reduce_kernel(const int32_t* __restrict__ deg, const double* __restrict__ colsum, int n,
                                    unsigned long long* __restrict__ red) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  atomicMax(&red[0], (unsigned long long)deg[j]);
  atomicMax(&red[1], (unsigned long long)__double_as_longlong(colsum[j]));
  atomicAdd(&red[2], (unsigned long long)deg[j]);
}

// exclusive prefix sum of deg[0..n) into ptr[0..n] (single block; n is at most a few 10^5)
__global__ void scan_kernel(const int32_t* __restrict__ deg, int n, int32_t* __restrict__ ptr) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = t * per, e = min(n, b + per);
  long long s = 0;
  for (int i = b; i < e; ++i) s += deg[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      long long v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  long long run = part[t];
  for (int i = b; i < e; ++i) {
    ptr[i] = (int32_t)run;
    run += deg[i];
  }
  if (e == n && b < e) ptr[n] = (int32_t)run;
  if (n == 0 && t == 0) ptr[0] = 0;
}

// successors of node v: {j : A[j][v] != 0} (edge v -> j), ascending j
__global__ void succ_fill_kernel(const uint8_t* __restrict__ A, int n, const int32_t* __restrict__ ptr,
                                 int32_t* __restrict__ idx) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int w = ptr[v];
  for (int j = 0; j < n; ++j)
    if (A[(long long)j * n + v]) idx[w++] = j;
}

// Hop distances from sampled sources and their spread within chunks of consecutive nodes (the
// split path's range screen).  One CTA per source: a level-synchronous BFS along the successor
// lists (dist: n ints per source, -1 = not reached; at most n levels), then, one warp per chunk
// of `chunk` consecutive nodes, the spread max d - min d over the chunk's reached nodes.  The
// largest spread over chunks and sources is atomicMax-ed into *out.  Sources: nodes
// b n / nsrc + n / (2 nsrc), b = blockIdx.x.
__global__ void __launch_bounds__(1024) chunk_spread_kernel(const int32_t* __restrict__ ptr,
                                                            const int32_t* __restrict__ succ, int n,
                                                            int nsrc, int chunk, int32_t* __restrict__ dist,
                                                            unsigned long long* out) {
  const int b = blockIdx.x, t = threadIdx.x;
  const int src = (int)(((long long)b * n) / nsrc + (n / nsrc) / 2);
  int32_t* d = dist + (long long)b * n;
  for (int v = t; v < n; v += blockDim.x) d[v] = (v == src) ? 0 : -1;
  __syncthreads();
  for (int L = 0; L < n; ++L) {
    int grew = 0;
    for (int v = t; v < n; v += blockDim.x) {
      if (d[v] != L) continue;
      const int e1 = ptr[v + 1];
      for (int e = ptr[v]; e < e1; ++e) {
        const int w = succ[e];
        if (d[w] < 0) {  // every writer of this level writes the same L + 1
          d[w] = L + 1;
          grew = 1;
        }
      }
    }
    if (!__syncthreads_or(grew)) break;
  }
  const int warp = t >> 5, lane = t & 31, nwarps = blockDim.x >> 5;
  const int nch = (n + chunk - 1) / chunk;
  for (int c = warp; c < nch; c += nwarps) {
    int lo = 0x7fffffff, hi = -1;
    const int v1 = min(n, (c + 1) * chunk);
    for (int v = c * chunk + lane; v < v1; v += 32) {
      const int x = d[v];
      if (x >= 0) {
        lo = min(lo, x);
        hi = max(hi, x);
      }
    }
    for (int o = 16; o; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0 && hi >= 0) atomicMax(out, (unsigned long long)(hi - lo));
  }
}

__global__ void copy_rows_kernel(const double* __restrict__ R, long long ldr, int rows, int cols,
                                 double* __restrict__ out, long long ldo) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  const int r = (int)(t / cols), c = (int)(t % cols);
  out[(long long)r * ldo + c] = R[(long long)r * ldr + c];
}

}  // namespace

cudaError_t rd_build_m(rd_ctx* h, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h->dRed, 0, 3 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->dDeg, 0, (size_t)h->n * sizeof(int32_t), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(h->dColsum, 0, (size_t)h->n * sizeof(double), s)) != cudaSuccess) return e;
  const int threads = 128;
  const int row_blocks = 16;
  const int rows_per_block = (h->N + row_blocks - 1) / row_blocks;
  dim3 grid((h->N + threads - 1) / threads, row_blocks);
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  build_m_kernel<<<grid, threads, 0, s>>>(h->dA, h->weighted ? h->dW : nullptr, h->n, h->N, rows_per_block,
                                          h->gamma, h->dLU, h->dDeg, h->dColsum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  build_reduce_kernel<<<(h->n + 255) / 256, 256, 0, s>>>(h->dDeg, h->dColsum, h->n, h->dRed);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

cudaError_t rd_build_succ(rd_ctx* h, cudaStream_t s) {
  // ptr lives after the degrees: dDeg[0..n) degrees, dDeg[n+1 .. 2n+1] prefix
  int32_t* ptr = h->dDeg + (h->n + 1);
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  scan_kernel<<<1, 1024, 0, s>>>(h->dDeg, h->n, ptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  succ_fill_kernel<<<(h->n + 127) / 128, 128, 0, s>>>(h->dA, h->n, ptr, h->dSucc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

cudaError_t rd_copy_rows_out(rd_ctx* h, const double* R, long long ldr, int rows, int cols,
                             double* out, long long ldo, cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  copy_rows_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(R, ldr, rows, cols,
                                                                                 out, ldo);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

cudaError_t rd_chunk_spread(rd_ctx* h, int nsrc, int chunk, int32_t* dist, unsigned long long* out,
                            cudaStream_t s) {
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  chunk_spread_kernel<<<nsrc, 1024, 0, s>>>(h->dDeg + (h->n + 1), h->dSucc, h->n, nsrc, chunk, dist, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}
