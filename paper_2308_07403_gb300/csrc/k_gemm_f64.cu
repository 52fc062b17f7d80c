// k_gemm_f64.cu -- the FP64 GEMM of the plain path.
//
// Every dense contraction of the plain path goes through this kernel: the trailing updates and
// the two panel products of the blocked LU, the off-diagonal products of the blocked
// triangular inverses, the final product Y = U^-1 L^-1 (with the R-distance decode fused into
// its epilogue), and the blocked goal solves.
//
// FP64 throughput on this part is two orders of magnitude below its BF16 tensor rate, so the
// kernel is bound by the FP64 pipe whatever the tiling: a 64x64 CTA tile with a 4x4 register
// micro-tile per thread and a 16-deep K step in shared memory keeps the pipe fed while the
// memory traffic stays three orders of magnitude below the HBM rate.  Small products (the low
// levels of the split path's recursion, the goal solves) switch to 32x32 or 16x16 tiles so that
// they still spread over every SM: with two FP64 FMAs per clock per SM, parallelism is what
// small FP64 products lack.
//
// Operands may be read through a "triangular view" of the packed storage: the strict lower
// part with an implied unit diagonal (L, L^-1) or the upper part including the diagonal
// (U, U^-1).  The view also bounds the K loop: a CTA skips the K range where its row (or
// column) strip of the triangular operand is zero, so triangular products cost what they
// should (n^3/3 for a triangle times a full matrix).
//
// In-place use: C may alias A's row strip or B's column strip of the same CTA (the panel
// products of the LU and the goal solves do this, flagged with `aliased`).  Every CTA reads all
// of its K range before its epilogue writes, and reads no other CTA's output, so this is safe
// when beta == 0 and one CTA owns the whole strip: aliased products keep the 64 x 64 tile.
#include "rd_internal.cuh"

namespace {

constexpr int BK = 16, NT = 256;

__device__ __forceinline__ double tri_load(const double* p, long long ld, int r, int c, int tri) {
  // r, c are indices inside the operand view; the view's diagonal is r == c
  if (tri == RD_TRI_LOWER_UNIT) {
    if (r < c) return 0.0;
    if (r == c) return 1.0;
  } else if (tri == RD_TRI_UPPER) {
    if (r > c) return 0.0;
  }
  return p[(long long)r * ld + c];
}

// T x T output tile per CTA (T = 64, 32 or 16), 256 threads on a 16 x 16 grid, each owning a
// (T/16) x (T/16) register micro-tile; K advances 16 at a time through shared memory with a
// register prefetch of the next step.
template <int T>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(rd_gemm_f64_args p0, rd_gemm_f64_args p1) {
  constexpr int R = T / 16;           // micro-tile edge
  constexpr int LA = T * BK / NT;     // elements of A (and of B) each thread stages per K step
  const rd_gemm_f64_args& p = (blockIdx.z == 0) ? p0 : p1;
  if (p.bg && p.bg[blockIdx.y].s == 0) return;  // a graph of a stacked batch without work in this pass
  // graph blockIdx.y of a stacked batch (strides 0 for one graph)
  const double* __restrict__ pA = p.A + (long long)blockIdx.y * p.a_gs;
  const double* __restrict__ pB = p.B + (long long)blockIdx.y * p.b_gs;
  double* pC = p.C + (long long)blockIdx.y * p.c_gs;
  const int tiles_n = p.N / T;
  const int tiles = (p.M / T) * tiles_n;
  const int tile = blockIdx.x;
  if (tile >= tiles) return;
  const int r0 = (tile / tiles_n) * T;
  const int c0 = (tile % tiles_n) * T;

  int kbeg = 0, kend = p.K;
  if (p.a_tri == RD_TRI_LOWER_UNIT) kend = min(kend, r0 + T);
  if (p.a_tri == RD_TRI_UPPER) kbeg = max(kbeg, r0);
  if (p.b_tri == RD_TRI_LOWER_UNIT) kbeg = max(kbeg, c0);
  if (p.b_tri == RD_TRI_UPPER) kend = min(kend, c0 + T);
  kbeg = kbeg / BK * BK;

  __shared__ double As[2][BK][T];
  __shared__ double Bs[2][BK][T];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // staging: A tile T rows x 16 k, B tile 16 k x T cols, LA consecutive elements per thread
  const int a_r = (tid * LA) / BK, a_k = (tid * LA) % BK;
  const int b_k = (tid * LA) / T, b_c = (tid * LA) % T;

  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;

  double ra[LA], rb[LA];
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      ra[e] = tri_load(pA, p.lda, r0 + a_r, k0 + a_k + e, p.a_tri);
      rb[e] = tri_load(pB, p.ldb, k0 + b_k, c0 + b_c + e, p.b_tri);
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      As[buf][a_k + e][a_r] = ra[e];
      Bs[buf][b_k][b_c + e] = rb[e];
    }
  };

  if (kbeg < kend) {
    load_regs(kbeg);
    store_regs(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = (k0 + BK) < kend;
      if (more) load_regs(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) {
        store_regs(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
  // every global read of this CTA's K range has been issued and consumed before any thread
  // reaches this barrier, so an epilogue that overwrites A's or B's strip is safe
  __syncthreads();

#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = r0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int c = c0 + tx + 16 * j;
      double v = p.alpha * acc[i][j];
      if (p.beta != 0.0) v = fma(p.beta, pC[(long long)r * p.ldc + c], v);
      if (p.store_c && r < p.c_rows && c < p.c_cols) pC[(long long)r * p.ldc + c] = v;
      if (p.D && r < p.d_rows && c < p.d_cols) {
        int32_t d;
        if (!isfinite(v)) {
          rd_set_status(p.status, RD_DEV_NONFINITE, r);
          d = RD_UNREACHABLE;
        } else {
          d = (r == c) ? 0 : rd_decode_entry(v, p.log_gamma, p.tau);
        }
        p.D[(long long)r * p.ldd + c] = d;
      }
    }
  }
}

}  // namespace

cudaError_t rd_gemm_f64(rd_ctx* h, const rd_gemm_f64_args* probs, int nprob, cudaStream_t s,
                        double flops) {
  if (nprob < 1 || nprob > 2) return cudaErrorInvalidValue;
  // the largest tile (64, 32 or 16) that still gives two waves of CTAs over the 152 SMs
  int T = 64;
  long long work = 0;
  bool aliased = false;
  // a stacked batch: every problem for every graph (graph 0's pointers, per-graph strides)
  rd_gemm_f64_args q[2];
  const int nb = h->nbatch > 1 ? h->nbatch : 1;
  for (int i = 0; i < nprob; ++i) {
    q[i] = probs[i];
    if (nb > 1) {
      if (q[i].D) return cudaErrorInvalidValue;  // no fused decode in stacked batches
      q[i].a_gs = rd_batch_stride(h, q[i].A);
      q[i].b_gs = rd_batch_stride(h, q[i].B);
      q[i].c_gs = rd_batch_stride(h, q[i].C);
      q[i].bg = h->dBatch;
    } else {
      q[i].a_gs = q[i].b_gs = q[i].c_gs = 0;
      q[i].bg = nullptr;
    }
  }
  probs = q;
  for (int i = 0; i < nprob; ++i) {
    const rd_gemm_f64_args& p = probs[i];
    if (p.M % 16 || p.N % 16 || p.K % BK || p.M < 0 || p.N < 0 || p.K < 0) return cudaErrorInvalidValue;
    if (p.M % 64 || p.N % 64) T = 16;
    if (p.aliased) {
      aliased = true;
      if (p.beta != 0.0 || (p.M != 64 && p.N != 64)) return cudaErrorInvalidValue;
    }
    work += (long long)p.M * p.N * nb;
  }
  if (aliased && T != 64) return cudaErrorInvalidValue;
  while (!aliased && T > 16 && work / ((long long)T * T) < 2 * 152) T /= 2;
  int maxtiles = 0;
  for (int i = 0; i < nprob; ++i) {
    const int t = (probs[i].M / T) * (probs[i].N / T);
    if (t > maxtiles) maxtiles = t;
  }
  if (maxtiles == 0) return cudaSuccess;
  dim3 grid(maxtiles, nb, nprob);
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_F64);
  if (e != cudaSuccess) return e;
  const rd_gemm_f64_args& q1 = nprob > 1 ? probs[1] : probs[0];
  if (T == 64)
    gemm_f64_kernel<64><<<grid, NT, 0, s>>>(probs[0], q1);
  else if (T == 32)
    gemm_f64_kernel<32><<<grid, NT, 0, s>>>(probs[0], q1);
  else
    gemm_f64_kernel<16><<<grid, NT, 0, s>>>(probs[0], q1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_F64, flops);
}
