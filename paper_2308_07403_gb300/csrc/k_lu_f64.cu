// k_lu_f64.cu -- blocked no-pivot LU, blocked triangular inverses and the inverse product with
// the fused decode, in FP64 (the plain path).
//
// The R-distance needs Y = M^-1 with M = I - X (Sec. 2 eq. Y-defined; Sec. 3.2).  Under the
// gain condition max_j sum_i X_ij < 1 (checked at load) M is a strictly column diagonally
// dominant M-matrix, so:
//   * Gaussian elimination without pivoting is stable: every Schur complement stays column
//     diagonally dominant and every pivot is positive;
//   * L and U have non-positive off-diagonal entries, and L^-1 >= 0, U^-1 >= 0 entrywise;
//   * Y = U^-1 L^-1 is a product of non-negative matrices.
// Every product below therefore adds terms of one sign (the only subtractions are on the
// diagonal of the Schur complements, bounded by the dominance margin), which is what keeps the
// tiny entries of Y (gamma^d for distance d) accurate relative to themselves.
//
// Work (2 N^3 flops in total): LU 2/3 N^3, two triangular inverses 1/3 N^3 each, the product
// 2/3 N^3.  Block size RD_BF = 64.
#include "rd_internal.cuh"

namespace {

constexpr int B = RD_BF;

// LU of the B x B diagonal block at (k0, k0) of LU, in place (strict lower = the multipliers of
// L, upper = U), by rank-1 elimination without pivoting.  One CTA of 256 threads.
//
// The FP64 pipe of one SM retires about two FMAs per clock, so the block is bound by the number
// of warp-level FP64 instructions issued, live lanes or not.  Thread t owns the 16 elements
// (r + 16 a, c + 16 b), r = t / 16, c = t % 16, a, b in 0..3: a cyclic distribution, so the
// shrinking active window of the elimination stays spread over every thread.  The 64 steps run
// as four chunks of 16 (template KB = k / 16), which makes the slot indices compile-time; slots
// left of or above the window are never touched, and a slot row whose two warp rows (2w, 2w+1)
// are both done is skipped by the whole warp.  The pivot row and column are published through
// shared memory (double-buffered: one barrier per step), with the reciprocal of the pivot.
struct LeafLuShared {
  double row[2][B];
  double col[2][B];
  double rcp[2];
};

template <int KB>
__device__ __forceinline__ void leaf_lu_chunk(double (&a)[4][4], LeafLuShared& sm, int r, int c,
                                              int w, int k0, int* status) {
#pragma unroll 1
  for (int kk = 0; kk < 16; ++kk) {
    const int bf = kk & 1;
    if (r == kk) {
#pragma unroll
      for (int b = KB; b < 4; ++b) sm.row[bf][c + 16 * b] = a[KB][b];
      if (c == kk) {
        const double p = a[KB][KB];
        const bool ok = (p > 0.0) && isfinite(p);
        if (!ok) rd_set_status(status, RD_DEV_PIVOT, k0 + 16 * KB + kk);
        sm.rcp[bf] = ok ? 1.0 / p : 0.0;
      }
    }
    if (c == kk) {
#pragma unroll
      for (int i = KB; i < 4; ++i) sm.col[bf][r + 16 * i] = a[i][KB];
    }
    __syncthreads();
    const double rp = sm.rcp[bf];
    double u[4];
#pragma unroll
    for (int b = KB; b < 4; ++b) u[b] = sm.row[bf][c + 16 * b];
#pragma unroll
    for (int i = KB; i < 4; ++i) {
      if (i == KB && 2 * w + 1 <= kk) continue;  // no row of this warp below the pivot
      const bool live_r = (i > KB) || (r > kk);
      const double l = sm.col[bf][r + 16 * i] * rp;
#pragma unroll
      for (int b = KB; b < 4; ++b) {
        if (b == KB && kk == 15) continue;       // no column right of the pivot in this slot
        if (live_r && ((b > KB) || (c > kk))) a[i][b] = fma(-l, u[b], a[i][b]);
      }
      if (live_r && c == kk) a[i][KB] = l;
    }
  }
}

// (a stacked batch: graph blockIdx.x, its matrix gs doubles further, its status in bg)
__global__ void __launch_bounds__(256) leaf_lu_kernel(double* __restrict__ LU, long long ld, int k0,
                                                      int* status, long long gs, rd_batch_graph* bg) {
  static_assert(B == 64, "the leaf kernels are laid out for 64 x 64 blocks");
  __shared__ LeafLuShared sm;
  const int t = threadIdx.x, r = t >> 4, c = t & 15, w = t >> 5;
  if (bg) {
    if (bg[blockIdx.x].s == 0) return;  // no split work for this graph in this pass
    status = bg[blockIdx.x].status;
  }
  double* blk = LU + (long long)blockIdx.x * gs + (long long)k0 * ld + k0;
  double a[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int b = 0; b < 4; ++b) a[i][b] = blk[(long long)(r + 16 * i) * ld + c + 16 * b];
  leaf_lu_chunk<0>(a, sm, r, c, w, k0, status);
  leaf_lu_chunk<1>(a, sm, r, c, w, k0, status);
  leaf_lu_chunk<2>(a, sm, r, c, w, k0, status);
  leaf_lu_chunk<3>(a, sm, r, c, w, k0, status);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int b = 0; b < 4; ++b) blk[(long long)(r + 16 * i) * ld + c + 16 * b] = a[i][b];
}

// Inverses of the two triangular factors of the factored diagonal block at (k0, k0), written to
// the same block of T (strict lower = L^-1, upper = U^-1).  The 2 B columns are independent
// problems: column j of L^-1 solves L x = e_j by forward substitution, column j of U^-1 solves
// U z = e_j by back substitution.  One warp per column, lanes owning rows l and l + 32; each
// step's pivot entry reaches the warp by shuffle and the factor is read from shared memory
// (padded rows: column reads are conflict-free).  32 CTAs of 4 warps: CTAs 0..15 take the
// columns of L^-1, 16..31 those of U^-1, so the FP64 work is spread over 32 SMs.
// (a stacked batch: graph blockIdx.y, its matrices gs doubles further)
__global__ void __launch_bounds__(128) leaf_inv_kernel(const double* __restrict__ LU,
                                                       double* __restrict__ T, long long ld, int k0, long long gs,
                                                       const rd_batch_graph* bg) {
  __shared__ double f[B][B + 1];
  __shared__ double rcp[B];
  const int t = threadIdx.x, lane = t & 31;
  if (bg && bg[blockIdx.y].s == 0) return;
  LU += (long long)blockIdx.y * gs;
  T += (long long)blockIdx.y * gs;
  const double* blk = LU + (long long)k0 * ld + k0;
  for (int e = t; e < B * B; e += blockDim.x) f[e / B][e % B] = blk[(long long)(e / B) * ld + e % B];
  const bool lower = blockIdx.x < 16;
  __syncthreads();
  if (!lower && t < B) rcp[t] = 1.0 / f[t][t];
  __syncthreads();
  const int j = 4 * (blockIdx.x & 15) + (t >> 5);
  double x0 = (lane == j) ? 1.0 : 0.0, x1 = (lane + 32 == j) ? 1.0 : 0.0;
  double* tb = T + (long long)k0 * ld + k0;
  if (lower) {
    // x_i -= L_iq x_q for i > q, q = j .. B-2 (x_q is final once step q starts)
    for (int q = j; q < B - 1; ++q) {
      const double xq = __shfl_sync(0xffffffffu, q < 32 ? x0 : x1, q & 31);
      if (q < 31 && lane > q) x0 = fma(-f[lane][q], xq, x0);
      if (lane + 32 > q) x1 = fma(-f[lane + 32][q], xq, x1);
    }
    if (lane > j) tb[(long long)lane * ld + j] = x0;
    if (lane + 32 > j) tb[(long long)(lane + 32) * ld + j] = x1;
  } else {
    // z_q = z_q / U_qq, then z_i -= U_iq z_q for i < q, q = j .. 0
    for (int q = j; q >= 0; --q) {
      const double zq = __shfl_sync(0xffffffffu, q < 32 ? x0 : x1, q & 31) * rcp[q];
      if (lane == q) x0 = zq;
      if (lane + 32 == q) x1 = zq;
      if (lane < q) x0 = fma(-f[lane][q], zq, x0);
      if (q > 32 && lane + 32 < q) x1 = fma(-f[lane + 32][q], zq, x1);
    }
    if (lane <= j) tb[(long long)lane * ld + j] = x0;
    if (lane + 32 <= j) tb[(long long)(lane + 32) * ld + j] = x1;
  }
}

rd_gemm_f64_args blank() {
  rd_gemm_f64_args a{};
  a.store_c = 1;
  a.alpha = 1.0;
  a.beta = 0.0;
  return a;
}

}  // namespace

cudaError_t rd_lu_diag(rd_ctx* h, int k0, cudaStream_t s) {
  cudaError_t e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  const int nb = h->nbatch > 1 ? h->nbatch : 1;
  const long long gs = nb > 1 ? (long long)h->N * h->N : 0;
  leaf_lu_kernel<<<nb, 256, 0, s>>>(h->dLU, h->N, k0, h->dStatus, gs, nb > 1 ? h->dBatch : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  leaf_inv_kernel<<<dim3(32, nb), 128, 0, s>>>(h->dLU, h->dT, h->N, k0, gs, nb > 1 ? h->dBatch : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

// Right-looking blocked LU: for each diagonal block k, factor it (and invert its factors),
// form the row panel U_kR = L_kk^-1 M_kR and the column panel L_Rk = M_Rk U_kk^-1, then
// update the trailing matrix M_RR -= L_Rk U_kR.
cudaError_t rd_lu_f64(rd_ctx* h, cudaStream_t s) {
  const long long N = h->N;
  double* LU = h->dLU;
  double* T = h->dT;
  cudaError_t e;
  for (int k0 = 0; k0 < N; k0 += B) {
    if ((e = rd_lu_diag(h, k0, s)) != cudaSuccess) return e;
    const int rest = (int)(N - k0 - B);
    if (rest == 0) break;
    rd_gemm_f64_args pr[2];
    // row panel: C(B x rest) = Linv_kk (B x B, lower unit view of T) * M_kR, in place
    pr[0] = blank();
    pr[0].A = T + k0 * N + k0; pr[0].lda = N; pr[0].a_tri = RD_TRI_LOWER_UNIT;
    pr[0].B = LU + k0 * N + k0 + B; pr[0].ldb = N;
    pr[0].C = LU + k0 * N + k0 + B; pr[0].ldc = N;
    pr[0].M = B; pr[0].N = rest; pr[0].K = B;
    pr[0].c_rows = B; pr[0].c_cols = rest; pr[0].aliased = 1;
    // column panel: C(rest x B) = M_Rk * Uinv_kk (upper view of T), in place
    pr[1] = blank();
    pr[1].A = LU + (k0 + B) * N + k0; pr[1].lda = N;
    pr[1].B = T + k0 * N + k0; pr[1].ldb = N; pr[1].b_tri = RD_TRI_UPPER;
    pr[1].C = LU + (k0 + B) * N + k0; pr[1].ldc = N;
    pr[1].M = rest; pr[1].N = B; pr[1].K = B;
    pr[1].c_rows = rest; pr[1].c_cols = B; pr[1].aliased = 1;
    const double fpan = 2.0 * rest * (B * (B - 1) / 2 + B * (B + 1) / 2);
    if ((e = rd_gemm_f64(h, pr, 2, s, fpan)) != cudaSuccess) return e;
    // trailing update
    rd_gemm_f64_args tu = blank();
    tu.A = LU + (k0 + B) * N + k0; tu.lda = N;
    tu.B = LU + k0 * N + k0 + B; tu.ldb = N;
    tu.C = LU + (k0 + B) * N + k0 + B; tu.ldc = N;
    tu.M = rest; tu.N = rest; tu.K = B;
    tu.alpha = -1.0; tu.beta = 1.0;
    tu.c_rows = rest; tu.c_cols = rest;
    if ((e = rd_gemm_f64(h, &tu, 1, s, 2.0 * rest * (double)rest * B)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Blocked triangular inverses by recursive halving of the diagonal range [lo, hi):
//   L = [[L11, 0], [L21, L22]]  ->  L^-1 = [[X11, 0], [-X22 L21 X11, X22]]
//   U = [[U11, U12], [0, U22]]  ->  U^-1 = [[V11, -V11 U12 V22], [0, V22]]
// The diagonal 64-blocks were inverted by the LU's diagonal kernel.  Each level runs the L and
// U products of a node in one launch (two problems).
static cudaError_t trtri_range(rd_ctx* h, int lo, int hi, cudaStream_t s) {
  if (hi - lo <= B) return cudaSuccess;
  const int half = ((hi - lo) / 2 + B - 1) / B * B;
  const int mid = lo + half;
  cudaError_t e;
  if ((e = trtri_range(h, lo, mid, s)) != cudaSuccess) return e;
  if ((e = trtri_range(h, mid, hi, s)) != cudaSuccess) return e;
  const long long N = h->N;
  const int m1 = mid - lo, m2 = hi - mid;
  double* LU = h->dLU;
  double* T = h->dT;
  double* SL = h->dS;                      // m2 x m1
  double* SU = h->dS + (long long)m1 * m2; // m1 x m2
  rd_gemm_f64_args p[2];
  // W_L = L21 (m2 x m1) * X11 (lower unit)
  p[0] = blank();
  p[0].A = LU + (long long)mid * N + lo; p[0].lda = N;
  p[0].B = T + (long long)lo * N + lo; p[0].ldb = N; p[0].b_tri = RD_TRI_LOWER_UNIT;
  p[0].C = SL; p[0].ldc = m1;
  p[0].M = m2; p[0].N = m1; p[0].K = m1; p[0].c_rows = m2; p[0].c_cols = m1;
  // W_U = U12 (m1 x m2) * V22 (upper)
  p[1] = blank();
  p[1].A = LU + (long long)lo * N + mid; p[1].lda = N;
  p[1].B = T + (long long)mid * N + mid; p[1].ldb = N; p[1].b_tri = RD_TRI_UPPER;
  p[1].C = SU; p[1].ldc = m2;
  p[1].M = m1; p[1].N = m2; p[1].K = m2; p[1].c_rows = m1; p[1].c_cols = m2;
  const double t1 = (double)m1 * (m1 + 1) / 2, t2 = (double)m2 * (m2 + 1) / 2;
  const double fl = 2.0 * (m2 * t1 + m1 * t2);  // a full block times a triangle, for L and U
  if ((e = rd_gemm_f64(h, p, 2, s, fl)) != cudaSuccess) return e;
  // X21 = -X22 (lower unit) * W_L ;  X12 = -V11 (upper) * W_U
  p[0] = blank();
  p[0].A = T + (long long)mid * N + mid; p[0].lda = N; p[0].a_tri = RD_TRI_LOWER_UNIT;
  p[0].B = SL; p[0].ldb = m1;
  p[0].C = T + (long long)mid * N + lo; p[0].ldc = N;
  p[0].M = m2; p[0].N = m1; p[0].K = m2; p[0].alpha = -1.0; p[0].c_rows = m2; p[0].c_cols = m1;
  p[1] = blank();
  p[1].A = T + (long long)lo * N + lo; p[1].lda = N; p[1].a_tri = RD_TRI_UPPER;
  p[1].B = SU; p[1].ldb = m2;
  p[1].C = T + (long long)lo * N + mid; p[1].ldc = N;
  p[1].M = m1; p[1].N = m2; p[1].K = m1; p[1].alpha = -1.0; p[1].c_rows = m1; p[1].c_cols = m2;
  return rd_gemm_f64(h, p, 2, s, fl);
}

cudaError_t rd_trtri_f64(rd_ctx* h, cudaStream_t s) { return trtri_range(h, 0, h->N, s); }

// Y = U^-1 L^-1 (upper view times lower-unit view of T; the K loop of tile (I, J) starts at
// max(I, J)) with the decode D = ceil(log(Y)/log(gamma) - tau) in the epilogue.
cudaError_t rd_trmm_decode_f64(rd_ctx* h, int32_t* D, double* Y, cudaStream_t s) {
  const long long N = h->N;
  rd_gemm_f64_args p = blank();
  p.A = h->dT; p.lda = N; p.a_tri = RD_TRI_UPPER;
  p.B = h->dT; p.ldb = N; p.b_tri = RD_TRI_LOWER_UNIT;
  p.M = (int)N; p.N = (int)N; p.K = (int)N;
  p.C = Y; p.ldc = h->n; p.store_c = Y != nullptr; p.c_rows = h->n; p.c_cols = h->n;
  p.D = D; p.ldd = h->n; p.d_rows = h->n; p.d_cols = h->n;
  p.log_gamma = log(h->gamma); p.tau = h->tau; p.status = h->dStatus;
  // sum over (i, j) of the N - max(i, j) products of the upper-times-lower product
  const double Nd = (double)N;
  return rd_gemm_f64(h, &p, 1, s, 2.0 * Nd * (Nd + 1) * (2 * Nd + 1) / 6.0);
}
