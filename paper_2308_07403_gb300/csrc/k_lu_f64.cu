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

// LU of the B x B diagonal block at (k0, k0) of LU (in place), then the inverses of its unit
// lower factor and of its upper factor, written to the same block of T (strict lower = L^-1,
// upper = U^-1).  One CTA of 256 threads; thread t keeps the 4 x 4 tile at rows 4 (t / 16),
// columns 4 (t % 16) of every matrix in registers.  Each elimination step publishes the pivot
// row and column through shared memory (double-buffered, so one barrier per step) and one
// thread forms the reciprocal of the pivot.  The two triangular inverses run in the same
// 64-step loop: L^-1 by forward elimination (step q), U^-1 by back substitution (step 63 - q).
__global__ void __launch_bounds__(256) lu_diag_kernel(double* __restrict__ LU, double* __restrict__ T,
                                                      long long ld, int k0, int* status) {
  __shared__ double rowb[2][B], colb[2][B], recip[2];
  __shared__ double xrow[2][B], lcol[2][B], zrow[2][B], ucol[2][B], zrecip[2];
  const int t = threadIdx.x;
  const int r0 = 4 * (t / 16), c0 = 4 * (t % 16);
  double a[4][4];
  double* blk = LU + (long long)k0 * ld + k0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a[i][j] = blk[(long long)(r0 + i) * ld + c0 + j];

  // ---- LU without pivoting
  for (int k = 0; k < B; ++k) {
    const int bf = k & 1;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      if (r0 + ii != k) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        rowb[bf][c0 + j] = a[ii][j];
        if (c0 + j == k) {
          const double p = a[ii][j];
          const bool ok = (p > 0.0) && isfinite(p);
          if (!ok) rd_set_status(status, RD_DEV_PIVOT, k0 + k);
          recip[bf] = ok ? 1.0 / p : 0.0;
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (c0 + jj != k) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) colb[bf][r0 + i] = a[i][jj];
    }
    __syncthreads();
    const double ip = recip[bf];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gi = r0 + i;
      if (gi <= k) continue;
      const double l = colb[bf][gi] * ip;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gj = c0 + j;
        if (gj > k) a[i][j] = fma(-l, rowb[bf][gj], a[i][j]);
        else if (gj == k) a[i][j] = l;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) blk[(long long)(r0 + i) * ld + c0 + j] = a[i][j];

  // ---- L^-1 (x) and U^-1 (z), both starting from the identity
  double x[4][4], z[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) x[i][j] = z[i][j] = (r0 + i == c0 + j) ? 1.0 : 0.0;
  for (int st = 0; st < B; ++st) {
    const int bf = st & 1;
    const int q1 = st, q2 = B - 1 - st;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      if (r0 + ii == q1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) xrow[bf][c0 + j] = x[ii][j];
      }
      if (r0 + ii == q2) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          zrow[bf][c0 + j] = z[ii][j];
          if (c0 + j == q2) zrecip[bf] = 1.0 / a[ii][j];
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (c0 + jj == q1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) lcol[bf][r0 + i] = a[i][jj];
      }
      if (c0 + jj == q2) {
#pragma unroll
        for (int i = 0; i < 4; ++i) ucol[bf][r0 + i] = a[i][jj];
      }
    }
    __syncthreads();
    const double dq = zrecip[bf];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gi = r0 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gj = c0 + j;
        if (gi > q1 && gj <= q1) x[i][j] = fma(-lcol[bf][gi], xrow[bf][gj], x[i][j]);
        if (gj >= q2) {
          if (gi < q2)
            z[i][j] = fma(-ucol[bf][gi], zrow[bf][gj] * dq, z[i][j]);
          else if (gi == q2)
            z[i][j] *= dq;
        }
      }
    }
  }
  double* tb = T + (long long)k0 * ld + k0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) tb[(long long)(r0 + i) * ld + c0 + j] = (r0 + i > c0 + j) ? x[i][j] : z[i][j];
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
  if ((e = rd_prof_begin(h, s, false)) != cudaSuccess) return e;
  lu_diag_kernel<<<1, 256, 0, s>>>(h->dLU, h->dT, h->N, k0, h->dStatus);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, false, 0.0);
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
