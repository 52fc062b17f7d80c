// k_goal.cu -- goal rows of Y on the resident LU factors, and the greedy next hop.
//
// Local mode of the paper (Sec. 4.2): greedy descent on R toward goal g uses the g-th row of
// Y (Theorem 4's proof reads Y_gj for the neighbours j of the current node).  Row g of Y
// solves y^T M = e_g^T, i.e. M^T y = e_g; with M = L U this is two block triangular solves in
// row-vector form, run for up to 64 goals at once (the rows of R, 64 x N):
//   forward  (U):  for K = 0 ..:    R_K = R_K U_KK^-1 ;  R_J -= R_K U_KJ   (J > K)
//   backward (L):  for K = .. 0:    R_K = R_K L_KK^-1 ;  R_J -= R_K L_KJ   (J < K)
// The diagonal-block inverses come from the factorisation (packed in T).  Each step is one
// in-place 64x64 product and one 64 x (remaining) update on the FP64 GEMM kernel.
#include "rd_internal.cuh"

namespace {

constexpr int B = RD_BF;

__global__ void init_rhs_kernel(double* __restrict__ R, long long N, const int32_t* __restrict__ goals,
                                int k, int n, int* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= RD_MAX_GOALS * N) return;
  const int c = (int)(t / N);
  const long long j = t % N;
  const int g = c < k ? goals[c] : -1;
  if (c < k && j == 0) rd_goal_ok(g, n, c, status);  // a goal outside [0, n) leaves its row zero
  R[t] = (c < k && g == j && j < n) ? 1.0 : 0.0;
}

// next[c*n + i]: see rd_greedy_next in rd.h.  One thread per (goal, node).
__global__ void greedy_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ, int n,
                              const int32_t* __restrict__ goals, int k, const double* __restrict__ Y,
                              int32_t* __restrict__ next, int* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)k * n) return;
  const int c = (int)(t / n), i = (int)(t % n);
  const int g = goals[c];
  if (!(g >= 0 && g < n)) {  // a goal outside [0, n): no next hops for it
    if (i == 0) rd_goal_ok(g, n, c, status);
    next[t] = -1;
    return;
  }
  const double* y = Y + (long long)c * n;
  int best = -1;
  if (i == g) {
    best = g;
  } else {
    double bv = 0.0;
    bool hasg = false;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
      const int j = succ[q];
      if (j == g) hasg = true;
      if (j == i) continue;
      const double v = y[j];
      if (best < 0 || v > bv) {
        best = j;
        bv = v;
      }
    }
    if (hasg) best = g;
  }
  next[t] = best;
}

rd_gemm_f64_args blank() {
  rd_gemm_f64_args a{};
  a.store_c = 1;
  a.alpha = 1.0;
  return a;
}

}  // namespace

cudaError_t rd_goal_f64(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s) {
  const long long N = h->N;
  double* R = h->dR;
  const double* LU = h->dLU;
  const double* T = h->dT;
  const long long total = RD_MAX_GOALS * N;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  init_rhs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(R, N, dgoals, k, h->n, h->dStatus);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  const double fdiag_u = 2.0 * RD_MAX_GOALS * (B * (B + 1) / 2);
  const double fdiag_l = 2.0 * RD_MAX_GOALS * (B * (B - 1) / 2);
  const int nb = (int)(N / B);
  for (int K = 0; K < nb; ++K) {  // y^T U = e^T
    rd_gemm_f64_args p = blank();
    p.A = R + K * B; p.lda = N;
    p.B = T + (long long)K * B * N + K * B; p.ldb = N; p.b_tri = RD_TRI_UPPER;
    p.C = R + K * B; p.ldc = N;
    p.M = RD_MAX_GOALS; p.N = B; p.K = B; p.c_rows = RD_MAX_GOALS; p.c_cols = B; p.aliased = 1;
    if ((e = rd_gemm_f64(h, &p, 1, s, fdiag_u)) != cudaSuccess) return e;
    const int rest = (int)(N - (K + 1) * B);
    if (rest == 0) continue;
    rd_gemm_f64_args u = blank();
    u.A = R + K * B; u.lda = N;
    u.B = LU + (long long)K * B * N + (K + 1) * B; u.ldb = N;
    u.C = R + (K + 1) * B; u.ldc = N;
    u.M = RD_MAX_GOALS; u.N = rest; u.K = B; u.alpha = -1.0; u.beta = 1.0;
    u.c_rows = RD_MAX_GOALS; u.c_cols = rest;
    if ((e = rd_gemm_f64(h, &u, 1, s, 2.0 * RD_MAX_GOALS * B * rest)) != cudaSuccess) return e;
  }
  for (int K = nb - 1; K >= 0; --K) {  // y^T L = w^T
    rd_gemm_f64_args p = blank();
    p.A = R + K * B; p.lda = N;
    p.B = T + (long long)K * B * N + K * B; p.ldb = N; p.b_tri = RD_TRI_LOWER_UNIT;
    p.C = R + K * B; p.ldc = N;
    p.M = RD_MAX_GOALS; p.N = B; p.K = B; p.c_rows = RD_MAX_GOALS; p.c_cols = B; p.aliased = 1;
    if ((e = rd_gemm_f64(h, &p, 1, s, fdiag_l)) != cudaSuccess) return e;
    if (K == 0) continue;
    rd_gemm_f64_args u = blank();
    u.A = R + K * B; u.lda = N;
    u.B = LU + (long long)K * B * N; u.ldb = N;
    u.C = R; u.ldc = N;
    u.M = RD_MAX_GOALS; u.N = K * B; u.K = B; u.alpha = -1.0; u.beta = 1.0;
    u.c_rows = RD_MAX_GOALS; u.c_cols = K * B;
    if ((e = rd_gemm_f64(h, &u, 1, s, 2.0 * RD_MAX_GOALS * B * (K * B))) != cudaSuccess) return e;
  }
  return rd_copy_rows_out(h, R, N, k, h->n, out, h->n, s);
}

// The greedy walk of Sec. 4.2 toward goal c from start[c], one thread per goal: follow the next
// hops (next[c n + x], the output of the greedy step) until a node is its own next hop (the goal),
// a node has none (-1), or max_len steps.  path[c (max_len + 1) + t] = the node after t steps, -1
// past the end; len[c] = the steps taken to the goal, or -1 if the walk did not reach it.
__global__ void walk_kernel(const int32_t* __restrict__ next, int n, int k, const int32_t* __restrict__ start,
                            int max_len, int32_t* __restrict__ path, int32_t* __restrict__ len) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  int32_t* p = path + (long long)c * (max_len + 1);
  const int32_t* nx = next + (long long)c * n;
  int x = start[c];
  int t = 0, steps = -1;
  if (x >= 0 && x < n) {
    p[0] = x;
    for (; t <= max_len; ++t) {
      const int y = nx[x];
      if (y == x) {  // the goal: its own next hop
        steps = t;
        break;
      }
      if (y < 0 || y >= n || t == max_len) break;  // dead end, or out of steps
      x = y;
      p[t + 1] = x;
    }
    ++t;  // entries 0..t-1 are set
  }
  for (int q = (x >= 0 && x < n) ? t : 0; q <= max_len; ++q) p[q] = -1;
  len[c] = steps;
}

cudaError_t rd_walk(rd_ctx* h, const int32_t* dnext, int k, const int32_t* dstart, int max_len, int32_t* dpath,
                    int32_t* dlen, cudaStream_t s) {
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  walk_kernel<<<1, 64, 0, s>>>(dnext, h->n, k, dstart, max_len, dpath, dlen);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

cudaError_t rd_greedy(rd_ctx* h, const int32_t* dgoals, int k, const double* yrows, int32_t* next,
                      cudaStream_t s) {
  const long long total = (long long)k * h->n;
  if (total == 0) return cudaSuccess;
  const int32_t* ptr = h->dDeg + (h->n + 1);
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  greedy_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ptr, h->dSucc, h->n, dgoals, k, yrows,
                                                                next, h->dStatus);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}
