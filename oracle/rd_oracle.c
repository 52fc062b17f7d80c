/*
 * rd_oracle.c -- plain, slow, single-threaded CPU reference of the R-distance method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this library.  It shares no code, header, table or helper with the CUDA
 * library in paper_2308_07403_gb300/csrc, and the CUDA path never calls it.
 *
 * What it computes (Jing & Meister, "A fast algorithm for All-Pairs-Shortest-Paths suitable
 * for neural networks"):
 *   Sec. 2, adjacency definition: A[i][j] != 0 iff edge j -> i (the transposed convention).
 *   Sec. 2, Y-defined / Sec. 3.1, inverse:   Y = (I - gamma A)^-1.
 *   Sec. 3.2:                                Y = (I - X)^-1 with X = gamma^W elementwise.
 *   Sec. 2, R-defined and Sec. 4.1, rounded-distance-function:  D = ceil(log_gamma Y).
 *   Sec. 3.1, Y-series:                      Y = sum_k gamma^k A^k  (series fixpoint below).
 *   Sec. 3.1, D-defined and shortest-path counts S (BFS below).
 *   Sec. 4.2, descent rule:                  next hop = argmax over successors of Y[g][j].
 *
 * Y is the plain definition of a matrix inverse, so the dense oracle is that definition
 * written out: an unblocked right-looking LU without pivoting (M is strictly column
 * diagonally dominant when gamma * Delta < 1, so no pivoting is needed and every pivot is
 * positive), followed by one forward and one back substitution per column of the identity.
 * No blocking, fusion or reordering.
 *
 * Readings where the paper is silent (listed with the rest in the design notes):
 *   - decode snap: D = ceil(log(Y)/log(gamma) - tau).  The paper writes the plain ceil; when
 *     Y is an exact power of gamma (a unique path with no longer walks) R is an integer in
 *     exact arithmetic and rounding would flip the ceil.  tau (1e-9 by default) absorbs that.
 *   - diagonal D[i][i] is forced to 0; Y <= 0 (unreachable, or underflow below the smallest
 *     double, Sec. 5.1) decodes to RDO_UNREACHABLE (INT32_MAX); a decoded value that would
 *     not fit in int32 is clamped to INT32_MAX - 1.
 *   - any nonzero byte of A counts as an edge.
 *
 * Built with -ffp-contract=off so x86-64 and aarch64 hosts produce the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RDO_UNREACHABLE INT32_MAX

/* ---- operator ----------------------------------------------------------------------- */

/* M = I - gamma * [A != 0]   (Sec. 2, Y-defined).  Row-major n x n. */
void rdo_build_m(const uint8_t* A, int64_t n, double gamma, double* M) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double x = A[i * n + j] ? gamma : 0.0;
      M[i * n + j] = (i == j ? 1.0 : 0.0) - x;
    }
}

/* M = I - X, X[i][j] = gamma^W[i][j] where A[i][j] != 0, else 0   (Sec. 3.2). */
void rdo_build_m_weighted(const uint8_t* A, const float* W, int64_t n, double gamma, double* M) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double x = A[i * n + j] ? pow(gamma, (double)W[i * n + j]) : 0.0;
      M[i * n + j] = (i == j ? 1.0 : 0.0) - x;
    }
}

/* Largest column sum of X = I - M (off the identity): sum_i X[i][j].  For the unweighted
 * operator this is gamma * Delta, Delta the largest out-degree (Theorem 2's definition). */
double rdo_max_column_sum(const double* M, int64_t n) {
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double x = (i == j ? 1.0 : 0.0) - M[i * n + j];
      s += x;
    }
    if (s > best) best = s;
  }
  return best;
}

/* ---- dense inverse -------------------------------------------------------------------- */

/* In-place LU without pivoting: on return the strict lower triangle holds L (unit diagonal
 * implied) and the upper triangle holds U, with M = L U.  Returns 0, or k+1 if pivot k is not
 * a positive finite number. */
int64_t rdo_lu_nopivot(double* M, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    double p = M[k * n + k];
    if (!(p > 0.0) || !isfinite(p)) return k + 1;
    for (int64_t i = k + 1; i < n; ++i) M[i * n + k] = M[i * n + k] / p;
    for (int64_t i = k + 1; i < n; ++i) {
      double l = M[i * n + k];
      if (l == 0.0) continue;
      double* row = M + i * n;
      const double* prow = M + k * n;
      for (int64_t j = k + 1; j < n; ++j) row[j] = row[j] - l * prow[j];
    }
  }
  return 0;
}

/* Y = M^-1 from the LU factors: for each column j of the identity, forward substitution
 * with the unit lower L, then back substitution with U. */
void rdo_inverse_from_lu(const double* LU, int64_t n, double* Y) {
  double* z = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double* y = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int64_t k = j; k < i; ++k) s = s - LU[i * n + k] * z[k];
      z[i] = (i < j) ? 0.0 : s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = z[i];
      for (int64_t k = i + 1; k < n; ++k) s = s - LU[i * n + k] * y[k];
      y[i] = s / LU[i * n + i];
    }
    for (int64_t i = 0; i < n; ++i) Y[i * n + j] = y[i];
  }
  free(z);
  free(y);
}

/* Rows g of Y for each goal: solve M^T y = e_g as U^T w = e_g (forward), L^T y = w (back).
 * Out[c*n + j] = Y[goals[c]][j]. */
void rdo_goal_rows(const double* LU, int64_t n, const int32_t* goals, int64_t k, double* out) {
  double* w = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (int64_t c = 0; c < k; ++c) {
    int64_t g = goals[c];
    double* y = out + c * n;
    for (int64_t i = 0; i < n; ++i) {
      double s = (i == g) ? 1.0 : 0.0;
      for (int64_t q = 0; q < i; ++q) s = s - LU[q * n + i] * w[q];
      w[i] = s / LU[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = w[i];
      for (int64_t q = i + 1; q < n; ++q) s = s - LU[q * n + i] * y[q];
      y[i] = s;
    }
  }
  free(w);
}

/* ---- decode --------------------------------------------------------------------------- */

static int32_t decode_one(double y, double lg, double tau) {
  if (!(y > 0.0)) return RDO_UNREACHABLE;
  double r = log(y) / lg - tau;
  double c = ceil(r);
  if (c >= 2147483646.0) return RDO_UNREACHABLE - 1;
  if (c <= -2147483647.0) return -2147483647;
  return (int32_t)c;
}

/* D[i][j] = ceil(log(Y[i][j]) / log(gamma) - tau), D[i][i] = 0, sentinel for Y <= 0.
 * Returns the number of non-finite Y entries (those decode to the sentinel as well). */
int64_t rdo_decode(const double* Y, int64_t n, double gamma, double tau, int32_t* D) {
  double lg = log(gamma);
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double y = Y[i * n + j];
      if (!isfinite(y)) {
        ++bad;
        D[i * n + j] = RDO_UNREACHABLE;
        continue;
      }
      D[i * n + j] = (i == j) ? 0 : decode_one(y, lg, tau);
    }
  return bad;
}

/* Decode one vector y of length n that is row (or column) `diag` of Y: same rule as
 * rdo_decode, with entry `diag` forced to 0. */
void rdo_decode_vector(const double* y, int64_t n, int64_t diag, double gamma, double tau,
                       int32_t* D) {
  double lg = log(gamma);
  for (int64_t j = 0; j < n; ++j)
    D[j] = (j == diag) ? 0 : (isfinite(y[j]) ? decode_one(y[j], lg, tau) : RDO_UNREACHABLE);
}

/* Whole method: build M, LU, inverse, decode.  Y_out may be NULL.
 * Returns 0, -1 on allocation failure, -2 on non-finite Y, or k+1 for a bad pivot k. */
int64_t rdo_rdistance(const uint8_t* A, const float* W, int64_t n, double gamma, double tau,
                      int32_t* D, double* Y_out) {
  size_t nn = (size_t)n * (size_t)n;
  double* M = (double*)malloc((nn ? nn : 1) * sizeof(double));
  double* Y = Y_out ? Y_out : (double*)malloc((nn ? nn : 1) * sizeof(double));
  if (!M || !Y) {
    free(M);
    if (!Y_out) free(Y);
    return -1;
  }
  if (W)
    rdo_build_m_weighted(A, W, n, gamma, M);
  else
    rdo_build_m(A, n, gamma, M);
  int64_t st = rdo_lu_nopivot(M, n);
  if (st == 0) {
    rdo_inverse_from_lu(M, n, Y);
    if (rdo_decode(Y, n, gamma, tau, D) != 0) st = -2;
  }
  free(M);
  if (!Y_out) free(Y);
  return st;
}

/* ---- sparse helpers ------------------------------------------------------------------- */

typedef struct {
  int64_t* ptr; /* n+1 */
  int32_t* idx;
  float* w; /* NULL when unweighted */
} adjlist;

/* by_row = 1: list k with A[v][k] != 0 (in-neighbours of v: edges k -> v).
 * by_row = 0: list k with A[k][v] != 0 (out-neighbours of v: edges v -> k). */
static int build_adj(const uint8_t* A, const float* W, int64_t n, int by_row, adjlist* g) {
  g->ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g->ptr) return -1;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      if (A[i * n + j]) g->ptr[(by_row ? i : j) + 1]++;
  for (int64_t v = 0; v < n; ++v) g->ptr[v + 1] += g->ptr[v];
  int64_t nnz = g->ptr[n];
  g->idx = (int32_t*)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
  g->w = W ? (float*)malloc((size_t)(nnz ? nnz : 1) * sizeof(float)) : NULL;
  int64_t* fill = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  if (!g->idx || !fill || (W && !g->w)) return -1;
  memcpy(fill, g->ptr, (size_t)n * sizeof(int64_t));
  if (by_row) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j)
        if (A[i * n + j]) {
          int64_t p = fill[i]++;
          g->idx[p] = (int32_t)j;
          if (W) g->w[p] = W[i * n + j];
        }
  } else {
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < n; ++i)
        if (A[i * n + j]) {
          int64_t p = fill[j]++;
          g->idx[p] = (int32_t)i;
          if (W) g->w[p] = W[i * n + j];
        }
  }
  free(fill);
  return 0;
}

static void free_adj(adjlist* g) {
  free(g->ptr);
  free(g->idx);
  free(g->w);
}

/* Partial sums of the series Y = sum_k X^k (Sec. 3.1, Y-series; Sec. 3.2 for X = gamma^W),
 * applied to one unit vector, iterated until the partial sum stops changing in FP64:
 *   transpose = 0:  y <- e_j + X y      converges to column j of Y   (y_i = Y[i][j])
 *   transpose = 1:  y <- e_j + X^T y    converges to row j of Y      (y_i = Y[j][i])
 * Every term is non-negative and the iterates are non-decreasing, so the loop reaches a
 * fixpoint.  Returns the iteration count, or -1 if max_iter was reached first. */
int64_t rdo_series_vector(const uint8_t* A, const float* W, int64_t n, double gamma, int64_t j,
                          int transpose, int64_t max_iter, double* y) {
  adjlist g;
  if (build_adj(A, W, n, transpose ? 0 : 1, &g) != 0) return -2;
  double* xv = (double*)malloc((size_t)(g.ptr[n] ? g.ptr[n] : 1) * sizeof(double));
  for (int64_t p = 0; p < g.ptr[n]; ++p) xv[p] = W ? pow(gamma, (double)g.w[p]) : gamma;
  double* nxt = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
  for (int64_t i = 0; i < n; ++i) y[i] = (i == j) ? 1.0 : 0.0;
  int64_t it = 0;
  int64_t result = -1;
  while (it < max_iter) {
    ++it;
    int changed = 0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t p = g.ptr[i]; p < g.ptr[i + 1]; ++p) s = s + xv[p] * y[g.idx[p]];
      double v = ((i == j) ? 1.0 : 0.0) + s;
      nxt[i] = v;
      if (v != y[i]) changed = 1;
    }
    memcpy(y, nxt, (size_t)n * sizeof(double));
    if (!changed) {
      result = it;
      break;
    }
  }
  free(nxt);
  free(xv);
  free_adj(&g);
  return result;
}

/* Breadth-first search along out-edges (edge v -> i iff A[i][v] != 0) from each source.
 * dist[s*n + i] = shortest distance from srcs[s] to i  (= D[i][srcs[s]], Sec. 3.1 D-defined),
 * count[s*n + i] = number of distinct shortest paths (= S[i][srcs[s]]), as a double
 * (exact below 2^53).  Unreachable: dist = INT32_MAX, count = 0. */
int rdo_bfs(const uint8_t* A, int64_t n, const int32_t* srcs, int64_t nsrc, int32_t* dist,
            double* count) {
  adjlist g;
  if (build_adj(A, NULL, n, 0, &g) != 0) return -1;
  int32_t* queue = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  for (int64_t s = 0; s < nsrc; ++s) {
    int32_t* d = dist + s * n;
    double* c = count ? count + s * n : NULL;
    for (int64_t i = 0; i < n; ++i) {
      d[i] = RDO_UNREACHABLE;
      if (c) c[i] = 0.0;
    }
    int32_t src = srcs[s];
    d[src] = 0;
    if (c) c[src] = 1.0;
    int64_t head = 0, tail = 0;
    queue[tail++] = src;
    while (head < tail) {
      int32_t v = queue[head++];
      for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) {
        int32_t i = g.idx[p];
        if (d[i] == RDO_UNREACHABLE) {
          d[i] = d[v] + 1;
          queue[tail++] = i;
        }
        if (c && d[i] == d[v] + 1) c[i] = c[i] + c[v];
      }
    }
  }
  free(queue);
  free_adj(&g);
  return 0;
}

/* Greedy next hop (Sec. 4.2, descent rule, run as ascent on Y as in Theorem 4's proof):
 * for goal g = goals[c] and node i, next[c*n + i] =
 *   g                                  if i == g or g is a successor of i,
 *   argmax_{j : edge i -> j} Yrows[c*n + j]   otherwise (smallest j among equal maxima),
 *   -1                                 if i has no successor. */
void rdo_greedy_next(const uint8_t* A, int64_t n, const int32_t* goals, int64_t k,
                     const double* Yrows, int32_t* next) {
  for (int64_t c = 0; c < k; ++c) {
    int64_t g = goals[c];
    const double* y = Yrows + c * n;
    for (int64_t i = 0; i < n; ++i) {
      int32_t best = -1;
      if (i == g || A[g * n + i]) {
        best = (int32_t)g;
      } else {
        for (int64_t j = 0; j < n; ++j) {
          if (!A[j * n + i] || j == i) continue;
          if (best < 0 || y[j] > y[best]) best = (int32_t)j;
        }
      }
      next[c * n + i] = best;
    }
  }
}

/* Dijkstra (weighted shortest distances from each source along out-edges), O(n^2) per
 * source with a linear scan for the minimum.  dist[s*n + i] = distance srcs[s] -> i,
 * +infinity when unreachable. */
int rdo_dijkstra(const uint8_t* A, const float* W, int64_t n, const int32_t* srcs, int64_t nsrc,
                 double* dist) {
  adjlist g;
  if (!W) return -1;
  if (build_adj(A, W, n, 0, &g) != 0) return -1;
  unsigned char* done = (unsigned char*)malloc((size_t)(n ? n : 1));
  for (int64_t s = 0; s < nsrc; ++s) {
    double* d = dist + s * n;
    for (int64_t i = 0; i < n; ++i) {
      d[i] = INFINITY;
      done[i] = 0;
    }
    d[srcs[s]] = 0.0;
    for (;;) {
      int64_t v = -1;
      for (int64_t i = 0; i < n; ++i)
        if (!done[i] && d[i] < INFINITY && (v < 0 || d[i] < d[v])) v = i;
      if (v < 0) break;
      done[v] = 1;
      for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) {
        int32_t i = g.idx[p];
        double nd = d[v] + (double)g.w[p];
        if (nd < d[i]) d[i] = nd;
      }
    }
  }
  free(done);
  free_adj(&g);
  return 0;
}
