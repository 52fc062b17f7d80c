// k_build.cu -- operator build (M = I - gamma A, or I - gamma^W), the gain check, and the
// successor lists used by the greedy next hop.
//
// Sec. 2 (eq. Y-defined) and Sec. 3.2 (X = gamma^W elementwise).  The gain check computes,
// for every column j, the out-degree Delta_j = sum_i [A_ij != 0] (Theorem 2's definition of
// Delta) and, for weighted graphs, the column sum of X; the host accepts the gain when the
// largest column sum of X is below one (strict column diagonal dominance of M).
//
// The build is an HBM-bound stream over the n x n byte matrix (and the N x N FP64 M): one thread
// per column walks down a block of rows, so a warp reads 32 consecutive bytes of a row per step
// and writes consecutive doubles of M.  The successor lists (8 warps per 32 columns) serve the
// greedy next hop, the split path's range screen (chunk_spread_kernel: BFS or Bellman-Ford
// spreads), its locality order (landmark_kernel, rcb_kernel: landmark and scored bisections into
// 64-node parts, permute_m_kernel) and the spectral-radius bracket of Theorem 1's condition
// (spectral_step_kernel).
#include <vector>

#include <cstring>

#include "rd_internal.cuh"

namespace {

// M for the rows of one row block; per-column edge counts and column sums are added with atomics
// (the column sums only feed the gain check, so their summation order does not matter).
// the edge j -> i exists: A_ij != 0 and, on a weighted graph, a finite weight (W_ij = +inf is the
// weight of a missing edge, Sec. 3.2: gamma^inf = 0)
__device__ __forceinline__ bool edge_on(const uint8_t* __restrict__ A, const float* __restrict__ W, long long at) {
  return A[at] != 0 && (!W || W[at] < __int_as_float(0x7f800000));
}

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
    if (i < n && j < n && edge_on(A, W, (long long)i * n + j)) {
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

// successors of node v: {j : A[j][v] != 0} (edge v -> j), ascending j; with W, also the edge weights.
// A block owns 32 consecutive columns (lane = column): its 8 warps split the rows into 8 ranges,
// count each column's non-zeros per range, offset the ranges by a prefix over the warps, and write
// in a second pass, so the lists come out in ascending j with coalesced row reads.
__global__ void __launch_bounds__(256) succ_fill_kernel(const uint8_t* __restrict__ A, const float* __restrict__ W,
                                                        int n, const int32_t* __restrict__ ptr,
                                                        int32_t* __restrict__ idx, float* __restrict__ wt) {
  __shared__ int cnt[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v = blockIdx.x * 32 + lane;
  const int rows = (n + 7) / 8, j0 = warp * rows, j1 = min(n, j0 + rows);
  int c = 0;
  if (v < n)
    for (int j = j0; j < j1; ++j) c += edge_on(A, W, (long long)j * n + v);
  cnt[warp][lane] = c;
  __syncthreads();
  if (v >= n) return;
  int w = ptr[v];
  for (int q = 0; q < warp; ++q) w += cnt[q][lane];
  for (int j = j0; j < j1; ++j)
    if (edge_on(A, W, (long long)j * n + v)) {
      if (W) wt[w] = W[(long long)j * n + v];
      idx[w++] = j;
    }
}

// Distances from sampled sources and their spread within chunks of consecutive positions (the split
// path's range screen; the node at position q is ord[q], or q without an order).  One CTA per
// source: a level-synchronous BFS along the successor lists (hop counts), or for a weighted graph
// (w != null, the weight of each successor edge) Bellman-Ford rounds of relaxation along them
// (float distances; at most n rounds; concurrent relaxations only lower a distance, so a round
// without a change ends it).  Then, one warp per chunk of `chunk` consecutive positions, the spread
// max d - min d over the chunk's reached nodes; the largest over chunks and sources goes to *out as
// the bits of a non-negative float (atomicMax).  Sources: nodes b n / nsrc + n / (2 nsrc).
__global__ void __launch_bounds__(1024) chunk_spread_kernel(const int32_t* __restrict__ ptr,
                                                            const int32_t* __restrict__ succ,
                                                            const float* __restrict__ w, int n, int nsrc,
                                                            int chunk, const int32_t* __restrict__ ord,
                                                            float* __restrict__ dist, unsigned long long* out) {
  const int b = blockIdx.x, t = threadIdx.x;
  const int src = (int)(((long long)b * n) / nsrc + (n / nsrc) / 2);
  float* d = dist + (long long)b * n;
  const float inf = __int_as_float(0x7f800000);
  for (int v = t; v < n; v += blockDim.x) d[v] = (v == src) ? 0.f : inf;
  __syncthreads();
  if (!w) {
    for (int L = 0; L < n; ++L) {
      int grew = 0;
      const float fl = (float)L;
      for (int v = t; v < n; v += blockDim.x) {
        if (d[v] != fl) continue;
        const int e1 = ptr[v + 1];
        for (int e = ptr[v]; e < e1; ++e) {
          const int x = succ[e];
          if (d[x] == inf) {  // every writer of this level writes the same L + 1
            d[x] = fl + 1.f;
            grew = 1;
          }
        }
      }
      if (!__syncthreads_or(grew)) break;
    }
  } else {
    for (int round = 0; round < n; ++round) {
      int changed = 0;
      for (int v = t; v < n; v += blockDim.x) {
        const float dv = d[v];
        if (dv == inf) continue;
        const int e1 = ptr[v + 1];
        for (int e = ptr[v]; e < e1; ++e) {
          const int x = succ[e];
          const float nd = dv + w[e];
          if (nd < d[x]) {  // non-negative floats order like their bit patterns
            atomicMin(reinterpret_cast<int*>(d + x), __float_as_int(nd));
            changed = 1;
          }
        }
      }
      if (!__syncthreads_or(changed)) break;
    }
  }
  const int warp = t >> 5, lane = t & 31, nwarps = blockDim.x >> 5;
  const int nch = (n + chunk - 1) / chunk;
  for (int c = warp; c < nch; c += nwarps) {
    float lo = inf, hi = -1.f;
    const int v1 = min(n, (c + 1) * chunk);
    for (int q = c * chunk + lane; q < v1; q += 32) {
      const float x = d[ord ? ord[q] : q];
      if (x != inf) {
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
      }
    }
    for (int o = 16; o; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0 && hi >= 0.f) atomicMax(out, (unsigned long long)__float_as_uint(hi - lo));
  }
}

// Block-wide exclusive prefix sum of one count per thread (blockDim.x <= 1024); returns the
// thread's offset and writes the total to *total.
__device__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
  *total = sh[nw - 1];
  __syncthreads();
  return before;
}

// Whole-graph BFS from `src` by one CTA (dist[v] = hops, -1 if not reached; at most n levels).
__device__ void cta_bfs(const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ, int n, int src,
                        int32_t* dist) {
  for (int v = threadIdx.x; v < n; v += blockDim.x) dist[v] = (v == src) ? 0 : -1;
  __syncthreads();
  for (int L = 0; L < n; ++L) {
    int grew = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      if (dist[v] != L) continue;
      for (int x = ptr[v]; x < ptr[v + 1]; ++x) {
        const int w = succ[x];
        if (dist[w] < 0) {  // every writer of this level writes L + 1
          dist[w] = L + 1;
          grew = 1;
        }
      }
    }
    if (!__syncthreads_or(grew)) break;
  }
}

// Smallest node maximising score[v] (score < 0: not a candidate); node 0 if there is none.
__device__ int cta_argmax(const int32_t* score, int n, int* sh) {
  long long best = -1;  // (score << 32) | (INT_MAX - v): the largest is the smallest v of the top score
  for (int v = threadIdx.x; v < n; v += blockDim.x)
    if (score[v] >= 0) best = max(best, ((long long)score[v] << 32) | (long long)(0x7fffffff - v));
  for (int o = 16; o; o >>= 1) best = max(best, (long long)__shfl_xor_sync(0xffffffffu, best, o));
  __shared__ long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long b = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, red[w]);
    *sh = b < 0 ? 0 : 0x7fffffff - (int)(b & 0xffffffffll);
  }
  __syncthreads();
  const int r = *sh;
  __syncthreads();
  return r;
}

// Landmark coordinates of the split path's locality order, by one CTA: L1 = the farthest node from
// node 0, L2 = the farthest from L1, L3 = the node farthest from both (largest min(d_L1, d_L2));
// each node gets cu = d_L1 - d_L3 and cv = d_L1 + d_L3 (on a mesh these are its two axes), or
// cv = -1 when L1 or L3 does not reach it.  d0..d3: n ints each of scratch.
__global__ void __launch_bounds__(1024) landmark_kernel(const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ succ, int n, int32_t* d0,
                                                        int32_t* d1, int32_t* d2, int32_t* cu, int32_t* cv) {
  __shared__ int sh;
  cta_bfs(ptr, succ, n, 0, d0);
  const int L1 = cta_argmax(d0, n, &sh);
  cta_bfs(ptr, succ, n, L1, d1);
  const int L2 = cta_argmax(d1, n, &sh);
  cta_bfs(ptr, succ, n, L2, d2);
  for (int v = threadIdx.x; v < n; v += blockDim.x) d0[v] = (d1[v] >= 0 && d2[v] >= 0) ? min(d1[v], d2[v]) : -1;
  __syncthreads();
  const int L3 = cta_argmax(d0, n, &sh);
  cta_bfs(ptr, succ, n, L3, d2);
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const bool r = d1[v] >= 0 && d2[v] >= 0;
    cu[v] = r ? d1[v] - d2[v] : 0;
    cv[v] = r ? d1[v] + d2[v] : -1;
  }
}

// ---- recursive bisection behind the split path's locality order ------------------------------
//
// A part (positions [b, e) of the order) is split into a first part of m0 = 64 ceil(m / 128)
// positions and the rest.  Unscored, along the landmark axis (cu or cv, see landmark_kernel) with
// the larger extent over the part.  Scored, along the best of four keys: the two landmark axes cu, cv (see
// landmark_kernel), and the hop distances d_a, d_b from the two ends of a double sweep inside the
// part (a farthest from the part's first node, b farthest from a).  Each key's split is scored by
// the larger double-sweep hop diameter of its two halves (a half that one BFS does not cover
// scores RCB_SPLIT_PENALTY more), and the best scoring key is applied (ties: in that order).  The
// landmark axes suit meshes with a Manhattan metric; the part-local distances suit king-move
// meshes, whose Chebyshev balls give a corner landmark's distance no row information (a cut by
// d_a alone leaves an L-shaped rest, which d_b then cuts from the other end).  Every BFS stays inside
// its part (or half), whose nodes carry the CTA's tag.

constexpr int RCB_SPLIT_PENALTY = 1 << 20;

// BFS inside the nodes L[q0..q1) that carry `tag_v`, from `src` (one of them): dist[v] = hops,
// -1 if not reached.  At most q1 - q0 levels.
__device__ void part_bfs(const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ, const int32_t* L, int q0,
                         int q1, const int32_t* tag, int tag_v, int src, int32_t* dist) {
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int v = L[q];
    dist[v] = (v == src) ? 0 : -1;
  }
  __syncthreads();
  for (int lev = 0; lev < q1 - q0; ++lev) {
    int grew = 0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const int v = L[q];
      if (dist[v] != lev) continue;
      for (int x = ptr[v]; x < ptr[v + 1]; ++x) {
        const int w = succ[x];
        if (tag[w] == tag_v && dist[w] < 0) {  // every writer of this level writes lev + 1
          dist[w] = lev + 1;
          grew = 1;
        }
      }
    }
    if (!__syncthreads_or(grew)) break;
  }
}

// The farthest reached node of L[q0..q1) (smallest position among ties), its distance, and
// whether some node was not reached.
struct Far {
  int node, dist, unreached;
};
__device__ Far part_farthest(const int32_t* L, int q0, int q1, const int32_t* dist) {
  __shared__ long long red[32];
  long long best = -1;  // (dist << 32) | (INT_MAX - q)
  int miss = 0;
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int d = dist[L[q]];
    if (d < 0) miss = 1;
    else best = max(best, ((long long)d << 32) | (long long)(0x7fffffff - q));
  }
  for (int o = 16; o; o >>= 1) best = max(best, (long long)__shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  miss = __syncthreads_or(miss);
  long long b = -1;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, red[w]);
  __syncthreads();
  Far f;
  f.node = b < 0 ? L[q0] : L[0x7fffffff - (int)(b & 0xffffffffll)];
  f.dist = b < 0 ? 0 : (int)(b >> 32);
  f.unreached = miss;
  return f;
}

// Double-sweep hop diameter of the half L[q0..q1) (nodes tagged tag_v), plus the penalty when it
// is not covered from its first node.
__device__ int half_score(const int32_t* ptr, const int32_t* succ, const int32_t* L, int q0, int q1, const int32_t* tag,
                          int tag_v, int32_t* dist) {
  if (q1 - q0 <= 1) return 0;
  part_bfs(ptr, succ, L, q0, q1, tag, tag_v, L[q0], dist);
  const Far f0 = part_farthest(L, q0, q1, dist);
  part_bfs(ptr, succ, L, q0, q1, tag, tag_v, f0.node, dist);
  const Far f1 = part_farthest(L, q0, q1, dist);
  return f1.dist + (f0.unreached ? RCB_SPLIT_PENALTY : 0);
}

// Stable split of Lin[b..e) into Lout: the m0 smallest keys first (ties in order of position),
// nodes without a key (key < 0) last; both parts keep their nodes' relative order.  Keys are
// counted in a histogram (hist: 2m + 2 ints; keys past 2m above the smallest share the last
// real bucket).
__device__ void part_split(const int32_t* Lin, int32_t* Lout, int b, int e, int m0, const int32_t* key,
                           int32_t* hist) {
  __shared__ int sh[32];
  __shared__ int sh_cut;
  __shared__ int sh_lo[32];
  const int m = e - b, t = threadIdx.x, T = blockDim.x;
  int lo = 0x7fffffff;
  for (int q = b + t; q < e; q += T) {
    const int k = key[Lin[q]];
    if (k >= 0) lo = min(lo, k);
  }
  for (int o = 16; o; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if ((t & 31) == 0) sh_lo[t >> 5] = lo;
  __syncthreads();
  lo = 0x7fffffff;
  for (int w = 0; w < (T >> 5); ++w) lo = min(lo, sh_lo[w]);
  const int cap = 2 * m;  // last real bucket; bucket cap + 1 holds nodes without a key
  auto key_of = [&](int q) {
    const int k = key[Lin[q]];
    return k < 0 ? cap + 1 : min(cap, k - lo);
  };
  for (int k = t; k < cap + 2; k += T) hist[k] = 0;
  __syncthreads();
  for (int q = b + t; q < e; q += T) atomicAdd(&hist[key_of(q)], 1);
  __syncthreads();
  // the cut key: the smallest k with count(key <= k) >= m0
  {
    const int nb = cap + 2, seg = (nb + T - 1) / T, k0 = t * seg, k1 = min(nb, k0 + seg);
    int c = 0;
    for (int k = k0; k < k1; ++k) c += hist[k];
    int tot;
    int before = block_exclusive_scan(c, sh, &tot);
    if (before < m0 && before + c >= m0) {
      for (int k = k0; k < k1; ++k) {
        before += hist[k];
        if (before >= m0) {
          sh_cut = k;
          break;
        }
      }
    }
    __syncthreads();
  }
  const int Ks = sh_cut;
  // contiguous segment of positions per thread, so that "earlier position" is a prefix count
  const int per = (m + T - 1) / T;
  const int q0 = min(e, b + t * per), q1 = min(e, q0 + per);
  int below = 0, tied = 0;
  for (int q = q0; q < q1; ++q) {
    const int k = key_of(q);
    below += (k < Ks);
    tied += (k == Ks);
  }
  int nbelow, ntied;
  block_exclusive_scan(below, sh, &nbelow);
  const int tied_before = block_exclusive_scan(tied, sh, &ntied);
  const int take = m0 - nbelow;  // tied nodes that join the first part, by position
  int first = 0;
  {
    int k = tied_before;
    for (int q = q0; q < q1; ++q) {
      const int key_q = key_of(q);
      const bool in0 = (key_q < Ks) || (key_q == Ks && k < take);
      if (key_q == Ks) ++k;
      first += in0;
    }
  }
  int nfirst;
  const int first_before = block_exclusive_scan(first, sh, &nfirst);
  {
    int k = tied_before, i0 = b + first_before, i1 = b + m0 + (q0 - b - first_before);
    for (int q = q0; q < q1; ++q) {
      const int key_q = key_of(q);
      const bool in0 = (key_q < Ks) || (key_q == Ks && k < take);
      if (key_q == Ks) ++k;
      if (in0)
        Lout[i0++] = Lin[q];
      else
        Lout[i1++] = Lin[q];
    }
  }
  __syncthreads();
}

// One depth of the bisection: CTA c splits the part [parts[2c], parts[2c+1]) of `ord`.  Scratch
// (n ints each, a CTA touching only its own nodes): tag, distP, distH, da, db, key; tmp (n ints);
// hist (2m + 2 ints per part at 2 b + 2 c).  Tags carry the depth, so a stale tag of another
// part never matches.
__global__ void __launch_bounds__(1024) rcb_kernel(const int32_t* __restrict__ parts, int depth, int n,
                                                   const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ,
                                                   const int32_t* __restrict__ cu, const int32_t* __restrict__ cv,
                                                   int32_t* ord, int32_t* tmp, int32_t* hist_all, int32_t* tag,
                                                   int32_t* distP, int32_t* distH, int32_t* da, int32_t* db,
                                                   int32_t* key, int scored) {
  const int b = parts[2 * blockIdx.x], e = parts[2 * blockIdx.x + 1];
  const int m = e - b, m0 = 64 * ((m + 127) / 128);
  const int t = threadIdx.x, T = blockDim.x;
  if (m0 >= m) return;
  int32_t* hist = hist_all + 2 * b + 2 * blockIdx.x;
  if (!scored) {  // the landmark axis with the larger extent over the part's reached nodes
    __shared__ int ext[4][32];
    int umin = 0x7fffffff, umax = -0x7fffffff, vmin = 0x7fffffff, vmax = -0x7fffffff;
    for (int q = b + t; q < e; q += T) {
      const int v = ord[q];
      if (cv[v] < 0) continue;
      umin = min(umin, cu[v]);
      umax = max(umax, cu[v]);
      vmin = min(vmin, cv[v]);
      vmax = max(vmax, cv[v]);
    }
    for (int o = 16; o; o >>= 1) {
      umin = min(umin, __shfl_xor_sync(0xffffffffu, umin, o));
      umax = max(umax, __shfl_xor_sync(0xffffffffu, umax, o));
      vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
      vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if ((t & 31) == 0) {
      ext[0][t >> 5] = umin;
      ext[1][t >> 5] = umax;
      ext[2][t >> 5] = vmin;
      ext[3][t >> 5] = vmax;
    }
    __syncthreads();
    for (int w = 0; w < (T >> 5); ++w) {
      umin = min(umin, ext[0][w]);
      umax = max(umax, ext[1][w]);
      vmin = min(vmin, ext[2][w]);
      vmax = max(vmax, ext[3][w]);
    }
    const bool use_u = (umax - umin) >= (vmax - vmin);
    for (int q = b + t; q < e; q += T) {
      const int v = ord[q];
      key[v] = cv[v] < 0 ? -1 : (use_u ? cu[v] + n : cv[v]);
    }
    __syncthreads();
    part_split(ord, tmp, b, e, m0, key, hist);
    for (int q = b + t; q < e; q += T) ord[q] = tmp[q];
    return;
  }
  const int tag0 = ((depth + 1) << 22) | ((int)blockIdx.x << 2);  // | 0 whole part, | 1, | 2 halves
  for (int q = b + t; q < e; q += T) tag[ord[q]] = tag0;
  __syncthreads();
  // the ends a, b of a double sweep inside the part and the part-local distances d_a, d_b
  part_bfs(ptr, succ, ord, b, e, tag, tag0, ord[b], distP);
  const Far fa = part_farthest(ord, b, e, distP);
  part_bfs(ptr, succ, ord, b, e, tag, tag0, fa.node, da);
  const Far fb = part_farthest(ord, b, e, da);
  part_bfs(ptr, succ, ord, b, e, tag, tag0, fb.node, db);
  constexpr int KEYS = 4;
  int best = 0, best_score = 0x7fffffff;
  for (int cand = 0; cand <= KEYS; ++cand) {
    const int use = cand < KEYS ? cand : best;  // the last pass applies the best key
    for (int q = b + t; q < e; q += T) {
      const int v = ord[q];
      key[v] = use == 0   ? (cv[v] >= 0 ? cu[v] + n : -1)
               : use == 1 ? (cv[v] >= 0 ? cv[v] : -1)
               : use == 2 ? da[v]
                          : db[v];
    }
    __syncthreads();
    part_split(ord, tmp, b, e, m0, key, hist);
    if (cand == KEYS) break;
    for (int q = b + t; q < e; q += T) tag[tmp[q]] = tag0 | (q < b + m0 ? 1 : 2);
    __syncthreads();
    const int s1 = half_score(ptr, succ, tmp, b, b + m0, tag, tag0 | 1, distH);
    const int s2 = half_score(ptr, succ, tmp, b + m0, e, tag, tag0 | 2, distH);
    const int sc = max(s1, s2);
    if (sc < best_score) {
      best_score = sc;
      best = cand;
    }
  }
  for (int q = b + t; q < e; q += T) ord[q] = tmp[q];
}

__global__ void iota_kernel(int n, int32_t* __restrict__ ord) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) ord[q] = q;
}

__global__ void inverse_perm_kernel(const int32_t* __restrict__ ord, int n, int32_t* __restrict__ pos) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) pos[ord[q]] = q;
}

// M'[i][j] = M[ord[i]][ord[j]] for i, j < n; the identity padding (rows/columns n..N-1) is kept
__global__ void permute_m_kernel(const double* __restrict__ M, const int32_t* __restrict__ ord, int n, int N,
                                 double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  out[t] = (i < n && j < n) ? M[(long long)ord[i] * N + ord[j]] : (i == j ? 1.0 : 0.0);
}

// (a stacked batch: graph blockIdx.y, R and out r_gs and o_gs doubles further)
__global__ void copy_rows_kernel(const double* __restrict__ R, long long ldr, int rows, int cols,
                                 double* __restrict__ out, long long ldo, long long r_gs, long long o_gs,
                                 const rd_batch_graph* bg) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  if (bg && bg[blockIdx.y].s == 0) return;
  R += (long long)blockIdx.y * r_gs;
  out += (long long)blockIdx.y * o_gs;
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
  succ_fill_kernel<<<(h->n + 31) / 32, 256, 0, s>>>(h->dA, h->weighted ? h->dW : nullptr, h->n, ptr, h->dSucc,
                                                    h->dSuccW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

// ---- spectral radius of X (the convergence condition of Theorem 1) ----------------------------
//
// Power iteration on B = X^T + I over the successor lists (a gather: y_j = x_j + sum over the
// successors i of j of X_ij x_i), which has the spectral radius rho(X) + 1 and keeps x positive.
// For a non-negative matrix and a positive vector, min_j (Bx)_j / x_j <= rho(B) <= max_j
// (Bx)_j / x_j (Collatz-Wielandt); the step reports both ratios and the largest y (bits of
// positive doubles, ordered as integers), one warp per node.
__global__ void spectral_step_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ,
                                     const float* __restrict__ w, double gamma, double log_gamma, int n,
                                     const double* __restrict__ x, double* __restrict__ y,
                                     unsigned long long* __restrict__ red) {
  const int lane = threadIdx.x & 31;
  const int j = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (j >= n) return;
  double acc = 0.0;
  for (int q = ptr[j] + lane; q < ptr[j + 1]; q += 32) {
    const double xe = w ? exp((double)w[q] * log_gamma) : gamma;
    acc += xe * x[succ[q]];
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double yj = x[j] + acc;
    y[j] = yj;
    const unsigned long long rb = (unsigned long long)__double_as_longlong(yj / x[j]);
    atomicMin(&red[0], rb);
    atomicMax(&red[1], rb);
    atomicMax(&red[2], (unsigned long long)__double_as_longlong(yj));
  }
}

__global__ void spectral_scale_kernel(const double* __restrict__ y, int n, const unsigned long long* __restrict__ red,
                                      double* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = y[j] / __longlong_as_double((long long)red[2]);
}

__global__ void fill_kernel(double* __restrict__ x, int n, double v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = v;
}

cudaError_t rd_copy_rows_out(rd_ctx* h, const double* R, long long ldr, int rows, int cols,
                             double* out, long long ldo, cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  const unsigned nb = h->nbatch > 1 ? (unsigned)h->nbatch : 1u;
  copy_rows_kernel<<<dim3((unsigned)((total + threads - 1) / threads), nb), threads, 0, s>>>(
      R, ldr, rows, cols, out, ldo, rd_batch_stride(h, R), rd_batch_stride(h, out), nb > 1 ? h->dBatch : nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

// Collatz-Wielandt bracket of rho(X) after `iters` steps (successor lists built; x, y: n doubles
// each, red: 3 words).  Synchronises once.
cudaError_t rd_spectral(rd_ctx* h, int iters, double* x, double* y, unsigned long long* red, double* lo, double* hi,
                        cudaStream_t s) {
  const int n = h->n;
  const int32_t* ptr = h->dDeg + (n + 1);
  const unsigned long long init[3] = {~0ull, 0ull, 0ull};
  unsigned long long out[3] = {0, 0, 0};
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, 1.0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  for (int it = 0; it < iters; ++it) {
    if ((e = cudaMemcpyAsync(red, init, sizeof(init), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
    spectral_step_kernel<<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, s>>>(
        ptr, h->dSucc, h->weighted ? h->dSuccW : nullptr, h->gamma, log(h->gamma), n, x, y, red);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
    if (it + 1 == iters) break;  // the last step's x is the one the ratios refer to
    if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
    spectral_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>(y, n, red, x);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  }
  if ((e = cudaMemcpyAsync(out, red, sizeof(out), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  double rmin, rmax;
  memcpy(&rmin, &out[0], sizeof(double));
  memcpy(&rmax, &out[1], sizeof(double));
  *lo = rmin - 1.0 > 0.0 ? rmin - 1.0 : 0.0;
  *hi = rmax - 1.0 > 0.0 ? rmax - 1.0 : 0.0;
  return cudaSuccess;
}

cudaError_t rd_chunk_spread(rd_ctx* h, int nsrc, int chunk, const int32_t* ord, int32_t* dist,
                            unsigned long long* out, cudaStream_t s) {
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  chunk_spread_kernel<<<nsrc, 1024, 0, s>>>(h->dDeg + (h->n + 1), h->dSucc, h->weighted ? h->dSuccW : nullptr, h->n,
                                            nsrc, chunk, ord, reinterpret_cast<float*>(dist), out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

// Locality order of the split path: landmark coordinates (landmark_kernel), then recursive
// bisection into parts of 64 consecutive positions (rcb_kernel, unscored or scored: see there),
// h->dOrd[position] = node,
// h->dPos[node] = position.  Scratch: 13 n ints of the N^2-int buffer dS (N >= 128, n <= N).  The part boundaries depend on n alone, so the host lists them;
// one launch per depth.
cudaError_t rd_locality_order(rd_ctx* h, int scored, cudaStream_t s) {
  const int n = h->n;
  int32_t* w = reinterpret_cast<int32_t*>(h->dS);  // free before the factorisation (>= N^2 ints)
  int32_t* d0 = w;
  int32_t* d1 = w + (size_t)n;
  int32_t* d2 = w + 2 * (size_t)n;
  int32_t* cu = w + 3 * (size_t)n;
  int32_t* cv = w + 4 * (size_t)n;
  int32_t* tmp = w + 5 * (size_t)n;
  int32_t* dparts = w + 6 * (size_t)n;  // < 4 n / 64 + 4 ints, then the histograms (< 2 n + n / 16 + 2)
  int32_t* tag = w + 9 * (size_t)n;
  int32_t* da = w + 10 * (size_t)n;
  int32_t* key = w + 11 * (size_t)n;
  int32_t* db = w + 12 * (size_t)n;
  std::vector<int32_t> all;             // every depth's list of parts to split, concatenated
  std::vector<std::pair<int, int>> depth_span;
  std::vector<std::pair<int, int>> cur{{0, n}};
  while (true) {
    std::vector<std::pair<int, int>> next;
    const int first = (int)all.size() / 2;
    for (auto& pr : cur) {
      const int m = pr.second - pr.first, m0 = 64 * ((m + 127) / 128);
      if (m0 >= m) continue;
      all.push_back(pr.first);
      all.push_back(pr.second);
      next.push_back({pr.first, pr.first + m0});
      next.push_back({pr.first + m0, pr.second});
    }
    const int count = (int)all.size() / 2 - first;
    if (count == 0) break;
    depth_span.push_back({first, count});
    cur.swap(next);
  }
  // histograms: 2 m + 2 ints per part at 2 b + 2 c, after the part list
  int32_t* hist = dparts + all.size() + 4;
  cudaError_t e;
  if (!all.empty() &&
      (e = cudaMemcpyAsync(dparts, all.data(), all.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  landmark_kernel<<<1, 1024, 0, s>>>(h->dDeg + (n + 1), h->dSucc, n, d0, d1, d2, cu, cv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, h->dOrd);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  for (size_t dep = 0; dep < depth_span.size(); ++dep) {
    const auto& d = depth_span[dep];
    if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
    rcb_kernel<<<d.second, 1024, 0, s>>>(dparts + 2 * d.first, (int)dep, n, h->dDeg + (n + 1), h->dSucc, cu, cv,
                                         h->dOrd, tmp, hist, tag, d0, d1, da, db, key, scored);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  }
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  inverse_perm_kernel<<<(n + 255) / 256, 256, 0, s>>>(h->dOrd, n, h->dPos);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the host list must outlive the copy: wait here (once per graph that needs the order)
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  return rd_prof_end(h, s, RD_PROF_NONE, 0.0);
}

// M' = P M P^T in place of M (through the inverse buffer, free before the factorisation)
cudaError_t rd_permute_m(rd_ctx* h, cudaStream_t s) {
  const long long NN = (long long)h->N * h->N;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  permute_m_kernel<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(h->dLU, h->dOrd, h->n, h->N, h->dT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  double* t = h->dLU;
  h->dLU = h->dT;
  h->dT = t;
  return cudaSuccess;
}

