"""Seeded synthetic graph generators shared by the tests, the bench and the oracle checks.

This module builds inputs only: adjacency matrices, edge weights and the gain recipes that
the workloads are quoted with.  It holds none of the R-distance arithmetic (no M, no inverse,
no decode), so the CUDA path and the CPU oracle can both draw their inputs from it without
sharing any of the method.

Conventions (paper Sec. 2, the adjacency definition and its footnote): the matrix is the
transpose of the usual graph-theory convention,

    A[i, j] = 1  iff there is a directed edge from node j to node i,

so column j lists the successors of j and the out-degree of j is the column sum.  Arrays are
numpy ``uint8`` of shape (n, n), C-contiguous (row-major).  Weighted graphs carry a float32
matrix ``W`` with the same orientation; W[i, j] is the weight of edge j -> i and is only
meaningful where A[i, j] = 1 (Sec. 3.2).

Workload recipes (seeds are ``SEED_BASE + config_index * 1000 + replica``):
  * ``er``      directed Erdos-Renyi: every ordered pair i != j independently with prob. p.
  * ``grid4``   4-neighbour grid with ``cols`` columns, node v = cols*r + c, truncated to n.
  * ``ws``      Watts-Strogatz ring: k nearest neighbours (k/2 per side), each ring edge
                rewired with probability ``beta`` to a uniform non-duplicate target;
                undirected (symmetric A).
  * ``grid8w``  8-neighbour (king-move) grid with independent per-directed-edge weights
                uniform in [wlo, whi] (float32).
  * ``er_weighted``  directed Erdos-Renyi with per-edge weights log-uniform in [wlo, whi].
plus small deterministic families used as closed-form pins (directed path, directed cycle,
complete graph, binary tree, the three-node path of Example 4.1).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2308_07403


def seed_for(config_index: int, replica: int = 0) -> int:
    """Seed of replica ``replica`` of workload ``config_index``."""
    return SEED_BASE + 1000 * int(config_index) + int(replica)


def _empty(n: int) -> np.ndarray:
    if n < 0:
        raise ValueError("n must be non-negative")
    return np.zeros((n, n), dtype=np.uint8)


def add_edge(A: np.ndarray, src: int, dst: int) -> None:
    """Record the directed edge src -> dst (sets A[dst, src])."""
    A[dst, src] = 1


def er(n: int, p: float, seed: int, chunk_rows: int = 512) -> np.ndarray:
    """Directed Erdos-Renyi graph; no self-loops.  Generated in row blocks to bound memory."""
    A = _empty(n)
    rng = np.random.default_rng(seed)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        A[r0:r1] = rng.random((r1 - r0, n)) < p
    np.fill_diagonal(A, 0)
    return A


def grid4(n: int, cols: int | None = None) -> np.ndarray:
    """4-neighbour grid, node v = cols*r + c for v < n (last row possibly partial); symmetric."""
    if cols is None:
        cols = max(1, int(np.ceil(np.sqrt(n))))
    A = _empty(n)
    v = np.arange(n)
    r, c = v // cols, v % cols
    right = v[(c + 1 < cols) & (v + 1 < n)]
    A[right + 1, right] = 1
    A[right, right + 1] = 1
    down = v[v + cols < n]
    A[down + cols, down] = 1
    A[down, down + cols] = 1
    del r
    return A


def grid8_weighted(rows: int, cols: int, seed: int, wlo: float = 1.0, whi: float = 4.0):
    """King-move grid rows x cols with per-directed-edge weights ~ U[wlo, whi] (float32).

    Returns (A, W); W is 0 where there is no edge.
    """
    n = rows * cols
    A = _empty(n)
    v = np.arange(n)
    r, c = v // cols, v % cols
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == 0 and dc == 0:
                continue
            ok = (r + dr >= 0) & (r + dr < rows) & (c + dc >= 0) & (c + dc < cols)
            src = v[ok]
            dst = src + dr * cols + dc
            A[dst, src] = 1
    rng = np.random.default_rng(seed)
    W = np.zeros((n, n), dtype=np.float32)
    ii, jj = np.nonzero(A)
    W[ii, jj] = rng.uniform(wlo, whi, size=ii.size).astype(np.float32)
    return A, W


def er_weighted(n: int, p: float, seed: int, wlo: float = 1.0, whi: float = 100.0):
    """Directed G(n, p) with per-edge weights log-uniform in [wlo, whi] (float32): the weighted
    graph family of the paper's Sec. 5 experiment (Fig. 3: p = 0.5, weights 1 to 100).

    Returns (A, W); W is 0 where there is no edge.
    """
    A = er(n, p, seed)
    rng = np.random.default_rng(seed + 1)
    W = np.zeros((n, n), dtype=np.float32)
    ii, jj = np.nonzero(A)
    W[ii, jj] = np.exp(rng.uniform(np.log(wlo), np.log(whi), size=ii.size)).astype(np.float32)
    return A, W


def ws(n: int, k: int, beta: float, seed: int) -> np.ndarray:
    """Undirected Watts-Strogatz small world (ring of n, k neighbours, rewiring prob. beta).

    Ring edges {u, u+m} for m = 1..k/2 are visited in the order (m outer, u inner); each is
    rewired with probability beta to {u, t}, t uniform among nodes that are neither u nor
    already adjacent to u.
    """
    if k % 2 or k >= n:
        raise ValueError("k must be even and < n")
    rng = np.random.default_rng(seed)
    adj = [set() for _ in range(n)]
    for u in range(n):
        for m in range(1, k // 2 + 1):
            w = (u + m) % n
            adj[u].add(w)
            adj[w].add(u)
    for m in range(1, k // 2 + 1):
        for u in range(n):
            w = (u + m) % n
            if rng.random() >= beta or w not in adj[u]:
                continue
            if len(adj[u]) >= n - 1:
                continue
            while True:
                t = int(rng.integers(n))
                if t != u and t not in adj[u]:
                    break
            adj[u].discard(w)
            adj[w].discard(u)
            adj[u].add(t)
            adj[t].add(u)
    A = _empty(n)
    for u in range(n):
        for w in adj[u]:
            A[w, u] = 1
    return A


def directed_path(n: int) -> np.ndarray:
    """0 -> 1 -> ... -> n-1."""
    A = _empty(n)
    for v in range(n - 1):
        add_edge(A, v, v + 1)
    return A


def directed_cycle(n: int) -> np.ndarray:
    """0 -> 1 -> ... -> n-1 -> 0."""
    A = _empty(n)
    for v in range(n):
        add_edge(A, v, (v + 1) % n)
    return A


def complete(n: int) -> np.ndarray:
    """Every ordered pair i != j is an edge."""
    A = np.ones((n, n), dtype=np.uint8)
    np.fill_diagonal(A, 0)
    return A


def binary_tree(n: int) -> np.ndarray:
    """Undirected binary tree on n nodes: node v joined to 2v+1 and 2v+2."""
    A = _empty(n)
    for v in range(n):
        for ch in (2 * v + 1, 2 * v + 2):
            if ch < n:
                add_edge(A, v, ch)
                add_edge(A, ch, v)
    return A


def path3() -> np.ndarray:
    """The undirected three-node path graph of Example 4.1."""
    return np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=np.uint8)


def symmetric_random(n: int, p: float, seed: int) -> np.ndarray:
    """Undirected Erdos-Renyi graph (upper triangle drawn, mirrored)."""
    rng = np.random.default_rng(seed)
    U = np.triu(rng.random((n, n)) < p, 1)
    return (U | U.T).astype(np.uint8)


def max_out_degree(A: np.ndarray) -> int:
    """Delta = max_j sum_i A[i, j] (Theorem 2's definition: largest column sum)."""
    if A.size == 0:
        return 0
    return int((A != 0).sum(axis=0, dtype=np.int64).max())


def gamma_small(A: np.ndarray) -> float:
    """Gain of the single-graph n=512 workload: 0.5 / (Delta + 1)."""
    return 0.5 / (max_out_degree(A) + 1)


def gamma_frac(A: np.ndarray, frac: float) -> float:
    """Gain at ``frac`` times the Theorem-4 bound 1/Delta (the n=8192 workloads use 0.5, 0.9)."""
    d = max_out_degree(A)
    if d == 0:
        raise ValueError("graph has no edges")
    return float(frac) / d


# ---- named workloads ---------------------------------------------------------------------

def workload_small(replica: int = 0):
    """n=512 directed ER graph, p=0.02, gain 0.5/(Delta+1)."""
    A = er(512, 0.02, seed_for(0, replica))
    return A, gamma_small(A)


LARGE_KINDS = ("er", "grid", "ws")
LARGE_FRACS = (0.5, 0.9)


def workload_large(kind: str, frac: float, n: int = 8192, replica: int = 0):
    """The dense n=8192 single-graph workloads: ER p=0.01, 90x91 grid, WS ring k=10 beta=0.1."""
    if kind == "er":
        A = er(n, 0.01, seed_for(1, replica))
    elif kind == "grid":
        A = grid4(n, cols=91)
    elif kind == "ws":
        A = ws(n, 10, 0.1, seed_for(1, replica) + 17)
    else:
        raise ValueError(kind)
    return A, gamma_frac(A, frac)


BATCH_KINDS = ("er", "grid", "ws")


def workload_batched(G: int = 4096, n_lo: int = 32, n_hi: int = 512, replica: int = 0):
    """The batched workload: G independent graphs, n uniform in [n_lo, n_hi], the kind uniform over
    ER (p = 4/n), a 4-neighbour grid with ceil(sqrt n) columns and Watts-Strogatz (k = min(10,
    n - 1 rounded down to even), beta = 0.1); gain 0.5 / (Delta + 1) per graph.  Returns the lists
    (kinds, n, A, gamma); graph g draws its own seed from the batch's generator."""
    rng = np.random.default_rng(seed_for(2, replica))
    kinds, ns, As, gs = [], [], [], []
    for _ in range(G):
        n = int(rng.integers(n_lo, n_hi + 1))
        kind = BATCH_KINDS[int(rng.integers(len(BATCH_KINDS)))]
        s = int(rng.integers(2**31 - 1))
        if kind == "er":
            A = er(n, 4.0 / n, s)
        elif kind == "grid":
            A = grid4(n, int(np.ceil(np.sqrt(n))))
        else:
            k = min(10, n - 1)
            k -= k % 2
            A = ws(n, k, 0.1, s)
        kinds.append(kind)
        ns.append(n)
        As.append(A)
        gs.append(gamma_small(A))
    return kinds, np.array(ns, dtype=np.int32), As, np.array(gs, dtype=np.float64)


def serving_pool(count: int = 128, n_lo: int = 64, n_hi: int = 4096, replica: int = 0):
    """The serving workload's graph pool: n log-uniform in [n_lo, n_hi], the kind uniform over ER
    (p = 4/n), a 4-neighbour grid with ceil(sqrt n) columns and Watts-Strogatz (k = 10, beta =
    0.1); gain 0.5 / (Delta + 1).  Returns a list of (A, gamma)."""
    rng = np.random.default_rng(seed_for(3, replica))
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        kind = BATCH_KINDS[int(rng.integers(len(BATCH_KINDS)))]
        s = int(rng.integers(2**31 - 1))
        if kind == "er":
            A = er(n, 4.0 / n, s)
        elif kind == "grid":
            A = grid4(n, int(np.ceil(np.sqrt(n))))
        else:
            A = ws(n, 10, 0.1, s)
        out.append((A, gamma_small(A)))
    return out


def gamma_weighted_bound(A: np.ndarray, W: np.ndarray) -> float:
    """Largest gain with max_j sum_i gamma^W_ij <= 1 over the edges (the weighted extension's
    counterpart of 1/Delta: strict column diagonal dominance of M = I - gamma^W), by bisection."""
    ii, jj = np.nonzero(A)
    w = W[ii, jj].astype(np.float64)
    n = A.shape[0]
    lo, hi = 0.0, 1.0
    for _ in range(80):
        g = 0.5 * (lo + hi)
        col = np.bincount(jj, weights=np.power(g, w), minlength=n)
        if col.max() <= 1.0:
            lo = g
        else:
            hi = g
    return lo


def workload_weighted(rows: int = 128, cols: int = 256, frac: float = 0.9, replica: int = 0):
    """Weighted local navigation: a rows x cols king-move grid (n = rows cols; 128 x 256 = 32768)
    with per-directed-edge weights uniform in [1, 4] (float32), gain frac x the weighted bound.
    Returns (A, W, gamma)."""
    A, W = grid8_weighted(rows, cols, seed_for(4, replica))
    return A, W, frac * gamma_weighted_bound(A, W)
