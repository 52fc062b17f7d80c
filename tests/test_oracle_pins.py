"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms (Example 4.1,
directed path and cycle, complete graph), exact rational arithmetic, the walk-count series,
breadth-first search (itself checked against scipy), the theorems of Sec. 4 and the
machine-precision bound of Sec. 5.1.  The last tests plant mistakes in the oracle's inputs to
show the pins would catch them.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2308_07403_gb300 import graphs

UNR = oracle.UNREACHABLE


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.maximum(np.abs(b), 1e-300)
    return float(np.max(np.abs(a - b) / den)) if a.size else 0.0


# ---- closed forms ---------------------------------------------------------------------

@pytest.mark.parametrize("g", [0.05, 0.2, 0.45, 0.6, 0.7])
def test_example_4_1_closed_form(oracle_lib, g):
    """Example 4.1: (I - gA)^-1 = [[1-g^2, g, g^2], [g, 1, g], [g^2, g, 1-g^2]] / (1 - 2g^2)."""
    Y = oracle.inverse(graphs.path3(), g)
    ref = np.array([[1 - g * g, g, g * g], [g, 1, g], [g * g, g, 1 - g * g]]) / (1 - 2 * g * g)
    assert rel_err(Y, ref) < 1e-14


def test_example_4_1_fails_near_critical_gain(oracle_lib):
    """Example 4.1: R_12 -> -inf as gamma -> 1/sqrt(2), so D_12 != 1 just below gamma_c."""
    D_ok = oracle.rdistance(graphs.path3(), 0.2)
    assert D_ok[0, 1] == 1 and D_ok[0, 2] == 2
    D_bad = oracle.rdistance(graphs.path3(), 0.7071)
    assert D_bad[0, 1] <= 0


@pytest.mark.parametrize("n,g", [(10, 0.3), (40, 0.05), (33, 0.6)])
def test_directed_path_exact_powers(oracle_lib, n, g):
    """Directed path 0->1->...: Y_ij = g^(i-j) for i >= j, else 0; D_ij = i - j exactly.

    R is an integer here in exact arithmetic, the case the decode snap exists for."""
    D, Y = oracle.rdistance(graphs.directed_path(n), g, want_y=True)
    i, j = np.indices((n, n))
    ref = np.where(i >= j, float(g) ** np.maximum(i - j, 0), 0.0)
    assert rel_err(Y[i >= j], ref[i >= j]) < 1e-13
    assert np.all(Y[i < j] == 0.0)
    assert np.array_equal(D, np.where(i >= j, i - j, UNR))


@pytest.mark.parametrize("n,g", [(7, 0.4), (25, 0.9), (64, 0.5)])
def test_directed_cycle(oracle_lib, n, g):
    """Directed cycle: Y_ij = g^((i-j) mod n) / (1 - g^n); D_ij = (i-j) mod n."""
    D, Y = oracle.rdistance(graphs.directed_cycle(n), g, want_y=True)
    i, j = np.indices((n, n))
    k = (i - j) % n
    ref = g ** k / (1 - g ** n)
    assert rel_err(Y, ref) < 1e-13
    assert np.array_equal(D, k)


@pytest.mark.parametrize("n,g", [(5, 0.1), (50, 0.015), (200, 0.004)])
def test_complete_graph_sherman_morrison(oracle_lib, n, g):
    """Complete graph A = J - I: M = (1+g)I - gJ, inverse by Sherman-Morrison."""
    Y = oracle.inverse(graphs.complete(n), g)
    off = g / ((1 + g) * (1 - (n - 1) * g))
    dia = (1 - (n - 2) * g) / ((1 + g) * (1 - (n - 1) * g))
    ref = np.full((n, n), off)
    np.fill_diagonal(ref, dia)
    assert rel_err(Y, ref) < 1e-13


# ---- exact rationals --------------------------------------------------------------------

def tiny_graphs():
    out = []
    for seed in range(6):
        n = 4 + seed
        A = graphs.er(n, 0.35, 100 + seed)
        out.append(A)
    out.append(graphs.path3())
    out.append(graphs.binary_tree(7))
    out.append(graphs.directed_path(6))
    return out


@pytest.mark.parametrize("idx", range(9))
def test_oracle_vs_exact_rationals(oracle_lib, idx):
    A = tiny_graphs()[idx]
    delta = max(1, graphs.max_out_degree(A))
    for q in (delta + 1, 2 * delta + 3, 7 * delta + 2):
        g = Fraction(1, q)
        Yx = exact.inverse(A.tolist(), g)
        Dx = np.array(exact.decode(Yx, g), dtype=np.int64)
        D, Y = oracle.rdistance(A, float(g), want_y=True)
        Yf = np.array([[float(v) for v in row] for row in Yx])
        assert rel_err(Y[Yf != 0], Yf[Yf != 0]) < 1e-13
        assert np.all(Y[Yf == 0] == 0.0)
        assert np.array_equal(D.astype(np.int64), Dx)


def test_weighted_oracle_vs_exact_integer_weights(oracle_lib):
    """Sec. 3.2: with positive integer weights, X = g^W and the same decode."""
    rng = np.random.default_rng(7)
    for n in (4, 6):
        A = graphs.er(n, 0.5, 900 + n)
        W = rng.integers(1, 4, size=(n, n)).astype(np.float32)
        W[A == 0] = 0
        g = Fraction(1, 9)
        Yx = exact.inverse(A.tolist(), g, W.astype(int).tolist())
        Yf = np.array([[float(v) for v in row] for row in Yx])
        D, Y = oracle.rdistance(A, float(g), W=W, want_y=True)
        assert rel_err(Y[Yf != 0], Yf[Yf != 0]) < 1e-12
        Dx = np.array(exact.decode(Yx, g))
        assert np.array_equal(D, Dx)


# ---- walk-count series (Sec. 3.1, Y-series) -------------------------------------------------

@pytest.mark.parametrize("seed", range(3))
def test_walk_count_series(oracle_lib, seed):
    n = 8
    A = graphs.er(n, 0.3, 300 + seed)
    delta = max(1, graphs.max_out_degree(A))
    g = 0.5 / delta
    K = 30
    N = exact.walk_counts(A.tolist(), K)
    partial = sum(np.array(N[k], dtype=np.float64) * g ** k for k in range(K + 1))
    tail = (g * delta) ** (K + 1) / (delta * (1 - g * delta))   # from N^(k) <= Delta^(k-1)
    Y = oracle.inverse(A, g)
    assert np.all(Y >= partial * (1 - 1e-14))
    assert np.all(Y - partial <= tail + 1e-14 * Y)


@pytest.mark.parametrize("kind", ["er", "grid", "ws", "tree"])
def test_series_fixpoint_matches_dense(oracle_lib, kind):
    """Two independent routes to Y: dense LU + solves vs the partial sums of the series."""
    n = 240
    if kind == "er":
        A = graphs.er(n, 0.03, 11)
    elif kind == "grid":
        A = graphs.grid4(n, 16)
    elif kind == "ws":
        A = graphs.ws(n, 6, 0.1, 12)
    else:
        A = graphs.binary_tree(n)
    g = graphs.gamma_frac(A, 0.9)
    Y = oracle.inverse(A, g)
    for j in (0, 17, n - 1):
        col, _ = oracle.series_vector(A, g, j)
        row, _ = oracle.series_vector(A, g, j, transpose=True)
        nz = Y[:, j] != 0
        assert rel_err(col[nz], Y[nz, j]) < 1e-12
        nz = Y[j, :] != 0
        assert rel_err(row[nz], Y[j, nz]) < 1e-12


# ---- BFS truth and theorems ------------------------------------------------------------------

def test_bfs_matches_scipy(oracle_lib):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(3):
        A = graphs.er(60, 0.05, 500 + seed)
        D, _ = oracle.bfs_all(A)
        # scipy's dist[s, t] is s -> t over edges G[s, t]; our edge j -> i is A[i, j], so G = A^T.
        ref = sp.shortest_path(A.T.astype(np.float64), unweighted=True, directed=True)
        ref = ref.T
        finite = np.isfinite(ref)
        assert np.array_equal(D[finite], ref[finite].astype(np.int32))
        assert np.all(D[~finite] == UNR)


@pytest.mark.parametrize("m", [3, 5, 8])
def test_grid_corner_path_count(oracle_lib, m):
    """Example 4.2: corner to corner of an m x m grid, D = 2m-2 and S = C(2m-2, m-1)."""
    A = graphs.grid4(m * m, m)
    dist, cnt = oracle.bfs(A, [0])
    assert dist[0, m * m - 1] == 2 * m - 2
    assert cnt[0, m * m - 1] == comb(2 * m - 2, m - 1)


def _diameter(D):
    return int(D[D != UNR].max())


def test_theorem2_sufficient_bound(oracle_lib):
    """Theorem 2: 0 < g < 1/(Delta + Delta^(d-1)) => D == BFS everywhere."""
    for seed in range(4):
        A = graphs.symmetric_random(40, 0.1, 40 + seed)
        Dt, _ = oracle.bfs_all(A)
        delta = graphs.max_out_degree(A)
        d = _diameter(Dt)
        g = 0.9 / (delta + delta ** (d - 1))
        assert g > 1e-300
        D = oracle.rdistance(A, g)
        assert np.array_equal(D, Dt)


def test_theorem3_trees(oracle_lib):
    """Theorem 3: on undirected trees, g < (-1 + sqrt(1 + 4 Delta (d+2))) / (2 Delta (d+2))."""
    for n in (15, 31, 63):
        A = graphs.binary_tree(n)
        Dt, _ = oracle.bfs_all(A)
        delta = graphs.max_out_degree(A)
        d = _diameter(Dt)
        gb = (-1 + np.sqrt(1 + 4 * delta * (d + 2))) / (2 * delta * (d + 2))
        D = oracle.rdistance(A, 0.98 * gb)
        assert np.array_equal(D, Dt)


def test_theorem1_redundant_paths_necessary(oracle_lib):
    """Theorem 1: with g >= 1/max S, the R-distance is not globally correct (grid example)."""
    m = 4
    A = graphs.grid4(m * m, m)
    Dt, S = oracle.bfs_all(A)
    smax = S.max()
    assert smax == comb(2 * m - 2, m - 1)
    g = 0.2  # 1/20 = 1/max S < 0.2 < 1/Delta = 0.25
    D = oracle.rdistance(A, g)
    assert not np.array_equal(D, Dt)
    # and the entry that realises max S is among the wrong ones
    i, j = np.unravel_index(np.argmax(S), S.shape)
    assert D[i, j] != Dt[i, j]


@pytest.mark.parametrize("kind", ["er", "grid", "ws"])
def test_bracket_Y(oracle_lib, kind):
    """S g^D <= Y (Y-series-trunc) and Y <= g^D Delta^(D-1)/(1 - g Delta) (Y-bracket)."""
    n = 150
    A = {"er": lambda: graphs.er(n, 0.04, 5), "grid": lambda: graphs.grid4(n, 12),
         "ws": lambda: graphs.ws(n, 6, 0.1, 6)}[kind]()
    g = graphs.gamma_frac(A, 0.5)
    delta = graphs.max_out_degree(A)
    Y = oracle.inverse(A, g)
    Dt, S = oracle.bfs_all(A)
    mask = (Dt != UNR) & (Dt >= 1)
    d = Dt[mask].astype(np.float64)
    lo = S[mask] * g ** d
    hi = g ** d * float(delta) ** (d - 1) / (1 - g * delta)
    y = Y[mask]
    assert np.all(y >= lo * (1 - 1e-12))
    assert np.all(y <= hi * (1 + 1e-12))
    assert np.all(Y[Dt == UNR] == 0.0)


def _walk(nxt, start, goal, n):
    seen = {start}
    v = start
    steps = 0
    while v != goal:
        v = int(nxt[v])
        steps += 1
        if v < 0 or v in seen or steps > n:
            return None
        seen.add(v)
    return steps


@pytest.mark.parametrize("kind", ["er", "grid", "tree"])
def test_theorem4_greedy_reaches_goal(oracle_lib, kind):
    """Theorem 4 and Cor. 4.1: for g < 1/Delta greedy ascent on Y reaches the goal without a
    cycle; on a tree the walk is the shortest path."""
    n = 120
    A = {"er": lambda: graphs.er(n, 0.06, 9), "grid": lambda: graphs.grid4(n, 11),
         "tree": lambda: graphs.binary_tree(n)}[kind]()
    g = graphs.gamma_frac(A, 0.95)
    Dt, _ = oracle.bfs_all(A)
    goals = np.array([0, 5, n // 2, n - 1], dtype=np.int32)
    rows = oracle.goal_rows(A, g, goals)
    nxt = oracle.greedy_next(A, goals, rows)
    for c, goal in enumerate(goals):
        for s in range(n):
            if Dt[goal, s] == UNR:
                continue
            steps = _walk(nxt[c], s, int(goal), n)
            assert steps is not None
            if kind == "tree":
                assert steps == Dt[goal, s]


def test_goal_rows_match_inverse(oracle_lib):
    A = graphs.er(200, 0.04, 21)
    g = graphs.gamma_frac(A, 0.9)
    Y = oracle.inverse(A, g)
    goals = np.array([3, 77, 199], dtype=np.int32)
    rows = oracle.goal_rows(A, g, goals)
    for c, goal in enumerate(goals):
        nz = Y[goal] != 0
        assert rel_err(rows[c, nz], Y[goal, nz]) < 1e-12


def test_machine_precision_cutoff(oracle_lib):
    """Sec. 5.1: a distance d is representable only while g^d exceeds the smallest double."""
    n, g = 60, 1e-6
    D, Y = oracle.rdistance(graphs.directed_path(n), g, want_y=True)
    i, j = np.indices((n, n))
    k = i - j
    normal = (k >= 0) & (k * np.log10(g) > -300)
    assert np.array_equal(D[normal], k[normal])
    gone = (k >= 0) & (k * np.log10(g) < -324.5)
    assert gone.any()
    assert np.all(Y[gone] == 0.0) and np.all(D[gone] == UNR)


def test_decode_special_values(oracle_lib):
    Y = np.array([[5.0, 0.0, -1.0], [0.5, 2.0, 1e-5], [1.0, 3.0, 1.0]])
    D = oracle.decode(Y, 0.1)
    assert D[0, 0] == 0 and D[1, 1] == 0 and D[2, 2] == 0
    assert D[0, 1] == UNR and D[0, 2] == UNR
    assert D[1, 0] == 1          # log_0.1(0.5) = 0.30 -> 1
    assert D[1, 2] == 5          # exact power 1e-5 stays 5 under the snap
    assert D[2, 0] == 0          # Y = 1 -> 0
    assert D[2, 1] == 0          # Y > 1: ceil of a negative R, kept literal


def test_dijkstra_matches_scipy(oracle_lib):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    A, W = graphs.grid8_weighted(6, 7, 3)
    dist = oracle.dijkstra(A, W, np.arange(A.shape[0], dtype=np.int32))
    G = np.where(A.T != 0, W.T, 0).astype(np.float64)
    ref = sp.shortest_path(G, method="D", directed=True)
    assert np.allclose(dist, ref, rtol=1e-6)


# ---- planted mistakes: the pins must catch them ----------------------------------------------

def test_planted_transpose_is_caught(oracle_lib):
    """Feeding A^T (the usual graph convention) breaks the directed-path pin."""
    n, g = 10, 0.3
    A = graphs.directed_path(n)
    D = oracle.rdistance(np.ascontiguousarray(A.T), g)
    i, j = np.indices((n, n))
    assert not np.array_equal(D, np.where(i >= j, i - j, UNR))


def test_planted_sign_is_caught(oracle_lib):
    """M = I + gA instead of I - gA breaks the complete-graph closed form."""
    n, g = 50, 0.015
    Y = oracle.inverse(graphs.complete(n), -g)
    off = g / ((1 + g) * (1 - (n - 1) * g))
    assert abs(Y[0, 1] - off) / off > 1e-3


def test_decode_vector_matches_matrix_decode(oracle_lib):
    A = graphs.er(90, 0.05, 4)
    g = graphs.gamma_frac(A, 0.9)
    D, Y = oracle.rdistance(A, g, want_y=True)
    for i in (0, 45, 89):
        assert np.array_equal(oracle.decode_vector(Y[i], i, g), D[i])
        assert np.array_equal(oracle.decode_vector(Y[:, i], i, g), D[:, i])


def test_spectral_radius_closed_forms():
    """rho(X) of Theorem 1's convergence condition, pinned by spectra known in closed form: a
    directed cycle (the n-th roots of unity: 1), the complete graph K_n (n - 1), a directed path
    (nilpotent: 0), the undirected path P_n (2 cos(pi / (n + 1))), Example 4.1's three-node path
    (sqrt 2), and the scaling rho(gamma A) = gamma rho(A)."""
    assert oracle.spectral_radius(graphs.directed_cycle(7)) == pytest.approx(1.0, abs=1e-12)
    assert oracle.spectral_radius(graphs.complete(5)) == pytest.approx(4.0, abs=1e-12)
    assert oracle.spectral_radius(graphs.directed_path(6)) == pytest.approx(0.0, abs=1e-12)
    assert oracle.spectral_radius(graphs.path3()) == pytest.approx(np.sqrt(2.0), abs=1e-12)
    n = 11
    P = np.zeros((n, n), np.uint8)
    for i in range(n - 1):
        P[i, i + 1] = P[i + 1, i] = 1
    assert oracle.spectral_radius(P) == pytest.approx(2.0 * np.cos(np.pi / (n + 1)), abs=1e-12)
    assert oracle.spectral_radius(P, 0.3) == pytest.approx(0.6 * np.cos(np.pi / (n + 1)), abs=1e-12)


def test_weighted_equals_subdivided_unweighted_graph(oracle_lib):
    """Sec. 3.2 for integer weights: Y_ij = sum_d N_ij^(d) gamma^d, N^(d) the number of walks of
    total weight d.  Replacing every edge of weight k by a chain of k unit edges through k - 1 new
    nodes (in- and out-degree one) maps those walks one to one onto the unit-step walks between
    the original nodes, so the weighted Y and D equal the unweighted ones of the subdivided graph
    on the original nodes -- a check of X = gamma^W that does not use that formula."""
    rng = np.random.default_rng(21)
    for n in (5, 8):
        A = graphs.er(n, 0.5, 700 + n)
        W = np.where(A != 0, rng.integers(1, 4, size=(n, n)), 0).astype(np.float32)
        rows = [(i, j, int(W[i, j])) for i, j in zip(*np.nonzero(A))]  # edge j -> i, weight k
        m = n + sum(k - 1 for _, _, k in rows)
        S = np.zeros((m, m), np.uint8)
        nxt = n
        for i, j, k in rows:
            prev = j
            for _ in range(k - 1):
                S[nxt, prev] = 1
                prev = nxt
                nxt += 1
            S[i, prev] = 1
        g = 1.0 / (graphs.max_out_degree(S) + 2)
        Dw, Yw = oracle.rdistance(A, g, W=W, want_y=True)
        Ds, Ys = oracle.rdistance(S, g, want_y=True)
        assert rel_err(Yw[Yw != 0], Ys[:n, :n][Yw != 0]) < 1e-12
        assert np.array_equal(Yw == 0, Ys[:n, :n] == 0)
        assert np.array_equal(Dw, Ds[:n, :n])


# ---- the gain check's quantity: the largest column sum of X ----------------------------------

def _out_star(n):
    """Node 0 -> every other node: out-degree n - 1 at node 0, in-degree at most 1."""
    A = np.zeros((n, n), dtype=np.uint8)
    A[1:, 0] = 1  # A[i, 0] = 1: the edge 0 -> i (Sec. 2's orientation)
    return A


@pytest.mark.parametrize("n,g", [(9, 0.1), (40, 0.02)])
def test_max_column_sum_is_gamma_times_out_degree(oracle_lib, n, g):
    """The gain check of Theorem 4 reads the largest column sum of X = gamma A, gamma times the
    largest OUT-degree Delta (column j of A lists the successors of j, Sec. 2).  Closed forms:
    the out-star (gamma (n - 1), against gamma for its transpose, the in-star, which a row sum
    would swap), the directed path (gamma), K_n (gamma (n - 1)), the directed cycle (gamma)."""
    star = _out_star(n)
    assert oracle.max_column_sum(oracle.build_m(star, g)) == pytest.approx(g * (n - 1), rel=1e-15)
    assert oracle.max_column_sum(oracle.build_m(np.ascontiguousarray(star.T), g)) == pytest.approx(g, rel=1e-15)
    assert oracle.max_column_sum(oracle.build_m(graphs.directed_path(n), g)) == pytest.approx(g, rel=1e-15)
    assert oracle.max_column_sum(oracle.build_m(graphs.directed_cycle(n), g)) == pytest.approx(g, rel=1e-15)
    gk = 0.9 / (n - 1)
    assert oracle.max_column_sum(oracle.build_m(graphs.complete(n), gk)) == pytest.approx(0.9, rel=1e-14)


def test_max_column_sum_weighted_geometric(oracle_lib):
    """Weighted (Sec. 3.2, X_ij = gamma^W_ij): node 0 -> node i with weight i (i = 1..m) gives a
    column sum of gamma + gamma^2 + ... + gamma^m = gamma (1 - gamma^m) / (1 - gamma); the other
    columns hold one edge i -> 0 of weight 7 (gamma^7)."""
    m, g = 12, 0.4
    n = m + 1
    A = _out_star(n)
    A[0, 1:] = 1
    W = np.zeros((n, n), dtype=np.float32)
    W[1:, 0] = np.arange(1, n, dtype=np.float32)
    W[0, 1:] = 7.0
    ref = g * (1 - g ** m) / (1 - g)
    assert oracle.max_column_sum(oracle.build_m(A, g, W)) == pytest.approx(ref, rel=1e-14)


def test_max_column_sum_er_and_the_gain_check(oracle_lib):
    """On a seeded directed ER graph the largest column sum is gamma Delta with Delta counted by
    hand from the edge list; at gamma = 1/Delta it reaches 1 (the boundary of Theorem 4's
    condition) and the no-pivot LU still has positive pivots just below it."""
    A = graphs.er(300, 0.03, 11)
    src = np.nonzero(A)[1]  # A[i, j] != 0: edge j -> i, so j is the source
    delta = int(np.bincount(src, minlength=300).max())
    ins = int(np.bincount(np.nonzero(A)[0], minlength=300).max())
    assert delta != ins  # the case separates out-degree from in-degree
    g = 0.999 / delta
    assert oracle.max_column_sum(oracle.build_m(A, g)) == pytest.approx(g * delta, rel=1e-14)
    assert oracle.max_column_sum(oracle.build_m(A, 1.0 / delta)) == pytest.approx(1.0, rel=1e-14)
    oracle.lu(A, g)  # raises on a non-positive pivot
