"""Parity of the split-precision path (BF16 digit products on the tensor cores) with the oracle.

D must equal the oracle's D exactly.  Y must agree entrywise within a relative 1e-10 at the
default 12 digits of 7 bits: the digit truncation leaves a relative 2^-84 of each operand
chunk's scale, the float-float (two FP32) accumulation carries about 2^-44 of each entry, and
the products are sign-definite, so each entry of Y keeps a relative error of a few 2^-44 times
the depth of the recursion (observed well below 1e-11).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YTOL = 1e-10
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def run(rd, A, g, slices=0, want_y=True):
    n = A.shape[0]
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    Y = torch.empty((n, n), dtype=torch.float64, device="cuda") if want_y else None
    with rd.Handle(At, g, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, slices)
        h.apsp(D, Y)
        h.sync()
        st = h.stats()
    torch.cuda.synchronize()
    return D.cpu().numpy(), (Y.cpu().numpy() if want_y else None), st


def rel_err(Yg, Yo):
    assert np.array_equal(Yg == 0, Yo == 0)
    nz = Yo != 0
    return float(np.max(np.abs(Yg[nz] - Yo[nz]) / np.abs(Yo[nz]))) if nz.any() else 0.0


# (name, graph and gain, digit count): the directed path puts a 2^-68 range of Y inside one
# 256-node chunk, which 12 digits of 7 bits cannot resolve to 1e-10; 15 digits do.
SLICES = {"dpath40": 15}
CASES = [
    ("er128", lambda: (graphs.er(128, 0.06, 1), None)),
    ("dpath40", lambda: (graphs.directed_path(40), 0.3)),
    ("complete64", lambda: (graphs.complete(64), 0.5 / 64)),
    ("grid200", lambda: (graphs.grid4(200, 15), None)),
    ("ws257", lambda: (graphs.ws(257, 6, 0.1, 3), None)),
    ("tree300", lambda: (graphs.binary_tree(300), None)),
    ("er512_small_workload", lambda: graphs.workload_small()),
    ("ws1000_ragged", lambda: (graphs.ws(1000, 10, 0.1, 9), None)),
]


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_split_matches_oracle(rd, name):
    A, g = dict(CASES)[name]()
    if g is None:
        g = graphs.gamma_frac(A, 0.9)
    Do, Yo = oracle.rdistance(A, g, want_y=True)
    s = SLICES.get(name, 12)
    Dg, Yg, st = run(rd, A, g, slices=s)
    assert st["precision"] == rd.RD_PREC_SPLIT_BF16 and st["slices"] == s
    err = rel_err(Yg, Yo)
    assert err < YTOL, err
    assert np.array_equal(Dg, Do), int(np.sum(Dg != Do))


def test_split_slice_count_controls_precision(rd):
    A, g = graphs.workload_small()
    _, Yo = oracle.rdistance(A, g, want_y=True)
    errs = {}
    for s in (4, 8, 12):
        _, Yg, st = run(rd, A, g, slices=s)
        assert st["slices"] == s
        errs[s] = rel_err(Yg, Yo)
    assert errs[4] > errs[8] > errs[12] or errs[12] < 1e-13
    assert errs[8] < 1e-6


def test_split_goal_rows_and_greedy(rd):
    n = 333
    A = graphs.grid4(n, 19)
    g = graphs.gamma_frac(A, 0.9)
    goals = np.array([0, 7, 100, n - 1], dtype=np.int32)
    rows_o = oracle.goal_rows(A, g, goals)
    rows = np.empty((goals.size, n))
    nxt = np.empty((goals.size, n), np.int32)
    with rd.Handle(A, g) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
    assert rel_err(rows, rows_o) < YTOL
    assert np.array_equal(nxt, oracle.greedy_next(A, goals, rows))


def test_split_rejects_bad_slice_counts(rd):
    A, g = graphs.workload_small()
    with rd.Handle(A, g) as h:
        for bad in (16, 1, -1):
            with pytest.raises(rd.RDError) as ei:
                h.set_precision(rd.RD_PREC_SPLIT_BF16, bad)
            assert ei.value.status == rd.RD_ERR_ARG
        D = np.empty((512, 512), np.int32)
        h.apsp(D)  # the handle is unharmed
        assert np.array_equal(D, oracle.rdistance(A, g))


def isolated_sources_path(n=200):
    """A directed path through every node but the range screen's 8 BFS sources (b n / 8 + n / 16),
    which are left isolated: every sampled BFS reaches nothing, so the screen sees no spread."""
    srcs = {(b * n) // 8 + (n // 8) // 2 for b in range(8)}
    chain = [v for v in range(n) if v not in srcs]
    A = np.zeros((n, n), np.uint8)
    for u, v in zip(chain, chain[1:]):
        A[v, u] = 1  # edge u -> v
    return A


def test_self_check_falls_back_to_fp64(rd):
    """A graph the screen misreads: a 192-node directed path at gain 0.125 spans 2^-573 within one
    256-node chunk, but the screen's sampled sources are isolated, so it picks 8 digits.  The far
    entries of Y are lost to the digit truncation, the residual of the sampled rows against M
    exposes it, and the library recomputes the graph in FP64 -- D stays exact."""
    A, g = isolated_sources_path(), 0.125
    Do = oracle.rdistance(A, g)
    Dg, _, st = run(rd, A, g, want_y=False)
    assert st["split_screen_bits"] == 0.0
    assert st["precision_used"] == rd.RD_PREC_FP64 and st["fallbacks"] >= 1
    assert st["split_residual"] > 1e-9
    assert np.array_equal(Dg, Do)


def weighted_split(rd, A, W, g, goals):
    """Goal rows, greedy next hops and the whole D / Y of a weighted graph with the digit count
    left to the library; returns the handle's stats and the outputs."""
    n = A.shape[0]
    D = np.empty((n, n), np.int32)
    Y = np.empty((n, n))
    rows = np.empty((goals.size, n))
    nxt = np.empty((goals.size, n), np.int32)
    with rd.Handle(A, g, W=W) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
        h.apsp(D, Y)
        st = h.stats()
    return st, D, Y, rows, nxt


def check_weighted(A, W, g, goals, D, Y, rows, nxt):
    Do, Yo = oracle.rdistance(A, g, W=W, want_y=True)
    assert rel_err(Y, Yo) < YTOL
    assert np.array_equal(D, Do)
    assert rel_err(rows, Yo[goals]) < YTOL
    assert np.array_equal(nxt, oracle.greedy_next(A, goals, rows))


@pytest.mark.parametrize("frac", [0.9, 0.5])
def test_weighted_king_grid(rd, frac):
    """Weighted extension (X = gamma^W, Sec. 3.3) on the split path: a 24 x 32 king-move grid with
    weights uniform in [1, 4] at frac x the weighted gain bound (about 2.2 and 3.0 bits of Y per
    unit of weight).  A 256-node run of the natural order spans 8 rows of the grid, so the screen
    takes the locality order (64-node parts, 64-wide chunks).  The landmark bisection cuts this mesh
    into strips (Chebyshev balls), so the scored bisection is built and taken.  At 0.5 the graph
    needs more than 15 digits, which only the locality order's chunks carry exactly (up to 22).  The result matches the
    oracle: Y within 1e-10, D exact, goal rows and greedy next hops equal."""
    A, W, gb = graphs.workload_weighted(24, 32, frac=1.0)
    g = frac * gb
    goals = np.array([0, 100, 383, 767], np.int32)
    st, D, Y, rows, nxt = weighted_split(rd, A, W, g, goals)
    # the landmark bisection cuts a king-move mesh into strips: the scored bisection is taken
    assert st["precision_used"] == rd.RD_PREC_SPLIT_BF16 and st["split_order"] == 2, st
    assert st["fallbacks"] <= 1 and 0 < st["split_residual"] < 1e-9, st
    if frac == 0.5:
        assert st["slices"] > 15, st
    check_weighted(A, W, g, goals, D, Y, rows, nxt)


@pytest.mark.parametrize("gamma", ["0.9 bound", "1e-7"])
def test_weighted_dense_random(rd, gamma):
    """The paper's weighted family (Sec. 5, Fig. 3: G(n, 0.5) with weights log-uniform in
    [1, 100]) at n = 768, at 0.9 x the weighted gain bound (Y spans about 11 bits: the screen's
    fewest digits, natural order) and at the paper's gamma = 1e-7 (Y spans about 70 bits: more
    than 12 digits, so the locality order's 64-wide chunks).  Split result, oracle parity."""
    A, W = graphs.er_weighted(768, 0.5, graphs.seed_for(4, 7))
    g = 0.9 * graphs.gamma_weighted_bound(A, W) if gamma == "0.9 bound" else 1e-7
    goals = np.array([3, 200, 511, 766], np.int32)
    st, D, Y, rows, nxt = weighted_split(rd, A, W, g, goals)
    assert st["precision_used"] == rd.RD_PREC_SPLIT_BF16 and 0 < st["split_residual"] < 1e-9, st
    if gamma == "0.9 bound":
        assert st["slices"] <= 9 and st["split_order"] == 0, st
    check_weighted(A, W, g, goals, D, Y, rows, nxt)


def screen_spread(A):
    """The range screen's hop spread from the oracle's BFS: sources b n / 8 + n / 16 (b < 8),
    chunks of 256 consecutive nodes, the largest max - min distance over a chunk's reached
    nodes."""
    n = A.shape[0]
    srcs = np.array([(b * n) // 8 + (n // 8) // 2 for b in range(8)], np.int32)
    dist, _ = oracle.bfs(A, srcs)
    worst = 0
    for row in dist:
        for c0 in range(0, n, 256):
            d = row[c0:c0 + 256]
            d = d[(d >= 0) & (d < np.iinfo(np.int32).max)]
            if d.size:
                worst = max(worst, int(d.max()) - int(d.min()))
    return worst


SCREEN_CASES = {  # (graph, gain): the branch follows from spread x log2(1/gamma)
    "grid1000x40": lambda: (graphs.grid4(1000, 40), None),   # ~95 bits natural: locality order
    "grid600x16": lambda: (graphs.grid4(600, 16), None),     # ~65 bits: 15 digits
    "dpath300_g0.85": lambda: (graphs.directed_path(300), 0.85),  # ~56 bits: 14 digits
    "dpath300_g0.9": lambda: (graphs.directed_path(300), 0.9),    # ~36 bits: 11 digits
    "tree700": lambda: (graphs.binary_tree(700), None),      # a few levels per chunk
    "ws1000": lambda: (graphs.ws(1000, 10, 0.1, 5), None),   # small world
    "er800": lambda: (graphs.er(800, 0.02, 2), None),        # small world
}


def screen_digits(bits):
    """The screen's digit count: the fewest (at least 8) whose 7 bits each cover the spread's bits
    plus 40 bits of result."""
    return max(8, int(np.ceil((bits + 40) / 7)))


@pytest.mark.parametrize("name", list(SCREEN_CASES))
def test_range_screen_matches_bfs(rd, name):
    """The screen's hop spread equals the one computed from the oracle's BFS (integer work: exact),
    the digit count, the node order or FP64 follow from it as documented, and D is exact on every
    branch."""
    A, g = SCREEN_CASES[name]()
    if g is None:
        g = graphs.gamma_frac(A, 0.9)
    spread = screen_spread(A)
    bits = spread * np.log2(1.0 / g)
    Dg, _, st = run(rd, A, g, want_y=False)
    if screen_digits(bits) <= 12:
        # the natural order suffices: the estimate is the BFS spread of 256-node runs, exactly
        assert st["split_order"] == 0
        assert st["split_screen_bits"] == pytest.approx(bits, rel=1e-12, abs=0.0)
        want = screen_digits(bits)
    elif st["split_order"] >= 1:
        # the locality order was taken: it needs fewer digits than the natural order, or the
        # natural order needs more than its 15 (the locality order carries up to 22)
        want = screen_digits(st["split_screen_bits"])
        assert want <= 22 and (want < screen_digits(bits) or screen_digits(bits) > 15)
    else:
        assert st["split_screen_bits"] == pytest.approx(bits, rel=1e-12, abs=0.0)
        want = screen_digits(bits)
    if st["split_order"] == 0 and want > 15:
        assert st["precision_used"] == rd.RD_PREC_FP64 and st["fallbacks"] == 0
    elif st["fallbacks"] == 0:
        assert st["precision_used"] == rd.RD_PREC_SPLIT_BF16 and st["slices"] == want
    assert np.array_equal(Dg, oracle.rdistance(A, g)), name


def test_locality_order_path(rd):
    """A 40-column grid: 256-node runs of the natural order span ~45 hops (95 bits at 0.9/Delta), so
    the library factors P M P^T with its locality order (compact 64-node parts, 64-wide chunks).
    D, Y, the goal rows and the greedy next hops must come back in the caller's node order."""
    A = graphs.grid4(1000, 40)
    g = graphs.gamma_frac(A, 0.9)
    Do, Yo = oracle.rdistance(A, g, want_y=True)
    Dg, Yg, st = run(rd, A, g)
    assert st["split_order"] == 1 and st["precision_used"] == rd.RD_PREC_SPLIT_BF16, st
    assert 0 < st["split_residual"] < 1e-9
    assert rel_err(Yg, Yo) < YTOL
    assert np.array_equal(Dg, Do)
    goals = np.array([0, 13, 500, 999], dtype=np.int32)
    rows = np.empty((goals.size, 1000))
    nxt = np.empty((goals.size, 1000), np.int32)
    with rd.Handle(A, g) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
        assert h.stats()["split_order"] == 1
    assert rel_err(rows, Yo[goals]) < YTOL
    assert np.array_equal(nxt, oracle.greedy_next(A, goals, rows))


@pytest.mark.parametrize("kind,frac", [(k, f) for k in graphs.LARGE_KINDS for f in graphs.LARGE_FRACS])
def test_split_full_size_D_identical(rd, kind, frac):
    """n = 8192: the D of the split mode hashes to the oracle's D.  ER and WS stay on the split
    path in their own node order; the 90 x 91 grid (a 256-node run of its natural order spans ~84
    hops of Y, and Y itself spans 2^-540) runs on the split path in the locality order, whose
    64-node parts span ~17 hops, with per-entry reference exponents in the accumulators."""
    p = os.path.join(HERE, "golden", f"large_{kind}_{frac}.json")
    if not os.path.exists(p):
        pytest.skip("golden file missing")
    with open(p) as f:
        rec = json.load(f)
    A, g = graphs.workload_large(kind, frac)
    Dg, _, st = run(rd, A, g, want_y=False)
    assert st["precision_used"] == rd.RD_PREC_SPLIT_BF16, st
    assert 0 < st["split_residual"] < 1e-9, st
    assert st["split_order"] == (1 if kind == "grid" else 0), st
    digest = hashlib.sha256(np.ascontiguousarray(Dg, dtype="<i4").tobytes()).hexdigest()
    if digest != rec["sha256_D"]:
        B = rec["block_rows"]
        bad = [b for b, hx in enumerate(rec["block_sha256_16"])
               if hashlib.sha256(np.ascontiguousarray(Dg[b * B:(b + 1) * B], dtype="<i4").tobytes())
               .hexdigest()[:16] != hx]
        pytest.fail(f"{len(bad)} of {len(rec['block_sha256_16'])} row blocks differ")


def test_goal_rows_follow_reloaded_graphs(rd):
    """The digits of the final L^-1 are reused between the inverse product, the self-check and the
    goal products of one factorisation.  Loading another graph of the same size (same buffers,
    same views), switching precision and back, and a second load must each give goal rows and D
    of the graph now resident: parity with the oracle after every change."""
    n = 1000
    goals = np.array([0, 17, 500, 999], np.int32)
    rows = np.empty((goals.size, n))
    D = np.empty((n, n), np.int32)
    cases = [graphs.er(n, 0.02, 11), graphs.ws(n, 10, 0.1, 12), graphs.er(n, 0.03, 13)]
    with rd.Handle(cases[0], graphs.gamma_frac(cases[0], 0.5)) as h:
        for step, A in enumerate(cases):
            g = graphs.gamma_frac(A, 0.5)
            if step:
                h.load(A, g)
            h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
            h.apsp(D)
            h.goal_solve(goals, rows)
            Do, Yo = oracle.rdistance(A, g, want_y=True)
            assert np.array_equal(D, Do), step
            assert rel_err(rows, Yo[goals]) < YTOL, step
            h.set_precision(rd.RD_PREC_FP64, 0)      # and back: the factors are recomputed
            h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
            h.goal_solve(goals, rows)
            assert rel_err(rows, Yo[goals]) < YTOL, step
        assert h.stats()["precision_used"] == rd.RD_PREC_SPLIT_BF16


def test_profiling_modes(rd):
    """rd_set_profiling: mode 1 brackets every dense-contraction launch (the split GEMM and the FP64
    products of the recursion's small nodes), mode 2 the split GEMM alone; another value is refused."""
    A, g = graphs.workload_small()
    n = A.shape[0]
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    At = torch.from_numpy(A).cuda()
    with rd.Handle(At, g, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        h.apsp(D)
        counts = {}
        for mode in (1, 2):
            rd.rd_set_profiling(h.h, mode)
            h.load(At, g)  # factored again: the recursion's products run, not just the inverse product
            h.apsp(D)
            h.sync()
            st = h.stats()
            counts[mode] = (st["prof_launches"], st["prof_split_launches"])
        with pytest.raises(rd.RDError) as ei:
            rd.rd_set_profiling(h.h, 3)
        assert ei.value.status == rd.RD_ERR_ARG
        rd.rd_set_profiling(h.h, 0)
    all1, split1 = counts[1]
    all2, split2 = counts[2]
    assert split1 > 0 and split1 == split2
    assert all1 > split1          # the FP64 products of the small nodes are counted too
    assert all2 == split2         # mode 2: the split GEMM alone
