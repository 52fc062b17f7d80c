"""Parity of the CUDA path (through the C ABI) with the CPU oracle on small and ragged sizes.

D must be bit-exact to the oracle's D.  Y must agree entrywise within a relative 1e-11:
both sides compute Y = M^-1 in FP64 with sign-definite products (every product adds terms
of one sign, see k_lu_f64.cu), so each entry carries a relative error of a few hundred ulp
at most (observed: ~1e-14), and exact zeros (unreachable pairs) stay exact zeros on both.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YTOL = 1e-11
UNR = oracle.UNREACHABLE


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def y_close(Yg, Yo):
    assert Yg.shape == Yo.shape
    assert np.array_equal(Yg == 0, Yo == 0)
    nz = Yo != 0
    if nz.any():
        err = np.max(np.abs(Yg[nz] - Yo[nz]) / np.abs(Yo[nz]))
        assert err < YTOL, err


def run_gpu(rd, A, g, W=None, device_io=True, precision=None):
    n = A.shape[0]
    if device_io:
        At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
        Wt = None if W is None else torch.from_numpy(np.ascontiguousarray(W)).cuda()
        D = torch.empty((n, n), dtype=torch.int32, device="cuda")
        Y = torch.empty((n, n), dtype=torch.float64, device="cuda")
    else:
        At, Wt = A, W
        D = np.empty((n, n), dtype=np.int32)
        Y = np.empty((n, n), dtype=np.float64)
    with rd.Handle(At, g, W=Wt, stream=torch.cuda.current_stream().cuda_stream) as h:
        if precision is not None:
            h.set_precision(*precision)
        h.apsp(D, Y)
        h.sync()
    if device_io:
        torch.cuda.synchronize()
        return D.cpu().numpy(), Y.cpu().numpy()
    return D, Y


CASES = [
    ("path3", lambda: (graphs.path3(), 0.2)),
    ("dpath40", lambda: (graphs.directed_path(40), 0.3)),
    ("dcycle17", lambda: (graphs.directed_cycle(17), 0.9)),
    ("complete64", lambda: (graphs.complete(64), 0.5 / 64)),
    ("er129", lambda: (graphs.er(129, 0.05, 1), None)),
    ("grid200", lambda: (graphs.grid4(200, 15), None)),
    ("ws257", lambda: (graphs.ws(257, 6, 0.1, 3), None)),
    ("tree300", lambda: (graphs.binary_tree(300), None)),
    ("er512_small_workload", lambda: graphs.workload_small()),
    ("grid700_ragged", lambda: (graphs.grid4(700, 26), None)),
]


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_apsp_matches_oracle(rd, name):
    A, g = dict(CASES)[name]()
    if g is None:
        g = graphs.gamma_frac(A, 0.9)
    Do, Yo = oracle.rdistance(A, g, want_y=True)
    Dg, Yg = run_gpu(rd, A, g)
    assert np.array_equal(Dg, Do), int(np.sum(Dg != Do))
    y_close(Yg, Yo)


def test_host_buffers_match_device_buffers(rd):
    A, g = graphs.workload_small(1)
    Dd, Yd = run_gpu(rd, A, g, device_io=True)
    Dh, Yh = run_gpu(rd, A, g, device_io=False)
    assert np.array_equal(Dd, Dh)
    assert np.array_equal(Yd, Yh)


def test_small_workload_bfs_agreement(rd):
    """n=512 workload: report (and bound) the fraction of D entries equal to BFS truth."""
    A, g = graphs.workload_small()
    Dg, _ = run_gpu(rd, A, g)
    Dt, _ = oracle.bfs_all(A)
    frac = float(np.mean(Dg == Dt))
    assert frac > 0.99, frac


def test_handle_reload_and_tau(rd):
    n = 150
    A1 = graphs.er(n, 0.05, 8)
    A2 = graphs.grid4(n, 13)
    g1, g2 = graphs.gamma_frac(A1, 0.5), graphs.gamma_frac(A2, 0.5)
    D = np.empty((n, n), np.int32)
    with rd.Handle(A1, g1) as h:
        h.apsp(D)
        assert np.array_equal(D, oracle.rdistance(A1, g1))
        h.load(A2, g2)
        h.apsp(D)
        assert np.array_equal(D, oracle.rdistance(A2, g2))
        rd.rd_set_tau(h.h, 1e-6)
        h.apsp(D)
        assert np.array_equal(D, oracle.rdistance(A2, g2, tau=1e-6))


def test_weighted_matches_oracle(rd):
    A, W = graphs.grid8_weighted(12, 15, 4)
    # largest column sum of gamma^W below one: 8 neighbours, weights >= 1
    g = 0.1
    Do, Yo = oracle.rdistance(A, g, W=W, want_y=True)
    Dg, Yg = run_gpu(rd, A, g, W=W)
    y_close(Yg, Yo)
    assert np.array_equal(Dg, Do)


@pytest.mark.parametrize("kind", ["er", "grid", "tree"])
def test_goal_rows_and_greedy(rd, kind):
    n = 333
    A = {"er": lambda: graphs.er(n, 0.03, 2), "grid": lambda: graphs.grid4(n, 19),
         "tree": lambda: graphs.binary_tree(n)}[kind]()
    g = graphs.gamma_frac(A, 0.9)
    goals = np.array([0, 7, 100, n - 1, 5], dtype=np.int32)
    k = goals.size
    rows_o = oracle.goal_rows(A, g, goals)
    At = torch.from_numpy(A).cuda()
    gt = torch.from_numpy(goals).cuda()
    rows = torch.empty((k, n), dtype=torch.float64, device="cuda")
    nxt = torch.empty((k, n), dtype=torch.int32, device="cuda")
    with rd.Handle(At, g, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.goal_solve(gt, rows)
        h.greedy_next(gt, rows, nxt)
        h.sync()
    torch.cuda.synchronize()
    rows_g = rows.cpu().numpy()
    nxt_g = nxt.cpu().numpy()
    y_close(rows_g, rows_o)
    # identical decisions on identical inputs
    assert np.array_equal(nxt_g, oracle.greedy_next(A, goals, rows_g))
    # the walk reaches the goal without a cycle (Theorem 4, Cor. 4.1); shortest on a tree
    Dt, _ = oracle.bfs_all(A)
    for c, goal in enumerate(goals):
        for s in range(n):
            v, seen, steps = s, {s}, 0
            while v != goal:
                v = int(nxt_g[c, v])
                steps += 1
                assert v >= 0 and v not in seen
                seen.add(v)
            if kind == "tree":
                assert steps == Dt[goal, s]


def test_goal_rows_host_pointers(rd):
    A, g = graphs.workload_small()
    goals = np.arange(0, 512, 8, dtype=np.int32)  # 64 goals, the maximum
    rows = np.empty((goals.size, 512))
    nxt = np.empty((goals.size, 512), np.int32)
    with rd.Handle(A, g) as h:
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
    y_close(rows, oracle.goal_rows(A, g, goals))
    assert np.array_equal(nxt, oracle.greedy_next(A, goals, rows))


def test_errors(rd):
    A = graphs.er(100, 0.05, 3)
    delta = graphs.max_out_degree(A)
    with pytest.raises(rd.RDError) as ei:
        rd.Handle(A, 1.0 / delta)  # gamma * Delta == 1: not strictly dominant
    assert ei.value.status == rd.RD_ERR_GAMMA
    with rd.Handle(A, 0.5 / delta) as h:
        rows = np.empty((1, 100))
        with pytest.raises(rd.RDError) as ei:
            h.goal_solve(np.array([100], np.int32), rows)
        assert ei.value.status == rd.RD_ERR_ARG
        with pytest.raises(rd.RDError):
            rd.rd_goal_solve(h.h, np.zeros(65, np.int32), 65, np.empty((65, 100)))
        with pytest.raises(rd.RDError):
            rd.rd_set_precision(h.h, 7, 0)
        # the handle still works after rejected calls
        D = np.empty((100, 100), np.int32)
        h.apsp(D)
        assert np.array_equal(D, oracle.rdistance(A, 0.5 / delta))


@pytest.mark.parametrize("precision", ["fp64", "split", "updated"])
def test_device_goal_out_of_range(rd, precision):
    """Goals in device memory are checked by the kernels that read them: a goal outside [0, n) is
    never used as an index, its row of Y stays zero and its next hops -1, the other goals' rows
    are the oracle's, and the next synchronising call returns RD_ERR_ARG naming the position.
    The handle stays usable afterwards.  ("updated": goal rows read from the resident Y that
    edge updates keep current.)"""
    A = graphs.er(200, 0.05, 4)
    n = A.shape[0]
    g = graphs.gamma_frac(A, 0.5)
    stream = torch.cuda.current_stream().cuda_stream
    bad = torch.tensor([5, n, 199, -3], dtype=torch.int32, device="cuda")
    ok_goals = np.array([5, 0, 199, 0], np.int32)
    rows = torch.full((4, n), -1.0, dtype=torch.float64, device="cuda")
    nxt = torch.full((4, n), -7, dtype=torch.int32, device="cuda")
    with rd.Handle(torch.from_numpy(A).cuda(), g, stream=stream) as h:
        if precision == "split":
            h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        if precision == "updated":
            Dd = torch.empty((n, n), dtype=torch.int32, device="cuda")
            i, j = next((i, j) for i in range(3, n) for j in range(4, n) if i != j and A[i, j] == 0)
            h.update_edge(i, j, True, Dd)   # a new edge j -> i
            A = A.copy()
            A[i, j] = 1
        h.goal_solve(bad, rows)
        with pytest.raises(rd.RDError) as ei:
            h.sync()
        assert ei.value.status == rd.RD_ERR_ARG
        msg = rd.rd_last_error(h.h)
        assert "position 1" in msg or "position 3" in msg  # the first bad goal recorded wins
        h.greedy_next(bad, rows, nxt)
        with pytest.raises(rd.RDError) as ei:
            h.sync()
        assert ei.value.status == rd.RD_ERR_ARG
        h.sync()  # reported once: the handle is usable again
        got, hops = rows.cpu().numpy(), nxt.cpu().numpy()
        ref = oracle.goal_rows(A, g, ok_goals)
        tol = YTOL if precision != "split" else 1e-10
        for c in (0, 2):
            nz = ref[c] != 0
            assert np.array_equal(got[c] == 0, ~nz)
            assert np.max(np.abs(got[c][nz] - ref[c][nz]) / ref[c][nz]) < tol
        assert np.all(got[1] == 0) and np.all(got[3] == 0)
        assert np.all(hops[1] == -1) and np.all(hops[3] == -1)
        ref_next = oracle.greedy_next(A, ok_goals[[0, 2]], got[[0, 2]])
        assert np.array_equal(hops[[0, 2]], ref_next)
        good = np.empty((2, n))
        h.goal_solve(np.array([5, 199], np.int32), good)
        assert np.array_equal(good, got[[0, 2]])


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("n", [1, 2, 65, 300])
def test_degenerate_graphs(rd, n, precision):
    """No edges at all (Y = I: D is 0 on the diagonal and the unreachable sentinel elsewhere) and a
    single node, in both precisions; goal rows are the unit rows and every greedy next hop is -1."""
    A = np.zeros((n, n), np.uint8)
    prec = (rd.RD_PREC_FP64, 0) if precision == "fp64" else (rd.RD_PREC_SPLIT_BF16, 0)
    D, Y = run_gpu(rd, A, 0.5, precision=prec)
    Do, Yo = oracle.rdistance(A, 0.5, want_y=True)
    assert np.array_equal(D, Do)
    assert np.array_equal(Y, np.eye(n)) and np.array_equal(Yo, np.eye(n))
    goals = np.arange(min(n, 4), dtype=np.int32)
    rows = np.empty((goals.size, n))
    nxt = np.empty((goals.size, n), np.int32)
    with rd.Handle(A, 0.5) as h:
        h.set_precision(*prec)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
    assert np.array_equal(rows, np.eye(n)[goals])
    assert np.array_equal(nxt, oracle.greedy_next(A, goals, rows))


def test_empty_graph_is_refused(rd):
    with pytest.raises(rd.RDError) as ei:
        rd.Handle(np.zeros((0, 0), np.uint8), 0.5)
    assert ei.value.status == rd.RD_ERR_ARG


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_infinite_weights_are_absent_edges(rd, precision):
    """W may be +inf on an edge (Sec. 3.2: the weight of a missing edge): gamma^inf = 0, so the
    result equals that of the graph without those edges, and the oracle's."""
    A, W, g = graphs.workload_weighted(12, 16)
    rng = np.random.default_rng(5)
    ii, jj = np.nonzero(A)
    cut = rng.random(ii.size) < 0.2
    Winf = W.copy()
    Winf[ii[cut], jj[cut]] = np.inf
    Acut = A.copy()
    Acut[ii[cut], jj[cut]] = 0
    prec = (rd.RD_PREC_FP64, 0) if precision == "fp64" else (rd.RD_PREC_SPLIT_BF16, 0)
    D, Y = run_gpu(rd, A, g, W=Winf, precision=prec)
    Do, Yo = oracle.rdistance(Acut, g, W=W, want_y=True)
    assert np.array_equal(D, Do)
    y_close(Y, Yo)
    # the greedy step never takes an edge of infinite weight
    goals = np.array([0, 77, 191], np.int32)
    rows = np.empty((goals.size, A.shape[0]))
    nxt = np.empty((goals.size, A.shape[0]), np.int32)
    with rd.Handle(A, g, W=Winf) as h:
        h.set_precision(*prec)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
    assert np.array_equal(nxt, oracle.greedy_next(Acut, goals, rows))


def test_zero_weight_breaks_the_gain_condition(rd):
    """A zero weight makes X_ij = gamma^0 = 1: the column sum of X reaches 1, refused."""
    A, W, g = graphs.workload_weighted(8, 8)
    W0 = W.copy()
    i, j = (int(x[0]) for x in np.nonzero(A))
    W0[i, j] = 0.0
    with pytest.raises(rd.RDError) as ei:
        rd.Handle(A, g, W=W0)
    assert ei.value.status == rd.RD_ERR_GAMMA
