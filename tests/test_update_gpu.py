"""Incremental edge updates (rd_update_edge, Sherman-Morrison on a resident Y): after every change
D equals the oracle's D of the changed graph; removals that cancel entries refactor; goal rows and
greedy next hops follow the changed graph; a change that breaks the gain condition is refused."""
import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def rel_err(a, b):
    nz = b != 0
    assert np.array_equal(a == 0, b == 0)
    return float(np.max(np.abs(a[nz] - b[nz]) / np.abs(b[nz]))) if nz.any() else 0.0


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_add_edges_match_oracle(rd, precision):
    A = graphs.er(300, 0.02, 5)
    g = 0.5 / (graphs.max_out_degree(A) + 3)  # room for a few more out-edges per node
    n = A.shape[0]
    rng = np.random.default_rng(1)
    D = np.empty((n, n), np.int32)
    Y = np.empty((n, n))
    with rd.Handle(A, g) as h:
        h.set_precision(rd.RD_PREC_FP64 if precision == "fp64" else rd.RD_PREC_SPLIT_BF16, 0)
        h.apsp(D)
        B = A.copy()
        for _ in range(6):
            while True:
                i, j = (int(x) for x in rng.integers(0, n, 2))
                if i != j and not B[i, j]:
                    break
            B[i, j] = 1
            h.update_edge(i, j, True, D, Y)
            Do, Yo = oracle.rdistance(B, g, want_y=True)
            assert np.array_equal(D, Do)
            assert rel_err(Y, Yo) < 1e-10
        st = h.stats()
    assert st["edge_updates"] == 6 and st["update_refactors"] == 0


def test_removing_a_bridge_refactors(rd):
    A = graphs.binary_tree(127)   # every edge is a bridge: removing one cuts a subtree off
    g = graphs.gamma_small(A)
    n = A.shape[0]
    D = np.empty((n, n), np.int32)
    with rd.Handle(A, g) as h:
        h.apsp(D)
        i, j = np.argwhere(A)[10]
        B = A.copy()
        B[i, j] = 0
        h.update_edge(int(i), int(j), False, D)
        st = h.stats()
        assert np.array_equal(D, oracle.rdistance(B, g))
        assert (D == rd.RD_UNREACHABLE).sum() > (oracle.rdistance(A, g) == rd.RD_UNREACHABLE).sum()
    assert st["update_refactors"] >= 1


def test_goal_rows_and_greedy_after_updates(rd):
    A = graphs.grid4(200, 15)
    g = 0.5 / (graphs.max_out_degree(A) + 2)
    n = A.shape[0]
    D = np.empty((n, n), np.int32)
    B = A.copy()
    goals = np.array([0, 77, 199], np.int32)
    rows = np.empty((goals.size, n))
    nxt = np.empty((goals.size, n), np.int32)
    with rd.Handle(A, g) as h:
        h.apsp(D)
        for (i, j) in ((50, 120), (120, 50), (3, 180)):  # shortcuts
            B[i, j] = 1
            h.update_edge(i, j, True, D)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
    assert rel_err(rows, oracle.goal_rows(B, g, goals)) < 1e-10
    assert np.array_equal(nxt, oracle.greedy_next(B, goals, rows))
    assert np.array_equal(D, oracle.rdistance(B, g))


def test_update_breaking_the_gain_is_refused(rd):
    A = graphs.complete(20)
    A[0, 1] = 0  # column 1 has one edge fewer
    g = 0.99 / 19  # gamma * 18 < 1, gamma * 19 < 1 ... but not with an added self-loop
    n = A.shape[0]
    D = np.empty((n, n), np.int32)
    with rd.Handle(A, g) as h:
        h.apsp(D)
        D0 = D.copy()
        h.update_edge(0, 1, True, D)           # column 1 back to 19 edges: 0.99 < 1, fine
        assert np.array_equal(D, oracle.rdistance(graphs.complete(20), g))
        with pytest.raises(rd.RDError) as ei:
            h.update_edge(1, 1, True, D)       # a self-loop makes column 1 sum to 20 g > 1
        assert ei.value.status == rd.RD_ERR_GAMMA
        h.update_edge(0, 1, False, D)          # back to A: the refusal changed nothing
        assert np.array_equal(D, D0)


def test_weighted_edge_reweight(rd):
    A, W, g = graphs.workload_weighted(12, 16)
    n = A.shape[0]
    D = np.empty((n, n), np.int32)
    with rd.Handle(A, g, W=W) as h:
        h.apsp(D)
        i, j = np.argwhere(A)[40]
        W2 = W.copy()
        W2[i, j] = 3.5 if W[i, j] < 2.5 else 1.5
        ok = np.bincount(np.nonzero(A)[1], weights=np.power(g, W2[np.nonzero(A)].astype(float)), minlength=n).max() < 1
        assert ok
        h.update_edge(int(i), int(j), True, D, w=float(W2[i, j]))
    assert np.array_equal(D, oracle.rdistance(A, g, W=W2))


@pytest.mark.parametrize("n,offset", [(300, 0), (300, 1), (301, 0)])
def test_update_into_device_views(rd, n, offset):
    """D as a device tensor: aligned with even n (two entries per access), a view 4 bytes into its
    buffer (not 8-byte aligned: one entry per access) and odd n; D equals the oracle's after each
    added edge."""
    A = graphs.er(n, 0.02, 9)
    g = 0.5 / (graphs.max_out_degree(A) + 3)
    rng = np.random.default_rng(4)
    buf = torch.empty(n * n + offset, dtype=torch.int32, device="cuda")
    D = buf[offset:].view(n, n)
    assert (D.data_ptr() % 8 == 0) == (offset == 0)
    with rd.Handle(A, g) as h:
        h.set_precision(rd.RD_PREC_FP64, 0)
        h.apsp(D)
        B = A.copy()
        for _ in range(3):
            while True:
                i, j = (int(x) for x in rng.integers(0, n, 2))
                if i != j and not B[i, j]:
                    break
            B[i, j] = 1
            h.update_edge(i, j, True, D)
            torch.cuda.synchronize()
            assert np.array_equal(D.cpu().numpy(), oracle.rdistance(B, g))
