"""rd_greedy_walk: the greedy walk of Sec. 4.2 along the next hops, against walks over the oracle's
next hops (a walk ends at the goal, the node that is its own next hop)."""
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


def host_walk(nxt, start, max_len):
    """(path, len) of one walk over a row of next hops."""
    path = [start]
    x = start
    for t in range(max_len + 1):
        y = int(nxt[x])
        if y == x:
            return path + [-1] * (max_len + 1 - len(path)), t
        if y < 0 or t == max_len:
            break
        x = y
        path.append(x)
    return path + [-1] * (max_len + 1 - len(path)), -1


@pytest.mark.parametrize("kind,device_io", [("er", True), ("grid", False), ("dpath", True)])
def test_walks_match_oracle_next_hops(rd, kind, device_io):
    if kind == "er":
        A = graphs.er(400, 0.02, 8)
    elif kind == "grid":
        A = graphs.grid4(500, 25)
    else:
        A = graphs.directed_path(300)   # nodes past the goal have no way to it: dead ends
    n = A.shape[0]
    g = graphs.gamma_frac(A, 0.5)
    goals = np.array([0, 57, n // 2, n - 1], np.int32)
    starts = np.array([n - 1, 3, n // 2, 10], np.int32)   # the third starts at its goal
    rows = np.empty((goals.size, n))
    nxt = np.empty((goals.size, n), np.int32)
    max_len = n // 2
    with rd.Handle(A, g) as h:
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
        if device_io:
            path_t = torch.empty((goals.size, max_len + 1), dtype=torch.int32, device="cuda")
            len_t = torch.empty(goals.size, dtype=torch.int32, device="cuda")
            h.greedy_walk(torch.from_numpy(nxt).cuda(), torch.from_numpy(starts).cuda(), max_len, path_t, len_t)
            torch.cuda.synchronize()
            path, length = path_t.cpu().numpy(), len_t.cpu().numpy()
        else:
            path = np.empty((goals.size, max_len + 1), np.int32)
            length = np.empty(goals.size, np.int32)
            h.greedy_walk(nxt, starts, max_len, path, length)
    ref_next = oracle.greedy_next(A, goals, rows)
    for c in range(goals.size):
        p, L = host_walk(ref_next[c], int(starts[c]), max_len)
        assert np.array_equal(path[c], p), (kind, c)
        assert length[c] == L, (kind, c)
    assert length[2] == 0   # started at the goal
    if kind == "dpath":
        assert length[0] == -1   # edges j -> j + 1 lead away from goal 0


def _walk(rd, h, nxt, starts, max_len, device_start):
    k = starts.size
    path = np.empty((k, max_len + 1), np.int32)
    length = np.empty(k, np.int32)
    st = torch.from_numpy(starts).cuda() if device_start else starts
    h.greedy_walk(torch.from_numpy(nxt).cuda(), st, max_len, path, length)
    return path, length


def test_walk_edge_cases_on_a_directed_path(rd):
    """Hand-computed walks on the directed path 0 -> 1 -> ... -> 19 toward goal 12: from 3 the walk
    is 3, 4, ..., 12 (9 steps).  max_len = 0 keeps the start only; a max_len shorter than the way
    ends the walk with exactly max_len + 1 nodes and length -1; a start at the goal has length 0
    even with max_len = 0; device starts outside [0, n) give an all -1 path and length -1."""
    A = graphs.directed_path(20)
    n, goal = 20, 12
    goals = np.full(4, goal, np.int32)
    with rd.Handle(A, 0.3) as h:
        rows = np.empty((4, n))
        nxt = np.empty((4, n), np.int32)
        h.goal_solve(goals, rows)
        h.greedy_next(goals, rows, nxt)
        starts = np.array([3, goal, 3, 3], np.int32)
        path, length = _walk(rd, h, nxt, starts, 0, device_start=False)
        assert path[:, 0].tolist() == [3, goal, 3, 3] and length.tolist() == [-1, 0, -1, -1]
        path, length = _walk(rd, h, nxt, starts, 4, device_start=True)
        assert path[0].tolist() == [3, 4, 5, 6, 7] and length[0] == -1
        assert path[1].tolist() == [goal, -1, -1, -1, -1] and length[1] == 0
        path, length = _walk(rd, h, nxt, starts, 9, device_start=False)
        assert path[0].tolist() == list(range(3, 13)) and length[0] == 9
        path, length = _walk(rd, h, nxt, starts, n, device_start=False)
        assert path[0].tolist() == list(range(3, 13)) + [-1] * (n + 1 - 10) and length[0] == 9
        bad = np.array([-1, n, 3, goal], np.int32)
        path, length = _walk(rd, h, nxt, bad, 6, device_start=True)
        assert path[0].tolist() == [-1] * 7 and path[1].tolist() == [-1] * 7
        assert length[:2].tolist() == [-1, -1] and length[3] == 0
        assert path[2].tolist() == [3, 4, 5, 6, 7, 8, 9] and length[2] == -1
        with pytest.raises(rd.RDError):  # host starts are checked on the host
            _walk(rd, h, nxt, bad, 6, device_start=False)
        with pytest.raises(ValueError):  # the binding checks shapes and dtypes
            h.greedy_walk(nxt[:, :10], starts, 4, np.empty((4, 5), np.int32), np.empty(4, np.int32))
        with pytest.raises(ValueError):
            h.greedy_walk(nxt, starts.astype(np.int64), 4, np.empty((4, 5), np.int32), np.empty(4, np.int32))
        with pytest.raises(ValueError):
            h.greedy_walk(nxt, starts, 4, np.empty((4, 4), np.int32), np.empty(4, np.int32))
