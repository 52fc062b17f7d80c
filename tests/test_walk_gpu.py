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
