"""Serving (rd_serve_*): every result is the same alone and in a concurrent mix (bit-exact: the
kernels are deterministic) and is the method's (D against the CPU oracle, goal rows against the
oracle's rows of Y); eviction under a small memory budget keeps results; a graph id resubmitted
at another size replaces its resident graph; goal solves reuse resident factors; bad and
oversized requests are refused on the host; a bounded wait runs out with RD_ERR_TIMEOUT."""
import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YTOL = {0: 1e-11, 1: 1e-10}  # goal rows: FP64 path, split path (digit count chosen by the library)


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def pool():
    """Requests over 8 graphs (ER, grid, WS; n from 64 to 1500), half of the graphs in FP64 and
    half in split precision, each graph with one full APSP and two goal-row requests, shuffled."""
    rng = np.random.default_rng(11)
    out = []
    for i, n in enumerate((64, 100, 200, 300, 513, 700, 1024, 1500)):
        kind = ("er", "grid", "ws")[i % 3]
        if kind == "er":
            A = graphs.er(n, 4.0 / n, 100 + i)
        elif kind == "grid":
            A = graphs.grid4(n, int(np.ceil(np.sqrt(n))))
        else:
            A = graphs.ws(n, 10, 0.1, 100 + i)
        out.append((i, A, graphs.gamma_small(A), i % 2))   # precision 0 = FP64, 1 = split
    reqs = []
    for gid, A, g, prec in out:
        reqs.append(("apsp", gid, A, g, None, prec))
        for _ in range(2):
            k = int(rng.integers(1, 65))
            goals = np.sort(rng.choice(A.shape[0], size=min(k, A.shape[0]), replace=False))
            reqs.append(("goals", gid, A, g, goals, prec))
    order = rng.permutation(len(reqs))
    return [reqs[i] for i in order]


def submit(srv, rd, req):
    kind, gid, A, g, goals, prec = req
    n = A.shape[0]
    if kind == "apsp":
        out = np.full((n, n), -7, np.int32)
        return srv.submit_apsp(gid, A, g, out, precision=prec), out
    out = np.full((goals.size, n), -7.0)
    return srv.submit_goals(gid, A, g, goals, out, precision=prec), out


@pytest.fixture(scope="module")
def oracle_results():
    """Per graph id: the oracle's D and Y (one CPU inverse per graph)."""
    res = {}
    for kind, gid, A, g, goals, prec in pool():
        if gid not in res:
            res[gid] = oracle.rdistance(A, g, want_y=True)
    return res


def check_against_oracle(req, out, oracle_results):
    kind, gid, A, g, goals, prec = req
    D, Y = oracle_results[gid]
    if kind == "apsp":
        assert np.array_equal(out, D), (gid, prec)
        return
    ref = Y[goals]
    assert np.array_equal(out == 0, ref == 0)
    nz = ref != 0
    err = np.max(np.abs(out[nz] - ref[nz]) / ref[nz])
    assert err < YTOL[prec], (gid, prec, err)


def test_serve_alone_equals_mix_and_the_oracle(rd, oracle_results):
    reqs = pool()
    alone = []
    with rd.Server(64 << 30, workers=1) as srv:
        for req in reqs:
            rid, out = submit(srv, rd, req)
            st, _ = srv.wait(rid)
            assert st == rd.RD_OK
            alone.append(out)
    with rd.Server(64 << 30, workers=4) as srv:
        live = [submit(srv, rd, req) for req in reqs]
        for (rid, out), ref in zip(live, alone):
            st, _ = srv.wait(rid)
            assert st == rd.RD_OK
            assert np.array_equal(out, ref)
        s = srv.stats()
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert s["max_inflight"] > 1          # the work overlapped
    assert s["reused"] >= len(reqs) - 8   # goal solves on resident factors
    # goal requests on graphs of at most 1024 nodes ran on the device loop, the rest on the host path
    assert s["loop_requests"] == sum(r[0] == "goals" and r[2].shape[0] <= 1024 for r in reqs)
    for req, out in zip(reqs, alone):     # and the results are the method's
        check_against_oracle(req, out, oracle_results)


def test_serve_small_budget_evicts_and_keeps_results(rd, oracle_results):
    reqs = pool()
    with rd.Server(300 << 20, workers=3) as srv:   # less than the pool's ~380 MB: graphs are evicted
        live = [submit(srv, rd, req) for req in reqs]
        for (rid, out), req in zip(live, reqs):
            assert srv.wait(rid)[0] == rd.RD_OK
            check_against_oracle(req, out, oracle_results)
        s = srv.stats()
    assert s["evictions"] > 0 and s["failed"] == 0


def test_serve_graph_id_reused_at_another_size(rd):
    """One graph id submitted with graphs of two sizes (and both precisions), beside another id's
    resident graph, under a 200 MB budget: the resident graph of the id is replaced each time
    (never evicted while in use, never freed twice), the other graph is evicted when room is
    needed, and every result is the oracle's."""
    small = graphs.er(300, 0.02, 5)
    large = graphs.ws(900, 10, 0.1, 6)
    cases = [(small, 0), (large, 1), (small, 1), (large, 0), (small, 0)]
    refs = {id(A): oracle.rdistance(A, graphs.gamma_small(A)) for A, _ in cases}
    other = graphs.grid4(1000, 32)
    with rd.Server(200 << 20, workers=2) as srv:
        Do = np.empty((1000, 1000), np.int32)
        assert srv.wait(srv.submit_apsp(3, other, graphs.gamma_small(other), Do))[0] == rd.RD_OK
        live = []
        for A, prec in cases:
            n = A.shape[0]
            out = np.full((n, n), -7, np.int32)
            live.append((srv.submit_apsp(7, A, graphs.gamma_small(A), out, precision=prec), out, A))
        for rid, out, A in live:
            assert srv.wait(rid)[0] == rd.RD_OK
            assert np.array_equal(out, refs[id(A)])
        s = srv.stats()
    assert s["failed"] == 0 and s["resident_graphs"] <= 2 and s["evictions"] >= 1


def test_serve_bounded_wait_times_out(rd):
    """rd_serve_wait_for gives up after its limit with RD_ERR_TIMEOUT while the request keeps
    running; a later wait returns its result.  One worker holds a large FP64 APSP, so a request
    queued behind it cannot complete within 1 ms."""
    big = graphs.er(4096, 4.0 / 4096, 9)
    small = graphs.er(64, 0.05, 10)
    with rd.Server(8 << 30, workers=1) as srv:
        Db = np.empty((4096, 4096), np.int32)
        Ds = np.empty((64, 64), np.int32)
        rb = srv.submit_apsp(1, big, graphs.gamma_small(big), Db, precision=rd.RD_PREC_FP64)
        rs = srv.submit_apsp(2, small, graphs.gamma_small(small), Ds, precision=rd.RD_PREC_FP64)
        with pytest.raises(rd.RDError) as ei:
            srv.wait(rs, timeout_ms=1.0)
        assert ei.value.status == rd.RD_ERR_TIMEOUT
        assert srv.wait(rb)[0] == rd.RD_OK
        assert srv.wait(rs, timeout_ms=60_000.0)[0] == rd.RD_OK
    assert np.array_equal(Ds, oracle.rdistance(small, graphs.gamma_small(small)))


def test_serve_rejects_bad_requests(rd):
    A = graphs.er(64, 0.05, 1)
    with rd.Server(1 << 30, workers=1) as srv:
        for bad in (lambda: srv.submit_goals(0, A, 0.01, np.arange(65), np.empty((65, 64))),
                    lambda: srv.submit_apsp(0, A, 1.5, np.empty((64, 64), np.int32))):
            with pytest.raises(rd.RDError) as ei:
                bad()
            assert ei.value.status == rd.RD_ERR_ARG
        with pytest.raises(ValueError):
            srv.submit_apsp(0, A, 0.01, np.empty((64, 64), np.int64))
    big = graphs.er(2048, 2.0 / 2048, 2)
    with rd.Server(64 << 20, workers=1) as srv:   # a 2048-node handle needs more than 64 MB
        with pytest.raises(rd.RDError) as ei:
            srv.submit_apsp(0, big, graphs.gamma_small(big), np.empty((2048, 2048), np.int32))
        assert ei.value.status == rd.RD_ERR_OOM


def test_serve_device_loop_bounded_wait_and_recovery(rd):
    """The device loop's failure path: a request whose descriptor is never marked ready makes the
    loop's bounded wait run out (RD_ERR_TIMEOUT, reported by the device), and the loop goes on
    serving: goal requests before and after are the oracle's rows."""
    A = graphs.ws(600, 10, 0.1, 12)  # (600 <= 1024: the loop serves it)
    g = graphs.gamma_small(A)
    goals = np.array([0, 17, 333, 599], np.int32)
    ref = oracle.goal_rows(A, g, goals)
    with rd.Server(4 << 30, workers=2) as srv:
        for precision in (rd.RD_PREC_FP64, rd.RD_PREC_SPLIT_BF16):
            out = np.empty((goals.size, 600))
            assert srv.wait(srv.submit_goals(5 + precision, A, g, goals, out, precision=precision))[0] == rd.RD_OK
            assert np.max(np.abs(out - ref) / ref) < YTOL[precision]
        assert srv.loop_check() == rd.RD_ERR_TIMEOUT
        out = np.empty((goals.size, 600))
        assert srv.wait(srv.submit_goals(5, A, g, goals, out, precision=rd.RD_PREC_FP64))[0] == rd.RD_OK
        assert np.max(np.abs(out - ref) / ref) < YTOL[0]
        s = srv.stats()
    assert s["loop_requests"] == 3 and s["failed"] == 0


def test_serve_large_goal_requests_take_the_host_path(rd):
    """Goal requests on graphs of more than 1024 nodes run through rd_goal_solve on the worker's
    stream: on the directed path 0 -> 1 -> ... the row of goal g is gamma^(g - j) for j <= g and 0
    beyond (the closed form of Y)."""
    n, gam = 4300, 0.9
    A = graphs.directed_path(n)
    goals = np.array([0, 5, 2000, n - 1], np.int32)
    out = np.empty((goals.size, n))
    with rd.Server(8 << 30, workers=1) as srv:
        assert srv.wait(srv.submit_goals(1, A, gam, goals, out, precision=rd.RD_PREC_FP64))[0] == rd.RD_OK
        s = srv.stats()
    assert s["loop_requests"] == 0
    j = np.arange(n)
    for c, g in enumerate(goals):
        ref = np.where(j <= g, float(gam) ** np.maximum(g - j, 0), 0.0)
        nz = ref > 0
        assert np.array_equal(out[c] == 0, ~nz)
        assert np.max(np.abs(out[c][nz] - ref[nz]) / ref[nz]) < 1e-11
