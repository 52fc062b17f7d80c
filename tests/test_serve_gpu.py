"""Serving (rd_serve_*): every result is the same alone and in a concurrent mix (bit-exact: the
kernels are deterministic), eviction under a small memory budget keeps results, goal solves reuse
resident factors, bad requests are refused on the host."""
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


def pool():
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
        out.append((i, A, graphs.gamma_small(A)))
    reqs = []
    for gid, A, g in out:
        reqs.append(("apsp", gid, A, g, None))
        for _ in range(2):
            k = int(rng.integers(1, 65))
            reqs.append(("goals", gid, A, g, np.sort(rng.choice(A.shape[0], size=min(k, A.shape[0]), replace=False))))
    order = rng.permutation(len(reqs))
    return [reqs[i] for i in order]


def submit(srv, rd, req):
    kind, gid, A, g, goals = req
    n = A.shape[0]
    if kind == "apsp":
        out = np.full((n, n), -7, np.int32)
        return srv.submit_apsp(gid, A, g, out), out
    out = np.full((goals.size, n), -7.0)
    return srv.submit_goals(gid, A, g, goals, out), out


def test_serve_alone_equals_mix(rd):
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
    for req, out in zip(reqs, alone):     # and the results are the method's
        kind, gid, A, g, goals = req
        if kind == "apsp" and A.shape[0] <= 700:
            assert np.array_equal(out, oracle.rdistance(A, g))


def test_serve_small_budget_evicts_and_keeps_results(rd):
    reqs = pool()
    with rd.Server(64 << 30, workers=1) as srv:
        ref = []
        for req in reqs:
            rid, out = submit(srv, rd, req)
            assert srv.wait(rid)[0] == rd.RD_OK
            ref.append(out)
    with rd.Server(300 << 20, workers=3) as srv:   # room for about one large handle at a time
        live = [submit(srv, rd, req) for req in reqs]
        for (rid, out), r in zip(live, ref):
            assert srv.wait(rid)[0] == rd.RD_OK
            assert np.array_equal(out, r)
        s = srv.stats()
    assert s["evictions"] > 0 and s["failed"] == 0


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
