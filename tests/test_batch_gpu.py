"""Batched graphs (rd_batch_*): every graph of a mixed batch in one launch, D bit-exact against the
oracle graph by graph, per-graph gain rejection, determinism across runs, argument errors."""
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


def mixed_batch():
    """The batched recipe's mix plus edge sizes (1, 2, 63, 64, 65, 128, 130, 512), closed-form
    families, and one graph whose gain breaks the column-sum bound."""
    kinds, n, As, g = graphs.workload_batched(40, 32, 512, replica=5)
    As, gs = list(As), list(g)
    for m in (1, 2, 63, 64, 65, 128, 130, 512):
        A = graphs.er(m, min(1.0, 4.0 / m), 77 + m)
        As.append(A)
        gs.append(graphs.gamma_small(A))
    for A, gam in ((graphs.directed_path(100), 0.3), (graphs.binary_tree(200), None),
                   (graphs.grid4(300, 17), None), (graphs.complete(40), 0.5 / 40)):
        As.append(A)
        gs.append(graphs.gamma_small(A) if gam is None else gam)
    bad = len(As)
    As.append(graphs.complete(20))
    gs.append(0.9)  # 0.9 * 19 >= 1: rejected
    ns = np.array([A.shape[0] for A in As], dtype=np.int32)
    return ns, As, np.array(gs), bad


def run(rd, ns, As, gs, fill=-7):
    with rd.Batch(ns, gs) as b:
        off = b.offsets()
        packed = np.zeros(int(off[-1]), dtype=np.uint8)
        for g, A in enumerate(As):
            packed[off[g]:off[g + 1]] = np.ascontiguousarray(A).ravel()
        A_dev = torch.from_numpy(packed).cuda()
        D_dev = torch.full((int(off[-1]),), fill, dtype=torch.int32, device="cuda")
        b.apsp(A_dev, D_dev, torch.cuda.current_stream().cuda_stream)
        st = b.status()
    return off, D_dev.cpu().numpy(), st


def test_batch_matches_oracle(rd):
    ns, As, gs, bad = mixed_batch()
    off, D, st = run(rd, ns, As, gs)
    for g, A in enumerate(As):
        n = int(ns[g])
        Dg = D[off[g]:off[g + 1]].reshape(n, n)
        if g == bad:
            assert st[g] == rd.RD_ERR_GAMMA
            assert (Dg == -7).all()  # untouched
            continue
        assert st[g] == rd.RD_OK, (g, n, st[g])
        assert np.array_equal(Dg, oracle.rdistance(A, float(gs[g]))), (g, n)


def test_batch_deterministic(rd):
    kinds, ns, As, gs = graphs.workload_batched(24, 32, 256, replica=6)
    off1, D1, st1 = run(rd, ns, As, gs)
    off2, D2, st2 = run(rd, ns, As, gs, fill=0)
    assert (st1 == rd.RD_OK).all() and (st2 == rd.RD_OK).all()
    assert np.array_equal(D1, D2)


def test_batch_rejects_bad_sizes(rd):
    for ns in ([0, 10], [10, rd.BATCH_MAX_N + 1]):
        with pytest.raises(rd.RDError) as ei:
            rd.Batch(np.array(ns), np.array([0.1, 0.1]))
        assert ei.value.status == rd.RD_ERR_ARG


# ---- the split variant (rd_batch_set_precision) ------------------------------------------------

def run_split(rd, ns, As, gs, autotune, fill=-7, graph_capture=False):
    """Pack, run in split mode (optionally as a captured CUDA graph, replayed twice), and return
    offsets, D, status, routes and the tuning record."""
    with rd.Batch(ns, gs) as b:
        b.set_precision(rd.RD_PREC_SPLIT_BF16, autotune)
        off = b.offsets()
        packed = np.zeros(int(off[-1]), dtype=np.uint8)
        for g, A in enumerate(As):
            packed[off[g]:off[g + 1]] = np.ascontiguousarray(A).ravel()
        A_dev = torch.from_numpy(packed).cuda()
        D_dev = torch.full((int(off[-1]),), fill, dtype=torch.int32, device="cuda")
        if graph_capture:
            s = torch.cuda.Stream()
            b.apsp(A_dev, D_dev, s.cuda_stream)   # warm-up outside the capture
            s.synchronize()
            D_dev.fill_(fill)
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, stream=s):
                b.apsp(A_dev, D_dev, torch.cuda.current_stream().cuda_stream)
            D_dev.fill_(fill)
            cg.replay()
            cg.replay()
            torch.cuda.synchronize()
        else:
            b.apsp(A_dev, D_dev, torch.cuda.current_stream().cuda_stream)
        st = b.status()
        routes = b.routes()
        tune = b.tuning()
        info = b.split_info()
    # the record agrees with the routes: a kept split result has its digit count (8..15) and one or
    # two passes; nothing else has digits
    kept = routes == 1
    assert ((info["digits"] >= 8) & (info["digits"] <= 15))[kept].all()
    assert np.isin(info["passes"][kept], (1, 2)).all()
    assert (info["digits"][~kept] == 0).all()
    return off, D_dev.cpu().numpy(), st, routes, tune


def test_batch_split_matches_oracle(rd):
    """Every size class forced onto the split path: D of every graph bit-exact against the oracle,
    whatever route it took (split kept, redone in FP64 after the residual check, screened to FP64);
    the gain-breaking graph is refused and its D left untouched; the ER and WS graphs of the larger
    classes stay on the split path, the wide grid is screened off it."""
    ns, As, gs, bad = mixed_batch()
    off, D, st, routes, tune = run_split(rd, ns, As, gs, autotune=False)
    for g, A in enumerate(As):
        n = int(ns[g])
        Dg = D[off[g]:off[g + 1]].reshape(n, n)
        if g == bad:
            assert st[g] == rd.RD_ERR_GAMMA and routes[g] == 4
            assert (Dg == -7).all()
            continue
        assert st[g] == rd.RD_OK, (g, n, st[g], routes[g])
        assert routes[g] in (1, 2, 3), (g, routes[g])
        assert np.array_equal(Dg, oracle.rdistance(A, float(gs[g]))), (g, n, routes[g])
    assert (routes == 1).sum() >= len(As) // 2, routes
    assert tune["split"] == [1 if c else 0 for c in tune["graphs"]]


def test_batch_split_autotune_and_graph_capture(rd):
    """The autotuned split variant captured in a CUDA graph and replayed twice: every graph equals
    the oracle; the tuning record has a measured time for both variants in every class present."""
    kinds, ns, As, gs = graphs.workload_batched(48, 200, 512, replica=7)
    off, D, st, routes, tune = run_split(rd, ns, As, gs, autotune=True, graph_capture=True)
    assert (st == rd.RD_OK).all()
    for g, A in enumerate(As):
        n = int(ns[g])
        assert np.array_equal(D[off[g]:off[g + 1]].reshape(n, n), oracle.rdistance(A, float(gs[g]))), (g, n)
    for c, cnt in enumerate(tune["graphs"]):
        if cnt:
            assert tune["ms_per_graph_fp64"][c] > 0 and tune["ms_per_graph_split"][c] > 0
            assert tune["split"][c] == int(tune["ms_per_graph_split"][c] < tune["ms_per_graph_fp64"][c])
