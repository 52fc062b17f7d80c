"""rd_apsp_noalloc: the APSP entry point for callers that must not allocate device memory.

Some callers cannot call cudaMalloc: their device memory is handed out up front by another
runtime, or they run inside another system's time-critical loop where the implicit device
synchronisation of an allocation is not acceptable.  rd_apsp_noalloc serves them from a fixed
device array declared in the library.  This test calls it through the C ABI twice in a row on
different graphs (so stale contents of the shared array would show) and checks each D against
the CPU oracle and against the handle-based rd_apsp: both must match exactly, the tolerance the
other parity tests use for D (an integer result).  It runs last (file name) and also passes
alone in a fresh process.
"""
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


def handle_D(rd, A, g):
    n = A.shape[0]
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    with rd.Handle(torch.from_numpy(A).cuda(), g, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.apsp(D)
        h.sync()
    torch.cuda.synchronize()
    return D.cpu().numpy()


def test_noalloc_matches_oracle_and_rd_apsp_twice(rd):
    cases = [graphs.workload_small(), (graphs.grid4(300, 17), None)]
    stream = torch.cuda.current_stream().cuda_stream
    for A, g in cases:
        if g is None:
            g = graphs.gamma_frac(A, 0.9)
        n = A.shape[0]
        At = torch.from_numpy(A).cuda()
        D = torch.full((n, n), -7, dtype=torch.int32, device="cuda")
        rd.rd_apsp_noalloc(At, n, g, D, stream)
        torch.cuda.synchronize()
        got = D.cpu().numpy()
        assert np.array_equal(got, oracle.rdistance(A, g))
        assert np.array_equal(got, handle_D(rd, A, g))


def test_noalloc_rejects_what_it_cannot_hold(rd):
    n = rd.NOALLOC_MAX_N + 1
    A = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(rd.RDError) as ei:
        rd.rd_apsp_noalloc(A, n, 0.1, D)
    assert ei.value.status == rd.RD_ERR_ARG
    assert "scratch" in rd.rd_last_error()
    # host buffers are refused: the caller passes device memory
    Ah = np.zeros((8, 8), np.uint8)
    Dh = np.zeros((8, 8), np.int32)
    with pytest.raises(rd.RDError):
        rd.rd_apsp_noalloc(Ah, 8, 0.1, Dh)
