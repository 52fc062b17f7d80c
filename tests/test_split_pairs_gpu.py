"""The split GEMM as CTA pairs (tcgen05 cta_group::2: a cluster of two CTAs per 256 x 128 output
tile, each CTA loading its own 128 rows of A and half of B, the leader issuing the MMAs for both;
used for products with 256-wide chunks) against the one-CTA kernel and the CPU oracle.

* n = 256 and 512: the only pair launch is the inverse product with the fused decode (the
  recursion's products run in FP64 up to 512 rows, and the 64-row self-check and goal products
  fill no pair), which never splits K, so the group sums and the epilogue's arithmetic are the
  same entry by entry: D and Y must be bit-identical to the one-CTA kernel's, and D the oracle's.
* n = 2048: every split product of 256 rows or more runs on pairs (with split K where tiles are
  few) in the natural order (256-wide chunks, ER); the grid runs in the locality order (64-wide
  chunks, one-CTA kernel): D must equal the oracle's and Y must stay within the split tolerance
  (1e-10) of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YTOL = 1e-10


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def run_split(rd, A, g, pairs, monkeypatch):
    """D, Y and stats of the split path (digits chosen by the library) with or without pairs."""
    monkeypatch.setenv("RD_SPLIT_CTA_PAIRS", "1" if pairs else "0")  # read by rd_create
    n = A.shape[0]
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    Y = torch.empty((n, n), dtype=torch.float64, device="cuda")
    with rd.Handle(torch.from_numpy(A).cuda(), g, stream=torch.cuda.current_stream().cuda_stream) as h:
        h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
        h.apsp(D, Y)
        h.sync()
        st = h.stats()
    torch.cuda.synchronize()
    return D.cpu().numpy(), Y.cpu().numpy(), st


@pytest.mark.parametrize("n", [256, 512])
def test_pairs_bit_identical_to_single_ctas(rd, n, monkeypatch):
    A = graphs.er(n, 8.0 / n, 31)
    g = graphs.gamma_frac(A, 0.5)
    D1, Y1, s1 = run_split(rd, A, g, True, monkeypatch)
    D0, Y0, s0 = run_split(rd, A, g, False, monkeypatch)
    assert s1["precision_used"] == rd.RD_PREC_SPLIT_BF16 and s1["slices"] == s0["slices"]
    assert np.array_equal(Y1.view(np.int64), Y0.view(np.int64))
    assert np.array_equal(D1, D0)
    assert np.array_equal(D1, oracle.rdistance(A, g))


@pytest.mark.parametrize("kind", ["er", "grid"])
def test_pairs_match_oracle(rd, kind, monkeypatch):
    n = 2048
    A = graphs.er(n, 0.01 * 8192 / n, 32) if kind == "er" else graphs.grid4(n, 46)
    g = graphs.gamma_frac(A, 0.5)
    D, Y, st = run_split(rd, A, g, True, monkeypatch)
    assert st["precision_used"] == rd.RD_PREC_SPLIT_BF16
    if kind == "grid":
        assert st["split_order"] != 0  # the locality order: 64-wide chunks
    Do, Yo = oracle.rdistance(A, g, want_y=True)
    assert np.array_equal(D, Do)
    assert np.array_equal(Y == 0, Yo == 0)
    nz = Yo != 0
    assert np.max(np.abs(Y[nz] - Yo[nz]) / Yo[nz]) < YTOL
