"""rd_split_stats, the split GEMM's cycle counters: the default library has none and says so
(RD_ERR_UNSUPPORTED); the diagnostic build (build(stats=True)) counts the roles of the decode
product consistently -- every wait is part of its role's total, every MMA warp ran its groups -- and
its D is still the oracle's.  The diagnostic library is loaded in a child process, since a process
holds one library at a time."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2308_07403_gb300 import build, graphs, rd
rd.load(build.build(stats=True))
import oracle
# n = 2048: enough tiles that the decode product runs without split K (the counters cover the
# launches that carry the decode)
n = 2048
A = graphs.er(n, 0.01, graphs.seed_for(3))
g = graphs.gamma_frac(A, 0.5)
D = torch.empty((n, n), dtype=torch.int32, device="cuda")
with rd.Handle(torch.from_numpy(A).cuda(), g, stream=torch.cuda.current_stream().cuda_stream) as h:
    h.set_precision(rd.RD_PREC_SPLIT_BF16, 0)
    h.apsp(D)
    h.sync()
    rd.rd_split_stats(reset=True)
    h.apsp(D)
    h.sync()
    c = rd.rd_split_stats()
ok = bool(np.array_equal(D.cpu().numpy(), oracle.rdistance(A, g)))
print(json.dumps({"stats": c, "D_equal": ok}))
"""


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def test_default_build_has_no_counters(rd):
    with pytest.raises(rd.RDError) as ei:
        rd.rd_split_stats()
    assert ei.value.status == rd.RD_ERR_UNSUPPORTED
    assert "RD_SPLIT_STATS" in rd.rd_last_error()


def test_diagnostic_build_counts_the_decode_product(rd):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    c = out["stats"]
    assert out["D_equal"]
    assert c["mma_warps"] > 0 and c["epilogue_warps"] >= c["mma_warps"] and c["mmas"] > 0
    assert c["groups"] >= c["mma_warps"]  # at least one digit group per tile
    assert c["mma_wait_accumulator"] + c["mma_wait_operands"] + c["mma_issue"] <= c["mma_cycles"]
    assert c["producer_wait_stage"] <= c["producer_cycles"]
    assert c["epilogue_wait_group"] + c["epilogue_renormalise"] <= c["epilogue_cycles"]
    # every MMA takes at least 64 cycles of the tensor pipe, and the MMA warp issues them all
    assert 64 * c["mmas"] <= c["mma_cycles"] * 1.05
