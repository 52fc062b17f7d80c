"""Write the stored expected values for the n=8192 single-graph workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generators; nothing here comes from the
CUDA path.  For each graph kind (ER p=0.01, 90x91 grid, WS ring k=10 beta=0.1) and gain
fraction (0.5 and 0.9 of 1/Delta) it stores, in ``large_<kind>_<frac>.json``:

  * the gain, Delta and the seed recipe,
  * sha256 of the oracle's D (int32 little-endian, row-major) and of each block of 64 rows,
  * the BFS-truth match fraction and the diameter,
  * the number of "fragile" entries: off-diagonal finite R with log_gamma(Y) - tau within
    1e-6 of an integer (the entries where a less accurate inverse could flip the ceil),
  * the smallest such distance observed (the decode margin).

Run:  python tests/golden/make_golden.py [kind frac ...]   (about 7 minutes per graph on one
core; graphs are independent and may be run in parallel processes).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2308_07403_gb300 import graphs  # noqa: E402

BLOCK = 64


def digest(D: np.ndarray) -> tuple[str, list[str]]:
    D = np.ascontiguousarray(D, dtype="<i4")
    full = hashlib.sha256(D.tobytes()).hexdigest()
    blocks = [hashlib.sha256(D[r:r + BLOCK].tobytes()).hexdigest()[:16]
              for r in range(0, D.shape[0], BLOCK)]
    return full, blocks


def one(kind: str, frac: float) -> dict:
    A, g = graphs.workload_large(kind, frac)
    n = A.shape[0]
    t0 = time.time()
    D, Y = oracle.rdistance(A, g, want_y=True)
    t_oracle = time.time() - t0
    full, blocks = digest(D)
    Dt, _ = oracle.bfs_all(A)
    match = float(np.mean(D == Dt))
    fin = Dt != oracle.UNREACHABLE
    diam = int(Dt[fin].max())
    off = ~np.eye(n, dtype=bool) & (Y > 0)
    r = np.log(Y[off]) / np.log(g) - oracle.TAU
    dist = np.abs(r - np.round(r))
    fragile = int(np.sum(dist < 1e-6))
    margin = float(dist.min()) if dist.size else 1.0
    return {
        "kind": kind, "frac": frac, "n": n, "gamma": repr(g), "delta": graphs.max_out_degree(A),
        "tau": oracle.TAU, "sha256_D": full, "block_rows": BLOCK, "block_sha256_16": blocks,
        "bfs_match_fraction": match, "diameter": diam, "fragile_1e-6": fragile,
        "min_decode_margin": margin, "y_min_positive": float(Y[Y > 0].min()),
        "oracle_seconds": round(t_oracle, 1),
        "generated_by": "tests/golden/make_golden.py (oracle only)",
    }


def main(argv):
    todo = []
    if argv:
        for i in range(0, len(argv), 2):
            todo.append((argv[i], float(argv[i + 1])))
    else:
        todo = [(k, f) for k in graphs.LARGE_KINDS for f in graphs.LARGE_FRACS]
    oracle.build()
    for kind, frac in todo:
        rec = one(kind, frac)
        path = os.path.join(HERE, f"large_{kind}_{frac}.json")
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
        print(kind, frac, rec["sha256_D"][:16], "match", rec["bfs_match_fraction"],
              "fragile", rec["fragile_1e-6"], "margin", rec["min_decode_margin"],
              "t", rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
