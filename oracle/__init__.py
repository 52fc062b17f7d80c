"""CPU oracle for the R-distance method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library never imports, links or calls it, and the two share no
code: the only common module is the seeded input generator
(``paper_2308_07403_gb300.graphs``), which holds no R-distance arithmetic.

Layers:
  * ``rd_oracle.c`` (plain C, single thread, FP64, built with ``-ffp-contract=off``): the
    dense definition Y = (I - gamma A)^-1 by unblocked no-pivot LU plus column solves, the
    decode D = ceil(log_gamma Y - tau), goal rows, the series fixpoint, BFS with shortest
    path counts, greedy next hop and Dijkstra.  Wrapped here with ctypes.
  * ``exact.py``: exact rational arithmetic for tiny graphs.

Every function cites the passage of the paper it follows; see ``rd_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rd_oracle.c")
LIB = os.path.join(HERE, "_build", "librd_oracle.so")
TAU = 1e-9
UNREACHABLE = 2**31 - 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rd_oracle.c into oracle/_build/librd_oracle.so with gcc (idempotent)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        sig = {
            "rdo_build_m": (None, [P, I64, D, P]),
            "rdo_build_m_weighted": (None, [P, P, I64, D, P]),
            "rdo_max_column_sum": (D, [P, I64]),
            "rdo_lu_nopivot": (I64, [P, I64]),
            "rdo_inverse_from_lu": (None, [P, I64, P]),
            "rdo_goal_rows": (None, [P, I64, P, I64, P]),
            "rdo_decode": (I64, [P, I64, D, D, P]),
            "rdo_decode_vector": (None, [P, I64, I64, D, D, P]),
            "rdo_rdistance": (I64, [P, P, I64, D, D, P, P]),
            "rdo_series_vector": (I64, [P, P, I64, D, I64, ctypes.c_int, I64, P]),
            "rdo_bfs": (ctypes.c_int, [P, I64, P, I64, P, P]),
            "rdo_greedy_next": (None, [P, I64, P, I64, P, P]),
            "rdo_dijkstra": (ctypes.c_int, [P, P, I64, P, I64, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u8(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint8)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    return A


def _f32(W, n):
    if W is None:
        return None
    W = np.ascontiguousarray(W, dtype=np.float32)
    if W.shape != (n, n):
        raise ValueError("W must match A")
    return W


def build_m(A, gamma: float, W=None) -> np.ndarray:
    """M = I - gamma A (Sec. 2) or M = I - gamma^W (Sec. 3.2)."""
    A = _u8(A)
    n = A.shape[0]
    M = np.empty((n, n), dtype=np.float64)
    W = _f32(W, n)
    if W is None:
        _load().rdo_build_m(_ptr(A), n, float(gamma), _ptr(M))
    else:
        _load().rdo_build_m_weighted(_ptr(A), _ptr(W), n, float(gamma), _ptr(M))
    return M


def spectral_radius(A, gamma: float = 1.0, W=None) -> float:
    """rho(X) for X = gamma A (or gamma^W on the edges): the largest eigenvalue modulus, from a
    dense eigenvalue routine (a library primitive).  Theorem 1: the walk series of Sec. 3.1
    converges iff rho(X) < 1.  Plain numpy, for tests."""
    n = np.asarray(A).shape[0]
    if n == 0:
        return 0.0
    X = np.asarray(A, dtype=np.float64) * gamma if W is None else \
        np.where(np.asarray(A) != 0, np.power(gamma, np.asarray(W, dtype=np.float64)), 0.0)
    return float(np.max(np.abs(np.linalg.eigvals(X))))


def max_column_sum(M: np.ndarray) -> float:
    M = np.ascontiguousarray(M, dtype=np.float64)
    return float(_load().rdo_max_column_sum(_ptr(M), M.shape[0]))


def lu(A, gamma: float, W=None) -> np.ndarray:
    """Packed no-pivot LU factors of M (strict lower = L, upper = U)."""
    M = build_m(A, gamma, W)
    st = _load().rdo_lu_nopivot(_ptr(M), M.shape[0])
    if st != 0:
        raise ArithmeticError(f"non-positive pivot at {st - 1}")
    return M


def inverse(A, gamma: float, W=None) -> np.ndarray:
    """Y = M^-1 via LU and column solves."""
    LU = lu(A, gamma, W)
    n = LU.shape[0]
    Y = np.empty((n, n), dtype=np.float64)
    _load().rdo_inverse_from_lu(_ptr(LU), n, _ptr(Y))
    return Y


def decode(Y: np.ndarray, gamma: float, tau: float = TAU) -> np.ndarray:
    """D = ceil(log_gamma Y - tau) with D_ii = 0 and the sentinel for Y <= 0."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    n = Y.shape[0]
    D = np.empty((n, n), dtype=np.int32)
    bad = _load().rdo_decode(_ptr(Y), n, float(gamma), float(tau), _ptr(D))
    if bad:
        raise ArithmeticError(f"{bad} non-finite entries of Y")
    return D


def decode_vector(y, diag: int, gamma: float, tau: float = TAU) -> np.ndarray:
    """Decode one row (or column) ``diag`` of Y."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    D = np.empty(y.size, dtype=np.int32)
    _load().rdo_decode_vector(_ptr(y), y.size, int(diag), float(gamma), float(tau), _ptr(D))
    return D


def rdistance(A, gamma: float, W=None, tau: float = TAU, want_y: bool = False):
    """The whole method on the CPU: returns D (and Y when ``want_y``)."""
    A = _u8(A)
    n = A.shape[0]
    W = _f32(W, n)
    D = np.empty((n, n), dtype=np.int32)
    Y = np.empty((n, n), dtype=np.float64) if want_y else None
    st = _load().rdo_rdistance(_ptr(A), _ptr(W), n, float(gamma), float(tau), _ptr(D), _ptr(Y))
    if st != 0:
        raise ArithmeticError(f"oracle status {st}")
    return (D, Y) if want_y else D


def goal_rows(A, gamma: float, goals, W=None) -> np.ndarray:
    """Rows g of Y for each goal, by transposed solves on the LU factors."""
    LU = lu(A, gamma, W)
    n = LU.shape[0]
    goals = np.ascontiguousarray(goals, dtype=np.int32)
    out = np.empty((goals.size, n), dtype=np.float64)
    _load().rdo_goal_rows(_ptr(LU), n, _ptr(goals), goals.size, _ptr(out))
    return out


def series_vector(A, gamma: float, j: int, transpose: bool = False, W=None,
                  max_iter: int = 1_000_000):
    """Column j (or row j with ``transpose``) of Y from the partial sums of sum_k X^k."""
    A = _u8(A)
    n = A.shape[0]
    W = _f32(W, n)
    y = np.empty(n, dtype=np.float64)
    it = _load().rdo_series_vector(_ptr(A), _ptr(W), n, float(gamma), int(j), int(bool(transpose)),
                                   int(max_iter), _ptr(y))
    if it < 0:
        raise ArithmeticError("series did not reach a fixpoint")
    return y, int(it)


def bfs(A, srcs):
    """Shortest distances and path counts from each source: (dist, count), rows = sources.

    dist[s, i] = D[i, srcs[s]] (distance srcs[s] -> i), count[s, i] = S[i, srcs[s]].
    """
    A = _u8(A)
    n = A.shape[0]
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    dist = np.empty((srcs.size, n), dtype=np.int32)
    cnt = np.empty((srcs.size, n), dtype=np.float64)
    if _load().rdo_bfs(_ptr(A), n, _ptr(srcs), srcs.size, _ptr(dist), _ptr(cnt)) != 0:
        raise MemoryError
    return dist, cnt


def bfs_all(A):
    """Full truth matrices in the paper's orientation: D[i, j] and S[i, j] (from j to i)."""
    n = _u8(A).shape[0]
    dist, cnt = bfs(A, np.arange(n, dtype=np.int32))
    return np.ascontiguousarray(dist.T), np.ascontiguousarray(cnt.T)


def greedy_next(A, goals, Yrows) -> np.ndarray:
    A = _u8(A)
    n = A.shape[0]
    goals = np.ascontiguousarray(goals, dtype=np.int32)
    Yrows = np.ascontiguousarray(Yrows, dtype=np.float64)
    nxt = np.empty((goals.size, n), dtype=np.int32)
    _load().rdo_greedy_next(_ptr(A), n, _ptr(goals), goals.size, _ptr(Yrows), _ptr(nxt))
    return nxt


def dijkstra(A, W, srcs) -> np.ndarray:
    A = _u8(A)
    n = A.shape[0]
    W = _f32(W, n)
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    dist = np.empty((srcs.size, n), dtype=np.float64)
    if _load().rdo_dijkstra(_ptr(A), _ptr(W), n, _ptr(srcs), srcs.size, _ptr(dist)) != 0:
        raise ValueError("dijkstra failed")
    return dist
