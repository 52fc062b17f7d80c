"""Python binding of librd.so (include/rd.h): argument marshalling only.

Every function below has the name of the C entry point it calls and forwards plain pointers
and sizes.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are passed
as device pointers, everything else as host pointers (the library copies host data itself).
No step of the R-distance runs in Python: if librd.so is missing the import of the library
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librd.so")

RD_OK = 0
RD_ERR_ARG = 1
RD_ERR_GAMMA = 2
RD_ERR_OOM = 3
RD_ERR_CUDA = 4
RD_ERR_NUMERIC = 5
RD_ERR_STATE = 6
RD_ERR_TIMEOUT = 7
RD_ERR_UNSUPPORTED = 8

RD_PREC_FP64 = 0
RD_PREC_SPLIT_BF16 = 1
RD_UNREACHABLE = 2**31 - 1
MAX_GOALS = 64
NOALLOC_MAX_N = 512
BATCH_MAX_N = 512
BATCH_CLASSES = 4

# every symbol declared in include/rd.h, with its ctypes signature
_P = ctypes.c_void_p
_SIGS = {
    "rd_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_P)]),
    "rd_create_weighted": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_P)]),
    "rd_load": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "rd_set_stream": (ctypes.c_int, [_P, _P]),
    "rd_set_precision": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "rd_set_tau": (ctypes.c_int, [_P, ctypes.c_double]),
    "rd_apsp": (ctypes.c_int, [_P, _P, _P]),
    "rd_goal_solve": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "rd_greedy_next": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "rd_spectral_radius": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "rd_greedy_walk": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P]),
    "rd_set_profiling": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rd_sync": (ctypes.c_int, [_P]),
    "rd_get_stats": (ctypes.c_int, [_P, _P]),
    "rd_last_error": (ctypes.c_char_p, [_P]),
    "rd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rd_destroy": (None, [_P]),
    "rd_apsp_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, _P, _P]),
    "rd_probe_mma": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]),
    "rd_split_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32, ctypes.c_int32]),
    "rd_update_edge": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P, _P]),
    "rd_batch_create": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "rd_batch_offsets": (ctypes.c_int, [_P, _P]),
    "rd_batch_apsp": (ctypes.c_int, [_P, _P, _P, _P]),
    "rd_batch_status": (ctypes.c_int, [_P, _P]),
    "rd_batch_destroy": (None, [_P]),
    "rd_batch_set_precision": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "rd_batch_routes": (ctypes.c_int, [_P, _P]),
    "rd_batch_split_info": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "rd_batch_tuning": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "rd_serve_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_P)]),
    "rd_serve_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "rd_serve_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
    "rd_serve_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double)]),
    "rd_serve_wait_for": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]),
    "rd_serve_stats": (ctypes.c_int, [_P, _P]),
    "rd_serve_loop_check": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "rd_serve_destroy": (None, [_P]),
}
RD_REQ_APSP = 0
RD_REQ_GOALS = 1


class rd_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_padded", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("slices", ctypes.c_int32), ("gamma", ctypes.c_double), ("max_column_sum", ctypes.c_double),
        ("tau", ctypes.c_double), ("ms_factor", ctypes.c_double), ("ms_inverse", ctypes.c_double),
        ("ms_goal", ctypes.c_double), ("ms_greedy", ctypes.c_double), ("bytes_device", ctypes.c_int64),
        ("launches", ctypes.c_int64), ("prof_launches", ctypes.c_int64), ("prof_ms", ctypes.c_double),
        ("prof_flops", ctypes.c_double), ("precision_used", ctypes.c_int32), ("fallbacks", ctypes.c_int32),
        ("split_residual", ctypes.c_double),
        ("split_screen_bits", ctypes.c_double),
        ("prof_split_launches", ctypes.c_int64), ("prof_split_ms", ctypes.c_double),
        ("prof_split_flops", ctypes.c_double),
        ("split_order", ctypes.c_int32),
        ("edge_updates", ctypes.c_int64), ("update_refactors", ctypes.c_int64),
        ("prof_update_launches", ctypes.c_int64), ("prof_update_ms", ctypes.c_double),
        ("prof_update_bytes", ctypes.c_double),
        ("prof_split_busy_ms", ctypes.c_double),
    ]


class RDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load librd.so (built by paper_2308_07403_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with `python -m paper_2308_07403_gb300.build` "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def status_string(st: int) -> str:
    return load().rd_status_string(int(st)).decode()


def _check(st: int, h=None):
    if st != RD_OK:
        msg = load().rd_last_error(h).decode(errors="replace")
        raise RDError(st, msg)


def _ptr(x):
    """(pointer, keepalive) of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data_as(ctypes.c_void_p), a


def _np_out(x):
    if isinstance(x, np.ndarray) and not x.flags.c_contiguous:
        raise ValueError("output arrays must be C-contiguous")


# ---- entry points (same names as the C ABI) -------------------------------------------------

def rd_create(A, n: int, gamma: float):
    h = ctypes.c_void_p()
    pa, keep = _ptr(A)
    _check(load().rd_create(pa, int(n), float(gamma), ctypes.byref(h)))
    del keep
    return h


def rd_create_weighted(A, W, n: int, gamma: float):
    h = ctypes.c_void_p()
    pa, ka = _ptr(A)
    pw, kw = _ptr(W)
    _check(load().rd_create_weighted(pa, pw, int(n), float(gamma), ctypes.byref(h)))
    del ka, kw
    return h


def rd_load(h, A, W, gamma: float):
    pa, ka = _ptr(A)
    pw, kw = _ptr(W)
    _check(load().rd_load(h, pa, pw, float(gamma)), h)


def rd_set_stream(h, stream_ptr: int):
    _check(load().rd_set_stream(h, ctypes.c_void_p(int(stream_ptr))), h)


def rd_set_precision(h, mode: int, slices: int = 0):
    _check(load().rd_set_precision(h, int(mode), int(slices)), h)


def rd_set_tau(h, tau: float):
    _check(load().rd_set_tau(h, float(tau)), h)


def _shape_dtype(x):
    return tuple(int(d) for d in x.shape), str(x.dtype).replace("torch.", "")


def rd_greedy_walk(h, next_hops, start, max_len: int, path, length, n: int | None = None):
    """Walks from start[c] along the next hops of goal c (next_hops: k x n), at most max_len steps.

    Shapes and dtypes are checked before the call (the library copies k n next hops in and
    k (max_len + 1) path entries out): next_hops int32 (k, n), start int32 (k,), path int32
    (k, max_len + 1), length int32 (k,).  n defaults to the handle's graph size."""
    _np_out(path)
    _np_out(length)
    if n is None:
        n = rd_get_stats(h)["n"]
    k = int(start.shape[0]) if len(start.shape) == 1 else -1
    want = {"next_hops": (next_hops, (k, int(n))), "start": (start, (k,)),
            "path": (path, (k, int(max_len) + 1)), "length": (length, (k,))}
    for name, (x, shape) in want.items():
        got, dt = _shape_dtype(x)
        if k < 1 or got != shape or dt != "int32":
            raise ValueError(f"{name} must be int32 of shape {shape}, got {dt} {got}")
    pn, kn = _ptr(next_hops)
    ps, ks = _ptr(start)
    pp, kp = _ptr(path)
    pl, kl = _ptr(length)
    _check(load().rd_greedy_walk(h, pn, k, ps, int(max_len), pp, pl), h)


def rd_spectral_radius(h, iters: int = 200):
    """(lo, hi): Collatz-Wielandt bracket of the spectral radius of X after `iters` power steps."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(load().rd_spectral_radius(h, int(iters), ctypes.byref(lo), ctypes.byref(hi)), h)
    return lo.value, hi.value


def rd_apsp(h, D, Y=None):
    _np_out(D)
    _np_out(Y)
    pd, kd = _ptr(D)
    py, ky = _ptr(Y)
    _check(load().rd_apsp(h, pd, py), h)


def rd_goal_solve(h, goals, k: int, Y_out):
    _np_out(Y_out)
    pg, kg = _ptr(goals)
    py, ky = _ptr(Y_out)
    _check(load().rd_goal_solve(h, pg, int(k), py), h)


def rd_greedy_next(h, goals, k: int, Yrows, nxt):
    _np_out(nxt)
    pg, kg = _ptr(goals)
    py, ky = _ptr(Yrows)
    pn, kn = _ptr(nxt)
    _check(load().rd_greedy_next(h, pg, int(k), py, pn), h)


def rd_set_profiling(h, on):
    """0 / False: off; 1 / True: every dense-contraction kernel; 2: the split GEMM alone."""
    _check(load().rd_set_profiling(h, int(on)), h)


def rd_sync(h):
    _check(load().rd_sync(h), h)


def rd_get_stats(h) -> dict:
    s = rd_stats()
    _check(load().rd_get_stats(h, ctypes.byref(s)), h)
    return {name: getattr(s, name) for name, _ in rd_stats._fields_}


def rd_last_error(h=None) -> str:
    return load().rd_last_error(h).decode(errors="replace")


def rd_destroy(h):
    if h:
        load().rd_destroy(h)


def rd_update_edge(h, i: int, j: int, present: bool, w: float, D, Y=None):
    """Edge j -> i present (weight w) or absent; D (and Y) of the changed graph."""
    _np_out(D)
    _np_out(Y)
    pd, kd = _ptr(D)
    py, ky = _ptr(Y)
    _check(load().rd_update_edge(h, int(i), int(j), 1 if present else 0, float(w), pd, py), h)


def rd_apsp_noalloc(A, n: int, gamma: float, D, stream_ptr: int = 0):
    """APSP without any device allocation (device A and D, n <= NOALLOC_MAX_N)."""
    pa, ka = _ptr(A)
    pd, kd = _ptr(D)
    _check(load().rd_apsp_noalloc(pa, int(n), float(gamma), pd, ctypes.c_void_p(int(stream_ptr))))


def rd_probe_mma(kind: int, batches: int = 4000):
    """(tera-ops/s, seconds) of back-to-back tcgen05 MMAs: kind 0 BF16 (K = 16), 1 INT8 (K = 32)."""
    r, s = ctypes.c_double(), ctypes.c_double()
    _check(load().rd_probe_mma(int(kind), int(batches), ctypes.byref(r), ctypes.byref(s)))
    return r.value, s.value


SPLIT_STATS_N = 13
SPLIT_STATS_FIELDS = ("mma_cycles", "mma_wait_accumulator", "mma_wait_operands", "mma_issue",
                      "producer_cycles", "producer_wait_stage", "epilogue_cycles", "epilogue_wait_group",
                      "epilogue_renormalise", "mma_warps", "epilogue_warps", "groups", "mmas")


def rd_split_stats(reset: bool = False):
    """The split GEMM's role cycle counters as a dict (a library built with stats=True only)."""
    buf = (ctypes.c_uint64 * SPLIT_STATS_N)()
    _check(load().rd_split_stats(buf, SPLIT_STATS_N, 1 if reset else 0))
    return dict(zip(SPLIT_STATS_FIELDS, (int(v) for v in buf)))


# ---- convenience wrapper ---------------------------------------------------------------------

class Handle:
    """Owns one rd_handle; methods forward to the entry points above."""

    def __init__(self, A, gamma: float, W=None, stream=None):
        n = int(A.shape[0])
        self.n = n
        self.h = rd_create(A, n, gamma) if W is None else rd_create_weighted(A, W, n, gamma)
        if stream is not None:
            rd_set_stream(self.h, stream)

    def load(self, A, gamma, W=None):
        rd_load(self.h, A, W, gamma)

    def set_precision(self, mode, slices=0):
        rd_set_precision(self.h, mode, slices)

    def apsp(self, D, Y=None):
        rd_apsp(self.h, D, Y)
        return D

    def update_edge(self, i, j, present, D, Y=None, w=1.0):
        rd_update_edge(self.h, i, j, present, w, D, Y)
        return D

    def goal_solve(self, goals, Y_out):
        rd_goal_solve(self.h, goals, int(goals.shape[0]), Y_out)
        return Y_out

    def greedy_next(self, goals, Yrows, nxt):
        rd_greedy_next(self.h, goals, int(goals.shape[0]), Yrows, nxt)
        return nxt

    def sync(self):
        rd_sync(self.h)

    def spectral_radius(self, iters=200):
        return rd_spectral_radius(self.h, iters)

    def greedy_walk(self, next_hops, start, max_len, path, length):
        rd_greedy_walk(self.h, next_hops, start, max_len, path, length, n=self.n)
        return path, length

    def stats(self):
        return rd_get_stats(self.h)

    def close(self):
        if self.h:
            rd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns one rd_batch_handle: G graphs of at most BATCH_MAX_N nodes, solved in one launch.

    n and gamma are host sequences; offsets() gives the packing of A (uint8) and D (int32):
    graph g occupies elements [off[g], off[g + 1]) = n_g * n_g entries, row-major."""

    def __init__(self, n, gamma):
        n = np.ascontiguousarray(n, dtype=np.int32)
        gamma = np.ascontiguousarray(gamma, dtype=np.float64)
        if n.shape != gamma.shape:
            raise ValueError("n and gamma must have the same length")
        self.G = int(n.size)
        h = ctypes.c_void_p()
        _check(load().rd_batch_create(n.ctypes.data_as(_P), gamma.ctypes.data_as(_P), self.G, ctypes.byref(h)))
        self.h = h

    def offsets(self):
        off = np.empty(self.G + 1, dtype=np.int64)
        _check(load().rd_batch_offsets(self.h, off.ctypes.data_as(_P)))
        return off

    def apsp(self, A, D, stream=None):
        """A, D: CUDA tensors (packed); the call is asynchronous on `stream` (cudaStream_t int)."""
        pa, ka = _ptr(A)
        pd, kd = _ptr(D)
        _check(load().rd_batch_apsp(self.h, pa, pd, ctypes.c_void_p(stream or 0)))
        return D

    def status(self):
        st = np.empty(self.G, dtype=np.int32)
        _check(load().rd_batch_status(self.h, st.ctypes.data_as(_P)))
        return st

    def set_precision(self, mode, autotune=True):
        _check(load().rd_batch_set_precision(self.h, int(mode), 1 if autotune else 0))

    def routes(self):
        """Per graph: 0 FP64 kernel, 1 split, 2 split redone in FP64, 3 screened to FP64, 4 gain failed."""
        r = np.empty(self.G, dtype=np.int32)
        _check(load().rd_batch_routes(self.h, r.ctypes.data_as(_P)))
        return r

    def split_info(self):
        """Per graph: digits of its kept split result, split passes, last residual, screen bits."""
        d = np.empty(self.G, np.int32)
        p = np.empty(self.G, np.int32)
        r = np.empty(self.G)
        sb = np.empty(self.G)
        _check(load().rd_batch_split_info(self.h, *(x.ctypes.data_as(_P) for x in (d, p, r, sb))))
        return {"digits": d, "passes": p, "residual": r, "screen_bits": sb}

    def tuning(self):
        """Per size class (n in (128 c, 128 (c + 1)]): graphs, on the split path, ms per graph of both variants."""
        g = np.empty(BATCH_CLASSES, np.int32)
        sp = np.empty(BATCH_CLASSES, np.int32)
        mf = np.empty(BATCH_CLASSES)
        ms = np.empty(BATCH_CLASSES)
        nl = np.zeros(1, np.int64)
        _check(load().rd_batch_tuning(self.h, *(x.ctypes.data_as(_P) for x in (g, sp, mf, ms, nl))))
        return {"graphs": g.tolist(), "split": sp.tolist(), "ms_per_graph_fp64": mf.tolist(),
                "ms_per_graph_split": ms.tolist(), "launches_last_run": int(nl[0])}

    def close(self):
        if self.h:
            load().rd_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class rd_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("graph_id", ctypes.c_int32), ("A", _P), ("n", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("goals", _P), ("k", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("D_out", _P), ("Y_out", _P)]


class rd_serve_report(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("resident_graphs", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("bytes_used", ctypes.c_int64), ("evictions", ctypes.c_int64), ("reused", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_int64), ("loop_requests", ctypes.c_int64)]


class Server:
    """Owns one rd_server_handle.  submit_* return an id; the numpy output array of a request stays
    referenced here until wait(id) returns (the library writes it when the request completes)."""

    def __init__(self, budget_bytes: int, workers: int = 4):
        h = ctypes.c_void_p()
        _check(load().rd_serve_create(int(budget_bytes), int(workers), ctypes.byref(h)))
        self.h = h
        self._live = {}

    def _submit(self, kind, graph_id, A, gamma, goals, out, precision):
        A = np.ascontiguousarray(A, dtype=np.uint8)
        r = rd_request()
        r.kind = kind
        r.graph_id = int(graph_id)
        r.A = A.ctypes.data_as(_P)
        r.n = int(A.shape[0])
        r.gamma = float(gamma)
        r.precision = int(precision)
        keep = [A, out]
        if goals is not None:
            goals = np.ascontiguousarray(goals, dtype=np.int32)
            r.goals = goals.ctypes.data_as(_P)
            r.k = int(goals.size)
            r.Y_out = out.ctypes.data_as(_P)
            keep.append(goals)
        else:
            r.D_out = out.ctypes.data_as(_P)
        rid = ctypes.c_int64()
        _check(load().rd_serve_submit(self.h, ctypes.byref(r), ctypes.byref(rid)))
        self._live[rid.value] = keep
        return rid.value

    @staticmethod
    def _host_out(x, dtype):
        if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags.c_contiguous):
            raise ValueError(f"outputs of a server request are C-contiguous numpy {np.dtype(dtype).name} arrays")
        return x

    def submit_apsp(self, graph_id, A, gamma, D_out, precision=RD_PREC_SPLIT_BF16):
        """D_out: C-contiguous int32 numpy array (n, n)."""
        return self._submit(RD_REQ_APSP, graph_id, A, gamma, None, self._host_out(D_out, np.int32), precision)

    def submit_goals(self, graph_id, A, gamma, goals, Y_out, precision=RD_PREC_SPLIT_BF16):
        """Y_out: C-contiguous float64 numpy array (k, n)."""
        return self._submit(RD_REQ_GOALS, graph_id, A, gamma, goals, self._host_out(Y_out, np.float64), precision)

    def poll(self, rid):
        d = ctypes.c_int32()
        _check(load().rd_serve_poll(self.h, int(rid), ctypes.byref(d)))
        return bool(d.value)

    def wait(self, rid, timeout_ms=None):
        """Returns (status, latency_ms); with timeout_ms, raises RDError(RD_ERR_TIMEOUT) when the
        request has not completed in time (it keeps running and can be waited for again)."""
        st = ctypes.c_int()
        lat = ctypes.c_double()
        if timeout_ms is None:
            _check(load().rd_serve_wait(self.h, int(rid), ctypes.byref(st), ctypes.byref(lat)))
        else:
            _check(load().rd_serve_wait_for(self.h, int(rid), float(timeout_ms), ctypes.byref(st),
                                            ctypes.byref(lat)))
        self._live.pop(int(rid), None)
        return st.value, lat.value

    def loop_check(self):
        """The device loop's failure path: the status it reports for a request whose descriptor is
        never marked ready (RD_ERR_TIMEOUT when its bounded wait ran out and it recovered)."""
        st = ctypes.c_int()
        _check(load().rd_serve_loop_check(self.h, ctypes.byref(st)))
        return st.value

    def stats(self):
        r = rd_serve_report()
        _check(load().rd_serve_stats(self.h, ctypes.byref(r)))
        return {name: getattr(r, name) for name, _ in r._fields_}

    def close(self):
        if self.h:
            load().rd_serve_destroy(self.h)
            self.h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
