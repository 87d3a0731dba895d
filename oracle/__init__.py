"""CPU oracle for delta-stepping SSSP -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never calls it and shares
no code with it. It wraps ``oracle.c`` (plain C, built with gcc) through ctypes:

* ``dijkstra``      binary-heap Dijkstra: the least-fixed-point definition;
* ``bellman_ford``  the fixed-point iteration written out;
* ``delta_ms``      delta-stepping in the vertex/edge set form (Fig. 1, right);
* ``delta_la``      delta-stepping in the linear-algebraic form (Fig. 1, left);
* ``floyd_warshall_i32``  all-pairs brute force for integer weights;
* ``check_invariants``    arc inequality, predecessor equality and minimality,
  realisability (a tight walk from the source reaches every reached vertex) and
  predecessor chains;
* ``bucket_index``  the exact bucket function floor(x / Delta) (Section III-B);
* ``tree_gradient`` dL/dw of L = sum_v c[v] * dist[v] by subtree sums of c over
  the shortest-path tree (float64), for float32 graphs;
* ``fd_arcs``       central differences of that loss with float64 distances,
  by local repair of the distances around each perturbed arc.

Every function takes a graph as (row_ptr int64[n+1], col int32[m], w int32|float32[m]).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

I32, F32 = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c (no FMA contraction, no fast-math) into a shared library beside it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class TraceRec(ctypes.Structure):
    _fields_ = [("bucket", ctypes.c_int64), ("round", ctypes.c_int64), ("vertex", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        c = ctypes
        vp = c.c_void_p
        sig = [c.c_int64, vp, vp, vp, c.c_int, c.c_int32, vp, vp]
        for name in ("or_dijkstra", "or_bellman_ford"):
            f = getattr(lib, name)
            f.restype = c.c_int
            f.argtypes = sig
        for name in ("or_delta_ms", "or_delta_la"):
            f = getattr(lib, name)
            f.restype = c.c_int
            f.argtypes = [c.c_int64, vp, vp, vp, c.c_int, c.c_int32, c.c_double, vp, vp,
                          vp, c.c_int64, c.POINTER(c.c_int64)]
        lib.or_floyd_warshall_i32.restype = c.c_int
        lib.or_floyd_warshall_i32.argtypes = [c.c_int64, vp, vp, vp, vp]
        lib.or_check_invariants.restype = c.c_int64
        lib.or_check_invariants.argtypes = [c.c_int64, vp, vp, vp, c.c_int, c.c_int32, vp, vp]
        lib.or_bucket_index.restype = c.c_int64
        lib.or_bucket_index.argtypes = [c.c_double, c.c_double]
        lib.or_fd_arcs.restype = c.c_int
        lib.or_fd_arcs.argtypes = [c.c_int64, vp, vp, vp, vp, vp, vp, c.c_int32, vp, vp, c.c_int64, c.c_double,
                                   vp, vp]
        lib.or_tree_gradient.restype = c.c_int
        lib.or_tree_gradient.argtypes = [c.c_int64, vp, vp, vp, c.c_int32, vp, vp, vp, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(row_ptr, col, w):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w)
    if w.dtype == np.float32:
        dt = F32
    elif w.dtype == np.int32:
        dt = I32
    else:
        raise TypeError(f"weights must be int32 or float32, got {w.dtype}")
    return row_ptr, col, w, dt


class PathOverflow(ValueError):
    """A path sum out of a reached vertex does not fit the weight type (int32 sum >=
    INT32_MAX, or a float32 sum that rounds to +inf): the solve has no result."""


def _check(rc: int, name: str):
    if rc == 4:
        raise PathOverflow(f"{name}: a path sum overflows the weight type")
    if rc != 0:
        raise ValueError(f"{name}: error code {rc} (1 = invalid input, 2 = out of memory)")


def _single(fname, row_ptr, col, w, src):
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    n = row_ptr.shape[0] - 1
    dist = np.empty(n, dtype=w.dtype)
    pred = np.empty(n, dtype=np.int32)
    rc = getattr(lib, fname)(n, _ptr(row_ptr), _ptr(col), _ptr(w), dt, int(src), _ptr(dist), _ptr(pred))
    _check(rc, fname)
    return dist, pred


def dijkstra(row_ptr, col, w, src):
    """Binary-heap Dijkstra: (dist, pred) by the least-fixed-point definition."""
    return _single("or_dijkstra", row_ptr, col, w, src)


def bellman_ford(row_ptr, col, w, src):
    """Sweep all arcs until nothing changes: (dist, pred)."""
    return _single("or_bellman_ford", row_ptr, col, w, src)


def _delta(fname, row_ptr, col, w, src, delta, trace):
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    n = row_ptr.shape[0] - 1
    dist = np.empty(n, dtype=w.dtype)
    pred = np.empty(n, dtype=np.int32)
    cap = 0
    buf = None
    tlen = ctypes.c_int64(0)
    if trace:
        cap = max(64, 8 * n + 64)
        buf = (TraceRec * cap)()
    rc = getattr(lib, fname)(n, _ptr(row_ptr), _ptr(col), _ptr(w), dt, int(src), float(delta),
                             _ptr(dist), _ptr(pred), ctypes.cast(buf, ctypes.c_void_p) if trace else None,
                             cap, ctypes.byref(tlen))
    _check(rc, fname)
    if not trace:
        return dist, pred
    if tlen.value < 0:
        raise RuntimeError(f"{fname}: trace overflow ({-tlen.value} records)")
    recs = [(buf[k].bucket, buf[k].round, buf[k].vertex) for k in range(tlen.value)]
    return dist, pred, recs


def delta_ms(row_ptr, col, w, src, delta, trace: bool = False):
    """Delta-stepping, set form (Fig. 1 right). With trace=True also returns the
    processing records [(bucket, round, vertex)], round >= 0 for light phases and
    -1 - r for the r-th heavy phase of a bucket."""
    return _delta("or_delta_ms", row_ptr, col, w, src, delta, trace)


def delta_la(row_ptr, col, w, src, delta, trace: bool = False):
    """Delta-stepping, linear-algebraic form on dense vectors (Fig. 1 left)."""
    return _delta("or_delta_la", row_ptr, col, w, src, delta, trace)


def floyd_warshall_i32(row_ptr, col, w):
    """All-pairs shortest distances for int32 weights (n <= 4096), INT32_MAX = no path."""
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    if dt != I32:
        raise TypeError("floyd_warshall_i32 needs int32 weights")
    n = row_ptr.shape[0] - 1
    out = np.empty((n, n), dtype=np.int32)
    _check(lib.or_floyd_warshall_i32(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(out)), "floyd_warshall")
    return out


def check_invariants(row_ptr, col, w, src, dist, pred) -> int:
    """Number of violated invariants (0 = a valid shortest-path labelling with the
    smallest-id predecessor rule)."""
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    n = row_ptr.shape[0] - 1
    dist = np.ascontiguousarray(dist, dtype=w.dtype)
    pred = np.ascontiguousarray(pred, dtype=np.int32)
    return int(lib.or_check_invariants(n, _ptr(row_ptr), _ptr(col), _ptr(w), dt, int(src),
                                       _ptr(dist), _ptr(pred)))


def bucket_index(x: float, delta: float) -> int:
    """floor(x / Delta) evaluated exactly (Section III-B's bucket definition)."""
    return int(_load().or_bucket_index(float(x), float(delta)))


def dijkstra_many(row_ptr, col, w, sources, threads: int | None = None):
    """Dijkstra from each source, one source per host thread (ctypes drops the GIL).
    Returns (list of dist, list of pred, threads used)."""
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, len(sources)))
    row_ptr, col, w, _ = _prep(row_ptr, col, w)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda s: dijkstra(row_ptr, col, w, s), sources))
    return [r[0] for r in res], [r[1] for r in res], threads


class CycleError(ValueError):
    """The predecessor graph has a cycle (zero-weight ties): no gradient."""


def tree_gradient(row_ptr, col, w, src, c, dist=None, pred=None, out=None):
    """dL/dw (float64[m], input arc order) of L = sum over reached v of c[v] * dist[v]
    for one source; dist/pred from ``dijkstra`` unless given. Adds into ``out``.
    The tree arc of v is the arc with the smallest input index among those whose
    sum reaches dist[v]."""
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    if dt != F32:
        raise TypeError("tree_gradient needs float32 weights")
    n = row_ptr.shape[0] - 1
    if dist is None or pred is None:
        dist, pred = dijkstra(row_ptr, col, w, src)
    dist = np.ascontiguousarray(dist, dtype=np.float32)
    pred = np.ascontiguousarray(pred, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float32)
    if c.shape[0] < n:
        raise ValueError("c needs n entries")
    g = out if out is not None else np.zeros(col.shape[0], dtype=np.float64)
    rc = lib.or_tree_gradient(n, _ptr(row_ptr), _ptr(col), _ptr(w), int(src), _ptr(dist),
                              _ptr(pred), _ptr(c), _ptr(g))
    if rc == 3:
        raise CycleError("predecessor graph has a cycle")
    _check(rc, "or_tree_gradient")
    return g


def tree_gradient_many(row_ptr, col, w, sources, cs, threads: int | None = None):
    """Sum over sources k of tree_gradient(..., sources[k], cs[k]); one source per thread."""
    threads = max(1, min(threads or os.cpu_count() or 1, len(sources)))
    row_ptr, col, w, _ = _prep(row_ptr, col, w)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda k: tree_gradient(row_ptr, col, w, sources[k], cs[k]),
                            range(len(sources))))
    return np.sum(parts, axis=0) if parts else np.zeros(col.shape[0])


def reverse_csr(row_ptr, col):
    """In-arcs of every vertex: (rrow int64[n+1], tails int32[m], input arc index int64[m])."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = row_ptr.shape[0] - 1
    order = np.argsort(col, kind="stable").astype(np.int64)
    tails = np.repeat(np.arange(n, dtype=np.int32), np.diff(row_ptr))[order]
    rrow = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(col, minlength=n), out=rrow[1:])
    return rrow, np.ascontiguousarray(tails, dtype=np.int32), np.ascontiguousarray(order)


def fd_arcs(row_ptr, col, w, src, c, arcs, eps=1e-3, rev=None):
    """Central differences (L(w + eps) - L(w - eps)) / (2 eps) of L = sum over reached x of
    c[x] * D[x], D the float64 distances from src, for each arc index in ``arcs``.
    Returns (fd float64[k], kink int32[k]): kink 1 where L is not linear within eps of
    w[e] (fd is then not the derivative), 2 where w[e] < eps (not tested)."""
    lib = _load()
    row_ptr, col, w, dt = _prep(row_ptr, col, w)
    if dt != F32:
        raise TypeError("fd_arcs needs float32 weights")
    n = row_ptr.shape[0] - 1
    rrow, tails, rarc = rev if rev is not None else reverse_csr(row_ptr, col)
    c = np.ascontiguousarray(c, dtype=np.float32)
    arcs = np.ascontiguousarray(arcs, dtype=np.int64)
    fd = np.zeros(arcs.shape[0], dtype=np.float64)
    kink = np.zeros(arcs.shape[0], dtype=np.int32)
    rc = lib.or_fd_arcs(n, _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(rrow), _ptr(tails), _ptr(rarc), int(src),
                        _ptr(c), _ptr(arcs), arcs.shape[0], float(eps), _ptr(fd), _ptr(kink))
    _check(rc, "or_fd_arcs")
    return fd, kink


def fd_arcs_many(row_ptr, col, w, sources, cs, arcs, eps=1e-3, threads: int | None = None):
    """Sum over sources k of fd_arcs(..., sources[k], cs[k], ...); a kink on any source
    marks the arc. One source per host thread."""
    threads = max(1, min(threads or os.cpu_count() or 1, len(sources)))
    row_ptr, col, w, _ = _prep(row_ptr, col, w)
    rev = reverse_csr(row_ptr, col)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda k: fd_arcs(row_ptr, col, w, sources[k], cs[k], arcs, eps, rev),
                            range(len(sources))))
    fd = np.sum([p[0] for p in parts], axis=0)
    kink = np.max([p[1] for p in parts], axis=0)
    return fd, kink
