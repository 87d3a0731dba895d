"""ctypes binding of the C ABI in ``include/dsssp.h`` (argument marshalling only).

The raw entry points keep the C names (``dsssp_graph_create``, ``dsssp_solve``,
...). ``Graph`` wraps a handle and takes / returns torch tensors: torch only
provides device memory and the current CUDA stream; every step of the solve
runs in the library's CUDA kernels. There is no CPU fallback: importing this
module fails when ``libdsssp.so`` has not been built.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsssp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1911_06895_gb300.build` "
                      "(the CUDA library is required; there is no fallback path)")

_lib = ctypes.CDLL(LIB_PATH)

# ---- status / enums (mirror include/dsssp.h) ----------------------------------------
DSSSP_OK = 0
DSSSP_ERR_INVALID_ARG = 1
DSSSP_ERR_BAD_GRAPH = 2
DSSSP_ERR_NEG_WEIGHT = 3
DSSSP_ERR_NOT_CONVERGED = 4
DSSSP_ERR_TIMEOUT = 5
DSSSP_ERR_CUDA = 6
DSSSP_ERR_NO_TAPE = 7
DSSSP_ERR_OOM = 8
DSSSP_ERR_UNSUPPORTED = 9
DSSSP_ERR_TOO_LARGE = 10
DSSSP_ERR_DEGENERATE = 11
DSSSP_ERR_OVERFLOW = 12

DSSSP_I32 = 0
DSSSP_F32 = 1
DSSSP_MODE_PERSISTENT = 0
DSSSP_MODE_STEPPED = 1
DSSSP_MODE_DENSE = 2
DSSSP_MODE_TEAM = 3
DSSSP_FLAG_ASYNC = 0x1
DSSSP_FLAG_NO_FUSE = 0x2
DSSSP_HOOK_NONE = 0
DSSSP_HOOK_STALL_BARRIER = 1
DSSSP_BATCH_TAPE = 0x1
DSSSP_BACKWARD_ACCUMULATE = 0x1
DSSSP_TUNE_SOLVE = 0
DSSSP_TUNE_BATCH = 1


class dsssp_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("mode", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("grid_size", ctypes.c_int32), ("solo_work", ctypes.c_int32),
                ("max_phases", ctypes.c_int64), ("timeout_ns", ctypes.c_int64), ("test_hook", ctypes.c_int32),
                ("team_blocks", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class dsssp_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "buckets", "light_phases", "heavy_phases", "rebin_phases", "vertices_light",
        "vertices_heavy", "arcs_light", "arcs_heavy", "far_scanned", "improvements", "ns_light",
        "ns_heavy", "ns_rebin", "ns_total", "ns_first_arrival", "ns_arrival_spread", "grid_size",
        "block_size")] + [("reserved", ctypes.c_int64 * 6)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


class dsssp_batch_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "buckets", "light_phases", "heavy_phases", "select_phases", "arcs_light", "arcs_heavy",
        "improvements", "far_scanned", "ns", "team", "vertices_light", "vertices_heavy")] + [
        ("reserved", ctypes.c_int64 * 4)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


class dsssp_tune_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("target", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("candidates", ctypes.c_double * 16), ("reserved", ctypes.c_int32 * 8)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def _fn(name, restype, argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = argtypes
    return f


dsssp_status_string = _fn("dsssp_status_string", ctypes.c_char_p, [ctypes.c_int])
dsssp_options_default = _fn("dsssp_options_default", ctypes.c_int, [ctypes.POINTER(dsssp_options)])
dsssp_graph_create = _fn("dsssp_graph_create", ctypes.c_int,
                         [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)])
dsssp_graph_destroy = _fn("dsssp_graph_destroy", ctypes.c_int, [_vp])
dsssp_graph_info = _fn("dsssp_graph_info", ctypes.c_int,
                       [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32)])
dsssp_prepare = _fn("dsssp_prepare", ctypes.c_int, [_vp, ctypes.c_double, _vp])
dsssp_solve = _fn("dsssp_solve", ctypes.c_int,
                  [_vp, _i32, ctypes.c_double, _vp, _vp, ctypes.POINTER(dsssp_options),
                   ctypes.POINTER(dsssp_stats), _vp])
dsssp_graph_sync = _fn("dsssp_graph_sync", ctypes.c_int, [_vp, _vp])
dsssp_solve_noalloc = _fn("dsssp_solve_noalloc", ctypes.c_int,
                          [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, _i32, ctypes.c_double, _vp, _vp, _vp])

_u32 = ctypes.c_uint32
dsssp_batch_create = _fn("dsssp_batch_create", ctypes.c_int,
                         [_vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _u32, ctypes.POINTER(dsssp_options), _vp,
                          ctypes.POINTER(_vp)])
dsssp_batch_run = _fn("dsssp_batch_run", ctypes.c_int, [_vp, _vp])
dsssp_batch_sync = _fn("dsssp_batch_sync", ctypes.c_int, [_vp, _vp, _vp])
dsssp_batch_destroy = _fn("dsssp_batch_destroy", ctypes.c_int, [_vp])
dsssp_solve_batched = _fn("dsssp_solve_batched", ctypes.c_int,
                          [_vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(dsssp_options), _vp, _vp])
dsssp_backward = _fn("dsssp_backward", ctypes.c_int, [_vp, _vp, _vp, _u32, _vp])
dsssp_autotune = _fn("dsssp_autotune", ctypes.c_int,
                     [_vp, _i32, _vp, _i32, ctypes.POINTER(dsssp_tune_options), _vp, _vp, _vp])
dsssp_tune_solo_work = _fn("dsssp_tune_solo_work", ctypes.c_int,
                           [_vp, _vp, _i32, ctypes.c_double, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double), _vp])
dsssp_tune_schedule = _fn("dsssp_tune_schedule", ctypes.c_int,
                          [_vp, _vp, _i32, ctypes.c_double, ctypes.POINTER(dsssp_options),
                           ctypes.POINTER(ctypes.c_double), _vp])
dsssp_tune_team_blocks = _fn("dsssp_tune_team_blocks", ctypes.c_int,
                             [_vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(_i32),
                              ctypes.POINTER(ctypes.c_double), _vp])

EXPORTED = ["dsssp_status_string", "dsssp_options_default", "dsssp_graph_create", "dsssp_graph_destroy",
            "dsssp_graph_info", "dsssp_prepare", "dsssp_solve", "dsssp_graph_sync", "dsssp_solve_noalloc",
            "dsssp_batch_create", "dsssp_batch_run", "dsssp_batch_sync", "dsssp_batch_destroy",
            "dsssp_solve_batched", "dsssp_backward", "dsssp_autotune", "dsssp_tune_team_blocks",
            "dsssp_tune_solo_work", "dsssp_tune_schedule"]

NOALLOC_MAX_VERTICES = 1 << 17


class DsssError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = dsssp_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


def check(status: int, what: str = "") -> None:
    if status != DSSSP_OK:
        raise DsssError(status, what)


def make_options(**kw) -> dsssp_options:
    o = dsssp_options()
    check(dsssp_options_default(ctypes.byref(o)))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(dt) -> int:
    import torch
    if dt in (np.float32, torch.float32):
        return DSSSP_F32
    if dt in (np.int32, torch.int32):
        return DSSSP_I32
    raise TypeError(f"weights must be int32 or float32, got {dt}")


@dataclass
class SolveResult:
    dist: "object"
    pred: "object"
    stats: dict | None


class Graph:
    """A graph handle on the current CUDA device (library-owned copy of the CSR).

    ``row_ptr`` int64[n+1], ``col`` int32[m], ``w`` int32[m] or float32[m], given as
    numpy arrays (copied from host memory) or CUDA torch tensors (copied on device).
    """

    def __init__(self, row_ptr, col, w, stream=None):
        import torch
        self._h = None
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        if on_dev:
            rp = row_ptr.contiguous(); cl = col.contiguous(); ww = w.contiguous()
            if rp.dtype != torch.int64 or cl.dtype != torch.int32:
                raise TypeError("row_ptr must be int64 and col int32")
            code = _dtype_code(ww.dtype)
            ptrs = (rp.data_ptr(), cl.data_ptr(), ww.data_ptr())
            n = rp.numel() - 1
            m = cl.numel()
            keep = (rp, cl, ww)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            ww = np.ascontiguousarray(w)
            code = _dtype_code(ww.dtype.type)
            ptrs = (rp.ctypes.data, cl.ctypes.data, ww.ctypes.data)
            n = rp.shape[0] - 1
            m = cl.shape[0]
            keep = (rp, cl, ww)
        h = ctypes.c_void_p()
        st = dsssp_graph_create(n, m, ptrs[0], ptrs[1], ptrs[2], code, 1 if on_dev else 0,
                                _stream_ptr(stream), ctypes.byref(h))
        del keep
        check(st, "dsssp_graph_create")
        self._h = h
        self.n, self.m, self.dtype_code = n, m, code

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            dsssp_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, delta: float, stream=None) -> None:
        """Light/heavy split for delta (cached in the handle)."""
        check(dsssp_prepare(self._h, float(delta), _stream_ptr(stream)), "dsssp_prepare")

    def solve(self, src: int, delta: float, dist=None, pred=None, options: dsssp_options | None = None,
              stats: bool = False, stream=None) -> SolveResult:
        """One delta-stepping solve; returns CUDA tensors dist (graph dtype) and pred (int32)."""
        import torch
        tdt = torch.float32 if self.dtype_code == DSSSP_F32 else torch.int32
        if dist is None:
            dist = torch.empty(self.n, dtype=tdt, device="cuda")
        if pred is None:
            pred = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if dist.dtype != tdt or dist.numel() < self.n or pred.dtype != torch.int32 or pred.numel() < self.n:
            raise TypeError("dist/pred have the wrong dtype or size")
        st = dsssp_stats() if stats else None
        rc = dsssp_solve(self._h, int(src), float(delta), ctypes.c_void_p(dist.data_ptr()),
                         ctypes.c_void_p(pred.data_ptr()), ctypes.byref(options) if options is not None else None,
                         ctypes.byref(st) if st is not None else None, _stream_ptr(stream))
        check(rc, "dsssp_solve")
        return SolveResult(dist, pred, st.as_dict() if st is not None else None)

    def sync(self, stream=None) -> None:
        check(dsssp_graph_sync(self._h, _stream_ptr(stream)), "dsssp_graph_sync")


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


class Batch:
    """A batch plan: ``len(sources)`` solves run together in one persistent launch.

    ``graphs`` is a Graph or a list of Graphs (one dtype, current device), ``deltas``
    one Delta per graph, ``sources`` one source per instance and ``src_graph`` the
    graph index of each instance (default: all on graph 0). Outputs are CUDA tensors
    ``dist[k]`` (graph dtype) and ``pred[k]`` (int32), allocated unless given; every
    ``run()`` rewrites them. ``tape=True`` records each instance's shortest-path tree
    for ``backward()`` (float32 graphs only).
    """

    def __init__(self, graphs, deltas, sources, src_graph=None, dist=None, pred=None, tape: bool = False,
                 options: dsssp_options | None = None, stream=None):
        import torch
        self._h = None
        self.graphs = list(graphs) if isinstance(graphs, (list, tuple)) else [graphs]
        deltas = list(deltas) if isinstance(deltas, (list, tuple, np.ndarray)) else [deltas]
        if len(deltas) != len(self.graphs):
            raise ValueError("one Delta per graph")
        self.sources = [int(s) for s in sources]
        k = len(self.sources)
        self.src_graph = [0] * k if src_graph is None else [int(g) for g in src_graph]
        if len(self.src_graph) != k:
            raise ValueError("one graph index per source")
        tdt = torch.float32 if self.graphs[0].dtype_code == DSSSP_F32 else torch.int32
        ns = [self.graphs[g].n if 0 <= g < len(self.graphs) else 1 for g in self.src_graph]
        self.dist = dist if dist is not None else [torch.empty(n, dtype=tdt, device="cuda") for n in ns]
        self.pred = pred if pred is not None else [torch.empty(n, dtype=torch.int32, device="cuda") for n in ns]
        if len(self.dist) != k or len(self.pred) != k:
            raise ValueError("one dist and pred tensor per source")
        for d, p, n in zip(self.dist, self.pred, ns):
            if d.dtype != tdt or d.numel() < n or p.dtype != torch.int32 or p.numel() < n:
                raise TypeError("dist/pred have the wrong dtype or size")
        gh = _ptr_array([g.handle.value for g in self.graphs])
        dl = (ctypes.c_double * len(deltas))(*[float(x) for x in deltas])
        sr = (ctypes.c_int32 * k)(*self.sources)
        sg = (ctypes.c_int32 * k)(*self.src_graph)
        dp = _ptr_array([d.data_ptr() for d in self.dist])
        pp = _ptr_array([p.data_ptr() for p in self.pred])
        h = ctypes.c_void_p()
        rc = dsssp_batch_create(gh, len(self.graphs), dl, k, sr, sg, dp, pp, DSSSP_BATCH_TAPE if tape else 0,
                                ctypes.byref(options) if options is not None else None, _stream_ptr(stream),
                                ctypes.byref(h))
        check(rc, "dsssp_batch_create")
        self._h = h
        self.tape = tape

    @property
    def handle(self):
        return self._h

    def run(self, stream=None) -> None:
        """Enqueue one run of every instance (one CUDA-graph launch); does not wait."""
        check(dsssp_batch_run(self._h, _stream_ptr(stream)), "dsssp_batch_run")

    def sync(self, stats: bool = False, stream=None):
        """Wait; raise on a device-side error; optionally return per-instance counters."""
        k = len(self.sources)
        st = (dsssp_batch_stats * k)() if stats else None
        check(dsssp_batch_sync(self._h, st, _stream_ptr(stream)), "dsssp_batch_sync")
        return [x.as_dict() for x in st] if stats else None

    def backward(self, c, grad_w, accumulate: bool = False, stream=None) -> None:
        """grad_w[g] (float32[m_g], input arc order) = dL/dw for L = sum_k sum_v c[k][v] * dist[k][v]."""
        import torch
        if len(c) != len(self.sources) or len(grad_w) != len(self.graphs):
            raise ValueError("one c per instance and one grad_w per graph")
        for ck, g in zip(c, self.src_graph):
            if ck.dtype != torch.float32 or not ck.is_cuda or ck.numel() < self.graphs[g].n:
                raise TypeError("c[k] must be a CUDA float32 tensor of n entries")
        for gw, g in zip(grad_w, self.graphs):
            if gw.dtype != torch.float32 or not gw.is_cuda or gw.numel() < g.m:
                raise TypeError("grad_w[g] must be a CUDA float32 tensor of m entries")
        rc = dsssp_backward(self._h, _ptr_array([x.data_ptr() for x in c]),
                            _ptr_array([x.data_ptr() for x in grad_w]),
                            DSSSP_BACKWARD_ACCUMULATE if accumulate else 0, _stream_ptr(stream))
        check(rc, "dsssp_backward")

    def close(self):
        if self._h is not None and self._h.value:
            dsssp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(graphs, deltas, sources, src_graph=None, options: dsssp_options | None = None,
                  stats: bool = False, stream=None):
    """One-shot batch: returns (dist list, pred list, stats list or None)."""
    b = Batch(graphs, deltas, sources, src_graph=src_graph, options=options, stream=stream)
    try:
        b.run(stream)
        st = b.sync(stats=stats, stream=stream)
        return b.dist, b.pred, st
    finally:
        b.close()


def autotune(graphs, sample_sources, target: str = "solve", candidates=None, refine: int = 2, stream=None):
    """Choose Delta per graph by timing sample solves on this GPU.

    ``sample_sources`` is one list of k sources per graph (or one list for a single
    graph); ``target`` is "solve" (dsssp_solve) or "batch" (instances of a batch).
    Returns (deltas, ms): the chosen Delta of each graph and the device time of its
    k samples at that Delta."""
    graphs = list(graphs) if isinstance(graphs, (list, tuple)) else [graphs]
    if graphs and not isinstance(sample_sources[0], (list, tuple, np.ndarray)):
        sample_sources = [sample_sources]
    k = len(sample_sources[0])
    if len(sample_sources) != len(graphs) or any(len(s) != k for s in sample_sources):
        raise ValueError("k sample sources per graph")
    o = dsssp_tune_options()
    o.struct_size = ctypes.sizeof(dsssp_tune_options)
    o.target = DSSSP_TUNE_BATCH if target == "batch" else DSSSP_TUNE_SOLVE
    o.refine = refine if refine != 0 else -1
    if candidates:
        o.n_candidates = len(candidates)
        for i, c in enumerate(candidates):
            o.candidates[i] = float(c)
    flat = (ctypes.c_int32 * (len(graphs) * k))(*[int(s) for ss in sample_sources for s in ss])
    dout = (ctypes.c_double * len(graphs))()
    mout = (ctypes.c_double * len(graphs))()
    check(dsssp_autotune(_ptr_array([g.handle.value for g in graphs]), len(graphs), flat, k, ctypes.byref(o),
                         dout, mout, _stream_ptr(stream)), "dsssp_autotune")
    return list(dout), list(mout)


def tune_team_blocks(graphs, deltas, sources, src_graph=None, stream=None):
    """Blocks per instance (1, 2, 4 or 8) at which this batch runs fastest; returns (team_blocks, ms)."""
    import torch
    graphs = list(graphs) if isinstance(graphs, (list, tuple)) else [graphs]
    deltas = list(deltas) if isinstance(deltas, (list, tuple, np.ndarray)) else [deltas]
    k = len(sources)
    sg = [0] * k if src_graph is None else [int(g) for g in src_graph]
    tdt = torch.float32 if graphs[0].dtype_code == DSSSP_F32 else torch.int32
    dist = [torch.empty(graphs[g].n, dtype=tdt, device="cuda") for g in sg]
    tb = _i32(0)
    ms = ctypes.c_double(0.0)
    check(dsssp_tune_team_blocks(_ptr_array([g.handle.value for g in graphs]), len(graphs),
                                 (ctypes.c_double * len(deltas))(*[float(x) for x in deltas]), k,
                                 (ctypes.c_int32 * k)(*[int(s) for s in sources]), (ctypes.c_int32 * k)(*sg),
                                 _ptr_array([d.data_ptr() for d in dist]), None, ctypes.byref(tb), ctypes.byref(ms),
                                 _stream_ptr(stream)), "dsssp_tune_team_blocks")
    return int(tb.value), float(ms.value)


def tune_solo_work(graph, sample_sources, delta, stream=None):
    """Solo threshold (dsssp_options.solo_work) at which single solves run fastest; returns (solo_work, ms)."""
    k = len(sample_sources)
    sw = _i32(0)
    ms = ctypes.c_double(0.0)
    check(dsssp_tune_solo_work(graph.handle, (ctypes.c_int32 * k)(*[int(s) for s in sample_sources]), k,
                               float(delta), ctypes.byref(sw), ctypes.byref(ms), _stream_ptr(stream)),
          "dsssp_tune_solo_work")
    return int(sw.value), float(ms.value)


def tune_schedule(graph, sample_sources, delta, stream=None):
    """Fastest scheme of single solves for one graph at one Delta (persistent with a solo
    threshold, or one thread-block cluster per solve); returns (options, ms)."""
    k = len(sample_sources)
    o = dsssp_options()
    ms = ctypes.c_double(0.0)
    check(dsssp_tune_schedule(graph.handle, (ctypes.c_int32 * k)(*[int(s) for s in sample_sources]), k,
                              float(delta), ctypes.byref(o), ctypes.byref(ms), _stream_ptr(stream)),
          "dsssp_tune_schedule")
    return o, float(ms.value)
