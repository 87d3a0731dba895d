"""dsssp_solve_noalloc: the entry point for callers that cannot allocate device
memory (an allocator they must not bypass, a memory budget fixed in advance, or
a context where cudaMalloc would synchronise or fail). It keeps its working
state in a fixed array inside the library instead.

The test calls it through the C ABI on device buffers and compares it with the
regular dsssp_solve on the same inputs, bit for bit, on two calls in a row (the
second call must not see the first call's state), and with the CPU oracle.
Further cases: a graph exactly at the vertex limit, a call after a rejected one
(the shared control words must start clean), an overflow, and a refusal while
the stream is being captured. This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import graphgen.workloads as W
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_06895_gb300 as ds
    return ds


def _noalloc(ds, g, src, delta):
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    ww = torch.from_numpy(g.w).cuda()
    tdt = torch.float32 if g.w.dtype == np.float32 else torch.int32
    code = ds.DSSSP_F32 if g.w.dtype == np.float32 else ds.DSSSP_I32
    dist = torch.empty(g.n, dtype=tdt, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = ds.dsssp_solve_noalloc(g.n, g.m, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(cl.data_ptr()),
                                ctypes.c_void_p(ww.data_ptr()), code, int(src), float(delta),
                                ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(pred.data_ptr()), stream)
    return rc, dist.cpu().numpy(), pred.cpu().numpy()


def _regular(ds, g, src, delta):
    h = ds.Graph(g.row_ptr, g.col, g.w)
    r = h.solve(src, delta)
    out = r.dist.cpu().numpy(), r.pred.cpu().numpy()
    h.close()
    return out


def _same(a, b):
    if a.dtype == np.float32:
        return np.array_equal(a.view(np.uint32), b.view(np.uint32))
    return np.array_equal(a, b)


def test_noalloc_matches_regular_solve_two_calls(ds):
    # call 1: R-MAT scale 14, int32 weights U{1..255}, Delta 32, hub source
    g1, srcs1, deltas1 = W.rmat14_int()
    # call 2: an fp32 R-MAT with a different size and source
    g2, srcs2, _ = W.rmat22_unit(scale=15, n_sources=1)
    for g, s, delta in ((g1, srcs1[0], deltas1[0]), (g2, srcs2[0], 0.1)):
        rc, d, p = _noalloc(ds, g, s, delta)
        assert rc == ds.DSSSP_OK, ds.dsssp_status_string(rc)
        d_ref, p_ref = _regular(ds, g, s, delta)
        assert _same(d, d_ref), f"{g.name}: distances differ"
        assert np.array_equal(p, p_ref), f"{g.name}: predecessors differ"
        d_or, p_or = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
        assert _same(d, d_or) and np.array_equal(p, p_or), f"{g.name}: differs from the oracle"


def test_noalloc_at_the_vertex_limit_matches_the_oracle(ds):
    """R-MAT scale 17 (n = 131,072 = the limit), fp32 U[0,1), every Delta of the sweep."""
    g, srcs, deltas = W.rmat22_unit(scale=17, n_sources=2)
    assert g.n == ds.NOALLOC_MAX_VERTICES
    for s in srcs:
        d_or, p_or = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
        for delta in deltas:
            rc, d, p = _noalloc(ds, g, s, delta)
            assert rc == ds.DSSSP_OK, ds.dsssp_status_string(rc)
            assert _same(d, d_or) and np.array_equal(p, p_or), f"source {s} delta {delta}"


def test_noalloc_call_after_rejected_calls(ds):
    """A malformed CSR, a negative weight and an overflow are rejected; the next call,
    on the same fixed array, is exact."""
    good, srcs, deltas = W.rmat14_int(scale=12)
    bad = graphgen.from_arcs(4, [(0, 1), (1, 2)], np.array([1, 2], np.int32), dtype=np.int32)
    bad.col = bad.col.copy()
    bad.col[1] = 9                                            # head out of range
    rc, _, _ = _noalloc(ds, bad, 0, 1.0)
    assert rc == ds.DSSSP_ERR_BAD_GRAPH
    neg = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([1.0, -2.0], np.float32), dtype=np.float32)
    rc, _, _ = _noalloc(ds, neg, 0, 1.0)
    assert rc == ds.DSSSP_ERR_NEG_WEIGHT
    big = np.iinfo(np.int32).max - 10
    ovf = graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([big, 20, 5], np.int32), dtype=np.int32)
    for delta in (4.0, 1e9):
        rc, _, _ = _noalloc(ds, ovf, 0, delta)
        assert rc == ds.DSSSP_ERR_OVERFLOW
    benign = graphgen.from_arcs(4, [(0, 1), (0, 2), (2, 1), (1, 3)],
                                np.array([big - 90, 1, 1, 200], np.int32), dtype=np.int32)
    rc, d, p = _noalloc(ds, benign, 0, 1e9)                   # overflows only before the fixed point
    assert rc == ds.DSSSP_OK and list(d) == [0, 2, 1, 202] and list(p) == [0, 2, 0, 1]
    rc, d, p = _noalloc(ds, good, srcs[0], deltas[0])
    assert rc == ds.DSSSP_OK
    d_or, p_or = oracle.dijkstra(good.row_ptr, good.col, good.w, srcs[0])
    assert _same(d, d_or) and np.array_equal(p, p_or)


def test_noalloc_refuses_a_capturing_stream(ds):
    """The call reads its status back to the host, so it cannot be recorded into a CUDA
    graph: while the stream is being captured it returns UNSUPPORTED and enqueues nothing."""
    g, srcs, deltas = W.rmat14_int(scale=10)
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    ww = torch.from_numpy(g.w).cuda()
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        cg.capture_begin()
        dist.fill_(0)                                          # the captured graph is not empty
        rc = ds.dsssp_solve_noalloc(g.n, g.m, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(cl.data_ptr()),
                                    ctypes.c_void_p(ww.data_ptr()), ds.DSSSP_I32, int(srcs[0]), float(deltas[0]),
                                    ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(pred.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream))
        cg.capture_end()
    assert rc == ds.DSSSP_ERR_UNSUPPORTED
    rc, d, p = _noalloc(ds, g, srcs[0], deltas[0])           # and the next call works
    assert rc == ds.DSSSP_OK


def test_noalloc_rejects_graphs_beyond_its_capacity(ds):
    n = ds.NOALLOC_MAX_VERTICES + 1
    g = graphgen.from_arcs(n, [(0, 1)], np.array([1], np.int32), dtype=np.int32)
    rc, _, _ = _noalloc(ds, g, 0, 1.0)
    assert rc == ds.DSSSP_ERR_TOO_LARGE
    assert b"fixed working memory" in ds.dsssp_status_string(rc)
