"""dsssp_solve_noalloc: the entry point for callers that cannot allocate device
memory (an allocator they must not bypass, a memory budget fixed in advance, or
a context where cudaMalloc would synchronise or fail). It keeps its working
state in a fixed array inside the library instead.

The test calls it through the C ABI on device buffers and compares it with the
regular dsssp_solve on the same inputs, bit for bit, on two calls in a row (the
second call must not see the first call's state). This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import graphgen.workloads as W

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


def test_noalloc_rejects_graphs_beyond_its_capacity(ds):
    n = ds.NOALLOC_MAX_VERTICES + 1
    g = graphgen.from_arcs(n, [(0, 1)], np.array([1], np.int32), dtype=np.int32)
    rc, _, _ = _noalloc(ds, g, 0, 1.0)
    assert rc == ds.DSSSP_ERR_TOO_LARGE
    assert b"fixed working memory" in ds.dsssp_status_string(rc)
