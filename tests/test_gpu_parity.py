"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Distances must match bit for bit (float32 and int32) and predecessors exactly:
the least fixed point of the rounded min-plus recurrence does not depend on
the relaxation order (see oracle/oracle.c), and the packed 64-bit atomicMin
keeps the smallest predecessor among equal distances.
"""
import json
import math
import os
import random

import numpy as np
import pytest

import graphgen
import graphgen.workloads as W
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INT_INF = np.iinfo(np.int32).max


@pytest.fixture(scope="module")
def ds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_06895_gb300 as ds
    return ds


def gpu_solve(ds, h, src, delta, **opt):
    o = ds.make_options(**opt) if opt else None
    r = h.solve(src, delta, options=o, stats=True)
    return r.dist.cpu().numpy(), r.pred.cpu().numpy(), r.stats


def assert_same(g, src, d, p, d_ref=None, p_ref=None, what=""):
    if d_ref is None:
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
    if d.dtype == np.float32:
        bad = np.flatnonzero(d.view(np.uint32) != d_ref.view(np.uint32))
    else:
        bad = np.flatnonzero(d != d_ref)
    assert bad.size == 0, f"{what}: {bad.size} distances differ, first {bad[:5]} gpu {d[bad[:5]]} ref {d_ref[bad[:5]]}"
    badp = np.flatnonzero(p != p_ref)
    assert badp.size == 0, f"{what}: {badp.size} predecessors differ, first {badp[:5]} gpu {p[badp[:5]]} ref {p_ref[badp[:5]]}"


# persistent, stepped, a small grid, heavy passes kept apart from the next bucket (DSSSP_FLAG_NO_FUSE),
# the full-vector form (DSSSP_MODE_DENSE), and one thread-block cluster per solve (DSSSP_MODE_TEAM)
MODES = [dict(), dict(mode=1), dict(grid_size=3, block_size=64), dict(flags=2), dict(mode=2), dict(mode=3),
         dict(mode=3, team_blocks=2)]


# ------------------------------------------------------------------ hand-built cases

def test_hand_traced_example(ds):
    with open(os.path.join(GOLDEN, "fig1_trace_example.json")) as f:
        doc = json.load(f)
    arcs = [(a, b) for a, b, _ in doc["arcs"]]
    g = graphgen.from_arcs(doc["n"], arcs, np.array([c for _, _, c in doc["arcs"]], np.int32), dtype=np.int32)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    for opt in MODES:
        d, p, _ = gpu_solve(ds, h, doc["source_vertex"], doc["delta"], **opt)
        assert list(d) == doc["dist"] and list(p) == doc["pred"], opt


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_random_small_graphs(ds, dtype):
    rng = random.Random(7 if dtype == np.int32 else 8)
    for trial in range(60):
        n = rng.randint(1, 60)
        p = rng.choice([0.02, 0.08, 0.2])
        arcs, ws = [], []
        for u in range(n):
            for v in range(n):
                if rng.random() < p:
                    arcs.append((u, v))
                    if dtype == np.int32:
                        ws.append(rng.choice([0, 1, 2, 3, 7, 40]))
                    else:
                        ws.append(rng.choice([0.0, 0.1, 0.2, 0.3, 1e-7, 2.5, rng.random()]))
        if arcs and rng.random() < 0.5:
            arcs += arcs[:3]
            ws += ws[:3]
        g = graphgen.from_arcs(n, arcs, np.array(ws, dtype=dtype), dtype=dtype)
        h = ds.Graph(g.row_ptr, g.col, g.w)
        src = rng.randrange(n)
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
        for delta in (1e-3, 0.25, 3.0, math.inf):
            for opt in MODES:
                d, pr, _ = gpu_solve(ds, h, src, delta, **opt)
                assert_same(g, src, d, pr, d_ref, p_ref, f"trial {trial} delta {delta} {opt}")
        h.close()


def test_edge_cases(ds):
    cases = []
    cases.append((graphgen.from_arcs(1, [], np.zeros(0, np.float32), dtype=np.float32), 0))   # one vertex
    cases.append((graphgen.from_arcs(5, [(1, 2), (2, 3)], np.array([1, 1], np.int32), dtype=np.int32), 0))
    cases.append((graphgen.from_arcs(4, [(0, 1), (1, 2), (2, 1), (2, 3), (3, 0)],
                                     np.array([0, 0, 0, 0.5, 0], np.float32), dtype=np.float32), 0))
    big = INT_INF - 10
    cases.append((graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([big, 9, 5], np.int32),
                                     dtype=np.int32), 0))                   # INT32_MAX - 1: the largest distance
    cases.append((graphgen.from_arcs(3, [(0, 1), (0, 2), (1, 2)], np.array([-0.0, 1.0, 0.0], np.float32),
                                     dtype=np.float32), 0))
    # a hub whose arcs span many warps' slices, zero-weight arcs into the source
    k = 5000
    rng = np.random.default_rng(3)
    hub_w = rng.integers(0, 50, k).astype(np.int32)
    arcs = [(0, 1 + i) for i in range(k)] + [(1 + i, 0) for i in range(0, k, 7)] + [(5, 1 + i) for i in range(k)]
    ws = np.concatenate([hub_w, np.zeros(len(range(0, k, 7)), np.int32), rng.integers(0, 9, k).astype(np.int32)])
    cases.append((graphgen.from_arcs(k + 1, arcs, ws, dtype=np.int32), 0))
    cases.append((graphgen.from_arcs(k + 1, arcs, ws, dtype=np.int32), 17))
    # a long path: thousands of buckets
    n = 3000
    wp = (np.random.default_rng(5).random(n - 1) * 10).astype(np.float32)
    cases.append((graphgen.from_arcs(n, [(i, i + 1) for i in range(n - 1)], wp, dtype=np.float32), 0))
    for ci, (g, src) in enumerate(cases):
        h = ds.Graph(g.row_ptr, g.col, g.w)
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
        for delta in (0.5, 4.0, 1e9):
            for opt in MODES:
                d, p, _ = gpu_solve(ds, h, src, delta, **opt)
                assert_same(g, src, d, p, d_ref, p_ref, f"case {ci} delta {delta} {opt}")
        h.close()


def test_huge_bucket_indices(ds):
    """Bucket indices past 2^32 and past INT64_MAX (a small Delta against large distances):
    every vertex is still processed. int32: key 1431655765 at Delta 1/3 is bucket 2^32 - 1;
    float32: 1e9 at Delta 1e-12 is bucket 1e21, which saturates."""
    cases = [
        (graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([1431655765, 5, 7], np.int32), dtype=np.int32),
         [1.0 / 3.0, 0.25, 0.1]),
        (graphgen.from_arcs(4, [(0, 1), (1, 2), (2, 3)], np.array([1e9, 1.0, 3e9], np.float32), dtype=np.float32),
         [1e-12, 1e-3, 1e-30]),
    ]
    for g, deltas in cases:
        h = ds.Graph(g.row_ptr, g.col, g.w)
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
        assert (p_ref >= 0).all()
        for delta in deltas:
            for opt in MODES:
                d, p, _ = gpu_solve(ds, h, 0, delta, **opt)
                assert_same(g, 0, d, p, d_ref, p_ref, f"delta {delta} {opt}")
        h.close()


def overflow_cases():
    """(graph, source, overflows?) -- reading R14: an overflow is a sum out of a reached
    vertex, at its final distance, that the weight type cannot hold."""
    big = INT_INF - 100
    out = []
    # a true overflow out of a final distance (int32 and fp32)
    out.append((graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([INT_INF - 10, 20, 5], np.int32),
                                   dtype=np.int32), 0, True))
    out.append((graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([3e38, 3e38], np.float32),
                                   dtype=np.float32), 0, True))
    # a sum that overflows only from a distance that later decreases: no overflow.
    # With one bucket (large Delta) vertex 1 is relaxed first at distance big, then at 2.
    out.append((graphgen.from_arcs(4, [(0, 1), (0, 2), (2, 1), (1, 3)], np.array([big, 1, 1, 200], np.int32),
                                   dtype=np.int32), 0, False))
    out.append((graphgen.from_arcs(4, [(0, 1), (0, 2), (2, 1), (1, 3)], np.array([3e38, 1.0, 1.0, 3e38], np.float32),
                                   dtype=np.float32), 0, False))
    # an overflowing arc out of an unreached vertex: ignored
    out.append((graphgen.from_arcs(3, [(0, 1), (2, 1)], np.array([1, INT_INF - 1], np.int32), dtype=np.int32),
                0, False))
    return out


def test_overflow_status(ds):
    for ci, (g, src, overflows) in enumerate(overflow_cases()):
        h = ds.Graph(g.row_ptr, g.col, g.w)
        if overflows:
            with pytest.raises(oracle.PathOverflow):
                oracle.dijkstra(g.row_ptr, g.col, g.w, src)
        else:
            d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
        for delta in (0.5, 4.0, 1e9, math.inf):
            for opt in MODES:
                if overflows:
                    tdt = torch.float32 if g.w.dtype == np.float32 else torch.int32
                    dist = torch.full((g.n,), 7, dtype=tdt, device="cuda")
                    pred = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
                    with pytest.raises(ds.DsssError) as e:
                        h.solve(src, delta, dist=dist, pred=pred, options=ds.make_options(**opt) if opt else None)
                    assert e.value.status == ds.DSSSP_ERR_OVERFLOW, (ci, delta, opt)
                    assert bool((dist == 7).all()) and bool((pred == 7).all()), "outputs written on overflow"
                else:
                    d, p, _ = gpu_solve(ds, h, src, delta, **opt)
                    assert_same(g, src, d, p, d_ref, p_ref, f"overflow case {ci} delta {delta} {opt}")
        if overflows:                                   # asynchronous: the status comes from sync()
            h.solve(src, 1.0, options=ds.make_options(flags=ds.DSSSP_FLAG_ASYNC))
            with pytest.raises(ds.DsssError) as e:
                h.sync()
            assert e.value.status == ds.DSSSP_ERR_OVERFLOW
            h.sync()
        h.close()


# ------------------------------------------------------------------ workload recipes

def test_rmat14_int_delta32(ds):
    """R-MAT scale 14, int32 U{1..255}, Delta 32, highest-out-degree source: every launch shape."""
    g, srcs, deltas = W.rmat14_int()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, srcs[0])
    for opt in MODES + [dict(grid_size=1), dict(block_size=128), dict(grid_size=7, block_size=32)]:
        d, p, st = gpu_solve(ds, h, srcs[0], deltas[0], **opt)
        assert_same(g, srcs[0], d, p, d_ref, p_ref, str(opt))
        assert st["buckets"] >= 1 and (st["arcs_light"] > 0 or (opt.get("mode") == 2 and st["light_phases"] > 0))
    # the other sources too
    for s in graphgen.random_sources(g, 6, 99):
        d, p, _ = gpu_solve(ds, h, int(s), deltas[0])
        assert_same(g, int(s), d, p, what=f"src {s}")


@pytest.mark.parametrize("delta", [0.01, 0.05, 0.1, 0.5])
def test_rmat_unit_weights_deltas(ds, delta):
    """The scale-22 recipe at scale 17 (oracle in seconds): fp32 U[0,1), four Deltas."""
    g, srcs, _ = W.rmat22_unit(scale=17, n_sources=3)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    for s in srcs:
        d, p, _ = gpu_solve(ds, h, s, delta)
        assert_same(g, s, d, p, what=f"src {s} delta {delta}")


@pytest.mark.parametrize("delta", [100.0, 1000.0, 10000.0])
def test_grid_int_deltas(ds, delta):
    """The 4096 x 4096 grid recipe at 300 x 300: high diameter, int32 U{1..1000}."""
    g, srcs, _ = W.grid4096(side=300)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
    for opt in (dict(), dict(mode=1)):
        if opt and delta == 100.0:
            continue           # the stepped mode is host-driven; skip its thousands of phases
        d, p, _ = gpu_solve(ds, h, 0, delta, **opt)
        assert_same(g, 0, d, p, d_ref, p_ref, f"delta {delta} {opt}")


@pytest.mark.parametrize("solo_work", [-1, 2048, 2**31 - 1])
def test_window_rebins_with_every_solo_threshold(ds, solo_work):
    """Re-bins of the bucket window (more than 32 buckets) with phases never solo (-1), solo when small (the
    default), and always solo (block 0 runs every phase and takes each next view, re-bin thresholds included,
    from its own serial step); fused and separate heavy passes."""
    cases = [(W.grid4096(side=200)[0], 0, 100.0), (W.rmat22_unit(scale=15, n_sources=1)[0], None, 0.005)]
    for g, src, delta in cases:
        if src is None:
            src = int(np.argmax(np.diff(g.row_ptr)))
        h = ds.Graph(g.row_ptr, g.col, g.w)
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
        for flags in (0, 2):
            d, p, st = gpu_solve(ds, h, src, delta, solo_work=solo_work, flags=flags)
            assert_same(g, src, d, p, d_ref, p_ref, f"{g.name} solo_work {solo_work} flags {flags}")
            assert st["rebin_phases"] > 0 and st["buckets"] > 32, st
        h.close()


def test_er_family_small(ds):
    for g, src in W.er_family(count=6, n_lo=1000, n_hi=20000):
        h = ds.Graph(g.row_ptr, g.col, g.w)
        d, p, _ = gpu_solve(ds, h, src, 0.1)
        assert_same(g, src, d, p, what=g.name)
        h.close()


def test_device_pointer_graph_and_async(ds):
    g, srcs, deltas = W.rmat14_int(scale=12)
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    ww = torch.from_numpy(g.w).cuda()
    h = ds.Graph(rp, cl, ww)
    o = ds.make_options(flags=ds.DSSSP_FLAG_ASYNC)
    r = h.solve(srcs[0], deltas[0], options=o)
    h.sync()
    assert_same(g, srcs[0], r.dist.cpu().numpy(), r.pred.cpu().numpy(), what="device-ptr async")


# ------------------------------------------------------------------ error paths (no fault)

def test_validation_errors(ds):
    g = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([1.0, -2.0], np.float32), dtype=np.float32)
    with pytest.raises(ds.DsssError) as e:
        ds.Graph(g.row_ptr, g.col, g.w)
    assert e.value.status == ds.DSSSP_ERR_NEG_WEIGHT
    g = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([1.0, np.nan], np.float32), dtype=np.float32)
    with pytest.raises(ds.DsssError) as e:
        ds.Graph(g.row_ptr, g.col, g.w)
    assert e.value.status == ds.DSSSP_ERR_NEG_WEIGHT
    g = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([1, 2], np.int32), dtype=np.int32)
    col = g.col.copy()
    col[1] = 7
    with pytest.raises(ds.DsssError) as e:
        ds.Graph(g.row_ptr, col, g.w)
    assert e.value.status == ds.DSSSP_ERR_BAD_GRAPH
    rp = g.row_ptr.copy()
    rp[1] = 5
    with pytest.raises(ds.DsssError) as e:
        ds.Graph(rp, g.col, g.w)
    assert e.value.status == ds.DSSSP_ERR_BAD_GRAPH
    h = ds.Graph(g.row_ptr, g.col, g.w)
    with pytest.raises(ds.DsssError) as e:
        h.solve(3, 1.0)
    assert e.value.status == ds.DSSSP_ERR_INVALID_ARG
    with pytest.raises(ds.DsssError) as e:
        h.solve(0, 0.0)
    assert e.value.status == ds.DSSSP_ERR_INVALID_ARG


def test_bounded_wait_times_out_and_context_survives(ds):
    """One block leaves before the first barrier (test hook): the others' bounded
    wait runs out, the solve returns DSSSP_ERR_TIMEOUT, outputs are untouched,
    and the next solve on the same context is correct."""
    g, srcs, deltas = W.rmat14_int(scale=11)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    dist = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
    pred = torch.full((g.n,), -5, dtype=torch.int32, device="cuda")
    o = ds.make_options(test_hook=ds.DSSSP_HOOK_STALL_BARRIER, timeout_ns=50_000_000, grid_size=4)
    with pytest.raises(ds.DsssError) as e:
        h.solve(srcs[0], deltas[0], dist=dist, pred=pred, options=o)
    assert e.value.status == ds.DSSSP_ERR_TIMEOUT
    assert int((dist != -5).sum()) == 0 and int((pred != -5).sum()) == 0
    d, p, _ = gpu_solve(ds, h, srcs[0], deltas[0])
    assert_same(g, srcs[0], d, p, what="after timeout")
    # asynchronous flavour: the status surfaces at sync
    o.flags = ds.DSSSP_FLAG_ASYNC
    h.solve(srcs[0], deltas[0], options=o)
    with pytest.raises(ds.DsssError) as e:
        h.sync()
    assert e.value.status == ds.DSSSP_ERR_TIMEOUT
    h.sync()


def test_phase_cap_not_converged(ds):
    g, srcs, deltas = W.rmat14_int(scale=11)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    for mode in (0, 1, 3):
        with pytest.raises(ds.DsssError) as e:
            h.solve(srcs[0], deltas[0], options=ds.make_options(max_phases=3, mode=mode))
        assert e.value.status == ds.DSSSP_ERR_NOT_CONVERGED
    d, p, _ = gpu_solve(ds, h, srcs[0], deltas[0])
    assert_same(g, srcs[0], d, p, what="after cap")


# ------------------------------------------------------------------ full-size workloads

@pytest.fixture(scope="module")
def rmat22(ds):
    g, srcs, deltas = W.rmat22_unit()
    return g, srcs, deltas, ds.Graph(g.row_ptr, g.col, g.w)


def test_full_rmat22_every_source_every_delta_exact(ds, rmat22):
    """Full-size scale-22 R-MAT (fp32 U[0,1)), bench launch shape: all 64 sources at all four
    Deltas, whole arrays element by element against the oracle's Dijkstra."""
    g, srcs, deltas, h = rmat22
    for c0 in range(0, len(srcs), 16):
        chunk = srcs[c0:c0 + 16]
        refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, chunk)
        for s, d_ref, p_ref in zip(chunk, refd, refp):
            for delta in deltas:
                d, p, _ = gpu_solve(ds, h, s, delta)
                assert_same(g, s, d, p, d_ref, p_ref, f"source {s} delta {delta}")


def test_full_rmat22_dense_vector_form_exact(ds, rmat22):
    """The paper's full-vector form (DSSSP_MODE_DENSE) at full size: two sources, every Delta."""
    g, srcs, deltas, h = rmat22
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, srcs[:2])
    for s, d_ref, p_ref in zip(srcs[:2], refd, refp):
        for delta in deltas:
            d, p, st = gpu_solve(ds, h, s, delta, mode=2)
            assert_same(g, s, d, p, d_ref, p_ref, f"dense source {s} delta {delta}")
            assert st["light_phases"] > 0 and st["heavy_phases"] > 0


def test_full_grid4096_all_deltas_exact(ds):
    g, srcs, deltas = W.grid4096()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
    for delta in deltas:
        for opt in (dict(), dict(mode=3)):
            d, p, _ = gpu_solve(ds, h, 0, delta, **opt)
            assert_same(g, 0, d, p, d_ref, p_ref, f"delta {delta} {opt}")
