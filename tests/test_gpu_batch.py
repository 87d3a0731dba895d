"""Batched solves and the adjoint through the C ABI, against the CPU oracle.

Every instance of a batch must match the oracle's Dijkstra bit for bit
(distances) and exactly (predecessors), like a single solve. Gradients are
compared with the oracle's float64 subtree sums over the same tree (relative
error <= 1e-5 per arc) and, independently, with central differences of the
loss taken through the forward solve itself.
"""
import ctypes
import math

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


def same(d, p, d_ref, p_ref, what=""):
    if d.dtype == np.float32:
        bad = np.flatnonzero(d.view(np.uint32) != d_ref.view(np.uint32))
    else:
        bad = np.flatnonzero(d != d_ref)
    assert bad.size == 0, f"{what}: {bad.size} distances differ, first {bad[:5]} gpu {d[bad[:5]]} ref {d_ref[bad[:5]]}"
    badp = np.flatnonzero(p != p_ref)
    assert badp.size == 0, f"{what}: {badp.size} predecessors differ, first {badp[:5]}"


def batch(ds, hs, deltas, sources, src_graph=None, tape=False, **opt):
    o = ds.make_options(**opt) if opt else None
    b = ds.Batch(hs, deltas, sources, src_graph=src_graph, tape=tape, options=o)
    return b


def fetch(b):
    return [d.cpu().numpy() for d in b.dist], [p.cpu().numpy() for p in b.pred]


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("delta", [32.0, 1.0, math.inf])
def test_many_sources_int(ds, delta):
    g, srcs, _ = W.rmat14_int()
    sources = srcs + [int(s) for s in graphgen.random_sources(g, 23, 11)]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [delta], sources)
    b.run()
    st = b.sync(stats=True)
    ds_, ps_ = fetch(b)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for k, s in enumerate(sources):
        same(ds_[k], ps_[k], refd[k], refp[k], f"src {s} delta {delta}")
        assert st[k]["buckets"] >= 1
    b.close()
    h.close()


@pytest.mark.parametrize("delta", [0.01, 0.1, math.inf])
def test_many_sources_fp32(ds, delta):
    g, sources, _ = W.rmat22_unit(scale=16, n_sources=16)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [delta], sources)
    b.run()
    b.sync()
    ds_, ps_ = fetch(b)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for k, s in enumerate(sources):
        same(ds_[k], ps_[k], refd[k], refp[k], f"src {s} delta {delta}")


def test_one_team_reuses_its_memory(ds):
    """A single block solves every instance one after another, twice: stale stamps of
    earlier instances and earlier launches must never be mistaken for current ones."""
    g, sources, _ = W.rmat22_unit(scale=13, n_sources=12)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [0.05], sources, grid_size=1)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for rep in range(2):
        for d in b.dist:
            d.fill_(-1.0)
        b.run()
        st = b.sync(stats=True)
        ds_, ps_ = fetch(b)
        for k, s in enumerate(sources):
            same(ds_[k], ps_[k], refd[k], refp[k], f"rep {rep} src {s}")
            assert st[k]["team"] == 0
    b.close()


@pytest.mark.parametrize("team_blocks", [1, 2, 4, 8, 16])
def test_cluster_teams(ds, team_blocks):
    """An instance solved by a cluster of blocks sharing its control through distributed
    shared memory gives the same bits; few teams force several instances per team."""
    g, sources, _ = W.rmat22_unit(scale=15, n_sources=10)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for opt in (dict(team_blocks=team_blocks), dict(team_blocks=team_blocks, grid_size=2 * team_blocks)):
        for delta in (0.03, 0.3):
            b = batch(ds, h, [delta], sources, **opt)
            for rep in range(2):
                b.run()
                st = b.sync(stats=True)
                ds_, ps_ = fetch(b)
                for k, s in enumerate(sources):
                    same(ds_[k], ps_[k], refd[k], refp[k], f"{opt} delta {delta} rep {rep} src {s}")
            if "grid_size" in opt:
                assert max(x["team"] for x in st) <= 1
            b.close()


def test_cluster_teams_int32(ds):
    g, srcs, _ = W.rmat14_int()
    sources = srcs + [int(s) for s in graphgen.random_sources(g, 7, 21)]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for tb in (2, 8):
        b = batch(ds, h, [32.0], sources, team_blocks=tb)
        b.run()
        b.sync()
        ds_, ps_ = fetch(b)
        for k, s in enumerate(sources):
            same(ds_[k], ps_[k], refd[k], refp[k], f"int32 team_blocks {tb} src {s}")
        b.close()


def test_cluster_teams_tape_and_graphs(ds):
    g, sources, _ = W.rmat20_lognormal(scale=13, n_sources=6)
    cs = [graphgen.random_costs(g.n, 70 + k) for k in range(len(sources))]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    ref = oracle.tree_gradient_many(g.row_ptr, g.col, g.w, sources, cs)
    for tb in (4, 16):                          # 16: a non-portable cluster size, forward and adjoint
        b = batch(ds, h, [0.7], sources, tape=True, team_blocks=tb)
        b.run()
        b.sync()
        assert_grad_close(gpu_grad(ds, b, cs, g.m), ref, f"cluster tape {tb}")
        b.close()
    fam = W.er_family(count=10, n_lo=200, n_hi=30000)
    hs = [ds.Graph(x.row_ptr, x.col, x.w) for x, _ in fam]
    b = batch(ds, hs, [0.2] * len(fam), [s for _, s in fam], src_graph=list(range(len(fam))), team_blocks=2)
    b.run()
    b.sync()
    ds_, ps_ = fetch(b)
    for k, (x, s) in enumerate(fam):
        d_ref, p_ref = oracle.dijkstra(x.row_ptr, x.col, x.w, s)
        same(ds_[k], ps_[k], d_ref, p_ref, f"graph {k}")
    b.close()


def test_batch_run_inside_a_torch_cuda_graph(ds):
    """A batch run is one CUDA-graph launch with no allocation or host wait, so a caller can
    capture it in a graph of its own and replay it."""
    g, sources, _ = W.rmat22_unit(scale=13, n_sources=6)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [0.1], sources)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        b.run(side)                                      # warm-up outside the capture
    b.sync(stream=side)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=side):
        b.run(side)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for rep in range(2):
        for d in b.dist:
            d.fill_(-1.0)
        torch.cuda.synchronize()
        cg.replay()
        torch.cuda.synchronize()
        ds_, ps_ = fetch(b)
        for k, s in enumerate(sources):
            same(ds_[k], ps_[k], refd[k], refp[k], f"replay {rep} src {s}")
    b.sync()
    b.close()


def edge_graphs():
    out = []
    out.append((graphgen.from_arcs(1, [], np.zeros(0, np.float32), dtype=np.float32), 0, 1.0))
    out.append((graphgen.from_arcs(5, [(1, 2), (2, 3)], np.array([1, 1], np.float32), dtype=np.float32), 0, 1.0))
    out.append((graphgen.from_arcs(4, [(0, 1), (1, 2), (2, 1), (2, 3), (3, 0), (1, 1), (0, 1)],
                                   np.array([0, 0, 0, 0.5, 0, 0.25, 0.0], np.float32), dtype=np.float32), 0, 0.3))
    out.append((graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([3e38, 3e37], np.float32), dtype=np.float32),
                0, 1e38))                                 # 3.3e38: just below the float32 maximum
    k = 4000
    rng = np.random.default_rng(3)
    arcs = [(0, 1 + i) for i in range(k)] + [(1 + i, 0) for i in range(0, k, 7)] + [(5, 1 + i) for i in range(k)]
    ws = np.concatenate([rng.random(k), np.zeros(len(range(0, k, 7))), rng.random(k) * 0.1]).astype(np.float32)
    out.append((graphgen.from_arcs(k + 1, arcs, ws, dtype=np.float32), 0, 0.2))
    n = 2000
    wp = (np.random.default_rng(5).random(n - 1) * 10).astype(np.float32)
    out.append((graphgen.from_arcs(n, [(i, i + 1) for i in range(n - 1)], wp, dtype=np.float32), 0, 0.7))
    return out


def test_many_graphs_uneven_sizes(ds):
    """Graphs of very different sizes (ER family at small n, hand-built edge cases), a
    Delta per graph, several instances on some graphs, one launch."""
    graphs = [(g, s, d) for (g, s), d in zip(W.er_family(count=24, n_lo=50, n_hi=5000),
                                               np.geomspace(0.02, 2.0, 24))]
    graphs += edge_graphs()
    hs = [ds.Graph(g.row_ptr, g.col, g.w) for g, _, _ in graphs]
    sources, sg = [], []
    for gi, (g, s, _) in enumerate(graphs):
        sources.append(s)
        sg.append(gi)
    for gi in (0, 3, len(graphs) - 1):                   # more sources on a few graphs
        g = graphs[gi][0]
        for s in graphgen.random_sources(g, 3, 77 + gi):
            sources.append(int(s))
            sg.append(gi)
    b = batch(ds, hs, [d for _, _, d in graphs], sources, src_graph=sg)
    b.run()
    b.sync()
    ds_, ps_ = fetch(b)
    for k, (s, gi) in enumerate(zip(sources, sg)):
        g = graphs[gi][0]
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
        same(ds_[k], ps_[k], d_ref, p_ref, f"instance {k} graph {gi} src {s}")
    b.close()


def test_tape_forward_same_results(ds):
    g, sources, _ = W.rmat22_unit(scale=14, n_sources=8)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for tape in (False, True):
        b = batch(ds, h, [0.1], sources, tape=tape)
        b.run()
        b.sync()
        ds_, ps_ = fetch(b)
        for k, s in enumerate(sources):
            same(ds_[k], ps_[k], refd[k], refp[k], f"tape {tape} src {s}")
        b.close()


def test_phase_cap_and_errors(ds):
    g, sources, _ = W.rmat22_unit(scale=12, n_sources=4)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [0.01], sources, max_phases=3)
    b.run()
    with pytest.raises(ds.DsssError) as e:
        b.sync()
    assert e.value.status == ds.DSSSP_ERR_NOT_CONVERGED
    b.run()                                              # the plan stays usable
    with pytest.raises(ds.DsssError):
        b.sync()
    b.close()
    with pytest.raises(ds.DsssError) as e:               # source out of range
        ds.Batch(h, [0.1], [g.n])
    assert e.value.status == ds.DSSSP_ERR_INVALID_ARG
    b = batch(ds, h, [0.1], sources)                     # no tape: no backward
    b.run()
    b.sync()
    c = [torch.ones(g.n, device="cuda") for _ in sources]
    with pytest.raises(ds.DsssError) as e:
        b.backward(c, [torch.zeros(g.m, device="cuda")])
    assert e.value.status == ds.DSSSP_ERR_NO_TAPE
    b.close()
    gi = graphgen.from_arcs(3, [(0, 1)], np.array([1], np.int32), dtype=np.int32)
    hi = ds.Graph(gi.row_ptr, gi.col, gi.w)
    with pytest.raises(ds.DsssError) as e:               # a tape needs float32 weights
        ds.Batch(hi, [1.0], [0], tape=True)
    assert e.value.status == ds.DSSSP_ERR_UNSUPPORTED


def test_batch_overflow_status(ds):
    """Reading R14 in a batch: an instance whose path sums overflow fails the batch with
    DSSSP_ERR_OVERFLOW and leaves its own outputs alone; the other instances are exact."""
    big = np.iinfo(np.int32).max - 100
    g_ok = graphgen.from_arcs(4, [(0, 1), (0, 2), (2, 1), (1, 3)], np.array([big, 1, 1, 200], np.int32),
                              dtype=np.int32)                     # overflows only before the fixed point
    g_bad = graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([big + 90, 20, 5], np.int32),
                               dtype=np.int32)
    hs = [ds.Graph(g_ok.row_ptr, g_ok.col, g_ok.w), ds.Graph(g_bad.row_ptr, g_bad.col, g_bad.w)]
    for delta in (1e9, 4.0):
        b = batch(ds, hs, [delta, delta], [0, 0], src_graph=[0, 1])
        for d in b.dist:
            d.fill_(7)
        b.run()
        with pytest.raises(ds.DsssError) as e:
            b.sync()
        assert e.value.status == ds.DSSSP_ERR_OVERFLOW
        d_ref, p_ref = oracle.dijkstra(g_ok.row_ptr, g_ok.col, g_ok.w, 0)
        same(b.dist[0].cpu().numpy(), b.pred[0].cpu().numpy(), d_ref, p_ref, "instance without overflow")
        assert bool((b.dist[1] == 7).all()), "outputs of the overflowing instance were written"
        b.close()
    b = batch(ds, hs[:1], [1e9], [0, 0])                        # only the benign graph: no error
    b.run()
    b.sync()
    b.close()


# ------------------------------------------------------------------ adjoint

def gpu_grad(ds, b, cs, m):
    gw = torch.empty(m, dtype=torch.float32, device="cuda")
    b.backward([torch.from_numpy(c).cuda() for c in cs], [gw])
    b.sync()
    return gw.cpu().numpy().astype(np.float64)


def assert_grad_close(g, ref, what=""):
    err = np.abs(g - ref)
    tol = 1e-5 * np.abs(ref) + 1e-30
    bad = np.flatnonzero(err > tol)
    assert bad.size == 0, f"{what}: {bad.size} arcs off, first {bad[:5]} gpu {g[bad[:5]]} ref {ref[bad[:5]]}"
    assert np.linalg.norm(g - ref) <= 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("delta", [0.3, 2.0])
def test_backward_matches_oracle_gradient(ds, delta):
    g, sources, c0 = W.rmat20_lognormal(scale=14, n_sources=8)
    cs = [graphgen.random_costs(g.n, 1000 + k) for k in range(len(sources))]
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [delta], sources, tape=True)
    b.run()
    b.sync()
    ref = oracle.tree_gradient_many(g.row_ptr, g.col, g.w, sources, cs)
    gg = gpu_grad(ds, b, cs, g.m)
    assert np.count_nonzero(ref) > 1000
    assert_grad_close(gg, ref, f"delta {delta}")
    # accumulate adds into the output
    gw = torch.from_numpy(gg.astype(np.float32)).cuda()
    b.backward([torch.from_numpy(c).cuda() for c in cs], [gw], accumulate=True)
    b.sync()
    np.testing.assert_allclose(gw.cpu().numpy(), 2 * gg.astype(np.float32), rtol=1e-6)
    b.close()


def test_backward_special_cases(ds):
    # parallel arcs that both realise dist[2] (float32 sums round to 2^24): the tree arc is
    # the one with the smaller input index, whichever of them Delta calls light
    big = float(2 ** 24)
    for w1, w2 in ((1.0, 0.25), (0.25, 1.0), (0.5, 0.5)):
        g = graphgen.from_arcs(3, [(0, 1), (1, 2), (1, 2)], np.array([big, w1, w2], np.float32), dtype=np.float32)
        h = ds.Graph(g.row_ptr, g.col, g.w)
        for delta in (0.5, 4.0):
            b = batch(ds, h, [delta], [0], tape=True)
            b.run()
            b.sync()
            c = [np.array([0, 1, 3], np.float32)]
            got = gpu_grad(ds, b, c, g.m)
            np.testing.assert_array_equal(got, [4.0, 3.0, 0.0])
            np.testing.assert_array_equal(got, oracle.tree_gradient(g.row_ptr, g.col, g.w, 0, c[0]))
            b.close()
        h.close()
    # a zero-weight cycle in the predecessor graph: no gradient
    g = graphgen.from_arcs(4, [(0, 3), (3, 1), (3, 2), (1, 2), (2, 1)], np.array([1, 0, 0, 0, 0], np.float32),
                           dtype=np.float32)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [1.0], [0], tape=True)
    b.run()
    b.sync()
    b.backward([torch.ones(4, device="cuda")], [torch.zeros(g.m, device="cuda")])
    with pytest.raises(ds.DsssError) as e:
        b.sync()
    assert e.value.status == ds.DSSSP_ERR_DEGENERATE
    b.close()


def test_autograd_and_central_differences(ds):
    """torch.autograd through the library, then central differences of the loss taken
    through the forward solve itself (float32 distances, eps = 1e-3)."""
    from paper_1911_06895_gb300.autograd import shortest_path_distances
    g, sources, _ = W.rmat20_lognormal(scale=11, n_sources=4)
    rp = torch.from_numpy(g.row_ptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    w = torch.from_numpy(g.w).cuda().requires_grad_(True)
    c = torch.from_numpy(np.stack([graphgen.random_costs(g.n, 5 + k) for k in range(len(sources))])).cuda()
    delta = 1.0
    dist, pred = shortest_path_distances(w, rp, cl, sources, delta)
    ok = torch.isfinite(dist)
    loss = (c * torch.where(ok, dist, torch.zeros_like(dist))).double().sum()
    loss.backward()
    grad = w.grad.cpu().numpy().astype(np.float64)
    ref = oracle.tree_gradient_many(g.row_ptr, g.col, g.w, sources, [x for x in c.cpu().numpy()])
    assert_grad_close(grad, ref, "autograd")

    def loss_at(wv):
        with torch.no_grad():
            d, p = shortest_path_distances(wv, rp, cl, sources, delta)
            okk = torch.isfinite(d)
            return float((c.double() * torch.where(okk, d, torch.zeros_like(d)).double()).sum()), p

    base_pred = pred.clone()
    rng = np.random.default_rng(0)
    arcs = rng.choice(g.m, 150, replace=False)
    checked = 0
    for e in arcs:
        w0 = float(g.w[e])
        wp, wm = w.detach().clone(), w.detach().clone()
        wp[e] = w0 + 1e-3
        wm[e] = max(w0 - 1e-3, 0.0)
        hp = float(wp[e]) - w0
        hm = w0 - float(wm[e])
        lp, pp = loss_at(wp)
        lm, pm = loss_at(wm)
        if not (torch.equal(pp, base_pred) and torch.equal(pm, base_pred)):
            continue                                        # the tree changes within eps: a kink
        fd = (lp - lm) / (hp + hm)
        assert abs(fd - grad[e]) <= 2e-2 * abs(grad[e]) + 2e-3, (e, fd, grad[e])
        checked += 1
    assert checked >= 100


# ------------------------------------------------------------------ full-size workloads

def test_full_rmat20_256_sources(ds):
    """R-MAT scale 20, fp32 U[0,1), 256 sources in one launch: every instance exact."""
    g, sources = W.rmat20_unit()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [0.1], sources)
    b.run()
    b.sync()
    for c0 in range(0, 256, 64):
        refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources[c0:c0 + 64])
        for j in range(len(refd)):
            k = c0 + j
            same(b.dist[k].cpu().numpy(), b.pred[k].cpu().numpy(), refd[j], refp[j], f"src {sources[k]}")
    b.close()


def test_full_er_family_512(ds):
    """512 ER graphs, n log-uniform in [1e3, 2e5], one source each, one launch: all exact."""
    fam = W.er_family()
    hs = [ds.Graph(g.row_ptr, g.col, g.w) for g, _ in fam]
    b = batch(ds, hs, [0.1] * len(fam), [s for _, s in fam], src_graph=list(range(len(fam))))
    b.run()
    b.sync()
    ds_, ps_ = fetch(b)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor() as ex:
        refs = list(ex.map(lambda gs: oracle.dijkstra(gs[0].row_ptr, gs[0].col, gs[0].w, gs[1]), fam))
    for k, ((g, s), (d_ref, p_ref)) in enumerate(zip(fam, refs)):
        same(ds_[k], ps_[k], d_ref, p_ref, f"graph {k} ({g.name})")
    b.close()


def test_full_rmat20_lognormal_gradient(ds):
    """R-MAT scale 20, lognormal(0, 1) weights, 32 sources, c ~ U[0,1): forward exact on every
    source, gradient within 1e-5 (relative, per arc) of the oracle's float64 subtree sums."""
    g, sources, c = W.rmat20_lognormal()
    delta = 1.0
    cs = [c] * len(sources)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [delta], sources, tape=True)
    b.run()
    b.sync()
    ds_, ps_ = fetch(b)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    for k in range(len(sources)):
        same(ds_[k], ps_[k], refd[k], refp[k], f"src {sources[k]}")
    gg = gpu_grad(ds, b, cs, g.m)
    ref = oracle.tree_gradient_many(g.row_ptr, g.col, g.w, sources, cs)
    assert_grad_close(gg, ref, "scale 20")
    b.close()


def test_full_rmat20_lognormal_central_differences(ds):
    """The gradient check of the differentiable workload as specified: R-MAT scale 20,
    lognormal(0, 1) weights, 32 sources, c ~ U[0,1); central differences (eps = 1e-3) of
    the loss with float64 distances on the CPU, on 1,000 uniformly random arcs and on
    1,000 random arcs that carry gradient (tree arcs of some source). Arcs where the loss
    is not linear within eps (a kink) are excluded and counted."""
    g, sources, c = W.rmat20_lognormal()
    cs = [c] * len(sources)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    b = batch(ds, h, [1.0], sources, tape=True)
    b.run()
    b.sync()
    gg = gpu_grad(ds, b, cs, g.m)
    b.close()
    rng = np.random.default_rng(20)
    uniform = rng.choice(g.m, 1000, replace=False)
    carrying = rng.choice(np.flatnonzero(gg != 0.0), 1000, replace=False)
    # a tree arc with a large subtree is often within eps of a kink for one of the 32 sources
    for name, arcs, need in (("uniform", uniform, 950), ("tree arcs", carrying, 700)):
        fd, kink = oracle.fd_arcs_many(g.row_ptr, g.col, g.w, sources, cs, arcs, eps=1e-3)
        ok = kink == 0
        assert ok.sum() >= need, f"{name}: {int((~ok).sum())} arcs excluded"
        err = np.abs(gg[arcs][ok] - fd[ok])
        tol = 1e-5 * np.abs(fd[ok]) + 1e-6
        bad = np.flatnonzero(err > tol)
        assert bad.size == 0, (f"{name}: {bad.size} arcs off, first gpu {gg[arcs][ok][bad[:5]]} "
                               f"fd {fd[ok][bad[:5]]}")
        if name == "tree arcs":
            assert np.count_nonzero(fd[ok]) >= need


def test_batch_one_after_another_on_the_whole_gpu(ds):
    """team_blocks = -1: the plan runs its instances one after another with the grid-wide solver;
    same bits, counters filled, no tape, and a run refuses a stream being captured."""
    g, sources, _ = W.rmat22_unit(scale=15, n_sources=6)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    refd, refp, _ = oracle.dijkstra_many(g.row_ptr, g.col, g.w, sources)
    b = batch(ds, h, [0.1], sources, team_blocks=-1)
    for rep in range(2):
        b.run()
        st = b.sync(stats=True)
        ds_, ps_ = fetch(b)
        for k, s in enumerate(sources):
            same(ds_[k], ps_[k], refd[k], refp[k], f"rep {rep} src {s}")
    assert all(x["team"] == -1 and x["arcs_light"] + x["arcs_heavy"] > 0 and x["buckets"] >= 1 for x in st)
    s_ = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_):
        cg.capture_begin()
        b.dist[0].fill_(0)
        rc = ds.dsssp_batch_run(b.handle, ctypes.c_void_p(s_.cuda_stream))
        cg.capture_end()
    assert rc == ds.DSSSP_ERR_UNSUPPORTED
    b.close()
    with pytest.raises(ds.DsssError) as e:
        ds.Batch(h, [0.1], sources, tape=True, options=ds.make_options(team_blocks=-1))
    assert e.value.status == ds.DSSSP_ERR_UNSUPPORTED
