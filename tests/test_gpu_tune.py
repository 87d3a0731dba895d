"""The Delta autotuner: it returns a Delta from the candidates it tried, and
distances at the chosen Delta stay exact (Delta only orders the work)."""
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


def test_tune_single_solve_explicit_candidates(ds):
    g, srcs, _ = W.rmat14_int()
    h = ds.Graph(g.row_ptr, g.col, g.w)
    cands = [4.0, 16.0, 64.0, 256.0]
    sample = [int(s) for s in graphgen.random_sources(g, 3, 5)]
    (d,), (ms,) = ds.autotune(h, sample, target="solve", candidates=cands, refine=-1)
    assert d in cands and ms > 0
    r = h.solve(srcs[0], d)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, srcs[0])
    assert np.array_equal(r.dist.cpu().numpy(), d_ref) and np.array_equal(r.pred.cpu().numpy(), p_ref)


def test_tune_default_ladder_with_refinement(ds):
    g, srcs, _ = W.rmat22_unit(scale=14, n_sources=4)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    (d,), (ms,) = ds.autotune(h, srcs[:2], target="solve")
    mean_w = float(np.mean(g.w, dtype=np.float64))
    d0 = 4 * mean_w / (g.m / g.n)
    ratio = np.log2(d / d0)
    assert -3.75 <= ratio <= 3.75                    # within the ladder plus refinement steps
    assert abs(ratio * 4 - round(ratio * 4)) < 1e-9  # a quarter-power-of-two step from the start
    r = h.solve(srcs[2], d)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, srcs[2])
    assert np.array_equal(r.dist.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))


def test_tune_batch_per_graph(ds):
    fam = W.er_family(count=12, n_lo=500, n_hi=20000)
    hs = [ds.Graph(g.row_ptr, g.col, g.w) for g, _ in fam]
    sample = [[s] + [int(x) for x in graphgen.random_sources(g, 1, 9)] for g, s in fam]
    deltas, ms = ds.autotune(hs, sample, target="batch")
    assert len(deltas) == len(fam) and all(d > 0 for d in deltas) and all(t > 0 for t in ms)
    b = ds.Batch(hs, deltas, [s for _, s in fam], src_graph=list(range(len(fam))))
    b.run()
    b.sync()
    for k, (g, s) in enumerate(fam):
        d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
        assert np.array_equal(b.dist[k].cpu().numpy().view(np.uint32), d_ref.view(np.uint32)), k
        assert np.array_equal(b.pred[k].cpu().numpy(), p_ref), k
    b.close()


def test_tune_rejects_bad_arguments(ds):
    g, srcs, _ = W.rmat14_int(scale=10)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    with pytest.raises(ds.DsssError):
        ds.autotune(h, [g.n], target="solve")
    with pytest.raises(ds.DsssError):
        ds.autotune(h, srcs, target="solve", candidates=[-1.0])


def test_tune_team_blocks(ds):
    g, sources, _ = W.rmat22_unit(scale=15, n_sources=8)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    tb, ms = ds.tune_team_blocks(h, [0.1], sources)
    assert tb in (1, 2, 4, 8, 16, -1) and ms > 0
    b = ds.Batch(h, [0.1], sources, options=ds.make_options(team_blocks=tb))
    b.run()
    b.sync()
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, sources[0])
    assert np.array_equal(b.dist[0].cpu().numpy().view(np.uint32), d_ref.view(np.uint32))
    b.close()


def test_tune_solo_work(ds):
    g, sources, _ = W.rmat22_unit(scale=14, n_sources=3)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    sw, ms = ds.tune_solo_work(h, sources[:2], 0.05)
    assert sw in (-1, 512, 2048, 8192, 32768) and ms > 0
    r = h.solve(sources[2], 0.05, options=ds.make_options(solo_work=sw))
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, sources[2])
    assert np.array_equal(r.dist.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))


def test_tune_schedule_picks_a_scheme_and_it_is_exact(ds):
    """The schedule tuner times the persistent scheme at each solo threshold and the one-cluster
    scheme at 8 and 16 blocks; the options it returns solve exactly. On a high-diameter grid the
    one-cluster scheme is expected to win, on a small-world R-MAT the grid-wide one."""
    g, srcs, _ = W.grid4096(side=400)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    o, ms = ds.tune_schedule(h, [0, 1], 100.0)
    assert ms > 0 and o.mode in (ds.DSSSP_MODE_PERSISTENT, ds.DSSSP_MODE_TEAM)
    assert o.mode == ds.DSSSP_MODE_TEAM
    r = h.solve(0, 100.0, options=o)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
    assert np.array_equal(r.dist.cpu().numpy(), d_ref) and np.array_equal(r.pred.cpu().numpy(), p_ref)
    g, sources, _ = W.rmat22_unit(scale=16, n_sources=3)
    h = ds.Graph(g.row_ptr, g.col, g.w)
    o, ms = ds.tune_schedule(h, sources[:2], 0.5)
    r = h.solve(sources[2], 0.5, options=o)
    d_ref, p_ref = oracle.dijkstra(g.row_ptr, g.col, g.w, sources[2])
    assert np.array_equal(r.dist.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))
    assert np.array_equal(r.pred.cpu().numpy(), p_ref)
