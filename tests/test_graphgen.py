"""Seeded generators: determinism, shapes, and the structure each recipe promises."""
import numpy as np

import graphgen
import graphgen.workloads as W


def test_rmat_deterministic_and_simple():
    g1 = graphgen.rmat(10, 16, seed=3)
    g2 = graphgen.rmat(10, 16, seed=3)
    g3 = graphgen.rmat(10, 16, seed=4)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col, g2.col)
    assert not np.array_equal(g1.col, g3.col)
    assert g1.row_ptr[0] == 0 and g1.row_ptr[-1] == g1.m and np.all(np.diff(g1.row_ptr) >= 0)
    src = np.repeat(np.arange(g1.n), np.diff(g1.row_ptr))
    assert np.all(src != g1.col)                                  # no self-loops
    key = src.astype(np.int64) * g1.n + g1.col
    assert np.all(np.diff(key) > 0)                               # sorted, no repeats
    assert 0.5 * 16 * 1024 < g1.m <= 16 * 1024
    deg = g1.out_degree()
    assert deg.max() > 20 * deg.mean()                            # skewed (power-law-like)


def test_grid_drop_rate_and_neighbours():
    g = graphgen.grid(64, 48, drop_p=0.05, seed=3)
    full = 2 * (64 * 47 + 48 * 63)
    assert abs(g.m / full - 0.95) < 0.02
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    r1, c1 = np.divmod(src, 48)
    r2, c2 = np.divmod(g.col, 48)
    assert np.all(np.abs(r1 - r2) + np.abs(c1 - c2) == 1)


def test_weights_ranges():
    wi = graphgen.weights_int(100000, 1, 255, 1)
    assert wi.min() == 1 and wi.max() == 255
    wu = graphgen.weights_unit(100000, 2)
    assert wu.dtype == np.float32 and wu.min() >= 0 and wu.max() < 1
    assert np.all(wu * np.float32(2 ** 24) == np.floor(wu * np.float32(2 ** 24)))
    wl = graphgen.weights_lognormal(200000, 0.0, 1.0, 3)
    assert abs(np.mean(np.log(wl))) < 0.02 and abs(np.std(np.log(wl)) - 1) < 0.02


def test_workload_recipes_small():
    g, srcs, deltas = W.rmat14_int(scale=9)
    assert srcs == [graphgen.highest_outdegree_vertex(g)] and deltas == [32.0]
    assert g.w.dtype == np.int32
    g, srcs, deltas = W.rmat22_unit(scale=9, n_sources=8)
    assert len(set(srcs)) == 8 and all(g.out_degree()[s] >= 1 for s in srcs)
    assert deltas == [0.01, 0.05, 0.1, 0.5]
    fam = W.er_family(count=4, n_lo=100, n_hi=400)
    assert all(100 <= g.n <= 400 and 0.88 * 8 * g.n < g.m <= 8 * g.n for g, _ in fam)
