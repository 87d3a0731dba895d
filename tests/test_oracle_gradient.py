"""Pins of the oracle's weight gradient (tree_gradient) to facts outside it:
closed forms on paths and stars, central finite differences of the loss
computed with SciPy's float64 Dijkstra (a library routine, independent of the
oracle), detection of planted mistakes, the cycle case and the parallel-arc
reading. The gradient is the derivative of L = sum_v c[v] * dist[v] over reached
vertices; the paper defines distances only, so its pins are mathematical."""
import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def csr(n, arcs):
    arcs = sorted(arcs, key=lambda a: a[0])
    rp = np.zeros(n + 1, dtype=np.int64)
    for u, _, _ in arcs:
        rp[u + 1] += 1
    rp = np.cumsum(rp)
    col = np.array([a[1] for a in arcs], dtype=np.int32)
    w = np.array([a[2] for a in arcs], dtype=np.float32)
    return rp, col, w


def random_graph(rng, n, m):
    arcs = set()
    while len(arcs) < m:
        u, v = rng.integers(0, n, 2)
        if u != v:
            arcs.add((int(u), int(v)))
    arcs = sorted(arcs)
    w = np.exp(rng.normal(0.0, 1.0, len(arcs))).astype(np.float32)    # lognormal(0, 1), tie-free
    return csr(n, [(u, v, float(x)) for (u, v), x in zip(arcs, w)])


def loss64(rp, col, w64, src, c):
    n = rp.shape[0] - 1
    a = sp.csr_matrix((w64, col, rp), shape=(n, n))
    d, p = csgraph.dijkstra(a, directed=True, indices=src, return_predecessors=True)
    ok = np.isfinite(d)
    return float(np.sum(c.astype(np.float64)[ok] * d[ok])), p


def test_path_closed_form():
    rng = np.random.default_rng(1)
    n = 40
    rp, col, w = csr(n, [(i, i + 1, float(rng.uniform(0.1, 2))) for i in range(n - 1)])
    c = rng.uniform(0, 1, n).astype(np.float32)
    g = oracle.tree_gradient(rp, col, w, 0, c)
    want = np.array([c[i + 1:].astype(np.float64).sum() for i in range(n - 1)])
    np.testing.assert_allclose(g, want, rtol=1e-12)


def test_star_and_unreached():
    n = 8
    rp, col, w = csr(n, [(0, v, 0.5 + v) for v in range(1, 6)])      # 6, 7 unreached
    c = np.arange(n, dtype=np.float32) + 1
    g = oracle.tree_gradient(rp, col, w, 0, c)
    np.testing.assert_array_equal(g, c[1:6].astype(np.float64))


def test_off_tree_arcs_get_zero():
    # 0->1 (1), 0->2 (5), 1->2 (1): the arc 0->2 is not on the tree
    rp, col, w = csr(3, [(0, 1, 1.0), (0, 2, 5.0), (1, 2, 1.0)])
    c = np.array([0.0, 2.0, 3.0], dtype=np.float32)
    g = oracle.tree_gradient(rp, col, w, 0, c)
    # arcs sorted by tail: [0->1, 0->2, 1->2]
    np.testing.assert_array_equal(g, [5.0, 0.0, 3.0])


@pytest.mark.parametrize("seed", range(6))
def test_central_differences_with_scipy_float64(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = 60, 240
    rp, col, w = random_graph(rng, n, m)
    src = int(rng.integers(0, n))
    c = rng.uniform(0, 1, n).astype(np.float32)
    dist, pred = oracle.dijkstra(rp, col, w, src)
    g = oracle.tree_gradient(rp, col, w, src, c, dist, pred)
    w64 = w.astype(np.float64)
    _, p0 = loss64(rp, col, w64, src, c)
    reached = np.isfinite(dist)
    p_ref = np.where(reached, pred, -9999)
    p0 = np.where(reached, p0, -9999)
    p0[src] = src
    assert np.array_equal(p0, p_ref), "float32 and float64 trees differ on this seed"
    checked = 0
    for e in range(m):
        eps = min(1e-3, 0.5 * float(w[e]))
        wp, wm = w64.copy(), w64.copy()
        wp[e] += eps
        wm[e] -= eps
        lp, pp = loss64(rp, col, wp, src, c)
        lm, pm = loss64(rp, col, wm, src, c)
        pp[src] = src
        pm[src] = src
        if not (np.array_equal(np.where(reached, pp, -9999), p_ref)
                and np.array_equal(np.where(reached, pm, -9999), p_ref)):
            continue                                         # a kink: the tree changes within eps
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[e]) <= 1e-6 + 1e-9 * abs(g[e]), (e, fd, g[e])
        checked += 1
    assert checked >= int(0.9 * m)
    assert np.count_nonzero(g) >= 20


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(7)
    n, m = 60, 240
    rp, col, w = random_graph(rng, n, m)
    c = rng.uniform(0, 1, n).astype(np.float32)
    g = oracle.tree_gradient(rp, col, w, 0, c)
    w64 = w.astype(np.float64)
    e = int(np.argmax(g))                                    # a tree arc with a large subtree

    def fd(k, eps=1e-4):
        wp, wm = w64.copy(), w64.copy()
        wp[k] += eps
        wm[k] -= eps
        return (loss64(rp, col, wp, 0, c)[0] - loss64(rp, col, wm, 0, c)[0]) / (2 * eps)

    assert abs(fd(e) - g[e]) <= 1e-6 * (1 + abs(g[e]))
    dropped_self = g[e] - c[col[e]]                          # forgot the vertex's own weight c[v]
    assert abs(fd(e) - dropped_self) > 1e-3
    leaf = [k for k in range(m) if g[k] > 0 and abs(g[k] - c[col[k]]) < 1e-12]
    assert leaf, "no leaf arc"
    k = leaf[0]
    assert abs(fd(k) - 2 * g[k]) > 1e-3                      # double-counted leaf


def test_sum_over_sources_is_sum_of_singles():
    rng = np.random.default_rng(9)
    rp, col, w = random_graph(rng, 50, 200)
    srcs = [0, 3, 17]
    cs = [rng.uniform(0, 1, 50).astype(np.float32) for _ in srcs]
    many = oracle.tree_gradient_many(rp, col, w, srcs, cs, threads=2)
    single = sum(oracle.tree_gradient(rp, col, w, s, c) for s, c in zip(srcs, cs))
    np.testing.assert_allclose(many, single, rtol=0, atol=1e-12)


def test_zero_weight_cycle_is_rejected():
    # 0->3 (1); 3->1, 3->2, 1->2, 2->1 all 0: pred[1] = 2 and pred[2] = 1 (smallest id), a cycle
    rp, col, w = csr(4, [(0, 3, 1.0), (3, 1, 0.0), (3, 2, 0.0), (1, 2, 0.0), (2, 1, 0.0)])
    dist, pred = oracle.dijkstra(rp, col, w, 0)
    assert pred[1] == 2 and pred[2] == 1
    with pytest.raises(oracle.CycleError):
        oracle.tree_gradient(rp, col, w, 0, np.ones(4, dtype=np.float32))


def test_parallel_arcs_smallest_input_index():
    """Reading R11 on a hand-computed case. d[1] = 2^24; row 1 holds two parallel arcs
    1->2: input index 1 with w = 1.0 and input index 2 with w = 0.25. In float32 both
    sums round to 2^24 (the spacing there is 2; ties go to even), so both realise d[2]
    and L has a kink in either weight. The tree arc is the one with the smaller input
    index, whatever Delta would call light or heavy: dL/dw = [c1 + c2, c2, 0]."""
    big = float(2 ** 24)
    rp = np.array([0, 1, 3, 3], dtype=np.int64)
    col = np.array([1, 2, 2], dtype=np.int32)
    for w1, w2 in ((1.0, 0.25), (0.25, 1.0), (0.5, 0.5)):
        w = np.array([big, w1, w2], dtype=np.float32)
        dist, pred = oracle.dijkstra(rp, col, w, 0)
        assert dist[2] == np.float32(big) and pred[2] == 1
        g = oracle.tree_gradient(rp, col, w, 0, np.array([0, 1, 3], dtype=np.float32))
        np.testing.assert_array_equal(g, [4.0, 3.0, 0.0])


def test_tree_arc_rule_across_rows_follows_pred():
    """Two different tails reach d[3] exactly (0->1->3 and 0->2->3, all sums exact):
    pred[3] = 1 (smallest id) and the tree arc is 1->3, the smaller input index."""
    rp, col, w = csr(4, [(0, 1, 1.0), (0, 2, 2.0), (1, 3, 2.0), (2, 3, 1.0)])
    dist, pred = oracle.dijkstra(rp, col, w, 0)
    assert dist[3] == 3.0 and pred[3] == 1
    g = oracle.tree_gradient(rp, col, w, 0, np.array([0, 1, 1, 1], dtype=np.float32))
    np.testing.assert_array_equal(g, [2.0, 1.0, 1.0, 0.0])


@pytest.mark.parametrize("seed", range(4))
def test_local_repair_differences_match_full_resolves(seed):
    """The oracle's central differences (local repair of the float64 distances) against
    full re-solves with SciPy's float64 Dijkstra, on every arc of random graphs."""
    rng = np.random.default_rng(300 + seed)
    n, m = 80, 400
    rp, col, w = random_graph(rng, n, m)
    src = int(rng.integers(0, n))
    c = rng.uniform(0, 1, n).astype(np.float32)
    eps = 1e-3
    arcs = np.arange(m)
    fd, kink = oracle.fd_arcs(rp, col, w, src, c, arcs, eps)
    w64 = w.astype(np.float64)
    linear = 0
    for e in range(m):
        if kink[e] == 2:
            assert w[e] < eps
            continue
        wp, wm = w64.copy(), w64.copy()
        wp[e] += eps
        wm[e] -= eps
        want = (loss64(rp, col, wp, src, c)[0] - loss64(rp, col, wm, src, c)[0]) / (2 * eps)
        assert abs(fd[e] - want) <= 1e-7 * (1 + abs(want)), (e, fd[e], want, kink[e])
        if kink[e] == 0:
            linear += 1
    assert linear >= int(0.8 * m)


def test_local_repair_flags_kinks_and_matches_subtree_sums():
    """Where no kink is flagged the central difference is the derivative: it equals the
    float64 subtree sum of c below the arc (hand-built: a path and a shortcut to its end)."""
    # 0 -> 1 -> 2 -> 3 (1 each) and a shortcut 0 -> 3 of 3.0005: within eps of the path
    rp, col, w = csr(4, [(0, 1, 1.0), (1, 2, 1.0), (2, 3, 1.0), (0, 3, 3.0005)])
    c = np.array([0, 1, 2, 4], dtype=np.float32)
    fd, kink = oracle.fd_arcs(rp, col, w, 0, c, np.arange(4), 1e-3)
    # arcs by tail: [0->1, 0->3, 1->2, 2->3]; raising any path arc by 1e-3 makes the
    # shortcut win for vertex 3, and lowering the shortcut by 1e-3 does too: every arc
    # is within eps of a kink
    assert list(kink) == [1, 1, 1, 1]
    # a shortcut 2e-3 away from winning: linear on both sides of every arc
    rp, col, w = csr(4, [(0, 1, 1.0), (1, 2, 1.0), (2, 3, 1.0), (0, 3, 3.002)])
    fd, kink = oracle.fd_arcs(rp, col, w, 0, c, np.arange(4), 1e-3)
    assert list(kink) == [0, 0, 0, 0]
    np.testing.assert_allclose(fd, [7.0, 0.0, 6.0, 4.0], rtol=1e-9)
