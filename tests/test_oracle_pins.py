"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each test ties the oracle to something independent of its own code:
brute-force walk enumeration, Floyd-Warshall, closed forms (BFS levels with the
paper's unit weights and Delta = 1, Manhattan distance on a full grid, prefix
sums on a path), SciPy's Dijkstra on integer weights, exact rational bucket
indices, a hand-traced schedule of Fig. 1, and planted mistakes that the
invariant checker must catch.
"""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import graphgen
import graphgen.workloads
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INT_INF = np.iinfo(np.int32).max


# --------------------------------------------------------------------------- helpers

def brute_force_walks(n, row_ptr, col, w, src):
    """Enumerate every walk from src with at most n arcs, summing left to right in
    the weight type's own arithmetic (fp32 rounding per arc / saturating int32).
    dist[v] = min over walks; pred[v] = smallest last hop among the optimal walks."""
    is_f = w.dtype == np.float32
    inf = np.float32(np.inf) if is_f else INT_INF
    best = [inf] * n
    last = [set() for _ in range(n)]
    best[src] = np.float32(0) if is_f else 0

    def add(a, b):
        if is_f:
            return np.float32(a) + np.float32(b)       # one binary32 rounding
        s = int(a) + int(b)
        return INT_INF if s >= INT_INF else s

    def rec(u, acc, depth):
        if depth == n:
            return
        for e in range(row_ptr[u], row_ptr[u + 1]):
            v = int(col[e])
            x = add(acc, w[e])
            if (is_f and np.isinf(x)) or (not is_f and x == INT_INF):
                continue
            if x < best[v]:
                best[v] = x
                last[v] = {u}
            elif x == best[v]:
                last[v].add(u)
            rec(v, x, depth + 1)

    rec(src, best[src], 0)
    dist = np.array(best, dtype=w.dtype)
    pred = np.array([min(last[v]) if last[v] else -1 for v in range(n)], dtype=np.int32)
    pred[src] = src
    return dist, pred


def random_tiny_graph(rng, n, p, dtype, zero_frac=0.15, ties=True):
    arcs, ws = [], []
    for u in range(n):
        for v in range(n):
            if rng.random() < p:
                arcs.append((u, v))
                if dtype == np.int32:
                    ws.append(0 if rng.random() < zero_frac else rng.choice([1, 2, 3, 5]) if ties
                              else rng.randint(1, 50))
                else:
                    ws.append(0.0 if rng.random() < zero_frac else
                              rng.choice([0.1, 0.2, 0.3, 0.7, 1e-8]) if ties else rng.random())
    # a parallel arc and a self-loop now and then (the ABI accepts both)
    if arcs and rng.random() < 0.3:
        arcs.append(arcs[0]); ws.append(ws[0] if dtype == np.int32 else ws[0] * 0.5)
    if rng.random() < 0.3:
        arcs.append((0, 0)); ws.append(1 if dtype == np.int32 else 0.25)
    return graphgen.from_arcs(n, arcs, ws, dtype=dtype)


def same_bits(a, b):
    return a.dtype == b.dtype and np.array_equal(a.view(np.uint32), b.view(np.uint32))


ALL_SOLVERS = ["dijkstra", "bellman_ford", "delta_ms", "delta_la"]


def solve(name, g, src, delta=1.0):
    if name in ("delta_ms", "delta_la"):
        return getattr(oracle, name)(g.row_ptr, g.col, g.w, src, delta)
    return getattr(oracle, name)(g.row_ptr, g.col, g.w, src)


# --------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_brute_force_tiny_graphs(dtype):
    rng = random.Random(1234 if dtype == np.int32 else 4321)
    checked = 0
    for trial in range(600):
        n = rng.randint(1, 7)
        g = random_tiny_graph(rng, n, rng.choice([0.25, 0.4, 0.6]), dtype)
        src = rng.randrange(n)
        d_bf, p_bf = brute_force_walks(n, g.row_ptr, g.col, g.w, src)
        for name in ALL_SOLVERS:
            for delta in ([1.0] if name in ("dijkstra", "bellman_ford") else [0.05, 0.3, 2.0, math.inf]):
                d, p = solve(name, g, src, delta)
                assert same_bits(d, d_bf), (trial, name, delta, d, d_bf)
                assert np.array_equal(p, p_bf), (trial, name, delta, p, p_bf)
                checked += 1
    assert checked > 1000


def test_floyd_warshall_integer_all_sources():
    rng = random.Random(99)
    for trial in range(40):
        n = rng.randint(2, 24)
        g = random_tiny_graph(rng, n, 0.2, np.int32, ties=False)
        fw = oracle.floyd_warshall_i32(g.row_ptr, g.col, g.w)
        for s in range(n):
            for name in ALL_SOLVERS:
                d, _ = solve(name, g, s, delta=7.0)
                assert np.array_equal(d, fw[s]), (trial, s, name)


# --------------------------------------------------------------------------- closed forms

def test_bfs_levels_unit_weights_delta_one():
    """The paper's own setting (Section VI-A): unit weights and Delta = 1 give BFS levels."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = graphgen.rmat(11, 8, seed=21)
    g.w = np.ones(g.m, dtype=np.int32)
    src = graphgen.highest_outdegree_vertex(g)
    a = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
    hops = csgraph.shortest_path(a, directed=True, unweighted=True, indices=src)
    want = np.where(np.isinf(hops), INT_INF, hops).astype(np.int32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, src, delta=1.0)
        assert np.array_equal(d, want), name
        assert oracle.check_invariants(g.row_ptr, g.col, g.w, src, d, p) == 0


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_manhattan_full_grid(dtype):
    rows, cols = 23, 17
    g = graphgen.grid(rows, cols, drop_p=0.0, seed=1)
    g.w = np.ones(g.m, dtype=dtype)
    r, c = np.divmod(np.arange(g.n), cols)
    want = (r + c).astype(dtype)
    want_pred = np.where(r > 0, (r - 1) * cols + c, r * cols + c - 1).astype(np.int32)
    want_pred[0] = 0
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=3.0)
        assert np.array_equal(d, want), name
        assert np.array_equal(p, want_pred), name


def test_path_prefix_sums_fp32_rounding():
    """Left-to-right fp32 prefix sums (np.cumsum is sequential) on a path graph."""
    rng = np.random.default_rng(5)
    n = 3000
    w = (rng.random(n - 1) * 10.0).astype(np.float32)
    w[::7] = np.float32(1e-7)                  # increments that round away at large sums
    g = graphgen.from_arcs(n, [(i, i + 1) for i in range(n - 1)], w, dtype=np.float32)
    want = np.concatenate([[np.float32(0)], np.cumsum(w, dtype=np.float32)])
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=0.5)
        assert same_bits(d, want.astype(np.float32)), name
        assert np.array_equal(p, np.concatenate([[0], np.arange(n - 1)]).astype(np.int32))


def test_star_and_unreachable():
    arcs = [(0, k) for k in range(1, 9)] + [(9, 0)]
    w = np.array([5, 3, 0, 9, 1, 7, 2, 8, 4], dtype=np.int32)
    g = graphgen.from_arcs(10, arcs, w, dtype=np.int32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=2.0)
        assert list(d[1:9]) == [5, 3, 0, 9, 1, 7, 2, 8]
        assert d[9] == INT_INF and p[9] == -1 and p[0] == 0
        assert list(p[1:9]) == [0] * 8


def test_int32_overflow_is_an_error():
    """Reading R14: a sum >= INT32_MAX out of a reached vertex is an overflow, reported
    by every solver; one below it is an ordinary distance."""
    big = INT_INF - 10
    g = graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([big, 20, 5], np.int32), dtype=np.int32)
    for name in ALL_SOLVERS:
        with pytest.raises(oracle.PathOverflow):
            solve(name, g, 0, delta=100.0)
    g = graphgen.from_arcs(4, [(0, 1), (1, 2), (0, 3)], np.array([big, 9, 5], np.int32), dtype=np.int32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=100.0)
        assert d[1] == big and p[1] == 0
        assert d[2] == INT_INF - 1 and p[2] == 1            # the largest distance that fits
        assert d[3] == 5


def test_fp32_overflow_is_an_error():
    g = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([3e38, 3e38], np.float32), dtype=np.float32)
    for name in ALL_SOLVERS:
        with pytest.raises(oracle.PathOverflow):
            solve(name, g, 0, delta=1e38)     # the LA form steps through every bucket index


def test_overflow_only_counts_final_distances():
    """The overflow condition uses final distances: a long detour whose sum would not
    fit is irrelevant when a shorter path gives the vertex a small distance."""
    big = INT_INF - 100
    arcs = [(0, 1), (1, 2), (0, 2), (2, 3)]
    w = np.array([big, 50, 1, 200], np.int32)     # 0->1->2 gives big+50; 0->2 gives 1
    g = graphgen.from_arcs(4, arcs, w, dtype=np.int32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=100.0)
        assert list(d) == [0, big, 1, 201] and list(p) == [0, 0, 0, 2]


def test_overflow_out_of_an_unreached_vertex_is_ignored():
    big = INT_INF - 1
    g = graphgen.from_arcs(3, [(0, 1), (2, 1)], np.array([1, big], np.int32), dtype=np.int32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=10.0)
        assert list(d) == [0, 1, INT_INF] and list(p) == [0, 0, -1]


def test_zero_weight_from_source_and_zero_cycle():
    """Zero-weight arcs out of the source must relax (the paper's value-mask caveat,
    Section V-B, fails exactly when t_Req = 0); a zero cycle must not loop forever."""
    arcs = [(0, 1), (1, 2), (2, 1), (2, 3), (3, 0)]
    w = np.array([0.0, 0.0, 0.0, 0.5, 0.0], np.float32)
    g = graphgen.from_arcs(4, arcs, w, dtype=np.float32)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, 0, delta=0.25)
        assert list(d) == [0.0, 0.0, 0.0, 0.5]
        assert list(p) == [0, 0, 1, 2]


def test_newly_reached_vertex_enters_frontier():
    """A vertex first reached by a request (t was 'absent' = inf) must be put in the
    bucket -- the intersection pitfall the paper describes for eWiseMult (Section V-B)."""
    g = graphgen.from_arcs(3, [(0, 1), (1, 2)], np.array([1, 1], np.int32), dtype=np.int32)
    for name in ("delta_ms", "delta_la"):
        d, _ = solve(name, g, 0, delta=10.0)
        assert list(d) == [0, 1, 2]


def test_untouched_vertex_not_reintroduced():
    """A vertex with no request in a round must not re-enter the bucket -- the union
    pitfall of eWiseAdd in Section V-B. Checked on the trace: vertex 2 (no incoming
    light request after its first round) is processed exactly once."""
    g = graphgen.from_arcs(4, [(0, 1), (0, 2), (1, 3)], np.array([1, 1, 1], np.int32), dtype=np.int32)
    for name in ("delta_ms", "delta_la"):
        _, _, tr = getattr(oracle, name)(g.row_ptr, g.col, g.w, 0, 10.0, trace=True)
        light = [(b, r, v) for b, r, v in tr if r >= 0]
        assert sorted(v for _, _, v in light) == [0, 1, 2, 3]


# --------------------------------------------------------------------------- scipy

def test_scipy_dijkstra_integer_rmat():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g, srcs, deltas = graphgen.workloads.rmat14_int(scale=12)
    a = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.n, g.n))
    ref = csgraph.dijkstra(a, directed=True, indices=srcs[0])
    want = np.where(np.isinf(ref), INT_INF, ref).astype(np.int64)
    for name in ALL_SOLVERS:
        d, p = solve(name, g, srcs[0], deltas[0])
        assert np.array_equal(d.astype(np.int64), want), name
        assert oracle.check_invariants(g.row_ptr, g.col, g.w, srcs[0], d, p) == 0


def test_fp32_close_to_fp64_reference():
    """fp32 distances stay within path-length * 2^-24 relative of SciPy's fp64 result."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = graphgen.rmat(12, 16, seed=8)
    g.w = graphgen.weights_unit(g.m, 8)
    a = sp.csr_matrix((g.w.astype(np.float64) + 0.0, g.col, g.row_ptr), shape=(g.n, g.n))
    src = graphgen.highest_outdegree_vertex(g)
    ref = csgraph.dijkstra(a, directed=True, indices=src)
    d, _ = oracle.dijkstra(g.row_ptr, g.col, g.w, src)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(d))
    assert np.all(np.abs(d[fin] - ref[fin]) <= 64 * 2.0 ** -24 * np.maximum(ref[fin], 1e-30) + 1e-12)


# --------------------------------------------------------------------------- buckets

def test_bucket_index_exact_rational():
    rng = random.Random(7)
    cases = []
    for _ in range(3000):
        delta = rng.choice([0.1, 0.01, 1 / 3, 0.7, 3.0, 1e-3, rng.random() + 1e-9,
                            float(np.nextafter(1 / 3, 1)), float(np.nextafter(0.1, 0))])
        k = rng.randint(0, 5000)
        # fp32 values right at and around k*Delta
        base = np.float32(k * delta)
        for x in (base, np.nextafter(base, np.float32(0)), np.nextafter(base, np.float32(np.inf))):
            cases.append((float(x), delta))
        cases.append((float(np.float32(rng.random() * 100)), delta))
    cases += [(0.0, 0.1), (1.0, 0.1), (3.0, 1.0), (2.9999998, 1.0)]
    for x, delta in cases:
        want = math.floor(Fraction(x) / Fraction(delta))
        assert oracle.bucket_index(x, delta) == want, (x, delta)
    assert oracle.bucket_index(123.0, math.inf) == 0


# --------------------------------------------------------------------------- Fig. 1 trace

def _golden_graph(doc):
    arcs = [(a, b) for a, b, _ in doc["arcs"]]
    w = np.array([c for _, _, c in doc["arcs"]], dtype=np.int32)
    return graphgen.from_arcs(doc["n"], arcs, w, dtype=np.int32)


def test_hand_traced_fig1_schedule():
    with open(os.path.join(GOLDEN, "fig1_trace_example.json")) as f:
        doc = json.load(f)
    g = _golden_graph(doc)
    want = sorted(tuple(r) for r in doc["trace"])
    for name in ("delta_ms", "delta_la"):
        d, p, tr = getattr(oracle, name)(g.row_ptr, g.col, g.w, doc["source_vertex"], doc["delta"], trace=True)
        assert list(d) == doc["dist"], name
        assert list(p) == doc["pred"], name
        assert sorted(tr) == want, (name, sorted(tr))


@pytest.mark.parametrize("delta", [0.02, 0.1, 0.5])
def test_set_form_and_la_form_schedules_agree(delta):
    """Fig. 1 left and right describe the same schedule: same vertices per
    (bucket, round) and the same S per heavy phase on an R-MAT graph."""
    g = graphgen.rmat(9, 8, seed=3)
    g.w = graphgen.weights_unit(g.m, 3)
    src = graphgen.highest_outdegree_vertex(g)
    d1, p1, t1 = oracle.delta_ms(g.row_ptr, g.col, g.w, src, delta, trace=True)
    d2, p2, t2 = oracle.delta_la(g.row_ptr, g.col, g.w, src, delta, trace=True)
    assert same_bits(d1, d2) and np.array_equal(p1, p2)
    assert sorted(t1) == sorted(t2)


def test_delta_one_matches_dijkstra_integer():
    """Section VII: Delta = 1 on integer weights behaves like Dijkstra -- every
    light bucket holds one distance value; results equal Dijkstra's."""
    g, srcs, _ = graphgen.workloads.rmat14_int(scale=10)
    d0, p0 = oracle.dijkstra(g.row_ptr, g.col, g.w, srcs[0])
    d1, p1, tr = oracle.delta_ms(g.row_ptr, g.col, g.w, srcs[0], 1.0, trace=True)
    assert np.array_equal(d0, d1) and np.array_equal(p0, p1)
    for b, r, v in tr:                      # bucket index == distance of every processed vertex
        assert d1[v] == b


# --------------------------------------------------------------------------- invariants

def test_invariant_checker_catches_planted_mistakes():
    g, srcs, deltas = graphgen.workloads.rmat14_int(scale=10)
    s = srcs[0]
    d, p = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d, p) == 0
    reached = np.flatnonzero((d != INT_INF) & (np.arange(g.n) != s))
    v = int(reached[len(reached) // 2])
    d_bad = d.copy(); d_bad[v] += 1                       # one distance too large
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d_bad, p) > 0
    d_bad = d.copy(); d_bad[v] -= 1                       # one distance too small
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d_bad, p) > 0
    p_bad = p.copy(); p_bad[v] = (p[v] + 1) % g.n         # wrong predecessor
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d, p_bad) > 0
    p_bad = p.copy(); p_bad[s] = -1
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d, p_bad) > 0


def test_invariant_checker_catches_cyclic_labelling():
    """A labelling too small on a cycle of zero-effect arcs passes the arc inequality and
    the predecessor rules; realisability and the predecessor chains catch it."""
    # 0 -> 1 (5); 1 <-> 2 with zero weights; 2 -> 3 (1). Truth: d = [0, 5, 5, 6].
    arcs = [(0, 1), (1, 2), (2, 1), (2, 3)]
    for dtype, w in ((np.int32, [5, 0, 0, 1]), (np.float32, [5.0, 0.0, 0.0, 1.0])):
        g = graphgen.from_arcs(4, arcs, np.array(w, dtype), dtype=dtype)
        d, p = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
        assert oracle.check_invariants(g.row_ptr, g.col, g.w, 0, d, p) == 0
        bogus_d = np.array([0, 2, 2, 3], dtype)                      # 1 and 2 too small
        bogus_p = np.array([0, 2, 1, 2], np.int32)                   # each the other's pred
        assert oracle.check_invariants(g.row_ptr, g.col, g.w, 0, bogus_d, bogus_p) >= 3
    # the same trap with positive weights absorbed by float32 rounding (spacing 2 at 2^24)
    big = float(2 ** 24)
    g = graphgen.from_arcs(4, arcs, np.array([big + 8, 0.5, 0.5, 1.0], np.float32), dtype=np.float32)
    d, p = oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, 0, d, p) == 0
    bogus_d = np.array([0, big, big, big], np.float32)
    bogus_p = np.array([0, 2, 1, 2], np.int32)
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, 0, bogus_d, bogus_p) >= 3


def test_invariant_checker_accepts_a_legal_zero_weight_pred_cycle():
    """With zero weights the smallest-id rule can close a predecessor cycle on correct
    distances (source 2; 0 and 1 both at distance 1 and each other's smallest tight
    in-neighbour). Realisability holds, so the checker accepts it."""
    arcs = [(2, 0), (2, 1), (0, 1), (1, 0)]
    g = graphgen.from_arcs(3, arcs, np.array([1, 1, 0, 0], np.int32), dtype=np.int32)
    d, p = oracle.dijkstra(g.row_ptr, g.col, g.w, 2)
    assert list(d) == [1, 1, 0] and list(p) == [1, 0, 2]
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, 2, d, p) == 0
    p_bad = p.copy(); p_bad[0] = 2                               # not the smallest tight in-neighbour
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, 2, d, p_bad) > 0


def test_invariant_checker_catches_a_broken_chain_on_random_graphs():
    """Planted on large random labellings: a reached vertex whose only tight walk is
    removed by raising the source's outgoing distances is flagged (realisability)."""
    g = graphgen.rmat(10, 16, seed=23)
    g.w = graphgen.weights_unit(g.m, 23)
    s = int(graphgen.random_sources(g, 1, 23)[0])
    d, p = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d, p) == 0
    reached = np.flatnonzero(np.isfinite(d) & (np.arange(g.n) != s))
    v = int(reached[0])
    d_bad = d.copy(); d_bad[v] = np.float32(0.0)                  # v claims distance 0
    assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d_bad, p) > 0


def test_all_forms_agree_many_deltas_fp32():
    g = graphgen.rmat(10, 16, seed=17)
    g.w = graphgen.weights_unit(g.m, 17)
    for s in graphgen.random_sources(g, 3, 17):
        d0, p0 = oracle.dijkstra(g.row_ptr, g.col, g.w, s)
        assert oracle.check_invariants(g.row_ptr, g.col, g.w, s, d0, p0) == 0
        for delta in (1e-3, 0.05, 0.3, 2.0, math.inf):
            for name in ("delta_ms", "delta_la", "bellman_ford"):
                d, p = solve(name, g, s, delta)
                assert same_bits(d, d0) and np.array_equal(p, p0), (name, delta)


def test_rejects_bad_input():
    g = graphgen.from_arcs(2, [(0, 1)], np.array([-1.0], np.float32), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.dijkstra(g.row_ptr, g.col, g.w, 0)
    g = graphgen.from_arcs(2, [(0, 1)], np.array([np.nan], np.float32), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.delta_ms(g.row_ptr, g.col, g.w, 0, 1.0)
    g = graphgen.from_arcs(2, [(0, 1)], np.array([1.0], np.float32), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.delta_la(g.row_ptr, g.col, g.w, 5, 1.0)
