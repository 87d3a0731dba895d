"""Seeded synthetic graph and weight generators (inputs only).

This module holds none of the shortest-path arithmetic. It turns a seed into a
CSR graph (``row_ptr`` int64[n+1], ``col`` int32[m]) plus an edge-weight array,
and is the only code shared by the CPU oracle tests and the CUDA path.

Graphs stand in for the paper's real-world inputs (SNAP and GraphChallenge
graphs, Section VI-A), which are not available here:

* R-MAT (Chakrabarti et al. 2004), a/b/c/d = .57/.19/.19/.05, edge factor 16,
  vertices relabelled by a seeded permutation, self-loops and repeated arcs
  removed;
* a rows x cols 4-neighbour grid with each directed arc dropped independently;
* directed Erdos-Renyi G(n, m) draws.

All random numbers come from the counter-based splitmix64 hash in
``graphgen.c``, so a (generator, seed) pair gives the same graph on every host.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library beside it (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        c = ctypes
        lib.gg_hash.restype = c.c_uint64
        lib.gg_hash.argtypes = [c.c_uint64, c.c_uint64, c.c_uint64]
        lib.gg_rmat_edges.restype = None
        lib.gg_rmat_edges.argtypes = [c.c_int32, c.c_int64, c.c_double, c.c_double, c.c_double,
                                      c.c_uint64, i32p, i32p]
        lib.gg_permutation.restype = None
        lib.gg_permutation.argtypes = [c.c_int64, c.c_uint64, i32p]
        lib.gg_relabel.restype = None
        lib.gg_relabel.argtypes = [c.c_int64, i32p, i32p]
        lib.gg_grid_edges.restype = c.c_int64
        lib.gg_grid_edges.argtypes = [c.c_int32, c.c_int32, c.c_double, c.c_uint64, i32p, i32p]
        lib.gg_er_edges.restype = None
        lib.gg_er_edges.argtypes = [c.c_int64, c.c_int64, c.c_uint64, i32p, i32p]
        lib.gg_build_csr.restype = c.c_int64
        lib.gg_build_csr.argtypes = [c.c_int64, c.c_int64, i32p, i32p, i64p, i32p]
        lib.gg_weights_int.restype = None
        lib.gg_weights_int.argtypes = [c.c_int64, c.c_int32, c.c_int32, c.c_uint64, i32p]
        lib.gg_weights_unit.restype = None
        lib.gg_weights_unit.argtypes = [c.c_int64, c.c_uint64, f32p]
        lib.gg_weights_lognormal.restype = None
        lib.gg_weights_lognormal.argtypes = [c.c_int64, c.c_double, c.c_double, c.c_uint64, f32p]
        _lib = lib
    return _lib


def hash64(seed: int, stream: int, index: int) -> int:
    """The generator's counter-based 64-bit random word for (seed, stream, index)."""
    return int(_load().gg_hash(seed, stream, index))


# --------------------------------------------------------------------------- graphs

@dataclass
class Graph:
    """A directed graph in CSR form with one weight per arc.

    ``row_ptr[v]:row_ptr[v+1]`` indexes the out-arcs of ``v`` (row = out-edges,
    as in the paper's adjacency matrix, Section II-A); ``col`` holds heads,
    ``w`` holds int32 or float32 weights.
    """
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def csr_from_arcs(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sort arcs by (source, head), drop self-loops and repeats, return (row_ptr, col)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(src.shape[0], 1), dtype=np.int32)
    m = lib.gg_build_csr(n, src.shape[0], src, dst, row_ptr, col)
    if m < 0:
        raise MemoryError("gg_build_csr: allocation failed")
    return row_ptr, col[:m].copy()


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> Graph:
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale draws (before dedup)."""
    lib = _load()
    n = 1 << scale
    draws = edge_factor * n
    src = np.empty(draws, dtype=np.int32)
    dst = np.empty(draws, dtype=np.int32)
    lib.gg_rmat_edges(scale, draws, a, b, c, seed, src, dst)
    if permute:
        perm = np.empty(n, dtype=np.int32)
        lib.gg_permutation(n, seed, perm)
        lib.gg_relabel(draws, perm, src)
        lib.gg_relabel(draws, perm, dst)
    row_ptr, col = csr_from_arcs(n, src, dst)
    return Graph(n, row_ptr, col, name=f"rmat{scale}",
                 meta=dict(kind="rmat", scale=scale, edge_factor=edge_factor, a=a, b=b, c=c,
                           seed=seed, draws=draws))


def grid(rows: int, cols: int, drop_p: float = 0.05, seed: int = 3) -> Graph:
    """rows x cols 4-neighbour grid, both directions, each arc dropped with prob drop_p."""
    lib = _load()
    n = rows * cols
    cap = 4 * n
    src = np.empty(cap, dtype=np.int32)
    dst = np.empty(cap, dtype=np.int32)
    k = lib.gg_grid_edges(rows, cols, drop_p, seed, src, dst)
    row_ptr, col = csr_from_arcs(n, src[:k], dst[:k])
    return Graph(n, row_ptr, col, name=f"grid{rows}x{cols}",
                 meta=dict(kind="grid", rows=rows, cols=cols, drop_p=drop_p, seed=seed))


def erdos_renyi(n: int, m_draws: int, seed: int = 5) -> Graph:
    """Directed G(n, m): m_draws uniform ordered pairs, self-loops and repeats removed."""
    lib = _load()
    src = np.empty(m_draws, dtype=np.int32)
    dst = np.empty(m_draws, dtype=np.int32)
    lib.gg_er_edges(n, m_draws, seed, src, dst)
    row_ptr, col = csr_from_arcs(n, src, dst)
    return Graph(n, row_ptr, col, name=f"er{n}",
                 meta=dict(kind="er", n=n, draws=m_draws, seed=seed))


def from_arcs(n: int, arcs, weights=None, dtype=np.float32, name: str = "custom") -> Graph:
    """Build a Graph from an explicit arc list [(u, v), ...] (kept in given order per row).

    Unlike csr_from_arcs, self-loops and repeated arcs are KEPT; use for hand-built
    test graphs where those cases are wanted.
    """
    arcs = list(arcs)
    order = sorted(range(len(arcs)), key=lambda k: (arcs[k][0], k))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(len(arcs), dtype=np.int32)
    w = np.empty(len(arcs), dtype=dtype)
    for j, k in enumerate(order):
        u, v = arcs[k]
        row_ptr[u + 1] += 1
        col[j] = v
        if weights is not None:
            w[j] = weights[k]
    row_ptr = np.cumsum(row_ptr).astype(np.int64)
    return Graph(n, row_ptr, col, w if weights is not None else None, name=name)


# --------------------------------------------------------------------------- weights

def weights_int(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """int32 weights uniform in {lo, ..., hi}."""
    w = np.empty(m, dtype=np.int32)
    _load().gg_weights_int(m, lo, hi, seed, w)
    return w


def weights_unit(m: int, seed: int) -> np.ndarray:
    """float32 weights uniform in [0, 1) on the 2**-24 lattice (exact fp32 values, 0.0 possible)."""
    w = np.empty(m, dtype=np.float32)
    _load().gg_weights_unit(m, seed, w)
    return w


def weights_lognormal(m: int, mu: float, sigma: float, seed: int) -> np.ndarray:
    """float32 weights lognormal(mu, sigma), continuous sampling (ties have ~zero probability)."""
    w = np.empty(m, dtype=np.float32)
    _load().gg_weights_lognormal(m, mu, sigma, seed, w)
    return w


# --------------------------------------------------------------------------- sources

def highest_outdegree_vertex(g: Graph) -> int:
    """Vertex of largest out-degree, smallest id on ties."""
    return int(np.argmax(g.out_degree()))


def random_sources(g: Graph, k: int, seed: int, min_outdeg: int = 1) -> np.ndarray:
    """k distinct vertices with out-degree >= min_outdeg, drawn by the counter hash."""
    deg = g.out_degree()
    eligible = int(np.count_nonzero(deg >= min_outdeg))
    if eligible < k:
        raise ValueError(f"only {eligible} vertices have out-degree >= {min_outdeg}")
    out: list[int] = []
    seen: set[int] = set()
    i = 0
    while len(out) < k:
        v = hash64(seed, 7, i) % g.n
        i += 1
        if deg[v] >= min_outdeg and v not in seen:
            seen.add(v)
            out.append(int(v))
    return np.asarray(out, dtype=np.int32)


def random_costs(n: int, seed: int) -> np.ndarray:
    """Per-vertex loss coefficients c_v ~ U[0,1) in float32 (2**-24 lattice)."""
    return weights_unit(n, seed ^ 0xC05715)
