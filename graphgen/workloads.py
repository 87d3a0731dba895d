"""Named synthetic workloads shaped like the paper's inputs.

The paper runs on symmetric unit-weight SNAP / GraphChallenge graphs with
Delta = 1 (Section VI-A). Those files are not available, so these seeded
synthetic graphs stand in for them:

* ``rmat14_int``   R-MAT scale 14, edge factor 16, int32 weights U{1..255},
                   Delta = 32, source = highest out-degree vertex.
* ``rmat22_unit``  R-MAT scale 22, edge factor 16, fp32 weights U[0,1),
                   64 sources with out-degree >= 1, Delta in {0.01, 0.05, 0.1, 0.5}.
* ``grid4096``     4096 x 4096 grid, 4-neighbour arcs, 5 % of arcs dropped,
                   int32 weights U{1..1000}, corner source, Delta in {100, 1000, 10000}.
* ``rmat20_unit``  R-MAT scale 20, fp32 U[0,1), 256 sources (batched solve).
* ``er_family``    512 directed Erdos-Renyi graphs, n log-uniform in [1e3, 2e5],
                   8 n draws, fp32 U[0,1), one source each.
* ``rmat20_lognormal``  R-MAT scale 20, fp32 lognormal(0, 1), 32 sources,
                   per-vertex loss weights c_v ~ U[0,1).

Every builder takes a ``scale`` override so tests can build the same recipe
at a size the CPU oracle finishes in seconds.
"""
from __future__ import annotations

import math

import numpy as np

from . import (Graph, erdos_renyi, grid, hash64, highest_outdegree_vertex, random_costs,
               random_sources, rmat, weights_int, weights_lognormal, weights_unit)


def rmat14_int(scale: int = 14, seed: int = 1) -> tuple[Graph, list[int], list[float]]:
    g = rmat(scale, 16, seed=seed)
    g.w = weights_int(g.m, 1, 255, seed)
    g.name = f"rmat{scale}_int"
    return g, [highest_outdegree_vertex(g)], [32.0]


def rmat22_unit(scale: int = 22, n_sources: int = 64, seed: int = 2):
    g = rmat(scale, 16, seed=seed)
    g.w = weights_unit(g.m, seed)
    g.name = f"rmat{scale}_unit"
    return g, [int(s) for s in random_sources(g, n_sources, seed)], [0.01, 0.05, 0.1, 0.5]


def grid4096(side: int = 4096, seed: int = 3):
    g = grid(side, side, 0.05, seed)
    g.w = weights_int(g.m, 1, 1000, seed)
    g.name = f"grid{side}_int"
    return g, [0], [100.0, 1000.0, 10000.0]


def rmat20_unit(scale: int = 20, n_sources: int = 256, seed: int = 4):
    g = rmat(scale, 16, seed=seed)
    g.w = weights_unit(g.m, seed)
    g.name = f"rmat{scale}_unit"
    return g, [int(s) for s in random_sources(g, n_sources, seed)]


def er_family(count: int = 512, n_lo: float = 1e3, n_hi: float = 2e5, seed: int = 5):
    """count ER graphs; n = round(exp(U[ln n_lo, ln n_hi])), 8 n draws, one source each."""
    out = []
    for k in range(count):
        u = (hash64(seed, 11, k) >> 11) * (1.0 / 9007199254740992.0)
        n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        g = erdos_renyi(n, 8 * n, seed=seed * 1000003 + k)
        g.w = weights_unit(g.m, seed * 1000003 + k)
        g.name = f"er{n}"
        src = int(random_sources(g, 1, seed * 1000003 + k)[0])
        out.append((g, src))
    return out


def rmat20_lognormal(scale: int = 20, n_sources: int = 32, seed: int = 6):
    g = rmat(scale, 16, seed=seed)
    g.w = weights_lognormal(g.m, 0.0, 1.0, seed)
    g.name = f"rmat{scale}_lognormal"
    srcs = [int(s) for s in random_sources(g, n_sources, seed)]
    return g, srcs, random_costs(g.n, seed)
