"""The multi-GPU path of bench.py (weak scaling: independent sources per rank, no
collective on the data path, max-over-ranks timing), run as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import graphgen.workloads as W
    g, _, _ = W.rmat22_unit(scale=10, n_sources=4)
    srcs = bench.sources_for_rank(g, 8, rank)
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slower one
    out[rank] = (srcs, t, bench.job_gteps(g.m, 8, world, t))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, t0, v0), (s1, t1, v1) = res[0], res[1]
    assert t0 == t1 == 2.0                          # both see the slowest rank's time
    assert v0 == v1                                 # same whole-job value on every rank
    assert len(s0) == len(s1) == 8 and s0 != s1     # each rank has its own sources
    import bench
    assert bench.max_over_ranks(3.5) == 3.5         # no process group: identity
