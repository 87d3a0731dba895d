"""torch.autograd binding of the batched solve and its adjoint.

``shortest_path_distances(w, row_ptr, col, sources, delta)`` returns the (K, n)
distances from K sources on the directed CSR graph with float32 weights ``w``;
its backward gives dL/dw through the library's adjoint (``dsssp_backward``):
for every source, the upstream gradient of each reached vertex is summed over
that vertex's subtree of the shortest-path tree and lands on the subtree's root
arc. Entries of unreached vertices (distance +inf) receive no gradient. Both
directions run in the CUDA library; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import dsssp as _ds


class _ShortestPathDistances(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, row_ptr, col, sources, delta):
        if w.dtype != torch.float32 or not w.is_cuda:
            raise TypeError("w must be a CUDA float32 tensor")
        g = _ds.Graph(row_ptr, col, w.detach())
        srcs = [int(s) for s in sources]
        dist = torch.empty((len(srcs), g.n), dtype=torch.float32, device=w.device)
        pred = torch.empty((len(srcs), g.n), dtype=torch.int32, device=w.device)
        b = _ds.Batch(g, [float(delta)], srcs, dist=[dist[k] for k in range(len(srcs))],
                      pred=[pred[k] for k in range(len(srcs))], tape=True)
        b.run()
        b.sync()
        ctx.batch, ctx.graph, ctx.m = b, g, w.numel()
        ctx.mark_non_differentiable(pred)
        return dist, pred

    @staticmethod
    def backward(ctx, grad_dist, grad_pred):
        b, g = ctx.batch, ctx.graph
        grad_w = torch.empty(ctx.m, dtype=torch.float32, device=grad_dist.device)
        c = grad_dist.to(torch.float32).contiguous()
        b.backward([c[k] for k in range(c.shape[0])], [grad_w])
        b.sync()
        b.close()
        g.close()
        return grad_w, None, None, None, None


def shortest_path_distances(w, row_ptr, col, sources, delta):
    """Distances (K, n) and predecessors (K, n) from each source; differentiable in w."""
    return _ShortestPathDistances.apply(w, row_ptr, col, sources, delta)
