"""Source sharding across GPUs with one grid all-reduce (one process per GPU).

The history part of the evaluation (Sec. 3) is linear in the sources: the
grids spread from all the sources are the sum of the grids spread from any
partition of them.  So each rank binds a contiguous share of the volume
nodes, spreads them into a full-size grid (``lp_spread``), the ranks sum
their grids with one all-reduce (``lp_grid_buffers``), and every rank then
transforms, interpolates and adds the local part for its own share of the
targets (``lp_finish``).  The layer densities are bound on every rank (the
local part of each rank's targets needs them) but spread by rank 0 only, so
the sum counts the boundary nodes once.

The library calls and the all-reduce are arguments, so that the partition
and reduction logic can be exercised without a GPU.
"""
from __future__ import annotations

import numpy as np


def share(n, world, rank):
    """The contiguous share [lo, hi) of n items owned by rank (sizes differ
    by at most one, lower ranks first)."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def cuda_view(ptr, nbytes, dtype):
    """A torch tensor over device memory owned by the library (zero copy)."""
    import torch

    class _Buf:
        pass

    b = _Buf()
    item = 8 if dtype == "float64" else 4
    b.__cuda_array_interface__ = {"shape": (int(nbytes) // item,), "typestr": "<f8" if item == 8 else "<f4",
                                  "data": (int(ptr), False), "version": 3}
    return torch.as_tensor(b, device="cuda")


def torch_allreduce(t):
    import torch.distributed as dist
    dist.all_reduce(t)


class ShardedEvaluation:
    """One rank's part of a sharded V, S, D evaluation of `problem` (a dict
    as produced by workloads.configs) on an existing plan."""

    def __init__(self, lib, plan, problem, rank, world, allreduce=torch_allreduce, view=cuda_view,
                 to_device=None):
        self.lib, self.plan, self.p = lib, plan, problem
        self.rank, self.world = rank, world
        self.allreduce, self.view = allreduce, view
        self.dev = to_device or (lambda a: a)
        n = len(problem["src_w"])
        self.src = share(n, world, rank)
        self.tgt = share(len(problem["tgt_xy"]), world, rank)

    def bind(self):
        lo, hi = self.src
        p = self.p
        self.lib.lp_volume(self.plan, hi - lo, self.dev(p["src_xy"][lo:hi]), self.dev(p["src_w"][lo:hi]),
                           self.dev(p["src_f"][lo:hi]))
        self.outputs = "V"
        if p.get("sigma") is not None:
            self.lib.lp_single_layer(self.plan, self.dev(p["sigma"]))
            self.outputs += "S"
        if p.get("mu") is not None:
            self.lib.lp_double_layer(self.plan, self.dev(p["mu"]))
            self.outputs += "D"
        return self

    def spread(self):
        """This rank's sources onto full-size grids (the layers on rank 0)."""
        self.lib.lp_spread(self.plan, self.outputs, spread_layers=(self.rank == 0))

    def buffers(self):
        """Views of the buffers the ranks sum."""
        return [self.view(ptr, nbytes, dtype) for ptr, nbytes, dtype in self.lib.lp_grid_buffers(self.plan)]

    def reduce(self):
        for t in self.buffers():
            self.allreduce(t)

    def finish(self, out):
        """This rank's targets from the summed grids into out[k] (arrays over
        the rank's share of the targets, k in the bound outputs)."""
        lo, hi = self.tgt
        p = self.p
        self.lib.lp_finish(self.plan, hi - lo, self.dev(np.ascontiguousarray(p["tgt_xy"][lo:hi])),
                           self.dev(np.ascontiguousarray(p["tgt_jet"][lo:hi])),
                           *[out.get(k) for k in "VSD"])
        return out

    def evaluate(self, out):
        self.spread()
        self.reduce()
        return self.finish(out)
