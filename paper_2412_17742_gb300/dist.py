"""Several GPUs (one process per GPU, torch.distributed) on the binned distribution.

Two ways to share the work, both without a collective on the point path:

* independent tables or problems: ``shard_range(n_units, rank, world)`` deals each rank a
  contiguous block of units (tables of a parameter sweep, problems of a batch); nothing is
  exchanged;
* one table: the grid points are independent (each is one determinant, Sec. III Eq. q_d),
  and the inverse DFT that turns the grid into P(b) is linear, so rank r evaluates the slice
  ``shard_range(n_evaluated, r, world)`` of the evaluated half grid into a partial table and
  one all-reduce (sum) of prod(N_l + 1) doubles gives the whole table
  (``sharded_table``).

Slices of the half grid keep every conjugate pair G(w^-k) = conj G(w^k) on one rank: the
half grid holds one representative of each pair.  Where the large-matrix tree of block
eliminations serves the plan, a shard runs the subtrees of the first axis's roots that cover
its slice.

Gradients (``ShardedPlan.backward``): each rank's plan gives the gradient of its partial
table; the partial tables sum to the table, so the gradients sum to the gradient - one
all-reduce of each requested gradient array (the chain from the n x n adjoint to the
physical parameters is linear and the same on every rank).
"""
from __future__ import annotations

import numpy as np


def shard_range(n_units: int, rank: int, world: int):
    """Contiguous block [begin, end) of units for ``rank`` of ``world``; the blocks of all
    ranks partition [0, n_units) and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need 0 <= rank < world and n_units >= 0")
    return rank * n_units // world, (rank + 1) * n_units // world


def evaluated_points(cutoff, oversample: int = 1) -> int:
    """Points of the half grid a whole-table plan evaluates: prod over the axes but the last
    of R_l, times floor(R_last / 2) + 1, with R_l = oversample (N_l + 1)."""
    radix = [oversample * (int(c) + 1) for c in cutoff]
    return int(np.prod(radix[:-1], dtype=np.int64)) * (radix[-1] // 2 + 1)


def allreduce_table(table, group=None):
    """Sum the ranks' partial tables in place (one all-reduce of prod(N_l + 1) doubles)."""
    import torch.distributed as dist
    dist.all_reduce(table, op=dist.ReduceOp.SUM, group=group)
    return table


def sharded_table(prob, precision: int = 0, oversample: int = 1, group=None, stream=None):
    """The whole table P(b) of ``prob``, its grid shared by the ranks of ``group``: this rank
    evaluates its slice on its current CUDA device, then the partial tables are summed."""
    import torch.distributed as dist

    from . import Plan
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    begin, end = shard_range(evaluated_points(prob.cutoff, oversample), rank, world)
    if end <= begin:                       # more ranks than points: contribute zeros
        import torch
        table = torch.zeros(tuple(int(c) + 1 for c in prob.cutoff), dtype=torch.float64, device="cuda")
    else:
        with Plan(prob, precision=precision, oversample=oversample, shard=(begin, end)) as p:
            table = p.table(stream)
    return allreduce_table(table, group)


def allreduce_grads(grads, group=None):
    """Sum the ranks' partial gradients (a dict of numpy arrays, as Plan.backward returns) in
    place: one all-reduce per array (complex arrays as their real and imaginary parts)."""
    import torch
    import torch.distributed as dist
    for key in sorted(grads):
        a = np.ascontiguousarray(grads[key])
        t = torch.from_numpy(a.view(np.float64) if np.iscomplexobj(a) else a.astype(np.float64)).clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        v = t.numpy()
        grads[key] = v.view(np.complex128).reshape(a.shape) if np.iscomplexobj(a) else v.reshape(a.shape)
    return grads


class ShardedPlan:
    """One problem's grid shared by the ranks of ``group``: this rank's plan evaluates its
    slice of the evaluated half grid on its current CUDA device.  ``table()`` returns the whole
    table (partial tables all-reduced); ``backward(dL_dP, want)`` the whole gradient (partial
    gradients all-reduced) for the state of the last ``table()``."""

    def __init__(self, prob, precision: int = 0, oversample: int = 1, want_backward: bool = False, group=None):
        import torch.distributed as dist

        from . import Plan
        self.group = group
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        self.shape = tuple(int(c) + 1 for c in prob.cutoff)
        self.begin, self.end = shard_range(evaluated_points(prob.cutoff, oversample), rank, world)
        self.plan = None
        if self.end > self.begin:
            self.plan = Plan(prob, precision=precision, oversample=oversample, want_backward=want_backward,
                             shard=(self.begin, self.end))

    def table(self, stream=None):
        import torch
        if self.plan is None:              # more ranks than points: contribute zeros
            t = torch.zeros(self.shape, dtype=torch.float64, device="cuda")
        else:
            t = self.plan.table(stream)
        return allreduce_table(t, self.group)

    def backward(self, dL_dP, want=("r", "T", "alpha", "V"), stream=None):
        if self.plan is None:
            raise RuntimeError("a rank without points has no gradient to contribute")
        return allreduce_grads(self.plan.backward(dL_dP, stream, want), self.group)

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fock_node_count(photons) -> int:
    """Input nodes of a Fock-input problem: prod over the occupied inputs but the one with the
    fewest photons (lowest port on ties) of (p_k + 1)."""
    p = np.asarray(photons)
    occ = [j for j in range(len(p)) if p[j] > 0]
    if not occ:
        return 1
    held = min(occ, key=lambda j: (p[j], j))
    return int(np.prod([int(p[j]) + 1 for j in occ if j != held], dtype=np.int64))


def fock_sharded_table(prob, precision: int = 0, oversample: int = 1, group=None, stream=None):
    """The whole Fock-input table, its input nodes shared by the ranks of ``group``: this rank
    walks its node range on its current CUDA device, then the partial tables are summed."""
    import torch
    import torch.distributed as dist

    from . import FockPlan
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    begin, end = shard_range(fock_node_count(prob.photons), rank, world)
    if end <= begin:                       # more ranks than nodes: contribute zeros
        table = torch.zeros(tuple(int(c) + 1 for c in prob.cutoff), dtype=torch.float64, device="cuda")
    else:
        with FockPlan(prob, precision=precision, oversample=oversample, shard=(begin, end)) as p:
            table = p.table(stream)
    return allreduce_table(table, group)
