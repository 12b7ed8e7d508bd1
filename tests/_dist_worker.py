"""One rank of the world-size-2 gloo test (run as a subprocess by tests/test_dist.py).

Each rank builds the partial table of its shard of the evaluated half grid on the CPU from
the oracle's per-point log q (standing in for the device's partial table), the ranks sum
them with paper_2412_17742_gb300.dist.allreduce_table, and rank 0 saves the result; in the
"fock" mode the same over Fock-input node ranges, in the "grad" mode the partial gradients of
a linear loss summed with paper_2412_17742_gb300.dist.allreduce_grads.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2412_17742_gb300 import dist as gdist  # noqa: E402
from shard_tables import partial_table_cpu  # noqa: E402


def partial_loss_gradient(prob, pbar, begin, end, h=1e-6):
    """d/dr of sum_b pbar(b) P_[begin, end)(b) by central differences of the oracle."""
    g = np.zeros(prob.r.shape)
    for idx in np.ndindex(*prob.r.shape):
        vals = []
        for sgn in (1.0, -1.0):
            q = synth.Problem(prob.M, prob.K, prob.r.copy(), prob.T.copy(), prob.bin_of_mode, prob.cutoff)
            q.r[idx] += sgn * h
            vals.append(float((partial_table_cpu(q, oracle.binned(q)["logq"], begin, end) * pbar).sum()))
        g[idx] = (vals[0] - vals[1]) / (2 * h)
    return g


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    out = sys.argv[1]
    fock_mode = len(sys.argv) > 2 and sys.argv[2] == "fock"
    grad_mode = len(sys.argv) > 2 and sys.argv[2] == "grad"
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    if grad_mode:
        # gradients: each rank's partial gradient (central differences of the oracle's partial
        # table of its shard, standing in for a sharded plan's reverse pass), summed by
        # paper_2412_17742_gb300.dist.allreduce_grads
        prob = synth.config(0)
        n_eval = gdist.evaluated_points(prob.cutoff)
        begin, end = gdist.shard_range(n_eval, rank, world)
        pbar = np.random.default_rng(7).standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
        grads = {"r": partial_loss_gradient(prob, pbar, begin, end)}
        total = gdist.allreduce_grads(grads)
        if rank == 0:
            np.save(out, total["r"])
        dist.barrier()
        dist.destroy_process_group()
        return
    if fock_mode:
        # Fock inputs: the ranks split the input nodes (Gray-code order) and each contributes
        # the oracle's partial table of its range, standing in for a sharded Fock plan
        from oracle import fock
        fp = synth.random_fock_problem(np.random.default_rng(41), 5, [1, 2, 0, 1, 1], 2, 5)
        begin, end = gdist.shard_range(fock.node_count(fp.photons), rank, world)
        part = torch.from_numpy(fock.table(fp, node_range=(begin, end))["P"].copy())
    else:
        prob = synth.config(0)
        logq = oracle.binned(prob)["logq"]
        n_eval = gdist.evaluated_points(prob.cutoff)
        begin, end = gdist.shard_range(n_eval, rank, world)
        part = torch.from_numpy(partial_table_cpu(prob, logq, begin, end))
    total = gdist.allreduce_table(part)
    if rank == 0:
        np.save(out, total.numpy())
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
