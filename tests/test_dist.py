"""The N > 1 path on the CPU: shard arithmetic and the all-reduce of partial tables between
two real gloo ranks (subprocesses), checked against the oracle's whole table."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from paper_2412_17742_gb300 import dist as gdist
from shard_tables import partial_table_cpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("n", [0, 1, 5, 49, 3645])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_partition_the_units(n, world):
    blocks = [gdist.shard_range(n, r, world) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    for (b0, e0), (b1, e1) in zip(blocks, blocks[1:]):
        assert e0 == b1                                    # contiguous, no overlap, no gap
    sizes = [e - b for b, e in blocks]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        gdist.shard_range(n, world, world)


def test_evaluated_points_matches_the_half_grid():
    import paper_2412_17742_gb300 as gb
    for cut in ([6, 6], [8, 8, 8, 8], [3, 4, 2], [9], [0, 7]):
        assert gdist.evaluated_points(cut) == len(gb.evaluated_point_digits(np.array(cut)))


@pytest.mark.parametrize("world", [2, 3])
def test_partial_tables_sum_to_the_table(world):
    # the definition of a shard's partial table, summed over a partition, is the oracle's table
    prob = synth.config(0)
    res = oracle.binned(prob)
    n_eval = gdist.evaluated_points(prob.cutoff)
    total = sum(partial_table_cpu(prob, res["logq"], *gdist.shard_range(n_eval, r, world)) for r in range(world))
    assert np.abs(total - res["P"]).max() < 1e-13


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_world_size_2_allreduce(tmp_path):
    out = str(tmp_path / "table.npy")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "_dist_worker.py"), out],
                              env=dict(env, RANK=str(r)), stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
             for r in range(2)]
    logs = []
    for p in procs:
        try:
            logs.append(p.communicate(timeout=240)[0].decode(errors="replace"))
        except subprocess.TimeoutExpired:
            p.kill()
            raise
    assert all(p.returncode == 0 for p in procs), logs
    ref = oracle.binned(synth.config(0))["P"]
    assert np.abs(np.load(out) - ref).max() < 1e-13


def test_gloo_world_size_2_fock_node_shards(tmp_path):
    out = str(tmp_path / "fock_table.npy")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "_dist_worker.py"), out, "fock"],
                              env=dict(env, RANK=str(r)), stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
             for r in range(2)]
    logs = []
    for p in procs:
        try:
            logs.append(p.communicate(timeout=240)[0].decode(errors="replace"))
        except subprocess.TimeoutExpired:
            p.kill()
            raise
    assert all(p.returncode == 0 for p in procs), logs
    from oracle import fock
    fp = synth.random_fock_problem(np.random.default_rng(41), 5, [1, 2, 0, 1, 1], 2, 5)
    assert np.abs(np.load(out) - fock.table(fp)["P"]).max() < 1e-14


def test_gloo_world_size_2_partial_gradients(tmp_path):
    # each rank's gradient of its partial table (a sharded plan's reverse pass) summed by one
    # all-reduce per array equals the gradient of the whole table
    out = str(tmp_path / "grad.npy")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "_dist_worker.py"), out, "grad"],
                              env=dict(env, RANK=str(r)), stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
             for r in range(2)]
    logs = []
    for p in procs:
        try:
            logs.append(p.communicate(timeout=240)[0].decode(errors="replace"))
        except subprocess.TimeoutExpired:
            p.kill()
            raise
    assert all(p.returncode == 0 for p in procs), logs
    from _dist_worker import partial_loss_gradient
    prob = synth.config(0)
    pbar = np.random.default_rng(7).standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    whole = partial_loss_gradient(prob, pbar, 0, gdist.evaluated_points(prob.cutoff))
    assert np.abs(np.load(out) - whole).max() < 1e-8
