"""One table's grid split into shards (the multi-GPU decomposition), evaluated shard by
shard on one GPU: every shard's partial table against its CPU definition, and their sum
against the oracle's table, for each kernel family."""
import numpy as np
import pytest

import oracle
import synth
from paper_2412_17742_gb300 import dist as gdist
from shard_tables import partial_table_cpu

pytestmark = pytest.mark.gpu

CASES = [  # (name, problem, precision, tile override)
    ("warp_fp32r_n32", lambda: synth.config(1), 1, 0),
    ("smem_fp64_n32", lambda: synth.config(1), 0, 0),
    ("smem_fp32r_n50", lambda: synth.random_problem(np.random.default_rng(401), 25, 1, 2, [3, 4], displaced=True),
     1, 0),
    ("blk_fp32r_n120", lambda: synth.random_problem(np.random.default_rng(402), 60, 1, 2, [3, 2], displaced=True),
     1, 0),
    ("gmem_fp64_n120", lambda: synth.random_problem(np.random.default_rng(402), 60, 1, 2, [3, 2], displaced=True),
     0, 0),
    # the large-matrix tree: each shard runs the first-axis subtrees covering its slice
    ("btree_df32_n96_l3", lambda: synth.random_problem(np.random.default_rng(403), 12, 4, 3, [3, 4, 5], displaced=True,
                                                       internal_basis=True), 1, 13),
    ("btree_fp64_n96_l3", lambda: synth.random_problem(np.random.default_rng(403), 12, 4, 3, [3, 4, 5], displaced=True,
                                                       internal_basis=True), 0, 14),
    ("btree_df32_n130_l2", lambda: synth.random_problem(np.random.default_rng(404), 65, 1, 2, [4, 6]), 1, 13),
]


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name,make,precision,tile", CASES, ids=[c[0] for c in CASES])
def test_shard_tables_sum_to_the_table(cuda_lib, name, make, precision, tile, world):
    gb = cuda_lib
    prob = make()
    res = oracle.binned(prob)
    n_eval = gdist.evaluated_points(prob.cutoff)
    total = np.zeros(res["P"].shape)
    for r in range(world):
        b, e = gdist.shard_range(n_eval, r, world)
        with gb.Plan(prob, precision=precision, tile_override=tile, shard=(b, e)) as p:
            part = p.table().cpu().numpy()
            st, d = p.diagnostics()
        assert st == 0 and d["n_evaluated"] == (e - b) + (1 if b > 0 else 0)
        assert np.abs(part - partial_table_cpu(prob, res["logq"], b, e)).max() < 1e-10
        total += part
    assert np.abs(total - res["P"]).max() < 1e-10


def test_single_point_shards_and_errors(cuda_lib):
    gb = cuda_lib
    prob = synth.config(0)
    res = oracle.binned(prob)
    n_eval = gdist.evaluated_points(prob.cutoff)
    for b, e in ((0, 1), (n_eval - 1, n_eval), (7, 8)):
        with gb.Plan(prob, precision=1, shard=(b, e)) as p:
            part = p.table().cpu().numpy()
        assert np.abs(part - partial_table_cpu(prob, res["logq"], b, e)).max() < 1e-12
    for bad in ((3, 3), (5, 2), (-1, 4), (0, n_eval + 1)):
        with pytest.raises(gb.GbsbinError):
            gb.Plan(prob, shard=bad)


@pytest.mark.parametrize("world", [2, 3])
def test_shard_gradients_sum_to_the_gradient(cuda_lib, world):
    # the reverse pass of each shard's plan is the gradient of its partial table; summed over
    # a partition they give the whole plan's gradient (the sum an all-reduce forms)
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(405)
    prob = synth.random_problem(rng, 4, 2, 2, [4, 5], displaced=True, internal_basis=True)
    pbar = torch.from_numpy(rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))).cuda()
    want = ("r", "T", "alpha", "V")
    with gb.Plan(prob, want_backward=True) as p:
        p.table()
        whole = p.backward(pbar, want=want)
    n_eval = gdist.evaluated_points(prob.cutoff)
    total = {k: np.zeros_like(v) for k, v in whole.items()}
    for r in range(world):
        b, e = gdist.shard_range(n_eval, r, world)
        with gb.Plan(prob, want_backward=True, shard=(b, e)) as p:
            p.table()
            g = p.backward(pbar, want=want)
        for k in total:
            total[k] = total[k] + g[k]
    for k in whole:
        scale = max(1.0, float(np.abs(whole[k]).max()))
        assert np.abs(total[k] - whole[k]).max() < 1e-11 * scale, k
