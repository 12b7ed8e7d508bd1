"""Batched evaluation of many uneven problems in one persistent launch per kernel class."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def mixed_problems():
    rng = np.random.default_rng(701)
    specs = [  # (M, K, L, cutoff, displaced, internal basis)
        (4, 1, 2, [5, 4], False, False),       # n = 8   warp class (FP32R)
        (8, 1, 1, [40], True, False),          # n = 16
        (6, 2, 3, [3, 4, 2], True, True),      # n = 24
        (16, 1, 4, [2, 3, 2, 3], False, False),  # n = 32
        (12, 2, 2, [6, 5], True, True),        # n = 48  CTA, shared memory
        (32, 1, 2, [4, 4], False, False),      # n = 64
        (16, 3, 3, [2, 2, 3], True, True),     # n = 96
        (60, 1, 2, [3, 2], True, False),       # n = 120 CTA, L2 workspace (FP64) or blocked (FP32R)
        (40, 2, 1, [12], False, True),         # n = 160
    ]
    return [synth.random_problem(rng, M, K, L, cut, displaced=d, internal_basis=v) for M, K, L, cut, d, v in specs]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_tables_match_oracle(cuda_lib, precision):
    gb = cuda_lib
    probs = mixed_problems()
    with gb.Batch(probs, precision=precision) as b:
        outs = b.execute()
        kinds = set()
        for i, p in enumerate(probs):
            st, d = b.diagnostics(i)
            kinds.add(d["kernel_name"])
            assert st == 0 and d["n_bad_points"] == 0
            ref = oracle.binned(p)["P"]
            err = np.abs(outs[i].cpu().numpy() - ref).max()
            assert err <= 1e-10, (i, p.n, precision, err)
    if precision == 0:
        assert any(k.startswith("gmem") for k in kinds) and any(k.startswith("smem") for k in kinds)
    else:
        # warp kernel (n <= 32), shared memory (n <= 112), blocked on the L2 workspace above
        assert {"warp_fp32r", "smem_fp32r", "blk_fp32r"} <= kinds


def test_batch_autotune_and_graph_replay(cuda_lib):
    import torch
    gb = cuda_lib
    probs = mixed_problems()
    k, ppc, us = gb.gbsbin_autotune(32, 1)
    assert k in (2, 4, 5, 6, 7) and ppc >= 1 and us > 0
    with gb.Batch(probs, precision=1, autotune=True) as b:
        ref = [t.clone() for t in b.execute()]
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        for t in b.outputs:
            t.zero_()
        torch.cuda.synchronize()
        b.capture(s)
        b.replay(s)
        s.synchronize()
        for t, r in zip(b.outputs, ref):
            assert torch.equal(t, r)
        for i, p in enumerate(probs):
            assert np.abs(ref[i].cpu().numpy() - oracle.binned(p)["P"]).max() <= 1e-10


def test_full_batched_workload_sampled(cuda_lib):
    # 256 problems, M ~ U{8..48}, K ~ U{1..3}, L ~ U{1..4}, grids of 500-20000 points:
    # every table sums to 1, no bad pivots; sampled points of eight problems against the
    # oracle one by one
    gb = cuda_lib
    probs = synth.batch_config()
    with gb.Batch(probs, precision=1) as b:
        outs = b.execute()
        for i in range(len(probs)):
            st, d = b.diagnostics(i)
            assert st == 0 and d["n_bad_points"] == 0
            assert abs(d["sum_P"] - 1.0) < 1e-10
        rng = np.random.default_rng(702)
        for i in rng.choice(len(probs), 8, replace=False):
            p = probs[i]
            st, d = b.diagnostics(i)
            lq, _ = b.read_points(i, d["n_evaluated"])
            dig = gb.evaluated_point_digits(p.cutoff)
            pick = np.concatenate([[0], rng.choice(len(dig), 5, replace=False)])
            XA, gamma, labels = oracle.plan(p)
            ref, _, _ = oracle.logq_points(XA, gamma, labels, p.radix, dig[pick])
            assert np.abs(lq[pick] - ref).max() < 1e-9, (i, p.n)
        assert all(float(o.sum()) == pytest.approx(1.0, abs=1e-10) for o in outs)


def test_batch_problems_on_trees(cuda_lib):
    # problems large enough to run apart from the per-point queue take a tree of their own
    # (the small tree for n <= 64, the large-matrix tree above), beside per-point problems;
    # every table against the oracle, and the same tables from a captured graph
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(703)
    probs = [synth.random_problem(rng, 16, 2, 4, [4, 4, 4, 4], displaced=True),            # n = 64, small tree
             synth.random_problem(rng, 16, 3, 3, [6, 6, 6], displaced=True, internal_basis=True),   # n = 96, large
             synth.random_problem(rng, 4, 1, 2, [5, 4]),                                    # n = 8, queue
             synth.random_problem(rng, 60, 1, 2, [3, 2], displaced=True)]                   # n = 120, queue
    for precision, small, large in ((1, "tree_df32", "btree_df32"), (0, "tree_fp64", "btree_fp64")):
        with gb.Batch(probs, precision=precision) as b:
            ref = [t.clone() for t in b.execute()]
            kinds = [b.diagnostics(i)[1]["kernel_name"] for i in range(len(probs))]
            assert kinds[0] == small and kinds[1] == large, kinds
            assert "tree" not in kinds[2] and "tree" not in kinds[3], kinds
            for i, p in enumerate(probs):
                st, d = b.diagnostics(i)
                assert st == 0 and d["n_bad_points"] == 0
                assert np.abs(ref[i].cpu().numpy() - oracle.binned(p)["P"]).max() <= 1e-10, (i, precision)
            torch.cuda.synchronize()
            s = torch.cuda.Stream()
            for t in b.outputs:
                t.zero_()
            torch.cuda.synchronize()
            b.capture(s)
            b.replay(s)
            s.synchronize()
            for t, r in zip(b.outputs, ref):
                assert torch.equal(t, r)


def test_full_batched_workload_whole_tables(cuda_lib):
    # the 256-problem workload in both arithmetics: whole tables against the oracle element by
    # element (1e-10) for the 48 problems cheapest for the oracle and, in every kernel class the
    # batch uses, that class's cheapest problem (the trees, the one-group Hessenberg kernels and
    # the per-point kernels); log q at sampled points of 24 further problems one by one
    gb = cuda_lib
    probs = synth.batch_config()
    cost = sorted((p.n_points * (2 * p.M * p.K) ** 3, i) for i, p in enumerate(probs))
    for precision in (1, 0):
        with gb.Batch(probs, precision=precision) as b:
            outs = [t.cpu().numpy() for t in b.execute()]
            kinds = [b.diagnostics(i)[1]["kernel_name"] for i in range(len(probs))]
            pick = {i for _, i in cost[:48]}
            for kind in set(kinds):
                pick.add(min((c, i) for c, i in cost if kinds[i] == kind)[1])
            for i in sorted(pick):
                err = float(np.abs(outs[i] - oracle.binned(probs[i])["P"]).max())
                assert err <= 1e-10, (i, kinds[i], precision, err)
            rng = np.random.default_rng(704 + precision)
            rest = [i for i in range(len(probs)) if i not in pick]
            for i in rng.choice(rest, 24, replace=False):
                p = probs[i]
                st, d = b.diagnostics(i)
                lq, _ = b.read_points(i, d["n_evaluated"])
                dig = gb.evaluated_point_digits(p.cutoff)
                sel = np.concatenate([[0, len(dig) - 1], rng.choice(len(dig), 4, replace=False)])
                XA, gamma, labels = oracle.plan(p)
                ref, _, _ = oracle.logq_points(XA, gamma, labels, p.radix, dig[sel])
                assert np.abs(lq[sel] - ref).max() < 1e-9, (i, kinds[i], precision)
        assert len(set(kinds)) >= 4, set(kinds)
