"""The large-matrix tree of block eliminations with Hessenberg leaves (kernels 13 and 14)
against the CPU oracle: every table entry (1e-10 absolute) and every evaluated log q (1e-9,
imaginary part included, so the square-root branch is checked at every point).

Cases cover one and several sub-steps per level (a level's pivots split when its pivot rows
exceed the shared-memory budget), groups of uneven and shuffled rows, two to four groups,
a radix-1 axis, an even and a radix-2 last axis, a two-row last group, displaced and
undisplaced states, internal modes with non-aligned bases, and both arithmetics.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10
LOGQ_TOL = 1e-9


def _flat_index(digits, radix):
    strides = np.ones(len(radix), dtype=np.int64)
    for l in range(len(radix) - 2, -1, -1):
        strides[l] = strides[l + 1] * radix[l + 1]
    return digits @ strides


def _problem(seed, M, K, L, cutoff, **kw):
    return synth.random_problem(np.random.default_rng(seed), M, K, L, cutoff, **kw)


CASES = [
    # n = 96, three groups of 32 rows, one sub-step per level
    ("n96_l3_disp_basis", lambda: _problem(901, 12, 4, 3, [3, 4, 5], displaced=True, internal_basis=True)),
    # n = 300, three groups of 100 rows: level 0 in three sub-steps, level 1 in two
    ("n300_l3_substeps", lambda: _problem(902, 150, 1, 3, [2, 2, 3], displaced=True)),
    # n = 200, two groups of 100 rows, undisplaced, even last radix
    ("n200_l2_even", lambda: _problem(903, 100, 1, 2, [4, 5])),
    # uneven, shuffled groups over four axes, one of radix 1
    ("n144_l4_shuffled", lambda: _problem(904, 36, 2, 4, [2, 0, 3, 2], displaced=True, shuffle_bins=True,
                                          internal_basis=True)),
    # a two-row last group (a single port), radix-2 last axis
    ("n130_last_group_two_rows", lambda: synth.Problem(
        65, 1, np.random.default_rng(905).uniform(0.2, 0.9, (65, 1)),
        np.sqrt(0.8) * synth.haar_unitary(65, np.random.default_rng(906)),
        np.array([0] * 64 + [1], np.int32), np.array([3, 1], np.int32),
        alpha=0.3 * np.ones((65, 1), complex))),
    # n = 60, three groups of 20 rows: too large a last group for the small tree
    ("n60_l3_last_group_20_rows", lambda: _problem(909, 30, 1, 3, [4, 3, 5], displaced=True)),
    # the largest matrix the library takes: n = 512, five groups of ~102 rows (five levels)
    ("n512_l5_max", lambda: _problem(911, 256, 1, 5, [1, 1, 2, 1, 2], displaced=True, r_range=(0.1, 0.4))),
    # the largest last group the shared-memory Householder reduction takes: 116 rows (n = 232)
    ("n232_last_group_116_rows", lambda: synth.Problem(
        116, 1, np.random.default_rng(907).uniform(0.2, 0.7, (116, 1)),
        np.sqrt(0.7) * synth.haar_unitary(116, np.random.default_rng(908)),
        np.array([0] * 58 + [1] * 58, np.int32), np.array([2, 3], np.int32),
        alpha=0.2 * np.ones((116, 1), complex))),
    # last groups above 116 rows: the Householder reduction in the Hessenberg buffer through L2,
    # leaves with six register slots per lane; n = 282 with groups of 144 and 138 rows, and the
    # largest last group, 192 rows (n = 224)
    ("n282_last_group_138_rows", lambda: synth.Problem(
        141, 1, np.random.default_rng(912).uniform(0.2, 0.6, (141, 1)),
        np.sqrt(0.6) * synth.haar_unitary(141, np.random.default_rng(913)),
        np.array([0] * 72 + [1] * 69, np.int32), np.array([2, 3], np.int32),
        alpha=0.2 * np.ones((141, 1), complex))),
    ("n224_last_group_192_rows", lambda: synth.Problem(
        112, 1, np.random.default_rng(914).uniform(0.2, 0.6, (112, 1)),
        np.sqrt(0.6) * synth.haar_unitary(112, np.random.default_rng(915)),
        np.array([0] * 16 + [1] * 96, np.int32), np.array([3, 2], np.int32),
        alpha=0.2 * np.ones((112, 1), complex))),
]


@pytest.mark.parametrize("kernel", [13, 14], ids=["df32", "fp64"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_btree_matches_oracle(cuda_lib, name, make, kernel):
    gb = cuda_lib
    prob = make()
    with gb.Plan(prob, precision=1 if kernel == 13 else 0, tile_override=kernel) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert d["kernel"] == kernel
    assert st == 0 and d["n_bad_points"] == 0
    res = oracle.binned(prob)
    ref = res["P"]
    err = float(np.abs(P - ref).max())
    assert err <= TOL, (name, kernel, err)
    dig = gb.evaluated_point_digits(prob.cutoff)
    full = res["logq"][_flat_index(dig, prob.radix)]
    assert np.abs(lq - full).max() < LOGQ_TOL, (name, kernel, np.abs(lq - full).max())
    assert abs(d["log_q1_re"] - res["logq"][0].real) < 1e-10
    assert d["min_pivot_re"] > 0 and np.all(mp > 0)
    assert d["launches"] >= 4


def test_btree_is_default_for_large_grids(cuda_lib):
    # the n = 192 workload takes the large-matrix tree in both precisions by default, and
    # repeated executes are bit-identical (no atomics on the path)
    gb = cuda_lib
    prob = synth.config(2)
    for precision, kernel in ((1, "btree_df32"), (0, "btree_fp64")):
        with gb.Plan(prob, precision=precision) as p:
            a = p.table().cpu().numpy()
            b = p.table().cpu().numpy()
            st, d = p.diagnostics()
        assert d["kernel_name"] == kernel and st == 0
        assert np.array_equal(a, b)


def test_btree_set_state(cuda_lib):
    # a new state on an existing plan re-uploads the permuted augmented matrix
    gb = cuda_lib
    a = _problem(907, 40, 2, 2, [3, 4], displaced=True, internal_basis=True)
    b = _problem(907, 40, 2, 2, [3, 4], displaced=True, internal_basis=True)
    b.r = b.r * 0.8
    with gb.Plan(a, precision=1, tile_override=13) as p:
        gb.gbsbin_plan_set_state(p.handle, b)
        Pb = p.table().cpu().numpy()
    assert np.abs(Pb - oracle.binned(b)["P"]).max() <= TOL


def test_btree_refuses_what_it_cannot_do(cuda_lib):
    gb = cuda_lib
    one_group = _problem(908, 40, 1, 1, 5)
    with pytest.raises(gb.GbsbinError) as e:
        gb.Plan(one_group, tile_override=14)
    assert e.value.status == 8
    big_last = synth.Problem(                                # last group of 194 rows > 192
        100, 1, np.full((100, 1), 0.3), np.sqrt(0.7) * synth.haar_unitary(100, np.random.default_rng(909)),
        np.array([0] * 3 + [1] * 97, np.int32), np.array([2, 2], np.int32))
    with pytest.raises(gb.GbsbinError) as e:
        gb.Plan(big_last, tile_override=13)
    assert e.value.status == 8


@pytest.mark.parametrize("precision,small,large", [(1, "tree_df32", "btree_df32"), (0, "tree_fp64", "btree_fp64")],
                         ids=["fp32pairs", "fp64"])
def test_trees_run_the_forward_of_a_reverse_pass(cuda_lib, precision, small, large):
    # plans with a reverse pass keep the tree for their forward (the reverse pass needs only
    # log q): the gradient matches a per-point plan's (the same recomputed reverse pass), for the
    # small tree (undisplaced: its DFT takes G, log q finished for the reverse pass) and the
    # large-matrix tree
    import torch
    gb = cuda_lib
    cases = [(_problem(911, 8, 2, 2, [4, 5], displaced=False), small, 4),     # n = 32
             (_problem(912, 40, 2, 2, [3, 4]), large, 6)]                      # n = 160
    for prob, kind, per_point in cases:
        rng = np.random.default_rng(913)
        pbar = torch.from_numpy(rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))).cuda()
        grads = []
        for tile in (0, per_point if precision else 3):
            with gb.Plan(prob, precision=precision, want_backward=True, tile_override=tile) as p:
                p.table()
                st, d = p.diagnostics()
                assert st == 0 and (d["kernel_name"] == kind) == (tile == 0), d["kernel_name"]
                grads.append(p.backward(pbar, want=("r", "T", "sigma1")))
        for k in grads[0]:
            scale = max(1.0, float(np.abs(grads[1][k]).max()))
            assert np.abs(grads[0][k] - grads[1][k]).max() < 1e-10 * scale, (kind, k)


def test_default_choice_for_small_matrices_with_large_groups(cuda_lib):
    # n = 60 with 20-row groups: the small tree does not apply (last group above 16 rows), the
    # large-matrix tree is the default in both arithmetics
    gb = cuda_lib
    prob = _problem(910, 30, 1, 3, [4, 3, 5], displaced=True)
    for precision, name in ((1, "btree_df32"), (0, "btree_fp64")):
        with gb.Plan(prob, precision=precision) as p:
            P = p.table().cpu().numpy()
            st, d = p.diagnostics()
        assert st == 0 and d["kernel_name"] == name, d["kernel_name"]
        assert np.abs(P - oracle.binned(prob)["P"]).max() <= 1e-10


def test_default_choice_above_the_shared_memory_householder(cuda_lib):
    # n = 282 with groups of 144 and 138 rows on a 21 x 21 grid (the shape of the 256-problem
    # batch's largest per-point problem): the large-matrix tree is now the default in both
    # arithmetics; log q at sampled evaluated points against the oracle one by one, the table's
    # total and the two arithmetics' tables against each other
    gb = cuda_lib
    prob = synth.Problem(
        141, 1, np.random.default_rng(916).uniform(0.3, 0.9, (141, 1)),
        np.sqrt(0.6) * synth.haar_unitary(141, np.random.default_rng(917)),
        np.array([0] * 72 + [1] * 69, np.int32), np.array([20, 20], np.int32),
        alpha=0.2 * np.ones((141, 1), complex))
    XA, gamma, labels = oracle.plan(prob)
    dig = gb.evaluated_point_digits(prob.cutoff)
    pick = np.concatenate([[0, 1, len(dig) - 1], np.random.default_rng(918).choice(len(dig), 9, replace=False)])
    ref, _, _ = oracle.logq_points(XA, gamma, labels, prob.radix, dig[pick])
    tables = []
    for precision, name in ((1, "btree_df32"), (0, "btree_fp64")):
        with gb.Plan(prob, precision=precision) as p:
            tables.append(p.table().cpu().numpy())
            st, d = p.diagnostics()
            lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
        assert st == 0 and d["kernel_name"] == name, d["kernel_name"]
        assert d["n_bad_points"] == 0 and abs(tables[-1].sum() - 1.0) < 1e-10
        assert np.abs(lq[pick] - ref).max() < LOGQ_TOL
    assert np.abs(tables[0] - tables[1]).max() < 1e-10
