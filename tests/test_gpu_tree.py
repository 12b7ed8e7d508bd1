"""The tree of block eliminations (kernel 11 in pairs of FP32, kernel 12 in FP64) against
the per-point FP64 kernel and the oracle: every evaluated log q and the table, on problems
with uneven and shuffled groups, displacement, internal modes, axes of radix 1 and 2 to 6
groups.  The pairs carry about 46 bits: log q within 1e-11, tables within 1e-12 of the
FP64 kernel; the FP64 tree differs from it by rounding order only (1e-12, 1e-13)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# (precision, kernel name, log q bound, table bound against the per-point FP64 kernel)
ARITH = [(1, "tree_df32", 1e-11, 1e-12), (0, "tree_fp64", 1e-12, 1e-13)]
ARITH_IDS = ["df32", "fp64"]


def _run(gb, prob, precision, tile_override=0):
    with gb.Plan(prob, precision=precision, tile_override=tile_override) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    return P, st, d, lq, mp


CASES = [
    ("m16_l4_n8", lambda: synth.config(1)),
    ("l2_disp", lambda: synth.random_problem(np.random.default_rng(201), 10, 1, 2, [6, 5], displaced=True)),
    ("l3_shuffled_disp_k2", lambda: synth.random_problem(np.random.default_rng(202), 6, 2, 3, [3, 4, 2],
                                                         displaced=True, internal_basis=True, shuffle_bins=True)),
    ("l6_radix1_axis", lambda: synth.random_problem(np.random.default_rng(203), 12, 1, 6, [2, 0, 1, 3, 1, 2],
                                                    displaced=True)),
    ("l4_k2_n64", lambda: synth.random_problem(np.random.default_rng(204), 16, 2, 4, [3, 2, 2, 4])),
    ("l2_uneven", lambda: synth.random_problem(np.random.default_rng(205), 9, 1, 2, [7, 9], shuffle_bins=True)),
]


@pytest.mark.parametrize("precision,kname,lq_tol,p_tol", ARITH, ids=ARITH_IDS)
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_tree_matches_per_point_and_oracle(cuda_lib, name, make, precision, kname, lq_tol, p_tol):
    prob = make()
    Pt, st, d, lq, mp = _run(cuda_lib, prob, precision)
    assert st == 0 and d["kernel_name"] == kname and d["n_bad_points"] == 0
    Pg, stg, dg, lqg, mpg = _run(cuda_lib, prob, 0, tile_override=3)       # per-point FP64 (workspace)
    assert stg == 0 and dg["kernel_name"] == "gmem_fp64"
    assert np.abs(lq - lqg).max() < lq_tol                                  # same log q, same branch
    assert np.abs(Pt - Pg).max() < p_tol
    assert d["min_pivot_re"] > 0
    res = oracle.binned(prob)
    sl = tuple(slice(0, int(c) + 1) for c in prob.cutoff)
    assert np.abs(Pt - res["P"][sl]).max() < 1e-10
    assert abs(d["log_q1_re"] - res["logq"][0].real) < 1e-10


@pytest.mark.parametrize("precision,kname,lq_tol,p_tol", ARITH, ids=ARITH_IDS)
def test_tree_state_change(cuda_lib, precision, kname, lq_tol, p_tol):
    a = synth.random_problem(np.random.default_rng(211), 8, 1, 3, [3, 2, 4], displaced=True)
    b = synth.random_problem(np.random.default_rng(212), 8, 1, 3, [3, 2, 4], displaced=True)
    with cuda_lib.Plan(a, precision=precision) as p:
        p.table()
        cuda_lib.gbsbin_plan_set_state(p.handle, b)
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
    assert st == 0 and d["kernel_name"] == kname
    sl = tuple(slice(0, int(c) + 1) for c in b.cutoff)
    assert np.abs(P - oracle.binned(b)["P"][sl]).max() < 1e-10


HARD = [
    # strong squeezing: |log det| large, the power-of-two exponents of P and P(1) differ by
    # odd and even amounts across the grid, windings of several turns
    ("strong_squeezing", lambda: synth.random_problem(np.random.default_rng(221), 8, 1, 4, [3, 3, 3, 4],
                                                      r_range=(1.2, 1.7), eta_range=(0.85, 0.99)), 1),
    ("oversampled", lambda: synth.random_problem(np.random.default_rng(222), 6, 1, 3, [2, 3, 2]), 3),
    ("last_group_16_rows", lambda: synth.random_problem(np.random.default_rng(223), 12, 2, 3, [3, 2, 4],
                                                        displaced=True, internal_basis=True), 1),
]


@pytest.mark.parametrize("precision,kname,lq_tol,p_tol", ARITH, ids=ARITH_IDS)
@pytest.mark.parametrize("name,make,oversample", HARD, ids=[c[0] for c in HARD])
def test_tree_hard_cases(cuda_lib, name, make, oversample, precision, kname, lq_tol, p_tol):
    prob = make()
    with cuda_lib.Plan(prob, precision=precision, oversample=oversample) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, _ = cuda_lib.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0 and d["kernel_name"] == kname
    radix = prob.radix * oversample
    res = oracle.binned(prob, radix=radix)
    sl = tuple(slice(0, int(c) + 1) for c in prob.cutoff)
    assert np.abs(P - res["P"][sl]).max() < 1e-10
    dig = cuda_lib.evaluated_point_digits(prob.cutoff, oversample)
    strides = np.ones(len(radix), dtype=np.int64)
    for l in range(len(radix) - 2, -1, -1):
        strides[l] = strides[l + 1] * radix[l + 1]
    assert np.abs(lq - res["logq"][dig @ strides]).max() < 1e-9
