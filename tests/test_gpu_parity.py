"""Parity of the CUDA path (through the C ABI) with the CPU oracle, on the GPU.

Bars:
* FP64 path: |P_gpu - P_oracle| <= 1e-10 absolute, element by element.
* FP32 + refinement path: the same 1e-10 bound.  One refinement step leaves an error of
  O(|K^^{-1} E|^2) in log det with |K^^{-1} E| ~ n eps32 ||K^{-1}||, measured at <= 2e-11
  for n <= 200 at the workloads here, and |Delta P| <= max_k |Delta G_k| <= |Delta log G|.
* log q at sampled grid points (full-size workloads, where the oracle cannot afford the
  whole grid): |Delta log q| <= 1e-9 (FP64) and 1e-9 (FP32R) including the imaginary part,
  so the square-root branch is checked too.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-10}
LOGQ_TOL = {0: 1e-9, 1: 1e-9}
PRECISIONS = [0, 1]


def gpu_table(gb, prob, precision, oversample=1, tile_override=0):
    with gb.Plan(prob, precision=precision, oversample=oversample, tile_override=tile_override) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    return P, st, d, lq, mp


def oracle_table(prob, oversample=1):
    radix = prob.radix * oversample
    res = oracle.binned(prob, radix=radix)
    sl = tuple(slice(0, int(c) + 1) for c in prob.cutoff)
    return res["P"][sl], res


def _flat_index(digits, radix):
    strides = np.ones(len(radix), dtype=np.int64)
    for l in range(len(radix) - 2, -1, -1):
        strides[l] = strides[l + 1] * radix[l + 1]
    return digits @ strides


SMALL = [
    ("m4_l2_n6", lambda: synth.config(0)),
    ("m16_l4_n8", lambda: synth.config(1)),
    ("disp_k2_basis_even", lambda: synth.random_problem(np.random.default_rng(101), 3, 2, 2, 5, displaced=True,
                                                        internal_basis=True)),
    ("l3_shuffled", lambda: synth.random_problem(np.random.default_rng(102), 6, 1, 3, [4, 3, 6], displaced=True,
                                                 shuffle_bins=True)),
    ("l1_n30", lambda: synth.random_problem(np.random.default_rng(103), 8, 1, 1, 30)),
    ("cutoff_zero_axis", lambda: synth.random_problem(np.random.default_rng(104), 4, 1, 2, [0, 7])),
    ("m1_k1", lambda: synth.random_problem(np.random.default_rng(105), 1, 1, 1, 9, displaced=True)),
    ("ragged_n50", lambda: synth.random_problem(np.random.default_rng(106), 25, 1, 2, [3, 4], displaced=True)),
    ("k3_m8_l4", lambda: synth.random_problem(np.random.default_rng(107), 8, 3, 4, [2, 3, 2, 1],
                                              internal_basis=True)),
]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_table_matches_oracle(cuda_lib, name, make, precision):
    prob = make()
    P, st, d, lq, mp = gpu_table(cuda_lib, prob, precision)
    ref, res = oracle_table(prob)
    assert st == 0 and d["n_bad_points"] == 0
    assert P.shape == ref.shape
    err = np.abs(P - ref).max()
    assert err <= TOL[precision], (name, precision, err)
    assert abs(d["sum_P"] - ref.sum()) < 1e-10
    assert d["min_pivot_re"] > 0
    # every evaluated point against the oracle's grid (the last axis is halved)
    dig = cuda_lib.evaluated_point_digits(prob.cutoff)
    full = res["logq"][_flat_index(dig, prob.radix)]
    assert np.abs(lq - full).max() < LOGQ_TOL[precision]
    assert abs(d["log_q1_re"] - res["logq"][0].real) < 1e-10


@pytest.mark.parametrize("precision", PRECISIONS)
def test_oversampled_table_is_unfolded(cuda_lib, precision):
    prob = synth.config(0)
    P, st, d, lq, mp = gpu_table(cuda_lib, prob, precision, oversample=8)
    ref, _ = oracle_table(prob, oversample=8)
    assert np.abs(P - ref).max() <= TOL[precision]
    from oracle import lhaf
    bf = lhaf.binned_brute_force(prob, 5)
    for b, v in bf.items():
        assert abs(P[b] - v) < 1e-10


@pytest.mark.parametrize("precision", PRECISIONS)
def test_global_workspace_kernel_matches(cuda_lib, precision):
    # n = 120 > shared-memory limit: the L2-resident workspace variants (the per-point
    # kernels for this size; the automatic choice here is the large-matrix tree)
    prob = synth.random_problem(np.random.default_rng(111), 60, 1, 2, [4, 3], displaced=True)
    P, st, d, lq, mp = gpu_table(cuda_lib, prob, precision, tile_override=3 if precision == 0 else 6)
    assert d["kernel_name"] == ("gmem_fp64" if precision == 0 else "blk_fp32r")
    ref, _ = oracle_table(prob)
    assert np.abs(P - ref).max() <= TOL[precision]
    # forcing the workspace variant on a small problem gives the shared-memory result
    small = synth.config(1)
    forced = 3 if precision == 0 else 4
    Pf, _, df, _, _ = gpu_table(cuda_lib, small, precision, tile_override=forced)
    Ps, _, ds, _, _ = gpu_table(cuda_lib, small, precision)
    assert df["kernel_name"].startswith("gmem") and not ds["kernel_name"].startswith("gmem")
    assert np.abs(Pf - Ps).max() < 1e-13


@pytest.mark.parametrize("kernel", [2, 4, 5, 6, 7])
def test_fp32r_kernel_variants_agree(cuda_lib, kernel):
    # every FP32 + refinement variant (CTA/shared memory, CTA/workspace, warp/registers)
    # meets the bound on the same small problems
    for prob in (synth.config(0), synth.config(1),
                 synth.random_problem(np.random.default_rng(131), 5, 3, 2, [3, 4], displaced=True,
                                      internal_basis=True)):
        P, st, d, lq, mp = gpu_table(cuda_lib, prob, 1, tile_override=kernel)
        ref, _ = oracle_table(prob)
        assert d["kernel"] == kernel
        assert np.abs(P - ref).max() <= TOL[1]


@pytest.mark.parametrize("kernel", [6, 7])
@pytest.mark.parametrize("M,K,displaced", [(17, 1, True), (32, 1, False), (49, 1, True), (48, 3, True),
                                           (70, 1, True), (192, 1, True)])
def test_blocked_kernel_sizes(cuda_lib, M, K, displaced, kernel):
    # the blocked kernel (32-wide panels, 64 x 32 residual blocks), trace updates on the CUDA
    # cores (6) or the tensor cores (7, 128 x 64 tiles), at n = 34 (one panel and a 2-row
    # tail), 64 (exact panels), 98 (ragged panel and residual block), 140 (two tensor M-tiles),
    # 288 (largest n of the batched workload, internal modes) and 384 (largest supported n)
    rng = np.random.default_rng(140 + M + K)
    prob = synth.random_problem(rng, M, K, 2, [2, 1], displaced=displaced, internal_basis=K > 1)
    P, st, d, lq, mp = gpu_table(cuda_lib, prob, 1, tile_override=kernel)
    assert st == 0 and d["kernel"] == kernel and d["n_bad_points"] == 0
    ref, res = oracle_table(prob)
    assert np.abs(P - ref).max() <= TOL[1]
    dig = cuda_lib.evaluated_point_digits(prob.cutoff)
    assert np.abs(lq - res["logq"][_flat_index(dig, prob.radix)]).max() < LOGQ_TOL[1]


def test_precisions_agree_and_repeatable(cuda_lib):
    prob = synth.config(1)
    P64, *_ = gpu_table(cuda_lib, prob, 0)
    P32, *_ = gpu_table(cuda_lib, prob, 1)
    P64b, *_ = gpu_table(cuda_lib, prob, 0)
    assert np.abs(P64 - P32).max() < 1e-10
    assert np.array_equal(P64, P64b)          # deterministic: no atomics in the path


@pytest.mark.parametrize("index", [2, 4])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_sampled(cuda_lib, index, precision):
    # full-size workloads (n = 192 with displacement and internal modes; n = 200): log q at
    # sampled points against the oracle one by one, and properties of the whole table
    prob = synth.config(index)
    P, st, d, lq, mp = gpu_table(cuda_lib, prob, precision)
    assert st == 0 and d["n_bad_points"] == 0
    assert abs(P.sum() - 1.0) < 1e-10
    assert P.min() > -1e-10
    XA, gamma, labels = oracle.plan(prob)
    dig = cuda_lib.evaluated_point_digits(prob.cutoff)
    rng = np.random.default_rng(index)
    pick = np.concatenate([[0, 1, len(dig) - 1], rng.choice(len(dig), 9, replace=False)])
    ref, _, _ = oracle.logq_points(XA, gamma, labels, prob.radix, dig[pick])
    assert np.abs(lq[pick] - ref).max() < LOGQ_TOL[precision]


def test_full_size_paths_agree(cuda_lib):
    prob = synth.config(2)
    P64, *_ = gpu_table(cuda_lib, prob, 0)
    P32, *_ = gpu_table(cuda_lib, prob, 1)
    assert np.abs(P64 - P32).max() < 1e-10


def test_set_state_matches_fresh_plan(cuda_lib):
    gb = cuda_lib
    a = synth.config(1)
    b = synth.config(1)
    b.r = b.r * 0.9
    with gb.Plan(a) as p:
        gb.gbsbin_plan_set_state(p.handle, b)
        Pb = p.table().cpu().numpy()
    ref, _ = oracle_table(b)
    assert np.abs(Pb - ref).max() < 1e-10


def test_execute_host_matches_device(cuda_lib):
    gb = cuda_lib
    prob = synth.config(1)
    with gb.Plan(prob, precision=1) as p:
        Pd = p.table().cpu().numpy()
        Ph = np.zeros(gb.gbsbin_plan_table_size(p.handle))
        gb.gbsbin_execute_host(p.handle, Ph)
    assert np.array_equal(Pd.reshape(-1), Ph)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32r"])
def test_pipelined_state_changes(cuda_lib, precision):
    # set_state + execute_host_async over alternating states into two pinned buffers with
    # one synchronisation per pair: every table equals the synchronous one of its state
    # (the two staging buffers let an upload proceed while the previous table is computed)
    import torch
    gb = cuda_lib
    probs = [synth.config(1), synth.config(1), synth.config(1)]
    probs[1].r = probs[1].r * 0.9
    probs[2].r = probs[2].r * 1.05
    args = [gb.ProblemArgs(q) for q in probs]
    with gb.Plan(probs[0], precision=precision) as p:
        ts = gb.gbsbin_plan_table_size(p.handle)
        sync = []
        for a in args:
            gb.gbsbin_plan_set_state(p.handle, a)
            out = np.zeros(ts)
            gb.gbsbin_execute_host(p.handle, out)
            sync.append(out)
        outs = [torch.zeros(ts, dtype=torch.float64).pin_memory() for _ in range(2)]
        stream = torch.cuda.current_stream()
        for step in range(7):
            k = step % 3
            gb.gbsbin_plan_set_state(p.handle, args[k], stream)
            gb.gbsbin_execute_host_async(p.handle, outs[step & 1], stream)
            if step & 1:
                torch.cuda.synchronize()
                for j, kk in ((0, (step - 1) % 3), (1, k)):
                    assert np.array_equal(outs[j].numpy(), sync[kk]), (step, j)
        torch.cuda.synchronize()
        assert np.array_equal(outs[0].numpy(), sync[6 % 3])
    for q, t in zip(probs, sync):
        ref, _ = oracle_table(q)
        assert np.abs(t.reshape(ref.shape) - ref).max() < 1e-10


def test_direct_covariance_input(cuda_lib):
    from oracle import state
    prob = synth.random_problem(np.random.default_rng(121), 4, 1, 2, 5, displaced=True)
    sigma1, zbar = state.sigma1_zbar(prob)

    class Direct:
        M, K, r, T = prob.M, prob.K, None, None
    d = Direct()
    d.sigma1, d.zbar, d.bin_of_mode, d.cutoff = sigma1, zbar, prob.bin_of_mode, prob.cutoff
    P, st, *_ = gpu_table(cuda_lib, d, 0)
    ref, _ = oracle_table(prob)
    assert np.abs(P - ref).max() < 1e-10


def test_errors_are_reported(cuda_lib):
    gb = cuda_lib
    prob = synth.config(0)
    bad = synth.config(0)
    bad.bin_of_mode = np.array([0, 0, 0, 0], np.int32)       # group 1 empty
    with pytest.raises(gb.GbsbinError) as e:
        gb.Plan(bad)
    assert e.value.status == 2
    bad = synth.config(0)
    bad.T = bad.T * 3.0                                        # gain: not a passive map
    with pytest.raises(gb.GbsbinError) as e:
        gb.Plan(bad)
    assert e.value.status == 4
    bad = synth.config(0)
    bad.cutoff = np.array([-1, 3], np.int32)
    with pytest.raises(gb.GbsbinError) as e:
        gb.Plan(bad)
    assert e.value.status == 3
    with gb.Plan(prob) as p:
        assert gb.gbsbin_plan_table_size(p.handle) == 49


def test_tensor_core_trace_full_size(cuda_lib):
    # n = 192 (displaced, internal modes): the trace updates on the tensor cores (3 x TF32)
    # give the same table as on the CUDA cores and as the FP64 path
    prob = synth.config(2)
    P6, st6, *_ = gpu_table(cuda_lib, prob, 1, tile_override=6)
    P7, st7, d7, *_ = gpu_table(cuda_lib, prob, 1, tile_override=7)
    P64, *_ = gpu_table(cuda_lib, prob, 0)
    assert st6 == 0 and st7 == 0 and d7["kernel_name"] == "blk_tc_fp32r"
    assert np.abs(P7 - P6).max() < 1e-10
    assert np.abs(P7 - P64).max() < 1e-10
