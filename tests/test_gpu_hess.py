"""One detector group (the total photon number of Sec. VIII): the Hessenberg path (one
reduction per state, O(n^2) per point, displacement through the reflected vectors) against
the oracle's LU, the general kernels, and the closed form of the uniform-loss setup of
Sec. VIII up to n = 512."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [  # (M, K, cutoff, internal basis, displaced)
    (4, 1, 12, False, False),      # n = 8
    (4, 1, 12, False, True),
    (15, 1, 30, False, True),      # n = 30: one ragged row block
    (32, 1, 20, False, False),     # n = 64
    (25, 2, 16, True, True),       # n = 100, internal modes
    (100, 1, 9, False, False),     # n = 200
    (100, 1, 9, False, True),
]


def _flat(digits, radix):
    strides = np.ones(len(radix), dtype=np.int64)
    for l in range(len(radix) - 2, -1, -1):
        strides[l] = strides[l + 1] * radix[l + 1]
    return digits @ strides


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("M,K,cut,basis,disp", CASES)
def test_one_group_matches_oracle(cuda_lib, M, K, cut, basis, disp, precision):
    gb = cuda_lib
    prob = synth.random_problem(np.random.default_rng(500 + M + K), M, K, 1, cut, internal_basis=basis,
                                displaced=disp)
    with gb.Plan(prob, precision=precision) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0 and d["kernel_name"] == ("hess_df32" if precision else "hess_fp64") and d["n_bad_points"] == 0
    res = oracle.binned(prob)
    assert np.abs(P - res["P"]).max() <= 1e-10
    dig = gb.evaluated_point_digits(prob.cutoff)
    assert np.abs(lq - res["logq"][_flat(dig, prob.radix)]).max() < 1e-9
    assert d["min_pivot_re"] > 0
    # the general FP64 kernel on the same problem gives the same table (the pairs path to the
    # oracle's bound)
    with gb.Plan(prob, precision=0, tile_override=3) as p:
        Pg = p.table().cpu().numpy()
    assert np.abs(P - Pg).max() < (1e-12 if precision == 0 else 1e-10)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("row", [0, 2, 4])
def test_uniform_loss_total_number_closed_form(cuda_lib, row, precision):
    # Sec. VIII setup (xi = 0.89, eta = 0.36, Haar U; M = 16, 64, 256 and the paper's N_max):
    # the total count is M independent lossy squeezed vacua, so log q(w) - log q(1) =
    # -(M/2) log[(1 - x(n+m))(1 - x(n-m))], x = w - 1, n = eta sinh^2 xi, m = eta sinh xi cosh xi
    gb = cuda_lib
    rows = [ln.split() for ln in open(__file__.replace("test_gpu_hess.py", "golden/e3_total_photon_setup.txt"))
            if ln.strip() and not ln.startswith("#")]
    M, Nmax = int(rows[row][0]), int(rows[row][1])
    xi, eta = 0.89, 0.36
    rng = np.random.default_rng(61 + row)
    prob = synth.Problem(M, 1, np.full((M, 1), xi), np.sqrt(eta) * synth.haar_unitary(M, rng),
                         np.zeros(M, np.int32), np.array([Nmax], np.int32))
    with gb.Plan(prob, precision=precision) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0 and d["kernel_name"] == ("hess_df32" if precision else "hess_fp64") and d["n"] == 2 * M
    w = np.exp(2j * np.pi * np.arange(Nmax + 1) / (Nmax + 1))
    n_, m_ = eta * np.sinh(xi) ** 2, eta * np.sinh(xi) * np.cosh(xi)
    x = w - 1
    G = ((1 - x * (n_ + m_)) * (1 - x * (n_ - m_))) ** (-M / 2.0)
    half = (Nmax + 1) // 2 + 1
    Gk = np.exp(lq - lq[0])
    assert np.abs(Gk - G[:half]).max() < (1e-11 if precision == 0 else 1e-10)
    assert np.abs(P - (np.fft.fft(G) / (Nmax + 1)).real).max() < (1e-12 if precision == 0 else 1e-10)
    assert abs(P.sum() - 1.0) < 1e-12


def test_one_group_state_changes_and_errors(cuda_lib):
    gb = cuda_lib
    rng = np.random.default_rng(520)
    two = synth.random_problem(rng, 6, 1, 2, [3, 4])
    for tile in (8, 16):                          # forcing the one-group path on two groups
        with pytest.raises(gb.GbsbinError):
            gb.Plan(two, tile_override=tile)
    # new states on a one-group plan: undisplaced, then displaced
    a = synth.random_problem(np.random.default_rng(521), 10, 1, 1, 14)
    b = synth.random_problem(np.random.default_rng(522), 10, 1, 1, 14)
    c = synth.random_problem(np.random.default_rng(523), 10, 1, 1, 14, displaced=True)
    with gb.Plan(a) as p:
        for new in (b, c):
            gb.gbsbin_plan_set_state(p.handle, new)
            Pn = p.table().cpu().numpy()
            st, d = p.diagnostics()
            assert st == 0 and d["kernel_name"] == "hess_fp64"
            assert np.abs(Pn - oracle.binned(new)["P"]).max() <= 1e-10


def test_hessenberg_table_matches_power_series(cuda_lib):
    # two evaluators of the total photon-number distribution: the roots-of-unity transform
    # of the one-group plan (Hessenberg kernel) and the power series of App. A (host); the
    # grid's folding is far below the bound at this squeezing (mean about 2 photons)
    gb = cuda_lib
    prob = synth.random_problem(np.random.default_rng(1001), 20, 1, 1, 40, displaced=True, r_range=(0.1, 0.35))
    with gb.Plan(prob) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
    assert st == 0 and d["kernel_name"] == "hess_fp64"
    ref = gb.gbsbin_total_photon_series(prob, 40)
    assert np.abs(P - ref).max() < 1e-12


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("M,cut,disp", [(80, 1400, True), (150, 1300, True), (200, 1300, False)])
def test_one_group_large_grids(cuda_lib, M, cut, disp, precision):
    # grids with enough points for a warp per point (n = 160, 300 and 400 with 701, 651 and 651
    # evaluated points: the 8-, 12- and 16-slot instantiations); the small-grid cases above run a
    # CTA per point from n = 128 on.  log q at sampled points against the oracle one by one, the
    # table's total and sign, and the two arithmetics' tables against each other
    gb = cuda_lib
    prob = synth.random_problem(np.random.default_rng(530 + M), M, 1, 1, cut, displaced=disp, r_range=(0.2, 0.7))
    with gb.Plan(prob, precision=precision) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, mp = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0 and d["kernel_name"] == ("hess_df32" if precision else "hess_fp64") and d["n_bad_points"] == 0
    assert abs(P.sum() - 1.0) < 1e-10 and P.min() > -1e-10
    XA, gamma, labels = oracle.plan(prob)
    dig = gb.evaluated_point_digits(prob.cutoff)
    pick = np.concatenate([[0, 1, len(dig) - 1], np.random.default_rng(M).choice(len(dig), 9, replace=False)])
    ref, _, _ = oracle.logq_points(XA, gamma, labels, prob.radix, dig[pick])
    assert np.abs(lq[pick] - ref).max() < 1e-9
    with gb.Plan(prob, precision=1 - precision) as p:
        Q = p.table().cpu().numpy()
    assert np.abs(P - Q).max() < 1e-10
