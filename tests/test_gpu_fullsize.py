"""Whole-table parity at full size (n = 192 and n = 200) and the n = 200 likelihood gradient
on the full 81 x 81 grid, against the CPU oracle.

* n = 192: 24 ports x 4 internal modes with non-aligned internal bases, displaced, three
  groups of eight detectors, N_l = 20 (9261 grid points; Sec. VI with App. B's bases).
* n = 200: 100 ports, two groups of 50, N_l = 80 (6561 grid points).

Every entry of the table is compared with the oracle's table (both paths, 1e-10 absolute),
and every evaluated log q with the oracle's per-point value (1e-9, imaginary part
included, so the square-root branch is checked at every point).  The oracle evaluates the
whole grid once per workload (about 2e11 flops on the host cores).
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


@pytest.fixture(scope="module")
def oracle_tables():
    cache = {}

    def get(index):
        if index not in cache:
            prob = synth.config(index)
            cache[index] = (prob, oracle.binned(prob))
        return cache[index]
    return get


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32r"])
@pytest.mark.parametrize("index", [2, 4], ids=["n192", "n200"])
def test_whole_table_matches_oracle(cuda_lib, oracle_tables, index, precision):
    gb = cuda_lib
    prob, res = oracle_tables(index)
    with gb.Plan(prob, precision=precision) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, _ = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0 and d["n_bad_points"] == 0
    ref = res["P"]
    assert P.shape == ref.shape
    err = float(np.abs(P - ref).max())
    assert err <= TOL, (index, precision, d["kernel_name"], err)
    dig = gb.evaluated_point_digits(prob.cutoff)
    full = res["logq"][_flat_index(dig, prob.radix)]
    assert np.abs(lq - full).max() < LOGQ_TOL
    assert abs(d["log_q1_re"] - res["logq"][0].real) < 1e-10
    assert abs(d["sum_P"] - ref.sum()) < 1e-10


@pytest.fixture(scope="module")
def nll_reference(oracle_tables):
    """The n = 200 negative log-likelihood of 10^6 multinomial draws from the oracle's table,
    and its Richardson-extrapolated central differences (oracle only) along a random direction
    in the 100 squeezings and along the transmission eta of T = sqrt(eta) U (the NLL is ~1e7
    in size, so h cannot be tiny)."""
    prob, res = oracle_tables(4)
    rng = np.random.default_rng(504)
    P0 = np.clip(res["P"], 0, None)
    counts = rng.multinomial(10 ** 6, P0.reshape(-1) / P0.sum()).reshape(P0.shape)

    def nll(q):
        P = oracle.binned(q)["P"]
        return float(-(counts * np.log(P)).sum())

    def copy_prob(q):
        return synth.Problem(q.M, q.K, q.r.copy(), q.T.copy(), q.bin_of_mode.copy(), q.cutoff.copy(),
                             notes=dict(q.notes))

    def richardson(shift, h=2e-4):
        def d(hh):
            return (nll(shift(hh)) - nll(shift(-hh))) / (2 * hh)
        return (4.0 * d(h / 2) - d(h)) / 3.0

    dr = rng.standard_normal(prob.r.shape)

    def shift_r(hh):
        q = copy_prob(prob)
        q.r = prob.r + hh * dr
        return q
    eta = prob.notes["eta"]

    def shift_eta(hh):
        q = copy_prob(prob)
        q.T = np.sqrt((eta + hh) / eta) * prob.T
        return q
    return dict(prob=prob, counts=counts, dr=dr, f_r=richardson(shift_r), f_eta=richardson(shift_eta),
                dT=prob.T / (2 * eta))      # T = sqrt(eta) U  =>  dT/deta = T / (2 eta)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
def test_full_grid_negative_log_likelihood_gradient(cuda_lib, nll_reference, precision):
    # n = 200 on the full 81 x 81 grid: the reverse pass (per-point inverse recomputed, FP64 or
    # pairs of FP32) along the two directions of the reference differences
    import torch
    gb = cuda_lib
    ref = nll_reference
    prob, counts = ref["prob"], ref["counts"]
    with gb.Plan(prob, precision=precision, want_backward=True) as p:
        Pg = p.table()
        dLdP = torch.from_numpy(-counts / Pg.cpu().numpy()).cuda()
        g = p.backward(dLdP, want=("r", "T"))
    got = float((g["r"] * ref["dr"]).sum())
    f = ref["f_r"]
    assert abs(got - f) <= 1e-4 + 1e-6 * abs(f), (got, f)
    got = float(np.real(np.sum(np.conj(g["T"]) * ref["dT"])))
    f = ref["f_eta"]
    assert abs(got - f) <= 1e-4 + 1e-6 * abs(f), (got, f)
