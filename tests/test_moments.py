"""Exact binned means, covariances and third and fourth cumulants (gbsbin_moments,
gbsbin_cumulants3, gbsbin_cumulants4; host FP64, no GPU) against textbook single-mode results
and against the central moments of the oracle's unfolded (oversampled) tables."""
import numpy as np
import pytest

import oracle
import synth
from oracle import state


@pytest.fixture(scope="module")
def gb():
    import paper_2412_17742_gb300 as gb
    try:
        gb.load()
    except RuntimeError:
        pytest.skip("library not built")
    return gb


def _one_mode(r, alpha=None, eta=1.0):
    return synth.Problem(1, 1, np.array([[r]]), np.array([[np.sqrt(eta)]], complex), np.zeros(1, np.int32),
                         np.array([5], np.int32), alpha=None if alpha is None else np.array([[alpha]], complex))


def test_squeezed_vacuum_and_coherent_state(gb):
    r = 0.7
    m, c = gb.gbsbin_moments(_one_mode(r))
    assert abs(m[0] - np.sinh(r) ** 2) < 1e-14
    assert abs(c[0, 0] - 2 * np.sinh(r) ** 2 * np.cosh(r) ** 2) < 1e-13   # variance of a squeezed vacuum
    a = 0.9 - 0.4j
    m, c = gb.gbsbin_moments(_one_mode(0.0, a))
    assert abs(m[0] - abs(a) ** 2) < 1e-14 and abs(c[0, 0] - abs(a) ** 2) < 1e-13   # Poisson
    # loss eta on a squeezed vacuum: mean eta sinh^2 r; the variance against the oracle's
    # unfolded table (its 400-point DFT carries ~1e-12 of rounding)
    m, c = gb.gbsbin_moments(_one_mode(r, eta=0.6))
    assert abs(m[0] - 0.6 * np.sinh(r) ** 2) < 1e-14
    P = oracle.binned(_one_mode(r, eta=0.6), radix=[400])["P"]
    k = np.arange(len(P))
    mu = (P * k).sum()
    assert abs(m[0] - mu) < 1e-10 and abs(c[0, 0] - ((P * k * k).sum() - mu * mu)) < 1e-9


@pytest.mark.parametrize("M,K,L,cut,disp,basis", [(4, 1, 2, 6, True, False), (3, 2, 2, 5, False, True),
                                                  (3, 2, 3, 4, True, True), (5, 1, 3, 4, True, False)])
def test_against_unfolded_tables(gb, M, K, L, cut, disp, basis):
    rng = np.random.default_rng(900 + M + K + L)
    prob = synth.random_problem(rng, M, K, L, cut, displaced=disp, internal_basis=basis, r_range=(0.1, 0.5))
    m, c = gb.gbsbin_moments(prob)
    P = oracle.binned(prob, radix=prob.radix * (12 if L <= 2 else 8))["P"]
    grids = np.meshgrid(*[np.arange(s) for s in P.shape], indexing="ij")
    assert abs(P.sum() - 1) < 1e-12
    mu = np.array([(P * g).sum() for g in grids])
    cov = np.array([[(P * gi * gj).sum() - mu[i] * mu[j] for j, gj in enumerate(grids)] for i, gi in enumerate(grids)])
    assert np.abs(m - mu).max() < 1e-10, (m, mu)
    assert np.abs(c - cov).max() < 1e-9, (c, cov)
    assert np.abs(c - c.T).max() < 1e-13


def test_means_match_closed_form(gb):
    # first moment per bin: sum_{j in group} (Sigma^(1)_jj + |zbar_j|^2), no table involved
    rng = np.random.default_rng(931)
    prob = synth.random_problem(rng, 12, 2, 3, 3, displaced=True, internal_basis=True, r_range=(0.5, 1.2))
    m, c = gb.gbsbin_moments(prob)
    s1, zbar = state.sigma1_zbar(prob)
    MK = prob.M * prob.K
    labels = np.repeat(prob.bin_of_mode, prob.K)
    expect = [sum((s1[i, i] + abs(zbar[i]) ** 2).real for i in range(MK) if labels[i] == l) for l in range(prob.L)]
    assert np.abs(m - np.array(expect)).max() < 1e-11
    assert np.all(np.linalg.eigvalsh(c) > 0)


def test_rejects_bad_input(gb):
    bad = synth.config(0)
    bad.bin_of_mode = np.array([0, 0, 0, 0], np.int32)
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_moments(bad)


# ------------------------------------------------------------------ third cumulants
def test_third_cumulant_single_modes(gb):
    # squeezed vacuum: log G(e^t) = -1/2 log(cosh^2 r - e^{2t} sinh^2 r), whose third
    # derivative at 0 is 4 s + 12 s^2 + 8 s^3 with s = sinh^2 r; coherent state: Poisson
    # (every cumulant is the mean)
    r = 0.6
    s = np.sinh(r) ** 2
    k3 = gb.gbsbin_cumulants3(_one_mode(r))
    assert abs(k3[0, 0, 0] - (4 * s + 12 * s * s + 8 * s ** 3)) < 1e-12
    a = 0.7 + 0.5j
    k3 = gb.gbsbin_cumulants3(_one_mode(0.0, a))
    assert abs(k3[0, 0, 0] - abs(a) ** 2) < 1e-13


@pytest.mark.parametrize("M,K,L,cut,disp,basis", [(4, 1, 2, 6, True, False), (3, 2, 2, 5, False, True),
                                                  (3, 1, 3, 4, True, False)])
def test_third_cumulants_against_unfolded_tables(gb, M, K, L, cut, disp, basis):
    # third cumulants are the third central moments of the unfolded table
    rng = np.random.default_rng(950 + M + K + L)
    prob = synth.random_problem(rng, M, K, L, cut, displaced=disp, internal_basis=basis, r_range=(0.1, 0.45))
    k3 = gb.gbsbin_cumulants3(prob)
    P = oracle.binned(prob, radix=prob.radix * (12 if L <= 2 else 8))["P"]
    grids = np.meshgrid(*[np.arange(sz) for sz in P.shape], indexing="ij")
    mu = [(P * g).sum() for g in grids]
    d = [g - m for g, m in zip(grids, mu)]
    ref = np.array([[[(P * d[i] * d[j] * d[k]).sum() for k in range(L)] for j in range(L)] for i in range(L)])
    assert np.abs(k3 - ref).max() < 1e-8, np.abs(k3 - ref).max()
    # symmetric in its three indices
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0)]:
        assert np.abs(k3 - k3.transpose(perm)).max() < 1e-12


# ------------------------------------------------------------------ fourth cumulants
def test_fourth_cumulant_single_modes(gb):
    # squeezed vacuum: the fourth derivative of -1/2 log(1 + s - s e^{2t}) at 0 is
    # 8 s (1 + s)(1 + 6 s + 6 s^2), s = sinh^2 r; coherent state: Poisson (every cumulant is
    # the mean); a squeezed displaced single mode: the fourth central moment minus 3 var^2
    # of its photon-number distribution (oracle table, unfolded)
    r = 0.6
    s = np.sinh(r) ** 2
    k4 = gb.gbsbin_cumulants4(_one_mode(r))
    assert abs(k4[0, 0, 0, 0] - 8 * s * (1 + s) * (1 + 6 * s + 6 * s * s)) < 1e-11
    a = 0.7 + 0.5j
    k4 = gb.gbsbin_cumulants4(_one_mode(0.0, a))
    assert abs(k4[0, 0, 0, 0] - abs(a) ** 2) < 1e-13
    prob = _one_mode(0.3, 0.4 - 0.2j, eta=0.8)
    # 32 bins: the squeezed tail is below 1e-16 there, and the table's roundoff weighted by
    # (b - mean)^4 stays near 1e-10 (a wider table amplifies it, a narrower one truncates)
    P = oracle.binned(prob, radix=np.array([32]))["P"]
    b = np.arange(P.shape[0])
    mu = (P * b).sum()
    m2, m4 = (P * (b - mu) ** 2).sum(), (P * (b - mu) ** 4).sum()
    assert abs(gb.gbsbin_cumulants4(prob)[0, 0, 0, 0] - (m4 - 3 * m2 * m2)) < 2e-9


def _central(P, L):
    grids = np.meshgrid(*[np.arange(sz) for sz in P.shape], indexing="ij")
    mu = [(P * g).sum() for g in grids]
    return [g - m for g, m in zip(grids, mu)]


@pytest.mark.parametrize("M,K,L,cut,disp,basis", [(4, 1, 2, 6, True, False), (3, 2, 2, 5, False, True),
                                                  (3, 1, 3, 4, True, False), (4, 1, 4, 3, True, False)])
def test_fourth_cumulants_against_unfolded_tables(gb, M, K, L, cut, disp, basis):
    # kappa_ijkl = mu_ijkl - mu_ij mu_kl - mu_ik mu_jl - mu_il mu_jk, central moments of the
    # unfolded table; the first three orders must agree with gbsbin_moments / cumulants3
    rng = np.random.default_rng(970 + M + K + L)
    prob = synth.random_problem(rng, M, K, L, cut, displaced=disp, internal_basis=basis, r_range=(0.1, 0.4))
    k4 = gb.gbsbin_cumulants4(prob)
    # the table's own accuracy bounds the reference: too few bins truncate the tail, too many
    # weight the table's roundoff by (b - mean)^4; these oversamplings sit near the optimum
    over = 6 if L <= 3 else 5
    P = oracle.binned(prob, radix=prob.radix * over)["P"]
    d = _central(P, L)
    c2 = np.array([[(P * d[i] * d[j]).sum() for j in range(L)] for i in range(L)])
    ref = np.zeros((L,) * 4)
    for i, j, k, l in np.ndindex(*(L,) * 4):
        ref[i, j, k, l] = ((P * d[i] * d[j] * d[k] * d[l]).sum()
                           - c2[i, j] * c2[k, l] - c2[i, k] * c2[j, l] - c2[i, l] * c2[j, k])
    assert np.abs(k4 - ref).max() < 1e-8 * max(1.0, np.abs(k4).max()), np.abs(k4 - ref).max()
    # symmetric in its four indices
    for perm in [(1, 0, 2, 3), (0, 2, 1, 3), (0, 1, 3, 2), (3, 1, 2, 0)]:
        assert np.abs(k4 - k4.transpose(perm)).max() < 1e-12


# ------------------------------------------------------------- joint cumulants of distinct groups
@pytest.mark.parametrize("M,K,L,disp,basis", [(4, 1, 4, True, False), (6, 2, 3, False, True), (5, 1, 5, True, False)])
def test_distinct_group_cumulants_match_the_tensors(gb, M, K, L, disp, basis):
    # orders 1-4 of the loop-Montrealer form against the mean, covariance and the
    # distinct-index entries of the third and fourth cumulant tensors
    import itertools
    rng = np.random.default_rng(1100 + M + K + L)
    prob = synth.random_problem(rng, M, K, L, 3, displaced=disp, internal_basis=basis, r_range=(0.2, 0.6))
    mean, cov = gb.gbsbin_moments(prob)
    k3, k4 = gb.gbsbin_cumulants3(prob), gb.gbsbin_cumulants4(prob)
    for l in range(L):
        assert abs(gb.gbsbin_cumulant_groups(prob, [l]) - mean[l]) < 1e-12
    for a, b in itertools.combinations(range(L), 2):
        assert abs(gb.gbsbin_cumulant_groups(prob, [a, b]) - cov[a, b]) < 1e-12
    for t in itertools.combinations(range(L), 3):
        assert abs(gb.gbsbin_cumulant_groups(prob, t) - k3[t]) < 1e-11
    for t in itertools.combinations(range(L), 4):
        assert abs(gb.gbsbin_cumulant_groups(prob, t) - k4[t]) < 1e-11


def test_fifth_joint_cumulant_against_unfolded_table(gb):
    # five groups of one mode: kappa_12345 = mu_12345 - sum over the 10 (pair, triple) splits of
    # mu_pair mu_triple, central moments of the oracle's unfolded table
    import itertools
    rng = np.random.default_rng(1200)
    prob = synth.random_problem(rng, 5, 1, 5, 2, displaced=True, r_range=(0.15, 0.4))
    P = oracle.binned(prob, radix=prob.radix * 5)["P"]
    d = _central(P, 5)
    mu = lambda idx: (P * np.prod([d[i] for i in idx], axis=0)).sum()
    ref = mu(range(5))
    for pair in itertools.combinations(range(5), 2):
        ref -= mu(pair) * mu([i for i in range(5) if i not in pair])
    got = gb.gbsbin_cumulant_groups(prob, range(5))
    assert abs(got - ref) < 1e-8 * max(1.0, abs(ref)), (got, ref)


def test_distinct_group_cumulant_errors(gb):
    prob = synth.random_problem(np.random.default_rng(1300), 3, 1, 3, 2)
    with pytest.raises(ValueError):
        gb.gbsbin_cumulant_groups(prob, [1, 1])
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_cumulant_groups(prob, [])
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_cumulant_groups(prob, [3])
