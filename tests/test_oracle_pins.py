"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties an oracle function to something other than itself: counting identities,
textbook single-mode distributions, brute-force loop Hafnians, closed-form generating
functions of limits named in the paper, a branch of log det that uses no LU, and an
independent DFT.  A dropped term, wrong sign, wrong index or transposed operand in the
oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import lhaf, state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- loop Hafnian itself
def test_lhaf_counts_matchings():
    # all-ones matrix: lhaf counts single-pair matchings with loops = involutions of m
    # elements (1, 1, 2, 4, 10, 26, 76, 232); haf (zero diagonal) of 2m vertices = (2m-1)!!
    involutions = [1, 1, 2, 4, 10, 26, 76, 232]
    for m in range(1, 8):
        assert abs(lhaf.lhaf_explicit(np.ones((m, m))) - involutions[m]) < 1e-9
    for m in range(1, 4):
        B = np.ones((2 * m, 2 * m)) - np.eye(2 * m)
        dfact = math.prod(range(2 * m - 1, 0, -2))
        assert abs(lhaf.lhaf_explicit(B) - dfact) < 1e-9


def test_lhaf_four_vertices_by_hand():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    a = a + a.T
    g = a.diagonal()
    expect = (g[0] * g[1] * g[2] * g[3]
              + a[0, 1] * g[2] * g[3] + a[0, 2] * g[1] * g[3] + a[0, 3] * g[1] * g[2]
              + a[1, 2] * g[0] * g[3] + a[1, 3] * g[0] * g[2] + a[2, 3] * g[0] * g[1]
              + a[0, 1] * a[2, 3] + a[0, 2] * a[1, 3] + a[0, 3] * a[1, 2])
    assert abs(lhaf.lhaf_explicit(a) - expect) < 1e-12


def test_lhaf_repeated_equals_expanded():
    rng = np.random.default_rng(2)
    for trial in range(12):
        s = int(rng.integers(2, 5))
        A = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
        A = A + A.T
        g = rng.standard_normal(s) + 1j * rng.standard_normal(s)
        mult = rng.integers(0, 3, s)
        if mult.sum() > 8:
            continue
        e = lhaf.lhaf_explicit(lhaf.expand(A, g, mult))
        r = lhaf.lhaf_repeated(A, g, mult)
        assert abs(e - r) <= 1e-11 * max(1.0, abs(e))


def test_lhaf_scaling_property():
    # Eq. lhaf_scaling: lhaf(diag(c) A diag(c), diag(c) gamma) = prod(c) lhaf(A, gamma)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3)) + 0j
    A = A + A.T
    g = rng.standard_normal(3) + 0j
    c = rng.uniform(0.5, 2.0, 3)
    mult = (2, 1, 1)
    base = lhaf.lhaf_repeated(A, g, mult)
    scaled = lhaf.lhaf_repeated(c[:, None] * A * c[None, :], c * g, mult)
    assert abs(scaled - np.prod(c ** np.array(mult)) * base) < 1e-12 * abs(base)


# ------------------------------------------------------- Fock probabilities (Sec. II)
def _single_mode_problem(r, alpha=None, eta=1.0):
    return synth.Problem(1, 1, np.array([[r]]), np.array([[np.sqrt(eta)]], dtype=complex),
                         np.array([0], dtype=np.int32), np.array([20], dtype=np.int32),
                         alpha=None if alpha is None else np.array([[alpha]], dtype=complex))


def _sq_vac(r, nmax):
    """Textbook squeezed vacuum: P(2m) = tanh^{2m} r (2m)! / (2^m m!)^2 / cosh r."""
    p = np.zeros(nmax + 1)
    for m in range(nmax // 2 + 1):
        p[2 * m] = np.tanh(r) ** (2 * m) * math.factorial(2 * m) / (2 ** m * math.factorial(m)) ** 2 / np.cosh(r)
    return p


def test_fock_single_mode_squeezed_vacuum():
    r = 0.7
    prob = _single_mode_problem(r)
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    A = state.xmat(2) @ XA
    pr0 = state.vacuum_probability(XA, gamma)
    ref = _sq_vac(r, 8)
    for nphot in range(9):
        assert abs(lhaf.fock_probability(A, gamma, pr0, (nphot,)) - ref[nphot]) < 1e-14


def test_fock_coherent_state():
    alpha = 0.8 - 0.5j
    prob = _single_mode_problem(0.0, alpha)
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    A = state.xmat(2) @ XA
    pr0 = state.vacuum_probability(XA, gamma)
    lam = abs(alpha) ** 2
    for nphot in range(8):
        ref = math.exp(-lam) * lam ** nphot / math.factorial(nphot)
        assert abs(lhaf.fock_probability(A, gamma, pr0, (nphot,)) - ref) < 1e-14


def test_adjacency_is_symmetric():
    rng = np.random.default_rng(4)
    prob = synth.random_problem(rng, 3, 2, 2, 4, displaced=True, internal_basis=True)
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    A = state.xmat(XA.shape[0]) @ XA
    assert np.abs(A - A.T).max() < 1e-13
    assert np.abs(sigma1 - sigma1.conj().T).max() < 1e-13
    # ||XA||_2 < 1 for a physical state (Sigma = Sigma^(0) + I/2 has eigenvalues > 1/2)
    assert np.linalg.norm(XA, 2) < 1.0


# -------------------------------------------- oracle vs brute force (Sec. VI definition)
BRUTE_CASES = [
    ("cfg_small", lambda: synth.config(0), 6),
    ("m3_displaced", lambda: synth.random_problem(np.random.default_rng(11), 3, 1, 2, 5, displaced=True), 5),
    ("m2_k2_basis", lambda: synth.random_problem(np.random.default_rng(12), 2, 2, 2, 5, internal_basis=True), 5),
    ("m3_l3_shuffled", lambda: synth.random_problem(np.random.default_rng(13), 3, 1, 3, 4, displaced=True,
                                                    shuffle_bins=True), 4),
    ("m2_k2_disp_basis", lambda: synth.random_problem(np.random.default_rng(14), 2, 2, 1, 6, displaced=True,
                                                      internal_basis=True), 5),
]


@pytest.mark.parametrize("name,make,total", BRUTE_CASES, ids=[c[0] for c in BRUTE_CASES])
def test_oracle_matches_brute_force(name, make, total):
    prob = make()
    bf = lhaf.binned_brute_force(prob, total)
    # grid large enough that the folded-in tail (~ tanh(r)^R) is below 1e-16
    over = int(np.ceil(96 / (int(prob.cutoff.min()) + 1)))
    Pu = oracle.unfolded(prob, oversample=over)
    for b, v in bf.items():
        if all(bi <= c for bi, c in zip(b, prob.cutoff)):
            assert abs(Pu[b] - v) < 1e-13, (b, Pu[b], v)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("index", [0, 1])
def test_normalisation_and_conjugate_symmetry(index):
    prob = synth.config(index)
    res = oracle.binned(prob)
    assert abs(res["P"].sum() - 1.0) < 1e-13
    assert res["imag_max"] < 1e-13
    assert res["min_pivot"] > 0.0 and res["status"].max() == 0
    # folded table is a distribution: nonnegative up to rounding
    assert res["P"].min() > -1e-14
    # G(omega^-k) = conj G(omega^k)
    R = prob.radix
    G = np.exp(res["logq"] - res["logq"][0]).reshape(tuple(R))
    neg = G[tuple(np.ix_(*[(-np.arange(r)) % r for r in R]))]
    assert np.abs(neg - G.conj()).max() < 1e-13


def test_mean_photon_number_per_bin():
    # first moment: sum_{j in Lambda_l} ( sum_{i,k} |T_ji|^2 sinh^2 r_ik + |(T_full alpha)_j|^2 )
    rng = np.random.default_rng(21)
    for K, disp in [(1, True), (2, False), (2, True)]:
        prob = synth.random_problem(rng, 4, K, 2, 7, displaced=disp, internal_basis=(K > 1))
        Pu = oracle.binned(prob, radix=prob.radix * 10)["P"]
        b = np.arange(Pu.shape[0])
        mean_num = [(Pu.sum(axis=1) * b).sum(), (Pu.sum(axis=0) * np.arange(Pu.shape[1])).sum()]
        Tf = state.full_transfer(prob)
        a = np.zeros(prob.M * prob.K, complex) if prob.alpha is None else prob.alpha.reshape(-1)
        disp_out = np.abs(Tf @ a) ** 2
        sq = np.sinh(prob.r.reshape(-1)) ** 2
        for l in range(2):
            ports = np.where(prob.bin_of_mode == l)[0]
            expect = sum((np.abs(prob.T[j, :]) ** 2 @ np.sinh(prob.r) ** 2).sum() for j in ports)
            expect += sum(disp_out[j * K:(j + 1) * K].sum() for j in ports)
            assert abs(mean_num[l] - expect) < 1e-10, (K, disp, l, mean_num[l], expect)
        del sq


# ---------------------------------------------------------------- closed forms
def test_lossless_pure_state_total_number():
    # Sec. IV: total photon number of a pure state through a lossless interferometer is the
    # convolution of the single-mode input distributions; odd totals vanish.
    rng = np.random.default_rng(31)
    M, N = 5, 24
    r = rng.uniform(0.3, 0.7, M)
    prob = synth.Problem(M, 1, r[:, None], synth.haar_unitary(M, rng), np.zeros(M, np.int32),
                         np.array([N], np.int32))
    conv = np.array([1.0])
    for ri in r:
        conv = np.convolve(conv, _sq_vac(ri, N))[: N + 1]
    P = oracle.unfolded(prob, oversample=6)
    assert np.abs(P - conv).max() < 1e-14
    assert np.abs(P[1::2]).max() < 1e-15


def test_fully_distinguishable_sources():
    # App. D limit: every source in its own internal mode -> no interference.  Each source
    # is a squeezed vacuum whose photons reach group l with probability
    # p_il = sum_{j in Lambda_l} |T_ji|^2, so G(w) = prod_i G_sq,i(1 + sum_l p_il (w_l - 1)),
    # G_sq(z) = 1 / (cosh r sqrt(1 - z^2 tanh^2 r)).
    rng = np.random.default_rng(41)
    M, L, N = 3, 2, 5
    rvals = rng.uniform(0.4, 0.9, M)
    r = np.diag(rvals)                           # K = M, source i squeezed in internal mode i
    T = np.sqrt(rng.uniform(0.5, 0.9, M))[:, None] * synth.haar_unitary(M, rng)
    prob = synth.Problem(M, M, r, T, np.array([0, 0, 1], np.int32), np.array([N, N], np.int32))
    G, logq, minre, st = oracle.pgf_grid(prob)
    R = prob.radix
    p = np.stack([(np.abs(T[prob.bin_of_mode == l, :]) ** 2).sum(axis=0) for l in range(L)], axis=1)
    ref = np.zeros(len(G), complex)
    for f, k in enumerate(itertools.product(*[range(x) for x in R])):
        w = np.exp(2j * np.pi * np.array(k) / R)
        z = 1 + p @ (w - 1)
        ref[f] = np.prod(1 / (np.cosh(rvals) * np.sqrt(1 - z ** 2 * np.tanh(rvals) ** 2)))
    assert np.abs(G - ref).max() < 1e-14


def test_coherent_inputs_are_poisson():
    # r = 0, alpha != 0: G(w) = exp(sum_l lambda_l (w_l - 1)), lambda_l = sum |(T alpha)_j|^2
    rng = np.random.default_rng(51)
    M, L = 4, 2
    T = np.sqrt(0.8) * synth.haar_unitary(M, rng)
    alpha = (rng.standard_normal(M) + 1j * rng.standard_normal(M))[:, None] * 0.7
    prob = synth.Problem(M, 1, np.zeros((M, 1)), T, np.array([0, 1, 1, 0], np.int32),
                         np.array([9, 9], np.int32), alpha=alpha)
    lam = [np.sum(np.abs(T @ alpha[:, 0])[prob.bin_of_mode == l] ** 2) for l in range(L)]
    P = oracle.unfolded(prob, oversample=6)
    for b0 in range(10):
        for b1 in range(10):
            ref = (math.exp(-lam[0]) * lam[0] ** b0 / math.factorial(b0)
                   * math.exp(-lam[1]) * lam[1] ** b1 / math.factorial(b1))
            assert abs(P[b0, b1] - ref) < 1e-14


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_uniform_loss_total_number_e3():
    # Sec. VIII (GBS total photon number): equal squeezing xi, T = sqrt(eta) U with Haar U.
    # Loss commutes with U, so the total count is M independent lossy squeezed vacua, each
    # with PGF [(1 - x(n+m))(1 - x(n-m))]^{-1/2}, x = w - 1, n = eta sinh^2 xi,
    # m = eta sinh xi cosh xi.  Parameters from the paper's printed setup.
    rows = _read_golden("e3_total_photon_setup.txt")
    xi, eta = 0.89, 0.36
    M, Nmax = int(rows[0][0]), int(rows[0][1])
    assert (M, Nmax) == (16, 27)
    rng = np.random.default_rng(61)
    prob = synth.Problem(M, 1, np.full((M, 1), xi), np.sqrt(eta) * synth.haar_unitary(M, rng),
                         np.zeros(M, np.int32), np.array([Nmax], np.int32))
    G, logq, minre, st = oracle.pgf_grid(prob)
    w = np.exp(2j * np.pi * np.arange(Nmax + 1) / (Nmax + 1))
    n_, m_ = eta * np.sinh(xi) ** 2, eta * np.sinh(xi) * np.cosh(xi)
    x = w - 1
    ref = ((1 - x * (n_ + m_)) * (1 - x * (n_ - m_))) ** (-M / 2.0)
    assert np.abs(G - ref).max() < 1e-13
    # folded table against an independent FFT of the closed form, and the mean
    P = oracle.binned(prob)["P"]
    assert np.abs(P - (np.fft.fft(ref) / (Nmax + 1)).real).max() < 1e-14
    Pbig = oracle.binned(prob, radix=[8 * (Nmax + 1)])["P"]
    mean = (Pbig * np.arange(len(Pbig))).sum()
    assert abs(mean - M * eta * np.sinh(xi) ** 2) < 1e-10
    assert abs(M * eta * np.sinh(xi) ** 2 - float(rows[0][2])) < 5e-3


def test_logdet_branch_matches_series():
    # R4: the sum of principal pivot logs is the branch continuous from w = 0; the series
    # -sum tr((D XA)^k)/k (Sec. IV, Eq. useful_series_expansions) uses no LU and no branch
    # choice.  Imaginary parts must agree exactly, not modulo 2 pi.  With gamma = 0,
    # log q = -1/2 log det(I - D XA).
    rng = np.random.default_rng(71)
    prob = synth.random_problem(rng, 20, 1, 2, 8, r_range=(0.8, 1.4), eta_range=(0.6, 0.9))
    XA, gamma, labels = oracle.plan(prob)
    norm = np.linalg.norm(XA, 2)
    terms = int(np.ceil(np.log(1e-17) / np.log(norm))) + 20
    logq, _, st = oracle.logq_grid(XA, np.zeros_like(gamma), labels, prob.radix)
    wrapped = 0
    for f, k in enumerate(itertools.product(*[range(x) for x in prob.radix])):
        d = np.exp(2j * np.pi * np.array(k) / prob.radix)[labels]
        series = oracle.logdet_series(XA, d, terms)
        assert abs(series - (-2.0 * logq[f])) < 1e-10, (k, series, -2 * logq[f])
        wrapped += abs(series.imag) > np.pi
    assert wrapped > 0      # the test exercises points beyond the principal branch


# ---------------------------------------------------------------- the DFT
@pytest.mark.parametrize("radix", [(7,), (3, 4), (2, 5, 3), (4, 1, 3)])
def test_dft_recovers_coefficients(radix):
    # G_k = sum_b c(b) omega^{k.b}  =>  (1/N) sum_k G_k omega^{-k.b} = c(b)
    rng = np.random.default_rng(sum(radix))
    R = np.array(radix)
    c = rng.standard_normal(tuple(R)) + 1j * rng.standard_normal(tuple(R))
    G = np.zeros(tuple(R), complex)
    for k in itertools.product(*[range(x) for x in R]):
        tot = 0j
        for b in itertools.product(*[range(x) for x in R]):
            tot += c[b] * np.exp(2j * np.pi * np.sum(np.array(k) * np.array(b) / R))
        G[k] = tot
    out = oracle.dft(G, R)
    assert np.abs(out - c).max() < 1e-13


def test_nonphysical_state_is_flagged():
    # ||XA|| > 1 breaks the accretivity that guarantees Re u_ii > 0; the oracle reports it
    n = 4
    XA = 1.5 * np.eye(n, dtype=complex)
    logq, minre, st = oracle.logq_grid(XA, np.zeros(n, complex), np.zeros(n, np.int32), np.array([3]))
    assert st[0] != 0 and minre[0] < 0


# ------------------------------------------ per-point evaluation at chosen grid points
@pytest.mark.parametrize("radix", [(3, 5), (4, 1, 6), (2, 3, 1, 5), (1, 7), (5, 2, 2, 3)])
def test_logq_points_matches_grid(radix):
    # oracle.logq_points maps digit rows to flat grid indices (last axis fastest) and
    # evaluates the same per-point LU as logq_grid: equal bits at every point, in any
    # order and with repeats; and, independently of the C code, exp(2 log q) equals
    # exp(gamma^T K^-1 D X gamma) / det K with K = I - D(w) XA formed by numpy (Sec. III,
    # Eq. q_d; the square removes the square root's branch)
    L = len(radix)
    rng = np.random.default_rng(600 + sum(radix))
    prob = synth.random_problem(rng, max(L, 3), 2, L, [r - 1 for r in radix], displaced=True,
                                internal_basis=True, shuffle_bins=True)
    XA, gamma, labels = oracle.plan(prob)
    R = np.array(radix, dtype=np.int64)
    full, minre_full, _ = oracle.logq_grid(XA, gamma, labels, R)
    npts = int(np.prod(R))
    flat = np.concatenate([rng.permutation(npts), rng.integers(0, npts, 5)])
    digits = np.stack(np.unravel_index(flat, tuple(radix)), axis=1)
    lq, minre, st = oracle.logq_points(XA, gamma, labels, R, digits)
    assert st.max() == 0
    assert np.array_equal(lq, full[flat]) and np.array_equal(minre, minre_full[flat])
    n = XA.shape[0]
    Xg = np.concatenate([gamma[n // 2:], gamma[:n // 2]])
    for idx in flat[:6]:
        k = np.unravel_index(idx, tuple(radix))
        w = np.array([np.exp(2j * np.pi * k[l] / radix[l]) for l in range(L)])[labels]
        K = np.eye(n) - w[:, None] * XA
        sq = np.exp(gamma @ np.linalg.solve(K, w * Xg)) / np.linalg.det(K)
        got = np.exp(2 * lq[np.where(flat == idx)[0][0]])
        assert abs(got - sq) <= 1e-12 * abs(sq), (radix, k, got, sq)


# ------------------------------------- fully distinguishable sources, one photon per port
def test_squeezed_pgf_taylor_matches_series():
    # Taylor coefficients of the single-mode squeezed vacuum's generating function about y0
    # against the direct sum_n P(n) C(n, j) y0^(n - j) with P(2k) = tanh^2k(r) (2k)! /
    # (4^k k!^2 cosh r)
    for r, y0 in ((0.7, 0.35), (0.3, 0.0), (1.1, 0.8)):
        t = math.tanh(r)
        P = np.zeros(400)
        for k in range(200):
            P[2 * k] = math.exp(2 * k * math.log(t) + math.lgamma(2 * k + 1) - k * math.log(4.0)
                                - 2 * math.lgamma(k + 1)) / math.cosh(r)
        a = oracle.squeezed_pgf_taylor(r, y0, 8)
        ref = [sum(P[n] * math.comb(n, j) * y0 ** (n - j) for n in range(j, 400)) for j in range(9)]
        assert np.abs(a - ref).max() < 1e-13


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_distinguishable_ones_matches_the_generic_oracle(M):
    # sources each in their own internal mode through a lossy interferometer: the positive
    # subset sum against the generic oracle's unfolded table (one group per detector)
    rng = np.random.default_rng(40 + M)
    r = rng.uniform(0.3, 0.8, M)
    T = np.sqrt(rng.uniform(0.4, 0.9, M))[:, None] * synth.haar_unitary(M, rng)
    prob = synth.Problem(M, M, np.diag(r), T, np.arange(M, dtype=np.int32), np.full(M, 1, np.int32))
    table = oracle.binned(prob, radix=np.full(M, 48 if M <= 3 else 28))["P"]
    assert abs(oracle.distinguishable_ones(r, T) - table[(1,) * M]) < 1e-12 * max(1.0, M)
