"""Pins of the Fock-input oracle (App. C) against definitions and closed forms (no GPU).

The generating-function table is tied to: the Hafnian definition of the density-matrix
diagonal (Eq. density_matrix_fock_circuit) summed over compatible patterns; the permanent
form (Eq. probs_fock_circuit) as a second, independent definition; a second generating-
function route (Ryser's permanent of B(z)); and closed forms - Hong-Ou-Mandel
interference, binomial totals under uniform loss, one mode, the per-group mean.  A dropped
weight, a transposed T, a wrong conjugation or an aliased extraction fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import fock


def _prob(M, T, photons, labels, cutoff):
    labels = np.asarray(labels, dtype=np.int32)
    L = int(labels.max()) + 1
    cut = np.array(np.broadcast_to(np.asarray(cutoff, dtype=np.int32), (L,)), dtype=np.int32)
    return synth.FockProblem(M, np.asarray(T, dtype=np.complex128), np.asarray(photons, dtype=np.int32),
                             labels, cut)


# ------------------------------------------------------------ Hafnian and permanent
def test_hafnian_and_permanent_counts():
    for m in range(1, 5):   # haf(J - I) on 2m vertices = (2m - 1)!!
        assert abs(fock.hafnian(np.ones((2 * m, 2 * m)) - np.eye(2 * m)) - math.prod(range(2 * m - 1, 0, -2))) < 1e-9
    assert fock.hafnian(np.ones((3, 3))) == 0
    for m in range(0, 7):   # perm(J) = m!
        assert abs(fock.permanent(np.ones((m, m))) - math.factorial(m)) < 1e-6
    rng = np.random.default_rng(2)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    brute = sum(np.prod([A[i, s[i]] for i in range(4)]) for s in itertools.permutations(range(4)))
    assert abs(fock.permanent(A) - brute) < 1e-12
    a = rng.standard_normal((4, 4))
    a = a + a.T
    by_hand = a[0, 1] * a[2, 3] + a[0, 2] * a[1, 3] + a[0, 3] * a[1, 2]
    assert abs(fock.hafnian(a) - by_hand) < 1e-12


def test_loss_channel_matrix_symmetric():
    rng = np.random.default_rng(4)
    T = 0.8 * synth.haar_unitary(3, rng)
    A = fock.loss_channel_matrix(T)
    assert A.shape == (12, 12)
    assert np.abs(A - A.T).max() < 1e-15


# ------------------------------------------------------------ the two definitions
@pytest.mark.parametrize("photons", [[1, 1, 0], [2, 0, 1], [1, 1, 1]])
def test_haf_and_perm_definitions_agree_and_normalise(photons):
    rng = np.random.default_rng(11 + sum(photons))
    fp = synth.random_fock_problem(rng, 3, photons, 1, sum(photons))
    N = fp.N
    tot_h = tot_p = 0.0
    for n in itertools.product(range(N + 1), repeat=3):
        if sum(n) > N:
            continue
        h = fock.density_diag_haf(fp.T, photons, n)
        p = fock.density_diag_perm(fp.T, photons, n)
        assert abs(h - p) < 1e-14
        assert h > -1e-15
        tot_h += h
        tot_p += p
    assert abs(tot_h - 1.0) < 1e-13 and abs(tot_p - 1.0) < 1e-13


def test_more_photons_than_detected_vanish():
    # a pattern with more output photons than inputs has zero probability
    rng = np.random.default_rng(5)
    fp = synth.random_fock_problem(rng, 2, [1, 1], 1, 2)
    assert abs(fock.density_diag_haf(fp.T, [1, 1], (2, 1))) < 1e-15


# ------------------------------------------------------------ generating function
@pytest.mark.parametrize("photons,L", [([1, 2, 0], 2), ([1, 1, 1], 3), ([0, 3, 0], 1), ([1, 0, 1, 1], 2)])
def test_table_matches_definition(photons, L):
    rng = np.random.default_rng(100 + 7 * L + len(photons))
    fp = synth.random_fock_problem(rng, len(photons), photons, L, sum(photons), shuffle_bins=True)
    brute = fock.binned_brute_force(fp)
    t = fock.table(fp)
    assert np.abs(t["P"] - brute).max() < 1e-13
    assert abs(t["P"].sum() - 1.0) < 1e-13
    assert t["imag_max"] < 1e-13


def test_table_matches_permanent_definition_larger():
    rng = np.random.default_rng(21)
    fp = synth.random_fock_problem(rng, 4, [2, 1, 0, 2], 2, 5)
    brute = fock.binned_brute_force(fp, fock.density_diag_perm)
    assert np.abs(fock.table(fp)["P"] - brute).max() < 1e-13


def test_folded_table_is_folded_brute_force():
    rng = np.random.default_rng(31)
    fp = synth.random_fock_problem(rng, 3, [1, 1, 1], 2, 1)          # N_l = 1 < N = 3
    full = fock.binned_brute_force(fp)                                # b_l in [0, 3]
    folded = np.zeros((2, 2))
    for b in itertools.product(range(4), repeat=2):
        folded[b[0] % 2, b[1] % 2] += full[b]
    assert np.abs(fock.table(fp)["P"] - folded).max() < 1e-13


@pytest.mark.parametrize("photons", [[3, 1, 2, 0, 1], [1, 1, 1, 1, 1, 1], [2, 2, 0, 0, 4]])
def test_two_generating_function_routes_agree(photons):
    # Ryser's permanent of B(z)[p, p] against the roots-of-unity extraction, on and off the
    # unit circle (the extraction is exact for any z: it only uses homogeneity in x)
    rng = np.random.default_rng(41 + len(photons))
    M = len(photons)
    fp = synth.random_fock_problem(rng, M, photons, 3, 2)
    nodes = fock.extraction_nodes(photons)
    for trial in range(4):
        rad = 1.0 if trial < 2 else 0.7
        z = rad * np.exp(2j * np.pi * rng.uniform(size=3))
        a = fock.pgf_permanent(fp, z)
        b = fock.pgf_extract(fp, z, nodes)
        assert abs(a - b) < 1e-13 * max(1.0, abs(a))


def test_extraction_nodes_hold_smallest_input():
    J, k0, others, X, W = fock.extraction_nodes([3, 0, 1, 2])
    assert J == [0, 2, 3] and k0 == 2 and others == [0, 3]
    assert X.shape == (4 * 3, 3) and np.all(X[:, 1] == 1.0)
    assert np.abs(W - X[:, 0] * X[:, 2]).max() < 1e-15
    J, k0, _, X, W = fock.extraction_nodes([0, 0])
    assert J == [] and k0 is None and X.shape == (1, 0)


# ------------------------------------------------------------ closed forms
def test_hong_ou_mandel():
    phi = 0.37
    T = np.array([[1.0, np.exp(1j * phi)], [1.0, -np.exp(1j * phi)]]) / np.sqrt(2.0)
    fp = _prob(2, T, [1, 1], [0, 1], 2)
    P = fock.table(fp)["P"]
    assert abs(P[1, 1]) < 1e-15
    assert abs(P[2, 0] - 0.5) < 1e-15 and abs(P[0, 2] - 0.5) < 1e-15
    # lossy arms: eta each; P(1,1) still 0 (balanced), one photon lost 2 eta (1 - eta)
    eta = 0.6
    fp = _prob(2, np.sqrt(eta) * T, [1, 1], [0, 1], 2)
    P = fock.table(fp)["P"]
    assert abs(P[1, 1]) < 1e-15
    assert abs(P[1, 0] + P[0, 1] - 2 * eta * (1 - eta)) < 1e-15
    assert abs(P[0, 0] - (1 - eta) ** 2) < 1e-15


@pytest.mark.parametrize("photons", [[2, 1, 1, 1, 0], [1, 1, 1, 1, 1]])
def test_uniform_loss_total_is_binomial(photons):
    # T^dag T = eta I: every photon survives independently whatever the interference
    rng = np.random.default_rng(61)
    eta = 0.55
    M = len(photons)
    fp = _prob(M, np.sqrt(eta) * synth.haar_unitary(M, rng), photons, [0] * M, sum(photons))
    N = fp.N
    P = fock.table(fp)["P"]
    ref = [math.comb(N, k) * eta ** k * (1 - eta) ** (N - k) for k in range(N + 1)]
    assert np.abs(P - ref).max() < 1e-14


def test_single_mode_is_binomial():
    eta = 0.3
    fp = _prob(1, [[np.sqrt(eta) * np.exp(0.9j)]], [4], [0], 4)
    P = fock.table(fp)["P"]
    ref = [math.comb(4, k) * eta ** k * (1 - eta) ** (4 - k) for k in range(5)]
    assert np.abs(P - ref).max() < 1e-15


def test_group_means():
    rng = np.random.default_rng(71)
    fp = synth.random_fock_problem(rng, 6, [1, 0, 2, 1, 0, 1], 3, 5, shuffle_bins=True)
    P = fock.table(fp)["P"]
    means = [sum(b[l] * P[b] for b in itertools.product(range(6), repeat=3)) for l in range(3)]
    assert np.abs(np.array(means) - fock.group_means(fp)).max() < 1e-13


def test_vacuum_input():
    rng = np.random.default_rng(81)
    fp = synth.random_fock_problem(rng, 3, [0, 0, 0], 2, 2)
    P = fock.table(fp)["P"]
    assert P[0, 0] == pytest.approx(1.0, abs=1e-15) and np.abs(P).sum() == pytest.approx(1.0, abs=1e-14)


def test_gray_code_walks_every_node_once_one_digit_at_a_time():
    radices = [3, 2, 4]
    seen = []
    prev = None
    for i in range(24):
        g = fock.gray_digits(i, radices)
        assert all(0 <= d < R for d, R in zip(g, radices))
        if prev is not None:
            diff = [abs(a - b) for a, b in zip(g, prev)]
            assert sorted(diff) == [0, 0, 1]
        seen.append(tuple(g))
        prev = g
    assert len(set(seen)) == 24


def test_node_shards_sum_to_the_table():
    rng = np.random.default_rng(91)
    fp = synth.random_fock_problem(rng, 5, [1, 2, 0, 1, 1], 2, 5)
    S = fock.node_count(fp.photons)
    assert S == 3 * 2 * 2
    full = fock.table(fp)["P"]
    parts = [fock.table(fp, node_range=(b, e))["P"] for b, e in [(0, 5), (5, 6), (6, 12)]]
    assert np.abs(sum(parts) - full).max() < 1e-15
