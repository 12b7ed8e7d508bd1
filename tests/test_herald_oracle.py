"""Pins of the heralded-state oracle (Sec. VII) against what the paper and the definition fix
(no GPU): the generating-function route against the brute-force sum of loop Hafnians of the
definition, Hermiticity, the trace against the binned table of the other oracle route, the
lossless two-mode squeezed vacuum (heralding n photons leaves |n> exactly) and the Fock-state
fidelities printed in Sec. VIII."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import herald

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fock_heralding_fidelities.txt")


def fock_setup(p, eta, xi=1.1):
    return synth.fock_heralding_source(p, eta, xi)


FOCK_ROLES = synth.FOCK_HERALD_ROLES


CASES = [
    # (name, problem, roles, heralding cutoffs, kept cutoff)
    ("one_group_traced", lambda: synth.random_problem(np.random.default_rng(801), 3, 1, 3, [2, 2, 2],
                                                      displaced=True), [0, -2, -1], [2], 3),
    ("two_groups_two_kept", lambda: synth.random_problem(np.random.default_rng(802), 4, 1, 4, [2, 2, 2, 2],
                                                         displaced=True), [0, 1, -2, -2], [1, 2], 2),
    ("grouped_internal", lambda: synth.random_problem(np.random.default_rng(803), 2, 2, 2, [2, 2],
                                                      displaced=True, internal_basis=True), [0, 0, -2, -1], [2], 3),
]


@pytest.mark.parametrize("name,make,roles,cutoff,cut", CASES, ids=[c[0] for c in CASES])
def test_table_matches_the_definition(name, make, roles, cutoff, cut):
    prob = make()
    rho, _ = herald.table(prob, roles, cutoff, cut, oversample=12)
    nk = sum(1 for r in roles if r == -2)
    rng = np.random.default_rng(11)
    for _ in range(6):
        b = [int(rng.integers(0, c + 1)) for c in cutoff]
        u = [int(rng.integers(0, cut + 1)) for _ in range(nk)]
        v = [int(rng.integers(0, cut + 1)) for _ in range(nk)]
        ref = herald.brute(prob, roles, b, u, v, tmax=18)
        got = rho[tuple(b) + tuple(u) + tuple(v)]
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (name, b, u, v, got, ref)


def test_hermitian_and_trace():
    prob = synth.random_problem(np.random.default_rng(804), 3, 1, 3, [2, 2, 2], displaced=True)
    roles = [0, -2, -1]
    rho, prb = herald.table(prob, roles, [2], 24, oversample=12)
    for b in range(3):
        assert np.abs(rho[b] - rho[b].conj().T).max() < 1e-13
        # Tr over the kept mode = Pr(b) of the binned oracle route (mode 0 its own group, the
        # rest one group summed out on a large grid)
        assert abs(np.trace(rho[b]).real - prb[b]) < 1e-9
    two = synth.Problem(prob.M, prob.K, prob.r, prob.T, np.array([0, 1, 1], np.int32), np.array([2, 2], np.int32),
                        alpha=prob.alpha)
    P = oracle.binned(two, radix=[36, 72])["P"]
    for b in range(3):
        assert abs(P[b].sum() - prb[b]) < 1e-12


def test_lossless_two_mode_squeezed_vacuum_heralds_fock_states():
    rho, prb = herald.table(fock_setup(1.0, 1.0), FOCK_ROLES, [4], 8, oversample=16)   # folding ~ tanh(1.1)^(2 R)
    for n in range(5):
        st = rho[n] / prb[n]
        expect = np.zeros_like(st)
        expect[n, n] = 1.0
        assert np.abs(st - expect).max() < 1e-12


def test_fock_heralding_fidelities_of_the_paper():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    cache = {}
    for p, eta, n, F in rows:
        key = (float(p), float(eta))
        if key not in cache:
            cache[key] = herald.table(fock_setup(*key), FOCK_ROLES, [3], 15, oversample=16)
        rho, prb = cache[key]
        n = int(n)
        got = np.sqrt((rho[n, n, n] / prb[n]).real)
        digits = len(F.split(".")[1])
        assert abs(got - float(F)) <= 0.5 * 10.0 ** (-digits) + 1e-12, (p, eta, n, got, F)
