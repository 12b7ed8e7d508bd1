"""Heralded states (Sec. VII) on the GPU against the oracle's generating-function route
(``oracle.herald.table``, itself pinned against the definition and the paper's printed
Fock-state fidelities): whole tables element by element, the heralding probabilities, the
fidelities of Sec. VIII from the GPU's own states, and diagnostics."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import herald
from test_herald_oracle import CASES, FOCK_ROLES, GOLDEN, fock_setup

pytestmark = pytest.mark.gpu


def _compare(gb, prob, roles, cutoff, cut, oversample, tol=1e-12):
    rho_ref, pr_ref = herald.table(prob, roles, cutoff, cut, oversample=oversample)
    with gb.HeraldPlan(prob, roles, cutoff, cut, oversample=oversample) as h:
        rho, pr = h.states()
        rho, pr = rho.cpu().numpy(), pr.cpu().numpy()
        d = h.diagnostics()
        assert d["status"] == 0 and d["n_bad_points"] == 0 and d["kernel_name"] == "herald_fp64"
        assert d["min_pivot_re"] > 0 and d["launches"] == 1 + len(cutoff)
        assert d["sum_P"] == pytest.approx(float(pr.sum()), rel=1e-14, abs=1e-300)
        rho_h, pr_h = h.states_host()
    assert rho.shape == rho_ref.shape and pr.shape == pr_ref.shape
    assert np.abs(rho - rho_ref).max() <= tol, np.abs(rho - rho_ref).max()
    assert np.abs(pr - pr_ref).max() <= tol
    assert np.array_equal(rho, rho_h) and np.array_equal(pr, pr_h)
    return rho, pr


@pytest.mark.parametrize("name,make,roles,cutoff,cut", CASES, ids=[c[0] for c in CASES])
def test_herald_tables_match_oracle(cuda_lib, name, make, roles, cutoff, cut):
    _compare(cuda_lib, make(), roles, cutoff, cut, oversample=4)


def test_fock_heralding_fidelities_from_the_gpu(cuda_lib):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    cache = {}
    for p, eta, n, F in rows:
        key = (float(p), float(eta))
        if key not in cache:
            cache[key] = _compare(cuda_lib, fock_setup(*key), FOCK_ROLES, [3], 15, oversample=16)
        rho, pr = cache[key]
        n = int(n)
        got = np.sqrt((rho[n, n, n] / pr[n]).real)
        digits = len(F.split(".")[1])
        assert abs(got - float(F)) <= 0.5 * 10.0 ** (-digits) + 1e-12, (p, eta, n, got, F)


def test_herald_large_state_ragged(cuda_lib):
    # 40 modes (n = 80): three heralding groups of uneven size and cutoff, two kept modes,
    # the rest traced; the elimination spans many 256-thread passes and a ragged tail
    rng = np.random.default_rng(806)
    prob = synth.random_problem(rng, 40, 1, 4, [1, 1, 1, 1], displaced=True)
    roles = [int(g) for g in rng.integers(0, 3, 40)]
    for m in range(3):
        roles[m] = m
    roles[10], roles[25] = -2, -2
    for m in (5, 17, 30, 31, 39):
        roles[m] = -1
    rho, pr = _compare(cuda_lib, prob, roles, [3, 1, 2], 4, oversample=1, tol=1e-11)
    # Hermitian per outcome: rho[b][u][v] = conj rho[b][v][u]
    R = rho.reshape(24, 25, 25)
    assert np.abs(R - np.conj(np.transpose(R, (0, 2, 1)))).max() < 1e-13


def test_herald_internal_modes_and_timing(cuda_lib):
    # two internal modes per port, grouped heralding over a port's both internal modes
    gb = cuda_lib
    rng = np.random.default_rng(807)
    prob = synth.random_problem(rng, 3, 2, 2, [2, 2], displaced=True, internal_basis=True)
    roles = [0, 0, 1, -1, -2, -2]
    _compare(gb, prob, roles, [2, 3], 3, oversample=2)
    with gb.HeraldPlan(prob, roles, [2, 3], 3, oversample=2, want_timing=True) as h:
        h.states()
        d = h.diagnostics()
        assert d["point_kernel_ms"] > 0 and d["n_points"] == 6 * 8 and d["n"] == 12
        assert d["log_q1_re"] == pytest.approx(-np.log(oracle.state.vacuum_probability(
            *oracle.state.adjacency(*oracle.state.sigma1_zbar(prob)))), rel=1e-12)
