"""Fine-grained Pr(n) of fully distinguishable states by App. D's finite differences with
rank-2 blocks (gbsbin_prob_distinguishable, host FP64, no GPU): the single squeezed mode's
closed form, patterns of a lossy three-source state against the oracle's fine-grained table
(one group per detector), and the structures it must reject."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def gb():
    import paper_2412_17742_gb300 as gb
    try:
        gb.load()
    except RuntimeError:
        pytest.skip("library not built")
    return gb


def _distinguishable(rng, M, cut, eta=(0.4, 0.9), r=(0.3, 0.7)):
    # source i squeezed in internal mode i only (K = M, aligned internal bases): every
    # internal mode carries one source
    rr = np.diag(rng.uniform(*r, M))
    T = np.sqrt(rng.uniform(*eta, M))[:, None] * synth.haar_unitary(M, rng)
    return synth.Problem(M, M, rr, T, np.arange(M, dtype=np.int32), np.full(M, cut, np.int32))


def test_single_squeezed_mode(gb):
    r = 0.8
    prob = synth.Problem(1, 1, np.array([[r]]), np.array([[1.0 + 0j]]), np.zeros(1, np.int32),
                         np.array([6], np.int32))
    for n in range(7):
        ref = 0.0 if n % 2 else (math.tanh(r) ** n * math.factorial(n)
                                 / (2 ** n * math.factorial(n // 2) ** 2) / math.cosh(r))
        assert abs(gb.gbsbin_prob_distinguishable(prob, [n]) - ref) < 1e-15


@pytest.mark.parametrize("seed", [1, 2])
def test_against_the_oracle_fine_grained_table(gb, seed):
    rng = np.random.default_rng(1400 + seed)
    M, cut = 3, 3
    prob = _distinguishable(rng, M, cut)
    table = oracle.binned(prob, radix=np.full(M, 32))["P"]       # one group per detector; 32 bins: unfolded to 1e-15
    for n in itertools.product(range(cut + 1), repeat=M):
        if sum(n) > 6:
            continue
        got = gb.gbsbin_prob_distinguishable(prob, list(n))
        assert abs(got - table[n]) < 1e-12, (n, got, table[n])


def test_gray_order_beyond_the_recompute_period(gb):
    # 6^4 = 1296 evaluation points: the incremental trace / norm updates run past the
    # recompute after 1024 points.  Each value lies within its own rounding-error estimate of
    # an unfolded oracle table (40 bins per detector), and a 20-photon pattern whose
    # alternating sum keeps fewer than three digits reports GBSBIN_ERR_PRECISION
    rng = np.random.default_rng(1600)
    prob = _distinguishable(rng, 4, 5, r=(0.6, 0.9))
    table = oracle.binned(prob, radix=np.full(4, 40))["P"]
    for n in [(5, 4, 3, 5), (2, 5, 5, 1), (2, 2, 2, 2)]:
        v, err = gb.gbsbin_prob_distinguishable(prob, list(n), with_error=True)
        assert err < 1e-3 * v and abs(v - table[n]) <= err + 1e-15, (n, v, err, table[n])
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable(prob, [5, 5, 5, 5])
    assert e.value.status == 10 and abs(e.value.value - table[5, 5, 5, 5]) <= e.value.abs_err


def test_cancelled_sum_is_flagged(gb):
    # 5^8 evaluation points, 32 photons: the alternating sum loses every digit (its rounded
    # value is even negative); the call says so instead of returning a probability
    big = _distinguishable(np.random.default_rng(1700), 8, 4, r=(0.2, 0.4))
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable(big, [4] * 8)
    assert e.value.status == 10 and abs(e.value.value) <= e.value.abs_err


def _m16_all_ones():
    rng = np.random.default_rng(1700)
    M = 16
    r = rng.uniform(0.5, 0.9, M)
    T = np.sqrt(rng.uniform(0.4, 0.9, M))[:, None] * synth.haar_unitary(M, rng)
    return synth.Problem(M, M, np.diag(r), T, np.arange(M, dtype=np.int32), np.full(M, 1, np.int32)), r, T


def test_ones_pattern_against_the_independent_sum(gb):
    # 16 sources, one photon per detector (2^16 evaluation points): App. D's alternating sum
    # against the positive subset sum of the sources' closed-form output distributions
    prob, r, T = _m16_all_ones()
    ref = oracle.distinguishable_ones(r, T)
    v, err = gb.gbsbin_prob_distinguishable(prob, [1] * 16, with_error=True)
    assert abs(v - ref) <= err and err < 1e-4 * ref, (v, ref, err)


def test_rejects_other_structures(gb):
    rng = np.random.default_rng(1500)
    indist = synth.random_problem(rng, 3, 1, 3, 2)                 # one internal mode, three sources
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable(indist, [1, 0, 1])
    assert e.value.status == 8
    disp = synth.random_problem(rng, 2, 1, 2, 2, displaced=True)
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_prob_distinguishable(disp, [1, 1])
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_prob_distinguishable(_distinguishable(rng, 2, 2), [1, -1])
    with pytest.raises(gb.GbsbinError) as e:                         # (2^21)^2 > 2^40 points
        gb.gbsbin_prob_distinguishable(_distinguishable(rng, 2, 2), [1 << 21, 1 << 21])
    assert e.value.status == 8
