"""The total photon-number distribution by the power series of App. A
(gbsbin_total_photon_series, host FP64, no GPU): closed forms for a lossless squeezed mode
and a lossy coherent state, the oracle's unfolded one-group table, and the totals of a
two-group oracle table (the series ignores the grouping)."""
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


def _one_mode(r, alpha=None, eta=1.0):
    return synth.Problem(1, 1, np.array([[r]]), np.array([[np.sqrt(eta)]], complex), np.zeros(1, np.int32),
                         np.array([5], np.int32), alpha=None if alpha is None else np.array([[alpha]], complex))


def test_squeezed_vacuum_and_lossy_coherent(gb):
    # lossless single-mode squeezed vacuum: Pr(2k) = tanh(r)^(2k) (2k)! / (4^k k!^2 cosh r), odd
    # counts vanish; coherent state through loss eta: Poisson with mean eta |alpha|^2
    r = 0.7
    P = gb.gbsbin_total_photon_series(_one_mode(r), 20)
    ref = np.zeros(21)
    for k in range(11):
        ref[2 * k] = math.tanh(r) ** (2 * k) * math.factorial(2 * k) / (4 ** k * math.factorial(k) ** 2) / math.cosh(r)
    assert np.abs(P - ref).max() < 1e-14
    a, eta = 0.9 - 0.4j, 0.6
    lam = eta * abs(a) ** 2
    P = gb.gbsbin_total_photon_series(_one_mode(0.0, a, eta), 15)
    ref = np.array([math.exp(-lam) * lam ** k / math.factorial(k) for k in range(16)])
    assert np.abs(P - ref).max() < 1e-15


@pytest.mark.parametrize("M,K,disp,basis", [(4, 1, True, False), (3, 2, False, True), (5, 1, True, False)])
def test_against_unfolded_one_group_table(gb, M, K, disp, basis):
    rng = np.random.default_rng(990 + M + K)
    prob = synth.random_problem(rng, M, K, 1, 6, displaced=disp, internal_basis=basis, r_range=(0.2, 0.6))
    N = 12
    ref = oracle.binned(prob, radix=np.array([64]))["P"][:N + 1]       # tail beyond 63 < 1e-16
    P = gb.gbsbin_total_photon_series(prob, N)
    assert np.abs(P - ref).max() < 1e-13, np.abs(P - ref).max()


def test_grouping_is_ignored(gb):
    rng = np.random.default_rng(999)
    prob = synth.random_problem(rng, 4, 1, 2, 5, displaced=True, r_range=(0.2, 0.5))
    T = oracle.binned(prob, radix=np.array([32, 32]))["P"]
    tot = np.zeros(T.shape[0] + T.shape[1] - 1)
    for b in np.ndindex(*T.shape):
        tot[sum(b)] += T[b]
    P = gb.gbsbin_total_photon_series(prob, 10)
    assert np.abs(P - tot[:11]).max() < 1e-13


def test_rejects_bad_input(gb):
    with pytest.raises(gb.GbsbinError):
        gb.gbsbin_total_photon_series(_one_mode(0.5), -1)
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_total_photon_series(_one_mode(0.5), (1 << 20) + 1)
    assert e.value.status == 8


@pytest.mark.parametrize("M,K", [(60, 1), (32, 2)], ids=["n120", "n128_internal"])
def test_large_states_on_the_threaded_host_algebra(gb, M, K):
    # n >= 96 runs the blocked, threaded Cholesky, triangular inverse and Gram product of the
    # host state algebra; the series it feeds matches the oracle's unfolded one-group table,
    # with the library's thread count and with one thread (bit-identical: every entry is
    # summed in the same order whatever the thread count)
    import subprocess
    import sys
    rng = np.random.default_rng(960 + M)
    prob = synth.random_problem(rng, M, K, 1, 12, displaced=True, internal_basis=K > 1, r_range=(0.1, 0.3),
                                eta_range=(0.2, 0.4))
    P = gb.gbsbin_total_photon_series(prob, 12)
    ref = oracle.binned(prob, radix=[64])["P"][:13]
    assert np.abs(P - ref).max() < 1e-12, np.abs(P - ref).max()
    code = ("import sys, numpy as np; sys.path[:0] = sys.argv[1:3]; import synth, paper_2412_17742_gb300 as gb; "
            f"p = synth.random_problem(np.random.default_rng({960 + M}), {M}, {K}, 1, 12, displaced=True, "
            f"internal_basis={K > 1}, r_range=(0.1, 0.3), eta_range=(0.2, 0.4)); "
            "sys.stdout.write(gb.gbsbin_total_photon_series(p, 12).tobytes().hex())")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code, root, os.path.join(root, "tests")], check=True,
                         capture_output=True, text=True, env=dict(os.environ, GBSBIN_HOST_THREADS="1")).stdout
    assert np.array_equal(np.frombuffer(bytes.fromhex(out), dtype=np.float64), P)
