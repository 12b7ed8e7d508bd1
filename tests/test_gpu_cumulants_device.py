"""Cumulants of orders 1-4 of the binned counts on the GPU (gbsbin_cumulants_device, Sec. VI
coarse-grained moments and cumulants; FP64, and the products in pairs of FP32) against textbook
single-mode results, the central moments of the oracle's unfolded tables, and the host
evaluators at the library's sizes."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_17742_gb300 as gb
    gb.load()
    return gb


def _one_mode(r, alpha=None, eta=1.0):
    return synth.Problem(1, 1, np.array([[r]]), np.array([[np.sqrt(eta)]], complex), np.zeros(1, np.int32),
                         np.array([5], np.int32), alpha=None if alpha is None else np.array([[alpha]], complex))


def test_single_modes(gb):
    # squeezed vacuum, s = sinh^2 r: mean s, variance 2 s (1 + s), third 4 s + 12 s^2 + 8 s^3,
    # fourth 8 s (1 + s)(1 + 6 s + 6 s^2) (derivatives of -1/2 log(1 + s - s e^{2t})); a coherent
    # state is Poisson: every cumulant is |alpha|^2
    r = 0.6
    s = np.sinh(r) ** 2
    k1, k2, k3, k4 = gb.gbsbin_cumulants_device(_one_mode(r))
    assert abs(k1[0] - s) < 1e-14
    assert abs(k2[0, 0] - 2 * s * (1 + s)) < 1e-13
    assert abs(k3[0, 0, 0] - (4 * s + 12 * s * s + 8 * s ** 3)) < 1e-12
    assert abs(k4[0, 0, 0, 0] - 8 * s * (1 + s) * (1 + 6 * s + 6 * s * s)) < 1e-11
    a = 0.7 + 0.5j
    for k in gb.gbsbin_cumulants_device(_one_mode(0.0, a)):
        assert abs(k.flat[0] - abs(a) ** 2) < 1e-13


def _central(P):
    grids = np.meshgrid(*[np.arange(sz) for sz in P.shape], indexing="ij")
    mu = np.array([(P * g).sum() for g in grids])
    return mu, [g - m for g, m in zip(grids, mu)]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("M,K,L,cut,disp,basis", [(4, 1, 2, 6, True, False), (3, 2, 2, 5, False, True),
                                                  (3, 1, 3, 4, True, False), (4, 1, 4, 3, True, False)])
def test_against_unfolded_tables(gb, M, K, L, cut, disp, basis, precision):
    # the cumulants are the central-moment combinations of the oracle's unfolded table:
    # kappa_ij = mu_ij, kappa_ijk = mu_ijk, kappa_ijkl = mu_ijkl - mu_ij mu_kl - mu_ik mu_jl - mu_il mu_jk
    rng = np.random.default_rng(970 + M + K + L)
    prob = synth.random_problem(rng, M, K, L, cut, displaced=disp, internal_basis=basis, r_range=(0.1, 0.4))
    k1, k2, k3, k4 = gb.gbsbin_cumulants_device(prob, precision=precision)
    over = 6 if L <= 3 else 5
    P = oracle.binned(prob, radix=prob.radix * over)["P"]
    mu, d = _central(P)
    c2 = np.array([[(P * d[i] * d[j]).sum() for j in range(L)] for i in range(L)])
    c3 = np.zeros((L,) * 3)
    c4 = np.zeros((L,) * 4)
    for i, j, k in np.ndindex(*(L,) * 3):
        c3[i, j, k] = (P * d[i] * d[j] * d[k]).sum()
    for i, j, k, l in np.ndindex(*(L,) * 4):
        c4[i, j, k, l] = ((P * d[i] * d[j] * d[k] * d[l]).sum()
                          - c2[i, j] * c2[k, l] - c2[i, k] * c2[j, l] - c2[i, l] * c2[j, k])
    assert np.abs(k1 - mu).max() < 1e-10
    assert np.abs(k2 - c2).max() < 1e-9
    assert np.abs(k3 - c3).max() < 1e-8
    assert np.abs(k4 - c4).max() < 1e-8 * max(1.0, np.abs(k4).max())
    for perm in [(1, 0, 2, 3), (0, 2, 1, 3), (0, 1, 3, 2), (3, 1, 2, 0)]:
        assert np.abs(k4 - k4.transpose(perm)).max() < 1e-12 * max(1.0, np.abs(k4).max())


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("case", ["n192", "ragged"])
def test_library_sizes_match_host(gb, case, precision):
    # the n = 192 workload (24 ports x 4 internal modes, three groups of 64 rows) and a ragged
    # n = 152 case (five groups of uneven size, a last 32-pivot block of 24 rows) against the
    # host evaluators (an FP64 Gauss-Jordan inverse and plain loops), relative to each tensor's
    # largest entry
    if case == "n192":
        prob = synth.config(2)
    else:
        rng = np.random.default_rng(4242)
        prob = synth.random_problem(rng, 38, 2, 5, 3, displaced=True, internal_basis=True, r_range=(0.4, 1.0))
        prob.bin_of_mode = np.array(rng.permutation(np.arange(38) % 5), np.int32)
    outs = gb.gbsbin_cumulants_device(prob, precision=precision)
    mean, cov = gb.gbsbin_moments(prob)
    host = [mean, cov, gb.gbsbin_cumulants3(prob), gb.gbsbin_cumulants4(prob)]
    for r, (dev, ref) in enumerate(zip(outs, host), start=1):
        scale = np.abs(ref).max()
        assert np.abs(dev - ref).max() < 1e-11 * scale, (r, np.abs(dev - ref).max(), scale)


def test_lower_orders_only(gb):
    # order 2 runs neither the Y_b products nor C_3 / C_4, and gives the same first two tensors
    prob = synth.config(1)
    m2, c2 = gb.gbsbin_cumulants_device(prob, order=2)
    m4, c4, _, _ = gb.gbsbin_cumulants_device(prob, order=4)
    assert np.array_equal(m2, m4) and np.array_equal(c2, c4)


def test_largest_matrix(gb):
    # n = 512 (M = 256, one internal mode), eight groups: finite, symmetric tensors whose means
    # match the closed form sum_{j in group} (Sigma^(1)_jj + |zbar_j|^2)
    from oracle import state
    rng = np.random.default_rng(77)
    prob = synth.random_problem(rng, 256, 1, 8, 2, displaced=True, r_range=(0.3, 0.9))
    (k1, k2, k3, k4), ms = gb.gbsbin_cumulants_device(prob, with_time=True)
    s1, zbar = state.sigma1_zbar(prob)
    labels = np.asarray(prob.bin_of_mode)
    expect = np.array([sum((s1[i, i] + abs(zbar[i]) ** 2).real for i in range(256) if labels[i] == l)
                       for l in range(8)])
    assert np.abs(k1 - expect).max() < 1e-10 * expect.max()
    assert np.all(np.isfinite(k4)) and ms > 0
    assert np.abs(k2 - k2.T).max() < 1e-12 * np.abs(k2).max()
    assert np.abs(k3 - k3.transpose(2, 0, 1)).max() < 1e-12 * np.abs(k3).max()
    assert np.all(np.linalg.eigvalsh(k2) > 0)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
def test_sixteen_groups_match_host(gb, precision):
    # the largest group count (L = 16, one port per group, n = 32): every coefficient launch and
    # the chain rule at their largest grids, against the host evaluators
    rng = np.random.default_rng(4343)
    prob = synth.random_problem(rng, 16, 1, 16, 2, displaced=True, r_range=(0.3, 0.8))
    prob.bin_of_mode = np.arange(16, dtype=np.int32)
    outs = gb.gbsbin_cumulants_device(prob, precision=precision)
    mean, cov = gb.gbsbin_moments(prob)
    host = [mean, cov, gb.gbsbin_cumulants3(prob), gb.gbsbin_cumulants4(prob)]
    for r, (dev, ref) in enumerate(zip(outs, host), start=1):
        assert dev.shape == (16,) * r
        assert np.abs(dev - ref).max() < 1e-11 * np.abs(ref).max(), (r, np.abs(dev - ref).max())


def test_rejects_other_precisions(gb):
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_cumulants_device(_one_mode(0.5), precision=2)
    assert e.value.status == 1
