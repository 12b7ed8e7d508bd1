"""The reverse pass along the large-matrix tree (per parent the inverse of the leading groups'
block and its products, per evaluated point the inverse of the last group's Schur complement)
against the per-point reverse pass (one n x n inverse per evaluated point) on the same state,
and against central differences of the oracle along physical directions."""
import numpy as np
import pytest

import oracle
import synth
from oracle import state

pytestmark = pytest.mark.gpu


def _grads(gb, prob, pbar, precision, tile):
    import torch
    with gb.Plan(prob, precision=precision, want_backward=True, tile_override=tile, want_timing=True) as p:
        p.table()
        g = p.backward(torch.from_numpy(pbar).cuda(), want=("r", "T", "alpha", "V", "sigma1", "zbar"))
        st, d = p.diagnostics()
        assert st == 0 and d["backward_kernel_ms"] > 0
    return g, d


def _problem(seed, M, K, L, cutoff, bins=None, **kw):
    rng = np.random.default_rng(seed)
    p = synth.random_problem(rng, M, K, L, cutoff, **kw)
    if bins is not None:
        p.bin_of_mode = np.asarray(bins, np.int32)
    return p


CASES = [
    # n = 96, three displaced groups of 32 rows with internal bases, uneven cutoffs
    ("n96_l3_disp_basis", lambda: _problem(1101, 12, 4, 3, [3, 4, 5], displaced=True, internal_basis=True)),
    # n = 160, two groups of 60 + 100 rows (last group larger), even last radix
    ("n160_l2_uneven", lambda: _problem(1102, 80, 1, 2, [4, 5], bins=[0] * 30 + [1] * 50, displaced=True)),
    # n = 200, two undisplaced groups of 100, one parent per first-axis root
    ("n200_l2", lambda: _problem(1103, 100, 1, 2, [6, 6])),
    # n = 240, a last group of 140 rows: the forward's Householder reduction through L2
    ("n240_last_group_140_rows", lambda: _problem(1104, 120, 1, 2, [5, 9], bins=[0] * 50 + [1] * 70,
                                                  displaced=True, r_range=(0.2, 0.6))),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_tree_reverse_pass_matches_per_point(cuda_lib, name, make, precision):
    gb = cuda_lib
    prob = make()
    rng = np.random.default_rng(1110)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    gt, dt = _grads(gb, prob, pbar, precision, 0)
    gp, dp = _grads(gb, prob, pbar, precision, 6 if precision else 3)
    assert dt["kernel_name"].startswith("btree") and dt["backward_path"] == 2, (dt["kernel_name"], dt["backward_path"])
    assert dp["backward_path"] == 1
    for k in gt:
        scale = max(1.0, float(np.abs(gp[k]).max()))
        assert np.abs(gt[k] - gp[k]).max() < 1e-10 * scale, (name, k, np.abs(gt[k] - gp[k]).max(), scale)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
def test_tree_reverse_pass_in_two_waves(cuda_lib, precision):
    # n = 288 with 450 first-axis roots: the parents' buffers (1.34 MB each) exceed one wave's
    # 512 MB, so the parents run in two waves into the same partials
    gb = cuda_lib
    prob = _problem(1104, 144, 1, 2, [449, 5], bins=[0] * 88 + [1] * 56, r_range=(0.1, 0.3))
    rng = np.random.default_rng(1111)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    gt, dt = _grads(gb, prob, pbar, precision, 0)
    gp, dp = _grads(gb, prob, pbar, precision, 6 if precision else 3)
    assert dt["backward_path"] == 2 and dp["backward_path"] == 1
    for k in ("r", "T", "sigma1"):
        scale = max(1.0, float(np.abs(gp[k]).max()))
        assert np.abs(gt[k] - gp[k]).max() < 1e-10 * scale, (k, np.abs(gt[k] - gp[k]).max(), scale)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
def test_tree_device_adjoints_along_a_physical_direction(cuda_lib, precision):
    # the adjoints S = dL/dXA, s = dL/dgamma of the tree's reverse pass against central
    # differences of the oracle along a direction in the squeezings (three groups, displaced)
    import torch
    gb = cuda_lib
    prob = _problem(1105, 12, 4, 3, [2, 3, 4], displaced=True, internal_basis=True)
    rng = np.random.default_rng(1112)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    dr = rng.standard_normal(prob.r.shape)
    h = 1e-5

    def shifted(t):
        q = synth.Problem(prob.M, prob.K, prob.r + t * dr, prob.T.copy(), prob.bin_of_mode.copy(),
                          prob.cutoff.copy(), alpha=prob.alpha.copy(), V=prob.V.copy())
        return q
    adj = [state.adjacency(*state.sigma1_zbar(shifted(t))) for t in (h, -h)]
    dXA = (adj[0][0] - adj[1][0]) / (2 * h)
    dg = (adj[0][1] - adj[1][1]) / (2 * h)
    f = (float((oracle.binned(shifted(h))["P"] * pbar).sum()) -
         float((oracle.binned(shifted(-h))["P"] * pbar).sum())) / (2 * h)
    with gb.Plan(prob, precision=precision, want_backward=True) as p:
        p.table()
        st, d = p.diagnostics()
        assert d["backward_path"] == 2
        S, s = p.backward_device(torch.from_numpy(pbar).cuda())
        torch.cuda.synchronize()
    got = float(np.real(np.sum(S.cpu().numpy() * dXA) + np.sum(s.cpu().numpy() * dg)))
    assert abs(got - f) <= 1e-7 + 1e-6 * abs(f), (got, f)
