"""The exact binned moments and cumulants (host FP64 algebra from the generating function's
derivatives at t = 0) against the same quantities read off the GPU's own tables: the large-matrix
tree at n = 96 and the small tree at n = 32, on grids large enough that the folded mass is
far below the bounds (an independent route: the roots-of-unity transform, not derivatives)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _central(P):
    L = P.ndim
    grids = np.meshgrid(*[np.arange(s) for s in P.shape], indexing="ij")
    mu = np.array([(P * g).sum() for g in grids])
    d = [g - m for g, m in zip(grids, mu)]
    cov = np.array([[(P * d[i] * d[j]).sum() for j in range(L)] for i in range(L)])
    k3 = np.array([[[(P * d[i] * d[j] * d[k]).sum() for k in range(L)] for j in range(L)] for i in range(L)])
    return mu, cov, k3


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("M,K,L,cut,over,kind", [(12, 4, 3, [24, 24, 24], 1, "btree"), (16, 1, 4, [16, 16, 16, 16], 1, "tree")],
                         ids=["n96_large_tree", "n32_small_tree"])
def test_moments_match_the_gpu_tables(cuda_lib, M, K, L, cut, over, kind, precision):
    gb = cuda_lib
    rng = np.random.default_rng(1201 + M)
    prob = synth.random_problem(rng, M, K, L, cut, displaced=True, internal_basis=K > 1, r_range=(0.1, 0.3),
                                eta_range=(0.3, 0.6))
    with gb.Plan(prob, precision=precision, oversample=over) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
    assert st == 0 and d["kernel_name"].startswith(kind), d["kernel_name"]
    # weak states on large grids: the mass folded back from beyond N_l is far below the bounds
    assert abs(P.sum() - 1.0) < 1e-12, 1.0 - P.sum()
    mu, cov, k3 = _central(P)
    m, c = gb.gbsbin_moments(prob)
    assert np.abs(m - mu).max() < 1e-9, (m, mu)
    assert np.abs(c - cov).max() < 1e-8
    assert np.abs(gb.gbsbin_cumulants3(prob) - k3).max() < 1e-7
