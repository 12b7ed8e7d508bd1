"""The inverse DFT (Sec. VI's coefficient extraction on the roots-of-unity grid) in its
two-phase form, taken for grids of three or more axes whose leading and trailing axis
blocks fit a CTA's shared memory (one grid barrier instead of one per axis): tables
against the oracle for every source of G the transform has (G written by the tree's
leaves, log q finished from the pivot records, log q per point, shards), on grids with
uneven radices, an even last radix (its self-conjugate column) and three axes."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _table(gb, prob, precision, tile=0):
    with gb.Plan(prob, precision=precision, tile_override=tile) as p:
        P = p.table().cpu().numpy()
        st, d = p.diagnostics()
    assert st == 0 and d["n_bad_points"] == 0
    return P, d


GRIDS = [
    # (name, problem): every one takes the two-phase form
    ("l4_radix9", lambda: synth.config(1)),
    ("l4_uneven_even_last", lambda: synth.random_problem(np.random.default_rng(601), 8, 1, 4, [8, 6, 7, 9],
                                                         displaced=True)),
    ("l3_long_first_axis", lambda: synth.random_problem(np.random.default_rng(602), 6, 1, 3, [40, 9, 9])),
]
# (precision, tile override): the trees (G from the leaves when undisplaced, else log q
# finished from the pivot records), the warp kernel (log q finished from its unfinished
# form) and the shared-memory FP64 kernel (log q per point)
PATHS = [(1, 0), (0, 0), (1, 5), (0, 1)]


@pytest.mark.parametrize("precision,tile", PATHS, ids=["tree_df32", "tree_fp64", "warp", "smem_fp64"])
@pytest.mark.parametrize("name,make", GRIDS, ids=[g[0] for g in GRIDS])
def test_two_phase_dft_tables(cuda_lib, name, make, precision, tile):
    prob = make()
    if tile == 5 and prob.n > 32:
        pytest.skip("warp kernel: n <= 32")
    P, d = _table(cuda_lib, prob, precision, tile)
    ref = oracle.binned(prob)
    sl = tuple(slice(0, int(c) + 1) for c in prob.cutoff)
    assert np.abs(P - ref["P"][sl]).max() < TOL
    assert abs(d["sum_P"] - 1.0) < 1e-12
    assert abs(d["log_q1_re"] - ref["logq"][0].real) < 1e-10
