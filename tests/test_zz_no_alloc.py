"""The allocation-free table entry point (for callers that must not call cudaMalloc, e.g.
under another framework's device-memory pool or in loops that cannot afford the device
synchronisation an allocation implies) gives the same table as gbsbin_execute.

Kept in its own file, collected last, so a run that stops at the first failure has run
every other test first.  It must pass alone in a fresh process and after the others."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _reference_and_logq(gb, prob, precision, oversample):
    with gb.Plan(prob, precision=precision, oversample=oversample) as p:
        ref = p.table().cpu().numpy()
        st, d = p.diagnostics()
        lq, _ = gb.gbsbin_read_points(p.handle, d["n_evaluated"])
    assert st == 0
    return ref, lq


def test_noalloc_table_matches_execute_twice(cuda_lib):
    import torch
    gb = cuda_lib
    cases = [
        (synth.config(1), 0, 1),
        (synth.random_problem(np.random.default_rng(301), 6, 2, 3, [4, 5, 3], displaced=True,
                              internal_basis=True), 1, 2),
    ]
    for prob, precision, over in cases:     # two calls in a row, different grids
        ref, lq = _reference_and_logq(gb, prob, precision, over)
        lq_dev = torch.from_numpy(lq.view(np.float64).copy()).cuda()
        out = torch.full(ref.shape, float("nan"), dtype=torch.float64, device="cuda")
        gb.gbsbin_table_from_logq_noalloc(prob.cutoff, over, lq_dev, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10


def test_noalloc_rejects_grids_beyond_its_scratch(cuda_lib):
    import torch
    gb = cuda_lib
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_table_from_logq_noalloc([600, 600], 1, dummy, dummy)   # 601 * 301 > 2^17 points
    assert e.value.status == 8
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_table_from_logq_noalloc([20000], 1, dummy, dummy)      # twiddles > 2^14
    assert e.value.status == 8

