"""App. D's fine-grained Pr(n) for fully distinguishable internal modes with the sum over the
evaluation points on the GPU (gbsbin_prob_distinguishable_device) against the host evaluator
(Gray-code order) and the oracle's fine-grained table."""
import itertools

import numpy as np
import pytest

import oracle
from test_distinguishable import _distinguishable

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2])
def test_device_matches_host_and_oracle(cuda_lib, seed):
    gb = cuda_lib
    rng = np.random.default_rng(1400 + seed)
    prob = _distinguishable(rng, 3, 3)
    table = oracle.binned(prob, radix=np.full(3, 32))["P"]
    for n in itertools.product(range(4), repeat=3):
        if sum(n) > 6:
            continue
        dev, de = gb.gbsbin_prob_distinguishable_device(prob, list(n), with_error=True)
        host = gb.gbsbin_prob_distinguishable(prob, list(n))
        assert abs(dev - host) <= 1e-14 * host + de and abs(dev - table[n]) < 1e-12, (n, dev, host, table[n])


def test_device_large_patterns(cuda_lib):
    gb = cuda_lib
    rng = np.random.default_rng(1600)
    prob = _distinguishable(rng, 4, 5, r=(0.6, 0.9))
    for n in [(5, 4, 3, 5), (2, 5, 5, 1)]:                          # 720 and 432 points
        dv, de = gb.gbsbin_prob_distinguishable_device(prob, list(n), with_error=True)
        hv, he = gb.gbsbin_prob_distinguishable(prob, list(n), with_error=True)
        assert abs(dv - hv) <= de + he, (n, dv, hv)
    # 5^8 = 390625 points, 32 photons: every thread walks several points of the grid-stride
    # loop, and the cancelled sum is flagged as on the host
    big = _distinguishable(np.random.default_rng(1700), 8, 4, r=(0.2, 0.4))
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable_device(big, [4] * 8)
    assert e.value.status == 10 and abs(e.value.value) <= e.value.abs_err
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable_device(prob, [20, 20, 20, 5])   # N = 65 > 64
    assert e.value.status == 8


def test_device_ones_pattern_against_the_independent_sum(cuda_lib):
    # 16 sources, one photon per detector: the device sum within its error estimate of the
    # positive subset sum, and of the host's Gray-code sum
    gb = cuda_lib
    from test_distinguishable import _m16_all_ones
    prob, r, T = _m16_all_ones()
    ref = oracle.distinguishable_ones(r, T)
    dv, de = gb.gbsbin_prob_distinguishable_device(prob, [1] * 16, with_error=True)
    hv, he = gb.gbsbin_prob_distinguishable(prob, [1] * 16, with_error=True)
    assert abs(dv - ref) <= de and abs(dv - hv) <= de + he, (dv, hv, ref, de)


def test_device_work_is_bounded(cuda_lib):
    # a sum whose estimated FP64 work is beyond ~30 s is refused before any launch
    gb = cuda_lib
    from test_distinguishable import _m16_all_ones
    prob, _, _ = _m16_all_ones()
    with pytest.raises(gb.GbsbinError) as e:                         # 4^16 points, ~6.5e13 operations
        gb.gbsbin_prob_distinguishable_device(prob, [3] * 16)
    assert e.value.status == 8
