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
        dev = gb.gbsbin_prob_distinguishable_device(prob, list(n))
        host = gb.gbsbin_prob_distinguishable(prob, list(n))
        assert abs(dev - host) < 1e-14 and abs(dev - table[n]) < 1e-12, (n, dev, host, table[n])


def test_device_large_patterns(cuda_lib):
    gb = cuda_lib
    rng = np.random.default_rng(1600)
    prob = _distinguishable(rng, 4, 5, r=(0.6, 0.9))
    for n in [(5, 5, 5, 5), (5, 4, 3, 5)]:                          # 1296 and 720 points
        assert abs(gb.gbsbin_prob_distinguishable_device(prob, list(n)) -
                   gb.gbsbin_prob_distinguishable(prob, list(n))) < 1e-10
    # 5^8 = 390625 points: every thread walks several points of the grid-stride loop
    big = _distinguishable(np.random.default_rng(1700), 8, 4, r=(0.2, 0.4))
    n = [4] * 8
    dev = gb.gbsbin_prob_distinguishable_device(big, n)
    assert np.isfinite(dev) and abs(dev - gb.gbsbin_prob_distinguishable(big, n)) < 1e-9
    with pytest.raises(gb.GbsbinError) as e:
        gb.gbsbin_prob_distinguishable_device(prob, [20, 20, 20, 5])   # N = 65 > 64
    assert e.value.status == 8
