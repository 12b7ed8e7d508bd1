"""Fock inputs through lossy circuits (App. C) on the GPU, through the C ABI.

Parity: the binned table of both kernels (FP64, and FP32 pairs) against the oracle's
roots-of-unity table element by element, |dP| <= 1e-10 (the FP64 kernel meets 1e-13),
on cases that cover repeated photons, vacuum and single-input problems, folded and
oversampled grids, shuffled groups and several node restarts.  At the benchmarked size
(16 photons, 32 ports, three groups) and at a size where every CTA walks several node
ranges (21 photons, 2^20 nodes), properties that hold at any size: total probability 1,
the per-group means sum_{i in l} sum_j |T_ij|^2 p_j, binomial totals under uniform loss,
and the two arithmetics against each other.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fock

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _gpu_table(gb, fp, precision, oversample=1):
    with gb.FockPlan(fp, precision=precision, oversample=oversample) as plan:
        P = plan.table().cpu().numpy()
        d = plan.diagnostics()
    assert d["status"] == 0
    return P, d


def _cases():
    rng = np.random.default_rng(177)
    c = []
    T = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    c.append(("hom", synth.FockProblem(2, T, np.array([1, 1], np.int32), np.array([0, 1], np.int32),
                                       np.array([2, 2], np.int32)), 1))
    c.append(("repeated", synth.random_fock_problem(rng, 5, [1, 2, 0, 1, 1], 2, 5, shuffle_bins=True), 1))
    c.append(("six_singles_l3", synth.random_fock_problem(rng, 6, [1] * 6, 3, 6), 1))
    c.append(("folded", synth.random_fock_problem(rng, 6, [1] * 6, 3, 3), 1))
    c.append(("oversampled", synth.random_fock_problem(rng, 4, [1, 1, 1, 0], 2, 2), 2))
    c.append(("vacuum", synth.random_fock_problem(rng, 3, [0, 0, 0], 2, 2), 1))
    c.append(("one_input", synth.random_fock_problem(rng, 3, [0, 3, 0], 2, 3), 1))
    c.append(("ten_singles", synth.random_fock_problem(rng, 12, [1] * 10 + [0, 0], 2, 10), 1))
    c.append(("four_groups", synth.random_fock_problem(rng, 8, [1, 0, 2, 1, 0, 1, 1, 0], 4, 4, shuffle_bins=True), 1))
    c.append(("twelve_singles_l1", synth.random_fock_problem(rng, 14, [1] * 12 + [0, 0], 1, 12), 1))
    return c


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "df32"])
@pytest.mark.parametrize("name,fp,oversample", _cases(), ids=[c[0] for c in _cases()])
def test_fock_parity(cuda_lib, name, fp, oversample, precision):
    ref = fock.table(fp, oversample)["P"]
    P, d = _gpu_table(cuda_lib, fp, precision, oversample)
    assert P.shape == ref.shape
    err = np.abs(P - ref).max()
    assert err <= (1e-13 if precision == 0 else TOL), (name, err)
    assert d["kernel"] == (9 if precision == 0 else 10)
    assert abs(d["sum_P"] - ref.sum()) < 1e-12


def test_fock_hom_exact(cuda_lib):
    T = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    fp = synth.FockProblem(2, T, np.array([1, 1], np.int32), np.array([0, 1], np.int32), np.array([2, 2], np.int32))
    for prec, tol in ((0, 1e-15), (1, 1e-13)):      # FP32 pairs carry about 46 bits
        P, _ = _gpu_table(cuda_lib, fp, prec)
        assert abs(P[1, 1]) < tol and abs(P[2, 0] - 0.5) < tol and abs(P[0, 2] - 0.5) < tol


def _group_means_from_table(P):
    out = []
    for l in range(P.ndim):
        marg = P.sum(axis=tuple(m for m in range(P.ndim) if m != l))
        out.append(float(np.dot(np.arange(P.shape[l]), marg)))
    return np.array(out)


def _totals(P):
    N = sum(s - 1 for s in P.shape)
    tot = np.zeros(N + 1)
    for b in np.ndindex(*P.shape):
        tot[sum(b)] += P[b]
    return tot


def test_fock_benchmark_size_properties(cuda_lib):
    fp = synth.fock_config()                                   # 16 photons, 32 ports, 3 groups
    P64, _ = _gpu_table(cuda_lib, fp, 0)
    Pdf, _ = _gpu_table(cuda_lib, fp, 1)
    assert np.abs(P64 - Pdf).max() < TOL
    for P in (P64, Pdf):
        assert abs(P.sum() - 1.0) < 1e-12
        assert np.abs(_group_means_from_table(P) - fock.group_means(fp)).max() < 1e-10
        assert P.min() > -1e-12


def test_fock_many_node_ranges_binomial_total(cuda_lib):
    # T = sqrt(eta) U: the total count is Binomial(N, eta) whatever the interference; 2^20
    # nodes make every CTA walk several node ranges in both arithmetics
    rng = np.random.default_rng(5)
    M, N, eta = 24, 21, 0.45
    photons = np.zeros(M, np.int32)
    photons[:N] = 1
    fp = synth.FockProblem(M, np.sqrt(eta) * synth.haar_unitary(M, rng), photons, synth.contiguous_bins(M, 2),
                           np.array([N, N], np.int32))
    ref = np.array([math.comb(N, k) * eta ** k * (1 - eta) ** (N - k) for k in range(N + 1)])
    tables = []
    for prec in (0, 1):
        P, _ = _gpu_table(cuda_lib, fp, prec)
        tot = _totals(P)
        assert np.abs(tot[:N + 1] - ref).max() < TOL
        assert np.abs(tot[N + 1:]).max() < TOL
        assert np.abs(_group_means_from_table(P) - fock.group_means(fp)).max() < 1e-9
        tables.append(P)
    assert np.abs(tables[0] - tables[1]).max() < TOL


def test_fock_set_transfer_and_host_execute(cuda_lib):
    rng = np.random.default_rng(9)
    fp = synth.random_fock_problem(rng, 6, [1, 1, 0, 2, 0, 1], 2, 5)
    fp2 = synth.random_fock_problem(rng, 6, [1, 1, 0, 2, 0, 1], 2, 5)
    with cuda_lib.FockPlan(fp, precision=1) as plan:
        plan.set_transfer(fp2.T)
        P_dev = plan.table().cpu().numpy()
        P_host = plan.table_host()
    assert np.array_equal(P_dev, P_host)
    assert np.abs(P_host - fock.table(fp2)["P"]).max() < TOL


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "df32"])
def test_fock_node_shards(cuda_lib, precision):
    # every shard's partial table against the oracle's partial table of the same node range,
    # and the shards of a partition summing to the whole table
    rng = np.random.default_rng(303)
    fp = synth.random_fock_problem(rng, 9, [1, 1, 2, 1, 0, 1, 1, 1, 0], 2, 8)
    S = fock.node_count(fp.photons)
    with cuda_lib.FockPlan(fp, precision=precision) as p:
        assert p.nodes() == S
        whole = p.table().cpu().numpy()
    cuts = [0, 1, S // 3, S - 7, S]
    total = np.zeros_like(whole)
    for b, e in zip(cuts[:-1], cuts[1:]):
        with cuda_lib.FockPlan(fp, precision=precision, shard=(b, e)) as p:
            part = p.table().cpu().numpy()
        ref = fock.table(fp, node_range=(b, e))["P"]
        assert np.abs(part - ref).max() < (1e-13 if precision == 0 else TOL)
        total += part
    assert np.abs(total - whole).max() < 1e-13
    for bad in [(-1, 3), (3, 3), (0, S + 1)]:
        with pytest.raises(cuda_lib.GbsbinError):
            cuda_lib.FockPlan(fp, precision=precision, shard=bad)
