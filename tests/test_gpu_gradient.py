"""Reverse pass (gbsbin_backward) against central finite differences of the CPU oracle.

The loss is linear in the table, L = sum_b pbar(b) P(b) with a fixed random pbar (any
loss reduces to this through dL/dP), except where a negative log-likelihood of a count
table is used.  Finite differences use h = 1e-6 on the oracle (FP64, |dP| ~ 1e-16), so
their error is ~1e-10; the bar is |g - g_fd| <= 1e-7 + 1e-6 |g_fd|.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import state

pytestmark = pytest.mark.gpu
H = 1e-6


def oracle_loss(prob, pbar):
    return float((oracle.binned(prob)["P"] * pbar).sum())


def oracle_loss_direct(sigma1, zbar, labels, radix, pbar):
    XA, gamma = state.adjacency(sigma1, zbar)
    logq, _, _ = oracle.logq_grid(XA, gamma, labels, radix)
    P = oracle.dft(np.exp(logq - logq[0]), radix).real
    return float((P * pbar).sum())


def copy_prob(p):
    return synth.Problem(p.M, p.K, p.r.copy(), p.T.copy(), p.bin_of_mode.copy(), p.cutoff.copy(),
                         alpha=None if p.alpha is None else p.alpha.copy(),
                         V=None if p.V is None else p.V.copy())


def fd(prob, pbar, name, idx, part):
    """d L / d (Re or Im) of prob.<name>[idx] by central differences."""
    vals = []
    for sgn in (1.0, -1.0):
        q = copy_prob(prob)
        arr = getattr(q, name)
        step = H if part == "re" else 1j * H
        arr[idx] = arr[idx] + sgn * step
        vals.append(oracle_loss(q, pbar))
    return (vals[0] - vals[1]) / (2 * H)


def gpu_grads(gb, prob, pbar, precision=0):
    import torch
    with gb.Plan(prob, precision=precision, want_backward=True) as p:
        p.table()
        g = p.backward(torch.from_numpy(pbar).cuda())
    return g


def close(g, f):
    return abs(g - f) <= 1e-7 + 1e-6 * abs(f)


@pytest.mark.parametrize("precision", [0, 1])
def test_physical_gradients_match_finite_differences(cuda_lib, precision):
    rng = np.random.default_rng(501)
    prob = synth.random_problem(rng, 3, 2, 2, [5, 4], displaced=True, internal_basis=True)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    g = gpu_grads(cuda_lib, prob, pbar, precision)
    for idx in np.ndindex(*prob.r.shape):
        f = fd(prob, pbar, "r", idx, "re")
        assert close(g["r"][idx], f), ("r", idx, g["r"][idx], f)
    for name in ("T", "alpha", "V"):
        arr = getattr(prob, name)
        for idx in np.ndindex(*arr.shape):
            fr, fi = fd(prob, pbar, name, idx, "re"), fd(prob, pbar, name, idx, "im")
            gv = g[name][idx]
            assert close(gv.real, fr) and close(gv.imag, fi), (name, idx, gv, fr, fi)


def test_gradients_without_displacement_three_groups(cuda_lib):
    rng = np.random.default_rng(502)
    prob = synth.random_problem(rng, 5, 1, 3, [3, 4, 2], shuffle_bins=True)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    g = gpu_grads(cuda_lib, prob, pbar)
    for idx in [(0, 0), (2, 0), (4, 0)]:
        assert close(g["r"][idx], fd(prob, pbar, "r", idx, "re"))
    for idx in [(0, 1), (3, 3), (4, 2)]:
        assert close(g["T"][idx].real, fd(prob, pbar, "T", idx, "re"))
        assert close(g["T"][idx].imag, fd(prob, pbar, "T", idx, "im"))
    assert np.abs(g["alpha"]).max() < 1e-12       # symmetric in alpha at alpha = 0


def test_covariance_and_mean_gradients_along_directions(cuda_lib):
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(503)
    prob = synth.random_problem(rng, 3, 1, 2, [4, 5], displaced=True)
    sigma1, zbar = state.sigma1_zbar(prob)
    n = sigma1.shape[0]
    labels = state.mode_labels(prob)

    class Direct:
        pass
    d = Direct()
    d.M, d.K, d.r, d.T = prob.M, prob.K, None, None
    d.sigma1, d.zbar, d.bin_of_mode, d.cutoff = sigma1, zbar, prob.bin_of_mode, prob.cutoff
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in prob.cutoff))
    with gb.Plan(d, want_backward=True) as p:
        p.table()
        g = p.backward(torch.from_numpy(pbar).cuda(), want=("sigma1", "zbar"))
    h = n // 2
    for _ in range(3):
        # a physical direction keeps the form [[N^T, Mm], [Mm^*, N]] (N Hermitian, Mm
        # symmetric), under which G(omega^-k) = conj G(omega^k) still holds
        Nd = rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h))
        Nd = Nd + Nd.conj().T
        Md = rng.standard_normal((h, h)) + 1j * rng.standard_normal((h, h))
        Md = Md + Md.T
        Hm = 0.05 * np.block([[Nd.T, Md], [Md.conj(), Nd]])
        f = (oracle_loss_direct(sigma1 + H * Hm, zbar, labels, prob.radix, pbar)
             - oracle_loss_direct(sigma1 - H * Hm, zbar, labels, prob.radix, pbar)) / (2 * H)
        got = float(np.real(np.sum(np.conj(g["sigma1"]) * Hm)))
        assert close(got, f), (got, f)
        u = rng.standard_normal(n // 2) + 1j * rng.standard_normal(n // 2)
        dz = np.concatenate([u, u.conj()])
        f = (oracle_loss_direct(sigma1, zbar + H * dz, labels, prob.radix, pbar)
             - oracle_loss_direct(sigma1, zbar - H * dz, labels, prob.radix, pbar)) / (2 * H)
        got = float(np.real(np.sum(np.conj(g["zbar"]) * dz)))
        assert close(got, f), (got, f)


def test_full_size_negative_log_likelihood_gradient(cuda_lib):
    # n = 200 (100 modes, 2 groups of 50) on a 21 x 21 grid: NLL of a count table; the
    # gradient along random directions in r and in the transmission eta of T = sqrt(eta) U
    import torch
    gb = cuda_lib
    prob = synth.config(4)
    prob.cutoff = np.array([20, 20], np.int32)
    rng = np.random.default_rng(504)
    P0 = oracle.binned(prob)["P"]
    counts = rng.multinomial(10 ** 6, np.clip(P0, 0, None).reshape(-1) / np.clip(P0, 0, None).sum()).reshape(P0.shape)

    def nll(q):
        P = oracle.binned(q)["P"]
        return float(-(counts * np.log(P)).sum())

    with gb.Plan(prob, want_backward=True) as p:
        Pg = p.table()
        dLdP = torch.from_numpy(-counts / Pg.cpu().numpy()).cuda()
        g = p.backward(dLdP, want=("r", "T"))
    # The NLL is ~1e7 in size, so h cannot be tiny (cancellation ~1e7 * 1e-16 / h); the
    # h^2 truncation term is removed by Richardson extrapolation over h and h/2.
    def richardson(shift, h=2e-4):
        def d(hh):
            return (nll(shift(hh)) - nll(shift(-hh))) / (2 * hh)
        return (4.0 * d(h / 2) - d(h)) / 3.0

    dr = rng.standard_normal(prob.r.shape)

    def shift_r(hh):
        q = copy_prob(prob)
        q.r = prob.r + hh * dr
        return q
    f = richardson(shift_r)
    got = float((g["r"] * dr).sum())
    assert abs(got - f) <= 1e-4 + 1e-6 * abs(f), (got, f)
    # eta: T = sqrt(eta) U  =>  dT/deta = T / (2 eta)
    eta = prob.notes["eta"]
    dT = prob.T / (2 * eta)
    got = float(np.real(np.sum(np.conj(g["T"]) * dT)))

    def shift_eta(hh):
        q = copy_prob(prob)
        q.T = np.sqrt((eta + hh) / eta) * prob.T
        return q
    f = richardson(shift_eta)
    assert abs(got - f) <= 1e-4 + 1e-6 * abs(f), (got, f)


def test_purity_gradient_two_internal_modes(cuda_lib):
    # Sec. VIII: second spectral mode with tanh^2(xi') = ((1-p)/p) tanh^2(xi); the
    # gradient in the purity p follows from dL/dr through dxi'/dp
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(505)
    M, p0 = 4, 0.8
    xi = rng.uniform(0.5, 0.9, M)

    def make(pur):
        xi2 = np.arctanh(np.sqrt((1 - pur) / pur) * np.tanh(xi))
        T = np.sqrt(0.85) * synth.haar_unitary(M, np.random.default_rng(7))
        return synth.Problem(M, 2, np.stack([xi, xi2], axis=1), T, np.array([0, 0, 1, 1], np.int32),
                             np.array([6, 6], np.int32))
    prob = make(p0)
    pbar = rng.standard_normal((7, 7))
    with gb.Plan(prob, want_backward=True) as p:
        p.table()
        g = p.backward(torch.from_numpy(pbar).cuda(), want=("r",))
    t = np.tanh(xi)
    s = np.sqrt((1 - p0) / p0)
    dxi2_dp = (t / (1 - (s * t) ** 2)) * (-0.5 / s) / p0 ** 2
    got = float((g["r"][:, 1] * dxi2_dp).sum())
    f = (oracle_loss(make(p0 + H), pbar) - oracle_loss(make(p0 - H), pbar)) / (2 * H)
    assert close(got, f), (got, f)


def test_autograd_function_matches(cuda_lib):
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(506)
    prob = synth.random_problem(rng, 3, 1, 2, [4, 4], displaced=True)
    pbar = torch.from_numpy(rng.standard_normal((5, 5))).cuda()
    r = torch.tensor(prob.r, dtype=torch.float64, requires_grad=True)
    T = torch.tensor(prob.T, dtype=torch.complex128, requires_grad=True)
    a = torch.tensor(prob.alpha, dtype=torch.complex128, requires_grad=True)
    with gb.Plan(prob, want_backward=True) as p:
        P = gb.binned_distribution(p, prob, r, T, a)
        (P * pbar).sum().backward()
        g = p.backward(pbar, want=("r", "T", "alpha"))
    assert np.allclose(r.grad.numpy(), g["r"], rtol=0, atol=1e-12)
    assert np.allclose(T.grad.numpy(), g["T"], rtol=0, atol=1e-12)
    assert np.allclose(a.grad.numpy(), g["alpha"], rtol=0, atol=1e-12)
    assert close(float(r.grad[1, 0]), fd(prob, pbar.cpu().numpy(), "r", (1, 0), "re"))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32pairs"])
@pytest.mark.parametrize("M,K,cutoff", [(21, 1, [3, 4]), (3, 7, [2, 3]), (171, 1, [1, 2])],
                         ids=["n42_ragged_block", "n42_internal", "n342_block8"])
def test_device_adjoints_along_a_physical_direction(cuda_lib, precision, M, K, cutoff):
    # the asynchronous adjoints S = dL/dXA, s = dL/dgamma (bilinear) against central differences
    # of the oracle along a direction in the squeezings: dL = Re(sum S dXA + sum s dgamma), with
    # dXA, dgamma the state algebra's own differences.  n = 42 runs blocks of 16, 16 and 10
    # pivots, n = 342 blocks of 8 with a ragged 4 x 4 tile edge
    import torch
    gb = cuda_lib
    rng = np.random.default_rng(505 + M)
    prob = synth.random_problem(rng, M, K, len(cutoff), cutoff, displaced=True, internal_basis=K > 1)
    pbar = rng.standard_normal(tuple(int(c) + 1 for c in cutoff))
    dr = rng.standard_normal(prob.r.shape)
    h = 1e-5

    def shifted(t):
        q = copy_prob(prob)
        q.r = prob.r + t * dr
        return q
    adj = [state.adjacency(*state.sigma1_zbar(shifted(t))) for t in (h, -h)]
    dXA = (adj[0][0] - adj[1][0]) / (2 * h)
    dg = (adj[0][1] - adj[1][1]) / (2 * h)
    f = (oracle_loss(shifted(h), pbar) - oracle_loss(shifted(-h), pbar)) / (2 * h)
    with gb.Plan(prob, precision=precision, want_backward=True, want_timing=True) as p:
        p.table()
        S, s = p.backward_device(torch.from_numpy(pbar).cuda())
        torch.cuda.synchronize()
        st, d = p.diagnostics()
        assert st == 0 and d["backward_kernel_ms"] > 0
        g = p.backward(torch.from_numpy(pbar).cuda(), want=("r",))
    S, s = S.cpu().numpy(), s.cpu().numpy()
    got = float(np.real(np.sum(S * dXA) + np.sum(s * dg)))
    assert abs(got - f) <= 1e-7 + 1e-6 * abs(f), (got, f)
    chained = float((g["r"] * dr).sum())
    assert abs(chained - got) <= 1e-9 + 1e-9 * abs(got), (chained, got)
