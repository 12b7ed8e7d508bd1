"""CPU partial tables of a shard of the evaluated half grid (test infrastructure).

The library's partial table of a shard [begin, end) is the half-grid inverse DFT applied
to G restricted to the shard: the complex transform over the axes but the last (full
radix), then the Hermitian last axis, P(b', b) = (1/N) (Re Y(b', 0) + sum_{k=1}^{H-1} c_k
Re(Y(b', k) w^{-k b})), c_k = 2 except c = 1 for k = R/2.  Written here from that
definition with numpy, G from per-point log q given on the full grid (row-major).
"""
import numpy as np


def partial_table_cpu(prob, logq_full, begin, end, oversample=1):
    radix = [oversample * (int(c) + 1) for c in prob.cutoff]
    nout = [int(c) + 1 for c in prob.cutoff]
    R, H = radix[-1], radix[-1] // 2 + 1
    lq = np.asarray(logq_full).reshape(radix)
    half = lq[..., :H].reshape(-1)                       # the evaluated half grid, in order
    g = np.exp(half - lq.reshape(-1)[0])
    mask = np.zeros(len(g), bool)
    mask[begin:end] = True
    h = np.where(mask, g, 0.0).reshape(radix[:-1] + [H])
    Y = h
    for ax, (Ra, na) in enumerate(zip(radix[:-1], nout[:-1])):
        k = np.arange(Ra)
        W = np.exp(-2j * np.pi * np.outer(np.arange(na), k) / Ra)   # (na, Ra)
        Y = np.moveaxis(np.tensordot(W, np.moveaxis(Y, ax, 0), axes=(1, 0)), 0, ax)
    b = np.arange(nout[-1])
    k = np.arange(H)
    c = np.where((k == 0) | (2 * k == R), 1.0, 2.0)
    W = c[None, :] * np.exp(-2j * np.pi * np.outer(b, k) / R)        # (nout, H)
    P = np.real(np.tensordot(Y, W.T, axes=(-1, 0))) / np.prod(radix)
    return P
