"""Heralded (conditional) states of a multimode Gaussian state (Sec. VII).
TEST INFRASTRUCTURE ONLY.

The modes (M K of them, external-major) are split into heralding modes (grouped: group l of
a heralding outcome b counts the photons of its modes), traced modes (discarded) and kept
modes (the heralded state's support).  The unnormalised heralded state has the elements
(Sec. VII, Eq. lhaf_heralded_offd_internal_1, with traced modes summed over)

    <v| rho(b) |u> = Pr(0) / sqrt(u! v!) sum_{n in K(b), t} lhaf(A_{(n,t,u) (+) (n,t,v)},
                     gamma_{...}) / (n! t!),

the first half of the repeated indices carrying the ket pattern (heralding n, traced t, kept
u) and the second half the bra pattern (n, t, v).

* :func:`brute` - that definition, loop Hafnians by the multiplicity recursion of
  :mod:`oracle.lhaf`, traced photon numbers summed up to ``tmax`` (tiny inputs only).
* :func:`table` - the same elements from the generating function.  With
  lhaf(A_p, gamma_p) = d^p exp(xi^T A xi / 2 + gamma^T xi) at xi = 0, the sum over the
  heralding and traced patterns with weights w^n / n! is the complex-Gaussian expectation of
  that exponential with xi = sqrt(w) (alpha, conj alpha) on those modes; for the kept modes
  the sum is the Taylor coefficient of x^u y^v times u! v!.  The expectation is, with D the
  heralding and traced indices (both halves), F the kept ones, D(w) = diag(w) (w = 1 on traced
  modes) and N(w) = (I - X D(w) A_DD)^{-1} X D(w),

    F(w; xi_F) = exp(xi_F^T M xi_F / 2 + l^T xi_F + e) / sqrt(det(I - X D(w) A_DD)),
    M = A_FF + A_DF^T N A_DF,   l = gamma_F + A_DF^T N gamma_D,   e = gamma_D^T N gamma_D / 2,

  so <v|rho(b)|u> = Pr(0) sqrt(u! v!) [w^b][x^u y^v] F.  Per point w of a roots-of-unity
  grid over the heralding groups: numpy's solve and eigenvalues (the branch of the square root
  from sum Log(1 - mu_i), each |mu_i| < 1), the Taylor coefficients of exp(quadratic) by the
  recurrence (p_i + 1) c_{p + e_i} = l_i c_p + sum_j M_ij c_{p - e_j}, then numpy's FFT over
  the grid gives the coefficient of w^b (folded modulo the grid: oversample to unfold).

Pinned by ``tests/test_herald_oracle.py``: :func:`table` against :func:`brute`, Hermiticity,
the trace against the binned table, the lossless two-mode squeezed vacuum (heralding n photons
gives |n> exactly) and the Fock-state fidelities printed in Sec. VIII.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import lhaf, state


def _adjacency(prob):
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    n = XA.shape[0]
    return state.xmat(n) @ XA, gamma, state.vacuum_probability(XA, gamma)


def _compositions(total, parts):
    """All non-negative integer vectors of length ``parts`` summing to ``total``."""
    if parts == 0:
        if total == 0:
            yield ()
        return
    for cuts in itertools.combinations(range(total + parts - 1), parts - 1):
        prev, out = -1, []
        for c in cuts:
            out.append(c - prev - 1)
            prev = c
        out.append(total + parts - 1 - prev - 1)
        yield tuple(out)


def brute(prob, roles, b, u, v, tmax=12):
    """<v|rho(b)|u> from the definition.  roles[m] >= 0: heralding group of mode m; -1: traced;
    -2: kept.  b: heralding outcome per group; u, v: kept-mode Fock indices in mode order."""
    A, gamma, pr0 = _adjacency(prob)
    nm = len(roles)
    groups = {}
    for m, r in enumerate(roles):
        if r >= 0:
            groups.setdefault(r, []).append(m)
    traced = [m for m, r in enumerate(roles) if r == -1]
    kept = [m for m, r in enumerate(roles) if r == -2]
    per_group = [list(_compositions(int(b[g]), len(groups[g]))) for g in sorted(groups)]
    total = 0.0 + 0.0j
    for combo in itertools.product(*per_group):
        nh = [0] * nm
        for g, s in zip(sorted(groups), combo):
            for m, c in zip(groups[g], s):
                nh[m] = c
        for tr in itertools.product(range(tmax + 1), repeat=len(traced)):
            if sum(tr) > tmax:
                continue
            first, second = list(nh), list(nh)
            for m, c in zip(traced, tr):
                first[m] = second[m] = c
            for m, a, c in zip(kept, u, v):
                first[m], second[m] = a, c
            weight = 1.0
            for c in [nh[m] for m in range(nm) if roles[m] >= 0] + list(tr):
                weight /= math.factorial(int(c))
            total += weight * lhaf.lhaf_repeated(A, gamma, tuple(first) + tuple(second))
    norm = 1.0
    for a, c in zip(u, v):
        norm *= math.sqrt(math.factorial(int(a)) * math.factorial(int(c)))
    return complex(pr0 * total / norm)


def _taylor_exp_quadratic(Mq, lq, cut):
    """Coefficients c_p, p in [0, cut]^n, of exp(x^T Mq x / 2 + lq^T x) (Mq symmetric)."""
    nf = len(lq)
    shape = (cut + 1,) * nf
    c = np.zeros(shape, complex)
    c[(0,) * nf] = 1.0
    order = sorted(itertools.product(range(cut + 1), repeat=nf), key=sum)
    for p in order[1:]:
        i = next(t for t in range(nf) if p[t] > 0)
        q = list(p)
        q[i] -= 1
        val = lq[i] * c[tuple(q)]
        for j in range(nf):
            if q[j] > 0:
                r = list(q)
                r[j] -= 1
                val += Mq[i, j] * c[tuple(r)]
        c[p] = val / p[i]
    return c


def table(prob, roles, cutoff, cut, oversample=4):
    """Unnormalised heralded elements for every heralding outcome b_l <= cutoff[l] and kept
    indices u, v <= cut: an array of shape (cutoff + 1 ...) + (cut + 1,) * (2 nkept), index
    [b..., u_1..u_k, v_1..v_k] = <v|rho(b)|u>; and the heralding probabilities Pr(b) (the trace
    over the kept modes, from the same expectation with the kept modes traced as well)."""
    A, gamma, pr0 = _adjacency(prob)
    nm = len(roles)
    L = len(cutoff)
    Dm = [m for m in range(nm) if roles[m] != -2]
    kept = [m for m in range(nm) if roles[m] == -2]
    D = Dm + [m + nm for m in Dm]
    F = kept + [m + nm for m in kept]
    radix = [oversample * (int(c) + 1) for c in cutoff]
    X2 = state.xmat(2 * len(Dm))
    ADD, ADF, AFF = A[np.ix_(D, D)], A[np.ix_(D, F)], A[np.ix_(F, F)]
    gD, gF = gamma[D], gamma[F]
    allD = list(range(nm)) + [m + nm for m in range(nm)]
    Xall = state.xmat(2 * nm)
    nf = len(F)
    G = np.zeros(tuple(radix) + (cut + 1,) * nf, complex)
    Gt = np.zeros(tuple(radix), complex)
    for k in itertools.product(*[range(r) for r in radix]):
        w = np.array([np.exp(2j * np.pi * k[roles[m]] / radix[roles[m]]) if roles[m] >= 0 else 1.0
                      for m in range(nm)])
        wD = np.concatenate([w[Dm], w[Dm]])
        K = np.eye(len(D)) - X2 @ (wD[:, None] * ADD)
        ld = np.sum(np.log(np.linalg.eigvals(K)))
        N = np.linalg.solve(K, X2 * wD[None, :])
        Mq = AFF + ADF.T @ N @ ADF
        lq = gF + ADF.T @ N @ gD
        e = 0.5 * gD @ N @ gD
        G[k] = _taylor_exp_quadratic(Mq, lq, cut) * np.exp(e - 0.5 * ld)
        # the heralding probability: every non-heralding mode traced (w = 1)
        wa = np.concatenate([w, w])
        Ka = np.eye(2 * nm) - Xall @ (wa[:, None] * A)
        lda = np.sum(np.log(np.linalg.eigvals(Ka)))
        Na = np.linalg.solve(Ka, Xall * wa[None, :])
        Gt[k] = np.exp(0.5 * gamma @ Na @ gamma - 0.5 * lda)
    for ax in range(L):
        G = np.fft.fft(G, axis=ax) / radix[ax]
        Gt = np.fft.fft(Gt, axis=ax) / radix[ax]
    sl = tuple(slice(0, int(c) + 1) for c in cutoff)
    fact = np.array([math.sqrt(math.factorial(i)) for i in range(cut + 1)])
    scale = np.ones((cut + 1,) * nf)
    for ax in range(nf):
        shape = [1] * nf
        shape[ax] = cut + 1
        scale = scale * fact.reshape(shape)
    rho = pr0 * G[sl] * scale
    return rho, (pr0 * Gt[sl]).real
