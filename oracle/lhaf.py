"""Brute-force loop Hafnians and Fock probabilities.  TEST INFRASTRUCTURE ONLY.

Only for tiny inputs: these are the combinatorial definitions the generating-function
route must reproduce.

* ``lhaf_explicit`` enumerates single-pair matchings with loops of a symmetric matrix
  whose diagonal already holds the loop weights (Sec. II, Eq. gen_loop_haf_def).
* ``lhaf_repeated`` evaluates lhaf(A_{n(+)n}, gamma_{n(+)n}) (Sec. II, the row/column
  repetition below Eq. vacuum_probability) without expanding the matrix: the first
  remaining copy of index i is matched to a loop (gamma_i), to another copy of i
  (A_ii), or to a copy of some later index j (A_ij), each copy being a distinct vertex.
* ``fock_probability`` is Eq. gbs_probability_distribution.
* ``binned_brute_force`` sums Fock probabilities over the compatible patterns of
  Eq. coarse_grained_subset (Sec. VI), the definition of P(b).
"""
from __future__ import annotations

import itertools
from functools import lru_cache
from math import factorial

import numpy as np

from . import state


def lhaf_explicit(B: np.ndarray) -> complex:
    """Sum over single-pair matchings with loops of vertices 0..m-1 (diag = loop weight)."""
    m = B.shape[0]

    def rec(free):
        if not free:
            return 1.0 + 0j
        v = free[0]
        rest = free[1:]
        tot = B[v, v] * rec(rest)                      # v matched to its loop
        for t, u in enumerate(rest):                  # v matched to u
            tot += B[v, u] * rec(rest[:t] + rest[t + 1:])
        return tot

    return complex(rec(tuple(range(m))))


def expand(A: np.ndarray, gamma: np.ndarray, mult) -> np.ndarray:
    """filldiag(A_{mult}, gamma_{mult}): index i repeated mult[i] times."""
    idx = [i for i, c in enumerate(mult) for _ in range(int(c))]
    B = A[np.ix_(idx, idx)].astype(np.complex128).copy()
    B[np.diag_indices(len(idx))] = np.asarray(gamma)[idx]
    return B


def lhaf_repeated(A: np.ndarray, gamma: np.ndarray, mult) -> complex:
    """lhaf of filldiag(A_mult, gamma_mult) by recursion over multiplicity vectors."""
    A = np.asarray(A, dtype=np.complex128)
    gamma = np.asarray(gamma, dtype=np.complex128)
    size = len(mult)

    @lru_cache(maxsize=None)
    def rec(m):
        i = next((t for t in range(size) if m[t] > 0), None)
        if i is None:
            return 1.0 + 0j
        m1 = list(m)
        m1[i] -= 1
        tot = gamma[i] * rec(tuple(m1))
        if m1[i] > 0:
            m2 = list(m1)
            m2[i] -= 1
            tot += m1[i] * A[i, i] * rec(tuple(m2))
        for j in range(i + 1, size):
            if m1[j] > 0:
                m2 = list(m1)
                m2[j] -= 1
                tot += m1[j] * A[i, j] * rec(tuple(m2))
        return tot

    return complex(rec(tuple(int(c) for c in mult)))


def fock_probability(A, gamma, pr0, s) -> float:
    """Pr(s) = Pr(0) lhaf(A_{s(+)s}, gamma_{s(+)s}) / prod s_i!  (Eq. gbs_probability_distribution)."""
    mult = tuple(s) + tuple(s)
    val = pr0 * lhaf_repeated(A, gamma, mult)
    for c in s:
        val /= factorial(int(c))
    return float(np.real(val))


def binned_brute_force(prob, total_max: int) -> dict:
    """P(b) for every coarse pattern with sum(b) <= total_max, by summing Fock
    probabilities of all fine patterns s over the M K modes (the internal modes of port j
    and all ports of group l are summed into b_l)."""
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    n = XA.shape[0]
    A = state.xmat(n) @ XA
    pr0 = state.vacuum_probability(XA, gamma)
    MK = prob.M * prob.K
    lab = np.repeat(np.asarray(prob.bin_of_mode), prob.K)
    L = prob.L
    out = {}
    for s in _patterns(MK, total_max):
        b = [0] * L
        for m, c in enumerate(s):
            b[lab[m]] += c
        out[tuple(b)] = out.get(tuple(b), 0.0) + fock_probability(A, gamma, pr0, s)
    return out


def _patterns(modes: int, total_max: int):
    for tot in range(total_max + 1):
        for cuts in itertools.combinations(range(tot + modes - 1), modes - 1):
            prev = -1
            s = []
            for c in cuts:
                s.append(c - prev - 1)
                prev = c
            s.append(tot + modes - 1 - prev - 1)
            yield tuple(s)
