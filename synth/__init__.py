"""Seeded synthetic workloads for binned photon statistics of Gaussian states.

This module only draws inputs: squeezing parameters, transfer matrices, displacements,
internal-mode bases, detector groupings and cutoffs.  It holds none of the method's
arithmetic (no covariance matrices, no generating functions), so both the CPU oracle and
the CUDA library can consume the same arrays without sharing any computation.

Physical model of a problem (Sec. II and Sec. VIII of arXiv:2412.17742):

* ``M`` external (spatial) modes, ``K`` internal modes per external mode.  Input port ``i``
  carries ``K`` independent single-mode squeezed states with real squeezing ``r[i, k]``,
  defined in an internal basis whose vectors are the columns of ``V[i]`` (``V=None`` means
  the identity for every port, i.e. all sources share one internal basis).
* ``alpha[i, k]`` displaces internal mode ``k`` of port ``i`` (``None`` = no displacement).
* ``T`` is the ``M x M`` (generally lossy, ``||T|| <= 1``) transfer matrix acting on the
  external index; it acts as ``T (x) I_K`` on the internal index.
* ``bin_of_mode[j]`` is the detector group ``Lambda_l`` of output port ``j``; ``cutoff[l]``
  is ``N_l``, giving a grid of ``prod(N_l + 1)`` roots-of-unity points.

Seeds follow ``177420 + config index`` so every consumer draws identical bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 177420


@dataclass
class Problem:
    """One binned-distribution problem (inputs only)."""

    M: int
    K: int
    r: np.ndarray                      # (M, K) float64
    T: np.ndarray                      # (M, M) complex128, row = output port
    bin_of_mode: np.ndarray            # (M,) int32, values in [0, L)
    cutoff: np.ndarray                 # (L,) int32, N_l >= 0
    alpha: Optional[np.ndarray] = None  # (M, K) complex128
    V: Optional[np.ndarray] = None      # (M, K, K) complex128, columns = internal basis
    name: str = ""
    notes: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return int(self.cutoff.shape[0])

    @property
    def n(self) -> int:
        return 2 * self.M * self.K

    @property
    def radix(self) -> np.ndarray:
        return (self.cutoff + 1).astype(np.int64)

    @property
    def n_points(self) -> int:
        return int(np.prod(self.radix))


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random ``n x n`` unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, Notices AMS 54, 592 (2007))."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def contiguous_bins(M: int, L: int) -> np.ndarray:
    """Detector groups of near-equal size over contiguous output ports."""
    edges = np.linspace(0, M, L + 1).round().astype(int)
    lab = np.zeros(M, dtype=np.int32)
    for l in range(L):
        lab[edges[l]:edges[l + 1]] = l
    return lab


def _schmidt_split(r_ext: np.ndarray, K: int) -> np.ndarray:
    """Per-source squeezing over K Schmidt modes with weights lambda_k ~ exp(-k/2),
    normalised, and r_{i,k} = r_i sqrt(lambda_k)."""
    lam = np.exp(-np.arange(K) / 2.0)
    lam = lam / lam.sum()
    return r_ext[:, None] * np.sqrt(lam)[None, :]


def config(index: int) -> Problem:
    """The five named workloads (index 0..4); index 3 returns the first problem of the
    batched workload, use :func:`batch_config` for all of it."""
    rng = np.random.default_rng(SEED_BASE + index)
    if index == 0:
        M, K = 4, 1
        r = rng.uniform(0.3, 0.8, M)[:, None]
        T = np.sqrt(0.7) * haar_unitary(M, rng)
        lab = np.array([0, 0, 1, 1], dtype=np.int32)
        return Problem(M, K, r, T, lab, np.array([6, 6], dtype=np.int32),
                       name="m4_k1_l2_n6")
    if index == 1:
        M, K = 16, 1
        r = rng.uniform(0.5, 1.2, M)[:, None]
        eta = rng.uniform(0.4, 0.9, M)
        U = haar_unitary(M, rng)
        T = np.sqrt(eta)[:, None] * U
        return Problem(M, K, r, T, contiguous_bins(M, 4), np.full(4, 8, dtype=np.int32),
                       name="m16_k1_l4_n8")
    if index == 2:
        M, K = 24, 4
        r = _schmidt_split(rng.uniform(0.5, 1.2, M), K)
        T = np.sqrt(0.6) * haar_unitary(M, rng)
        V = np.stack([haar_unitary(K, rng) for _ in range(M)])
        alpha = np.zeros((M, K), dtype=np.complex128)
        src = rng.choice(M, size=4, replace=False)
        alpha[src, 0] = np.sqrt(0.1 / 2.0) * (rng.standard_normal(4) + 1j * rng.standard_normal(4))
        return Problem(M, K, r, T, contiguous_bins(M, 3), np.full(3, 20, dtype=np.int32),
                       alpha=alpha, V=V, name="m24_k4_l3_n20_displaced")
    if index == 3:
        return batch_config()[0]
    if index == 4:
        M, K = 100, 1
        r = rng.uniform(0.8, 1.6, M)[:, None]
        T = np.sqrt(0.5) * haar_unitary(M, rng)
        return Problem(M, K, r, T, contiguous_bins(M, 2), np.full(2, 80, dtype=np.int32),
                       name="m100_k1_l2_n80", notes={"eta": 0.5})
    raise ValueError(f"no workload {index}")


def batch_config(count: int = 256, seed_index: int = 3) -> List[Problem]:
    """Uneven batch: M ~ U{8..48}, K ~ U{1..3}, L ~ U{1..4} (L <= M), r ~ U(0.3, 1.3),
    per-port loss eta ~ U(0.3, 0.95), Haar T; the grid size is drawn log-uniform in
    [500, 20000] and N_l = floor(N_pts^(1/L)) - 1 in every bin (at least 1)."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    out = []
    for p in range(count):
        M = int(rng.integers(8, 49))
        K = int(rng.integers(1, 4))
        L = int(min(rng.integers(1, 5), M))
        r = rng.uniform(0.3, 1.3, (M, K))
        eta = rng.uniform(0.3, 0.95, M)
        T = np.sqrt(eta)[:, None] * haar_unitary(M, rng)
        target = float(np.exp(rng.uniform(np.log(500.0), np.log(20000.0))))
        Nl = max(1, int(np.floor(target ** (1.0 / L))) - 1)
        out.append(Problem(M, K, r, T, contiguous_bins(M, L), np.full(L, Nl, dtype=np.int32),
                           name=f"batch{p}"))
    return out


def random_problem(rng: np.random.Generator, M: int, K: int, L: int, cutoff,
                   displaced: bool = False, internal_basis: bool = False,
                   r_range=(0.2, 0.9), eta_range=(0.3, 0.95),
                   shuffle_bins: bool = False) -> Problem:
    """Small random problem for tests."""
    r = rng.uniform(*r_range, (M, K))
    eta = rng.uniform(*eta_range, M)
    T = np.sqrt(eta)[:, None] * haar_unitary(M, rng)
    lab = contiguous_bins(M, L)
    if shuffle_bins:
        lab = rng.permutation(lab).astype(np.int32)
    cut = np.array(np.broadcast_to(np.asarray(cutoff, dtype=np.int32), (L,)), dtype=np.int32)
    alpha = None
    if displaced:
        alpha = 0.4 * (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K)))
    V = np.stack([haar_unitary(K, rng) for _ in range(M)]) if internal_basis else None
    return Problem(M, K, r, T, lab, cut, alpha=alpha, V=V, name=f"rand_m{M}_k{K}_l{L}")


# ---------------------------------------------------------------- Fock inputs (App. C)
@dataclass
class FockProblem:
    """Photon-number (Fock) inputs through a lossy linear circuit, binned outputs.

    ``photons[j]`` photons enter input port ``j`` of the ``M x M`` transfer matrix ``T``
    (row = output port, ``||T|| <= 1``); ``bin_of_mode[i]`` groups output port ``i``;
    ``cutoff[l]`` is ``N_l``."""

    M: int
    T: np.ndarray                      # (M, M) complex128, row = output port
    photons: np.ndarray                # (M,) int32 >= 0
    bin_of_mode: np.ndarray            # (M,) int32, values in [0, L)
    cutoff: np.ndarray                 # (L,) int32
    name: str = ""

    @property
    def L(self) -> int:
        return int(self.cutoff.shape[0])

    @property
    def N(self) -> int:
        return int(np.sum(self.photons))

    @property
    def radix(self) -> np.ndarray:
        return (self.cutoff + 1).astype(np.int64)


FOCK_SEED_INDEX = 50


def fock_config(N: int = 16, M: int = 32, L: int = 3) -> FockProblem:
    """Fock boson-sampling validation workload: single photons in input ports 0..N-1 of
    an M-port interferometer T = diag(sqrt(eta_i)) U (Haar U, output loss eta_i ~
    U(0.4, 0.9)), L contiguous detector groups, cutoff N_l = N (the whole table: no
    group can see more than N photons)."""
    rng = np.random.default_rng(SEED_BASE + FOCK_SEED_INDEX + N)
    eta = rng.uniform(0.4, 0.9, M)
    T = np.sqrt(eta)[:, None] * haar_unitary(M, rng)
    photons = np.zeros(M, dtype=np.int32)
    photons[:N] = 1
    return FockProblem(M, T, photons, contiguous_bins(M, L), np.full(L, N, dtype=np.int32),
                       name=f"fock_m{M}_n{N}_l{L}")


def random_fock_problem(rng: np.random.Generator, M: int, photons, L: int, cutoff,
                        eta_range=(0.3, 0.95), shuffle_bins: bool = False) -> FockProblem:
    """Small random Fock-input problem for tests (photons: a length-M sequence)."""
    eta = rng.uniform(*eta_range, M)
    T = np.sqrt(eta)[:, None] * haar_unitary(M, rng)
    lab = contiguous_bins(M, L)
    if shuffle_bins:
        lab = rng.permutation(lab).astype(np.int32)
    cut = np.array(np.broadcast_to(np.asarray(cutoff, dtype=np.int32), (L,)), dtype=np.int32)
    return FockProblem(M, T, np.asarray(photons, dtype=np.int32), lab, cut, name=f"fock_rand_m{M}_l{L}")


# ------------------------------------------------------------------ heralded states (Sec. VII-VIII)
FOCK_HERALD_ROLES = [0, 0, -2, -1]   # port 0 (both spectral modes) heralds; port 1: mode 2 kept, mode 3 traced


def fock_heralding_source(p: float, eta: float, xi: float = 1.1) -> Problem:
    """Sec. VIII's Fock-state source: two ports x two spectral modes, squeezing xi in spectral
    mode 1 and xi' with tanh^2 xi' = ((1 - p)/p) tanh^2 xi in mode 2 (Eq.
    relation_between_sqz_par, spectral purity p), through T = sqrt(eta) U with U the balanced
    beam splitter (1/sqrt 2) [[1, i], [i, 1]] (Eq. beam_splitter_unitary).  Roles
    FOCK_HERALD_ROLES: port 0 heralds with both spectral modes summed, spectral mode 1 of port 1
    is kept, its mode 2 traced."""
    xi2 = np.arctanh(np.sqrt((1 - p) / p) * np.tanh(xi)) if p < 1 else 0.0
    r = np.array([[xi, xi2], [xi, xi2]])
    T = np.sqrt(eta) * np.array([[1, 1j], [1j, 1]]) / np.sqrt(2)
    return Problem(2, 2, r, T, np.array([0, 1], np.int32), np.array([8, 8], np.int32))


def herald_config(seed: int = 17):
    """A larger heralding workload: 16 ports x 2 internal modes (64 x 64 matrices), displaced,
    non-aligned internal bases, Haar T with loss; two heralding groups of six ports each (both
    internal modes summed), cutoff 8 per group (81 grid points); the first internal mode of
    ports 12 and 13 kept (Fock cutoff 6: 7^4 coefficients per point), the rest traced.
    Returns (problem, roles, heralding cutoffs, Fock cutoff)."""
    rng = np.random.default_rng(seed)
    prob = random_problem(rng, 16, 2, 2, [8, 8], displaced=True, internal_basis=True, r_range=(0.4, 0.9),
                          eta_range=(0.6, 0.9))
    roles = []
    for port in range(16):
        for k in range(2):
            if port < 6:
                roles.append(0)
            elif port < 12:
                roles.append(1)
            elif port in (12, 13) and k == 0:
                roles.append(-2)
            else:
                roles.append(-1)
    return prob, roles, [8, 8], 6
