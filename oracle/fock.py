"""Fock inputs through a lossy linear circuit (arXiv:2412.17742, App. C).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the CUDA library never does.

Photon numbers p_j enter input port j of the M x M transfer matrix T (row = output port,
||T|| <= 1); the output ports are grouped into detector groups Lambda_1..Lambda_L.  N is
the total input photon number.  FP64 numpy throughout.

Definitions (App. C):

* ``loss_channel_matrix`` - the 4M x 4M symmetric matrix A_Phi of Eq. loss_channel_matrix
  (index blocks: input, output, input', output').
* ``density_diag_haf`` - <n|rho|n> = haf(A_Phi restricted to (p, n, p, n)) / (p! n!),
  Eq. density_matrix_fock_circuit with m = n; the Hafnian by memoised recursion over
  perfect matchings (tiny inputs only).
* ``density_diag_perm`` - the same element from the permanent of Eq. probs_fock_circuit,
  [[I - T^dag T, T^dag], [T, 0]] restricted to the multiplicities (p, n): the first
  index block is the input ports, the one I - T^dag T acts on, so it carries p (reading F1).
* ``binned_brute_force`` - P(b) = sum of <n|rho|n> over the patterns n compatible with b
  (Eq. coarse_grained_Fock), every pattern with |n| <= N enumerated.

The generating-function route (the method of Sec. VI on roots of unity, applied to the
generating function of App. C's diagonal elements):

* ``pgf_permanent`` - G(z) = sum_b P(b) z^b = perm(B(z)[p, p]) / prod_j p_j! with
  B(z) = I - T^dag (I - Z) T, Z = diag(z_label(i)) (reading F2: the generating function of
  Eq. probs_fock_circuit over the output patterns), by Ryser's formula on B with row and
  column j repeated p_j times.
* ``pgf_extract`` - the same G(z) as the coefficient of x^p in
  Q(x) = prod_j (sum_k B(z)_jk x_k)^{p_j}, taken with the finite-difference nodes of
  Sec. IV placed on roots of unity, x_k = exp(2 pi i g_k / (p_k + 1)) (reading F3): Q is
  homogeneous of degree N, so with one occupied input k0 of smallest p held at x_k0 = 1
  no other monomial aliases onto x^p; the weight x^{-p} equals prod_k x_k on these nodes.
* ``table`` - G on the roots-of-unity grid of the output groups by ``pgf_extract``, then the
  inverse DFT of :func:`oracle.dft` (Sec. VI, Eq. coarse_grained_prob): the folded table,
  exact (unfolded) when every N_l >= N.  For a range of the input nodes (in the reflected
  mixed-radix Gray order of ``gray_digits``) the partial table of their share of G, in the
  half-grid form of the DFT (see ``table``).

Pinned by ``tests/test_fock_oracle.py``: brute force through the Hafnian definition, the
two independent generating-function routes against each other, and closed forms (Hong-Ou-
Mandel, binomial totals under uniform loss, the single-mode case, the per-group mean).
"""
from __future__ import annotations

import itertools
from functools import lru_cache
from math import factorial

import numpy as np


def loss_channel_matrix(T: np.ndarray) -> np.ndarray:
    """A_Phi of App. C, Eq. loss_channel_matrix, for the M x M transfer matrix T."""
    T = np.asarray(T, dtype=np.complex128)
    M = T.shape[0]
    I = np.eye(M, dtype=np.complex128)
    Z = np.zeros((M, M), dtype=np.complex128)
    Td = T.conj().T
    return np.block([[Z, Td, I - Td @ T, Z],
                     [T.conj(), Z, Z, Z],
                     [I - T.T @ T.conj(), Z, Z, T.T],
                     [Z, Z, T, Z]])


def hafnian(A: np.ndarray) -> complex:
    """haf(A) = sum over perfect matchings of prod A_ij (memoised over vertex subsets)."""
    A = np.asarray(A, dtype=np.complex128)
    m = A.shape[0]
    if m % 2:
        return 0j

    @lru_cache(maxsize=None)
    def rec(mask: int) -> complex:
        if mask == 0:
            return 1.0 + 0j
        i = (mask & -mask).bit_length() - 1          # lowest free vertex
        rest = mask & ~(1 << i)
        tot = 0j
        r = rest
        while r:
            j = (r & -r).bit_length() - 1
            r &= r - 1
            tot += A[i, j] * rec(rest & ~(1 << j))
        return tot

    return complex(rec((1 << m) - 1))


def _repeat(blocks):
    """Index list: for each (offset, multiplicities) block, index offset + k repeated."""
    idx = []
    for off, mult in blocks:
        for k, c in enumerate(mult):
            idx += [off + k] * int(c)
    return idx


def _fact(v) -> float:
    return float(np.prod([factorial(int(c)) for c in v]))


def density_diag_haf(T: np.ndarray, p, n) -> float:
    """<n|rho|n> by Eq. density_matrix_fock_circuit (m = n)."""
    M = np.asarray(T).shape[0]
    A = loss_channel_matrix(T)
    idx = _repeat([(0, p), (M, n), (2 * M, p), (3 * M, n)])
    val = hafnian(A[np.ix_(idx, idx)]) if idx else 1.0 + 0j
    return float((val / (_fact(p) * _fact(n))).real)


def permanent(A: np.ndarray) -> complex:
    """Ryser's formula: perm A = (-1)^m sum_S (-1)^|S| prod_i sum_{j in S} A_ij."""
    A = np.asarray(A, dtype=np.complex128)
    m = A.shape[0]
    if m == 0:
        return 1.0 + 0j
    masks = np.arange(1, 1 << m, dtype=np.int64)
    sel = ((masks[:, None] >> np.arange(m)[None, :]) & 1).astype(np.float64)   # (2^m - 1, m)
    rows = sel @ A.T                                                              # row sums over S
    sign = np.where(np.sum(sel, axis=1) % 2 == 0, 1.0, -1.0)
    return complex((-1) ** m * np.sum(sign * np.prod(rows, axis=1)))


def density_diag_perm(T: np.ndarray, p, n) -> float:
    """<n|rho|n> by Eq. probs_fock_circuit, inputs carrying p in the first index block."""
    T = np.asarray(T, dtype=np.complex128)
    M = T.shape[0]
    Td = T.conj().T
    C = np.block([[np.eye(M) - Td @ T, Td], [T, np.zeros((M, M))]])
    idx = _repeat([(0, p), (M, n)])
    val = permanent(C[np.ix_(idx, idx)])
    return float((val / (_fact(p) * _fact(n))).real)


def _patterns(M: int, total_max: int):
    for n in itertools.product(range(total_max + 1), repeat=M):
        if sum(n) <= total_max:
            yield n


def binned_brute_force(fp, density=density_diag_haf) -> np.ndarray:
    """Unfolded P(b), 0 <= b_l <= N, by Eq. coarse_grained_Fock (every n with |n| <= N)."""
    N = int(np.sum(fp.photons))
    lab = np.asarray(fp.bin_of_mode)
    out = np.zeros((N + 1,) * fp.L)
    for n in _patterns(fp.M, N):
        b = [0] * fp.L
        for i, c in enumerate(n):
            b[lab[i]] += c
        out[tuple(b)] += density(fp.T, list(fp.photons), n)
    return out


def transfer_B(fp, z) -> np.ndarray:
    """B(z) = I - T^dag (I - Z) T with Z = diag(z_label(i)) over the output ports."""
    T = np.asarray(fp.T, dtype=np.complex128)
    zo = np.asarray(z, dtype=np.complex128)[np.asarray(fp.bin_of_mode)]
    return np.eye(fp.M) - T.conj().T @ ((1.0 - zo)[:, None] * T)


def pgf_permanent(fp, z) -> complex:
    """G(z) = perm(B(z)[p, p]) / prod p_j! (Ryser on the repeated matrix)."""
    B = transfer_B(fp, z)
    idx = _repeat([(0, fp.photons)])
    return permanent(B[np.ix_(idx, idx)]) / _fact(fp.photons)


def extraction_nodes(photons):
    """Occupied inputs J, the held input k0 (smallest p, lowest index), the other inputs
    and every node x (rows) of the roots-of-unity grid with its weight prod_k x_k."""
    p = np.asarray(photons)
    J = [j for j in range(len(p)) if p[j] > 0]
    if not J:
        return J, None, [], np.zeros((1, 0), dtype=np.complex128), np.ones(1, dtype=np.complex128)
    k0 = min(J, key=lambda j: (p[j], j))
    others = [j for j in J if j != k0]
    X, W = [], []
    for g in itertools.product(*[range(int(p[j]) + 1) for j in others]):
        x = {k0: 1.0 + 0j}
        w = 1.0 + 0j
        for j, gj in zip(others, g):
            x[j] = np.exp(2j * np.pi * gj / (int(p[j]) + 1))
            w *= x[j]
        X.append([x[j] for j in J])
        W.append(w)
    return J, k0, others, np.array(X, dtype=np.complex128), np.array(W, dtype=np.complex128)


def gray_digits(index: int, radices):
    """Digits of node ``index`` in the reflected mixed-radix Gray code over ``radices``
    (first digit fastest): n_d = floor(index / s_d) mod R_d, reflected (R_d - 1 - n_d) when
    floor(index / s_{d+1}) is odd, s_d = prod_{d' < d} R_d'."""
    g, stride = [], 1
    for R in radices:
        n = (index // stride) % R
        g.append(n if (index // (stride * R)) % 2 == 0 else R - 1 - n)
        stride *= R
    return g


def extraction_nodes_range(photons, begin: int, end: int):
    """As extraction_nodes, for the nodes [begin, end) in Gray-code order: the held input is
    the occupied one with the fewest photons (lowest port on ties), the digits run over the
    other occupied inputs in port order."""
    p = np.asarray(photons)
    J = [j for j in range(len(p)) if p[j] > 0]
    if not J:
        return J, None, [], np.zeros((1, 0), dtype=np.complex128), np.ones(1, dtype=np.complex128)
    k0 = min(J, key=lambda j: (p[j], j))
    others = [j for j in J if j != k0]
    radices = [int(p[j]) + 1 for j in others]
    X, W = [], []
    for i in range(begin, end):
        g = gray_digits(i, radices)
        x = {k0: 1.0 + 0j}
        w = 1.0 + 0j
        for j, gj, R in zip(others, g, radices):
            x[j] = np.exp(2j * np.pi * gj / R)
            w *= x[j]
        X.append([x[j] for j in J])
        W.append(w)
    return J, k0, others, np.array(X, dtype=np.complex128).reshape(len(X), len(J)), np.array(W, dtype=np.complex128)


def node_count(photons) -> int:
    p = np.asarray(photons)
    J = [j for j in range(len(p)) if p[j] > 0]
    if not J:
        return 1
    k0 = min(J, key=lambda j: (p[j], j))
    return int(np.prod([int(p[j]) + 1 for j in J if j != k0]))


def pgf_extract(fp, z, nodes=None, total=None) -> complex:
    """G(z) = [x^p] prod_j (B(z) x)_j^{p_j} by the roots-of-unity nodes (mean over them); with
    a subset of the nodes and ``total`` = the whole node count, that subset's share."""
    J, _, _, X, W = nodes if nodes is not None else extraction_nodes(fp.photons)
    if not J:
        return 1.0 + 0j
    B = transfer_B(fp, z)[np.ix_(J, J)]
    s = X @ B.T                                               # s[node, j] = (B x)_j
    pw = np.asarray(fp.photons)[J]
    F = np.prod(s ** pw[None, :], axis=1)
    return complex(np.sum(W * F) / (total if total else len(W)))


def pgf_grid(fp, radix=None, node_range=None) -> np.ndarray:
    """G(omega^k) on the roots-of-unity grid of the output groups (default N_l + 1); with
    node_range = (begin, end), only those nodes' share (Gray-code order)."""
    radix = fp.radix if radix is None else np.asarray(radix)
    total = None
    if node_range is None:
        nodes = extraction_nodes(fp.photons)
    else:
        nodes = extraction_nodes_range(fp.photons, *node_range)
        total = node_count(fp.photons)
    G = np.empty(tuple(int(r) for r in radix), dtype=np.complex128)
    for k in itertools.product(*[range(int(r)) for r in radix]):
        z = [np.exp(2j * np.pi * kl / int(r)) for kl, r in zip(k, radix)]
        G[k] = pgf_extract(fp, z, nodes, total)
    return G


def table(fp, oversample: int = 1, node_range=None) -> dict:
    """Folded table P~(b), 0 <= b_l <= N_l, on the grid oversample (N_l + 1) per axis.

    With node_range = (begin, end): the partial table of those nodes' share G_p of G, in the
    half-grid form of the inverse DFT - the last axis k <= R/2 only, weight 1 at k = 0 (and
    k = R/2 for even R) and 2 elsewhere, real part - which is exact for the whole G
    (G(-k) = conj G(k)); a node range's share alone has no such symmetry, so this is the
    form whose shares sum to the whole table over a partition of the nodes."""
    from . import dft
    radix = fp.radix * int(oversample)
    G = pgf_grid(fp, radix, node_range)
    if node_range is not None:
        R = int(radix[-1])
        c = np.zeros(R)
        c[:R // 2 + 1] = 2.0
        c[0] = 1.0
        if R % 2 == 0:
            c[R // 2] = 1.0
        G = G * c
    Pc = dft(G, radix)
    sl = tuple(slice(0, int(c) + 1) for c in fp.cutoff)
    return {"P": Pc.real[sl].copy(), "imag_max": float(np.abs(Pc.imag).max()), "G": G}


def group_means(fp) -> np.ndarray:
    """Mean count per group, sum_{i in group} sum_j |T_ij|^2 p_j (each photon reaches
    output i with probability |T_ij|^2, whatever the interference)."""
    T = np.asarray(fp.T)
    per_out = (np.abs(T) ** 2) @ np.asarray(fp.photons, dtype=np.float64)
    out = np.zeros(fp.L)
    for i, l in enumerate(fp.bin_of_mode):
        out[l] += per_out[i]
    return out
