"""Gaussian-state algebra of the oracle (numpy, FP64).  TEST INFRASTRUCTURE ONLY.

Builds, from a :class:`synth.Problem`, the normally ordered covariance Sigma^(1), the mean
vector z-bar, and from them the adjacency data XA and gamma of Sec. II:

* mode vector zeta = (a_1..a_n', a_1^dag..a_n'^dag), n' = M K, internal modes
  external-major: index (j, l) -> j K + l (Sec. VI, Eq. internal_mode_detection_pattern);
* Sigma^(s) = (1 - s)/2 I + [[N^T, Mm], [Mm^*, N]] with N_ij = <a_i^dag a_j>,
  Mm_ij = <a_i a_j> (Sec. II, covariance form); Sigma^(1) is the s = 1 member;
* A = X (I - Sigma^{-1}), gamma = X Sigma^{-1} z-bar, Sigma = Sigma^(-1) = I + Sigma^(1)
  (Eqs. defA, defgamma, x_matrix_husimi_cov), hence XA = I - Sigma^{-1};
* vacuum probability Pr(0) (Eq. vacuum_probability).

Propagation reading: a passive lossy map a_out = T_full a_in sends the normally ordered
moments to N_out = T_full^* N_in T_full^T and Mm_out = T_full Mm_in T_full^T, i.e.
Sigma^(1)_out = W Sigma^(1)_in W^dag with W = T_full (+) T_full^*; vacuum loss modes add
nothing to normally ordered moments.  T_full[(j,l),(i,k)] = T[j,i] V_i[l,k].
"""
from __future__ import annotations

import numpy as np


def full_transfer(prob) -> np.ndarray:
    """(M K) x (M K) transfer on the external (x) internal space: (T (x) I_K) blockdiag(V_i)."""
    M, K = prob.M, prob.K
    Tf = np.zeros((M * K, M * K), dtype=np.complex128)
    for j in range(M):
        for i in range(M):
            Vi = np.eye(K) if prob.V is None else prob.V[i]
            Tf[j * K:(j + 1) * K, i * K:(i + 1) * K] = prob.T[j, i] * Vi
    return Tf


def sigma1_zbar(prob):
    """Normally ordered covariance Sigma^(1) (n x n) and mean z-bar (n) of the output."""
    MK = prob.M * prob.K
    r = np.asarray(prob.r, dtype=np.float64).reshape(MK)
    # single-mode squeezed vacua: <b^dag b> = sinh^2 r, <b b> = sinh r cosh r
    N_in = np.diag(np.sinh(r) ** 2).astype(np.complex128)
    Mm_in = np.diag(np.sinh(r) * np.cosh(r)).astype(np.complex128)
    Tf = full_transfer(prob)
    N_out = Tf.conj() @ N_in @ Tf.T
    Mm_out = Tf @ Mm_in @ Tf.T
    sigma1 = np.block([[N_out.T, Mm_out], [Mm_out.conj(), N_out]])
    a = np.zeros(MK, dtype=np.complex128) if prob.alpha is None else \
        np.asarray(prob.alpha, dtype=np.complex128).reshape(MK)
    mean = Tf @ a
    zbar = np.concatenate([mean, mean.conj()])
    return sigma1, zbar


def xmat(n: int) -> np.ndarray:
    h = n // 2
    X = np.zeros((n, n))
    X[:h, h:] = np.eye(h)
    X[h:, :h] = np.eye(h)
    return X


def adjacency(sigma1: np.ndarray, zbar: np.ndarray):
    """XA = I - Sigma^{-1} and gamma = X Sigma^{-1} z-bar, Sigma = I + Sigma^(1)."""
    n = sigma1.shape[0]
    Sigma = np.eye(n) + sigma1
    Si = np.linalg.inv(Sigma)
    XA = np.eye(n) - Si
    gamma = xmat(n) @ (Si @ zbar)
    return XA, gamma


def mode_labels(prob) -> np.ndarray:
    """Detector group of each of the n rows of the mode vector."""
    lab = np.repeat(np.asarray(prob.bin_of_mode, dtype=np.int32), prob.K)
    return np.concatenate([lab, lab]).astype(np.int32)


def vacuum_probability(XA: np.ndarray, gamma: np.ndarray) -> float:
    """Pr(0) = exp(-1/2 gamma^T (I - XA)^{-1} X gamma) sqrt(det(I - XA))."""
    n = XA.shape[0]
    Kone = np.eye(n) - XA
    expo = gamma @ np.linalg.solve(Kone, xmat(n) @ gamma)
    sign, logdet = np.linalg.slogdet(Kone)
    val = np.exp(-0.5 * expo) * np.sqrt(sign) * np.exp(0.5 * logdet)
    return float(np.real(val))
