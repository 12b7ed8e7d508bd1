"""CPU oracle for binned photon-number distributions (arXiv:2412.17742).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library and its Python
binding never do, and they share no code with it.

Pieces:

* :mod:`oracle.state` - Gaussian-state algebra in numpy FP64 (Sigma^(1), z-bar, XA,
  gamma, Pr(0)); Sec. II and Sec. VIII (output covariance), Sec. VI (internal modes).
* ``gbs_oracle.c`` - the per-point evaluation of log q(A, gamma, D(w)) (Sec. III,
  Eq. q_d, with one w per detector group as in Sec. VI, Eq. Lamb_lhaf_master) by an
  unpivoted LU, and a direct, compensated inverse DFT; plain C, FP64, OpenMP over points.
* :mod:`oracle.lhaf` - brute-force loop Hafnians, Fock probabilities and binned sums
  (Sec. II, Eq. gbs_probability_distribution; Sec. VI, Eq. coarse_grained_prob).
* :func:`distinguishable_ones` - one photon per port for fully distinguishable sources (App. D's
  limit), from the sources' closed-form output generating functions by a positive subset
  dynamic programme (``gbs_oracle.c``).

Every function here is pinned by ``-m "not gpu"`` tests (brute force, closed forms,
invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

from . import state

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIBPATH = os.path.join(_LIBDIR, "libgbs_oracle.so")
_SRC = os.path.join(_HERE, "gbs_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in-tree (gcc, OpenMP, portable flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIBPATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_logq_grid.argtypes = [ctypes.c_int, dp, dp, ip, ctypes.c_int, ip, dp, dp, ip,
                                         ctypes.c_int]
        lib.oracle_logq_grid.restype = ctypes.c_int
        lib.oracle_logq_points.argtypes = [ctypes.c_int, dp, dp, ip, ctypes.c_int, ip,
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.c_long, dp, dp, ip,
                                           ctypes.c_int]
        lib.oracle_logq_points.restype = ctypes.c_int
        lib.oracle_dft.argtypes = [ctypes.c_int, ip, dp, dp]
        lib.oracle_dft.restype = ctypes.c_int
        lib.oracle_distinguishable_ones.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.oracle_distinguishable_ones.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def plan(prob):
    """Host-side data of a problem: XA, gamma and the row labels."""
    sigma1, zbar = state.sigma1_zbar(prob)
    XA, gamma = state.adjacency(sigma1, zbar)
    return XA, gamma, state.mode_labels(prob)


def logq_grid(XA, gamma, labels, radix, nthreads: int = 0):
    """log q at every point of the grid prod(radix) (flattened, last axis fastest).
    Returns (logq complex (N,), min Re pivot (N,), status (N,))."""
    lib = _load()
    XA = np.ascontiguousarray(XA, dtype=np.complex128)
    gamma = np.ascontiguousarray(gamma, dtype=np.complex128)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    radix = np.ascontiguousarray(radix, dtype=np.int32)
    npts = int(np.prod(radix.astype(np.int64)))
    logq = np.zeros(npts, dtype=np.complex128)
    minre = np.zeros(npts, dtype=np.float64)
    st = np.zeros(npts, dtype=np.int32)
    lib.oracle_logq_grid(XA.shape[0], _dp(XA.view(np.float64)), _dp(gamma.view(np.float64)),
                         _ip(labels), len(radix), _ip(radix), _dp(logq.view(np.float64)),
                         _dp(minre), _ip(st), int(nthreads))
    return logq, minre, st


def logq_points(XA, gamma, labels, radix, digits, nthreads: int = 0):
    """log q at the grid points whose digits are the rows of ``digits`` (count, L)
    (same per-point algorithm as :func:`logq_grid`).  Returns (logq, min pivot, status)."""
    lib = _load()
    XA = np.ascontiguousarray(XA, dtype=np.complex128)
    gamma = np.ascontiguousarray(gamma, dtype=np.complex128)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    radix = np.ascontiguousarray(radix, dtype=np.int32)
    digits = np.atleast_2d(np.asarray(digits, dtype=np.int64))
    strides = np.ones(len(radix), dtype=np.int64)
    for l in range(len(radix) - 2, -1, -1):
        strides[l] = strides[l + 1] * radix[l + 1]
    idx = np.ascontiguousarray(digits @ strides, dtype=np.int64)
    cnt = len(idx)
    logq = np.zeros(cnt, dtype=np.complex128)
    minre = np.zeros(cnt, dtype=np.float64)
    st = np.zeros(cnt, dtype=np.int32)
    lib.oracle_logq_points(XA.shape[0], _dp(XA.view(np.float64)), _dp(gamma.view(np.float64)), _ip(labels),
                           len(radix), _ip(radix), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), cnt,
                           _dp(logq.view(np.float64)), _dp(minre), _ip(st), int(nthreads))
    return logq, minre, st


def dft(values, radix) -> np.ndarray:
    """out(b) = (1/N) sum_k values(k) exp(-2 pi i k.b / R), table shaped like radix."""
    lib = _load()
    radix = np.ascontiguousarray(radix, dtype=np.int32)
    v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128).reshape(-1))
    out = np.zeros_like(v)
    rc = lib.oracle_dft(len(radix), _ip(radix), _dp(v.view(np.float64)), _dp(out.view(np.float64)))
    if rc != 0:
        raise RuntimeError(f"oracle_dft failed: {rc}")
    return out.reshape(tuple(int(r) for r in radix))


def pgf_grid(prob, radix=None, nthreads: int = 0):
    """G(omega^k) = q(omega^k) / q(1) on the grid (default radix N_l + 1)."""
    XA, gamma, labels = plan(prob)
    radix = prob.radix if radix is None else np.asarray(radix)
    logq, minre, st = logq_grid(XA, gamma, labels, radix, nthreads)
    return np.exp(logq - logq[0]), logq, minre, st


def binned(prob, radix=None, nthreads: int = 0) -> dict:
    """Folded binned table P~(b) on the grid ``radix`` (default N_l + 1).

    Returns a dict with ``P`` (real table), ``imag_max`` (max |Im P~|, a round-off
    diagnostic), ``logq`` (all points), ``min_pivot`` and ``status``."""
    G, logq, minre, st = pgf_grid(prob, radix, nthreads)
    radix = prob.radix if radix is None else np.asarray(radix)
    Pc = dft(G, radix)
    return {"P": Pc.real.copy(), "imag_max": float(np.abs(Pc.imag).max()), "logq": logq,
            "min_pivot": float(minre.min()), "status": st}


def unfolded(prob, oversample: int = 4, nthreads: int = 0) -> np.ndarray:
    """P(b) for 0 <= b_l <= N_l, from the folded table on a grid oversample x larger
    per axis (exact up to the probability mass beyond the larger grid)."""
    radix = prob.radix * oversample
    P = binned(prob, radix, nthreads)["P"]
    sl = tuple(slice(0, int(c) + 1) for c in prob.cutoff)
    return P[sl]


def squeezed_pgf_taylor(r: float, y0: float, order: int) -> np.ndarray:
    """Taylor coefficients a_j, j <= order, of a single-mode squeezed vacuum's photon-number
    generating function g(y) = (1 - tanh^2(r) y^2)^(-1/2) / cosh r (Sec. II) about y = y0.
    With u(x) = 1 - t^2 (y0 + x)^2 = u0 + u1 x + u2 x^2, the power w = u^(-1/2) follows from
    J. C. P. Miller's recurrence n u0 w_n = sum_{k=1}^{min(n,2)} (k (p + 1) - n) u_k w_{n-k},
    p = -1/2."""
    t2 = np.tanh(r) ** 2
    u = [1.0 - t2 * y0 * y0, -2.0 * t2 * y0, -t2]
    p = -0.5
    w = np.zeros(order + 1)
    w[0] = u[0] ** p
    for n in range(1, order + 1):
        acc = 0.0
        for k in (1, 2):
            if k <= n:
                acc += (k * (p + 1.0) - n) * u[k] * w[n - k]
        w[n] = acc / (n * u[0])
    return w / np.cosh(r)


def distinguishable_ones(r, T) -> float:
    """Probability of one photon on every output port for fully distinguishable sources
    (App. D's limit: source s in its own internal mode), r[s] the squeezing of source s and
    T (ports x sources) the lossy transfer matrix: the coefficient of z_1 ... z_M in
    prod_s g_s(1 - P_s + sum_k |T_ks|^2 z_k), by the positive subset dynamic programme of
    ``oracle_distinguishable_ones`` (``gbs_oracle.c``)."""
    T = np.asarray(T)
    M, S = T.shape
    pk = np.ascontiguousarray(np.abs(T) ** 2, dtype=np.float64)
    a = np.ascontiguousarray(np.stack([squeezed_pgf_taylor(float(r[s]), 1.0 - pk[:, s].sum(), M)
                                       for s in range(S)]), dtype=np.float64)
    out = ctypes.c_double()
    rc = _load().oracle_distinguishable_ones(M, S, _dp(pk), _dp(a), ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"oracle_distinguishable_ones failed: {rc}")
    return out.value


def logdet_series(XA, d, terms: int) -> complex:
    """log det(I - D XA) = -sum_{k>=1} tr((D XA)^k)/k (Sec. IV, Eq. useful_series_expansions),
    a branch that involves no LU: it converges because ||D XA|| = ||XA|| < 1."""
    B = np.asarray(d)[:, None] * np.asarray(XA)
    P = np.eye(B.shape[0], dtype=np.complex128)
    tot = 0.0 + 0j
    for k in range(1, terms + 1):
        P = P @ B
        tot -= np.trace(P) / k
    return complex(tot)
