// Host FP64 Gaussian-state algebra shared by the plan files (gbsbin_host.cpp defines it).
// Not part of the public ABI.
#pragma once

#include <complex>
#include <functional>
#include <vector>

#include "../../include/gbsbin.h"

namespace gbsbin {

// XA = I - Sigma^{-1}, gamma = X Sigma^{-1} z-bar and Xgamma = Sigma^{-1} z-bar of a problem's
// state (its physical description or sigma1 / zbar; Sec. II, Eqs. defA, defgamma); n = 2 M K.
// M, K and the state's pointers must have been checked.  ERR_ARG (non-finite input),
// ERR_NONPHYSICAL (not Hermitian, or Sigma - I/2 not positive definite).
int host_state(const gbsbin_problem* p, int n, std::vector<std::complex<double>>& XA,
               std::vector<std::complex<double>>& gamma, std::vector<std::complex<double>>& Xgamma);

// log q(A, gamma, 1) = 1/2 gamma^T (I - XA)^-1 X gamma - 1/2 log det(I - XA) (Sec. III, Eq. q_d
// at w = 1) by an unpivoted LU; every pivot has Re > 0 for a physical state, so the sum of
// principal logarithms is the branch continuous from XA = 0.  *minpiv (may be null) receives
// the smallest pivot real part.  Pr(0) = exp(-log q(1)).
std::complex<double> host_logq1(const std::vector<std::complex<double>>& XA,
                                const std::vector<std::complex<double>>& gamma,
                                const std::vector<std::complex<double>>& Xgamma, int n, double* minpiv);

// Host threads the state algebra uses: the hardware concurrency capped at 16, or the
// environment variable GBSBIN_HOST_THREADS.
int host_threads();
// fn(t, nthreads) for t = 0 .. nthreads - 1 on the pool's threads (the caller runs t = 0);
// returns when every call has returned.  One job at a time.
void parallel_run(int nthreads, const std::function<void(int, int)>& fn);

}  // namespace gbsbin
