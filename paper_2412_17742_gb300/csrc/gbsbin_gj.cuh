// CTA-wide dense building blocks of the reverse pass, over an arithmetic class Ar (ArF64 or
// ArDF, gbsbin_df.cuh): the in-place inverse of a matrix in global (L2-resident) memory by
// blocked Gauss-Jordan elimination without pivoting, and a staged product C (+)= +-A B with
// strided operands.  Both stage nb-wide panels in shared memory (Pc: m x nb, Rx: nb x m,
// Dg: nb x nb) and update the matrix in 4 x 4 register tiles.  Every thread of the CTA calls
// them; they end with a barrier.  A thread's 4 x 4 tile takes four consecutive rows and four
// columns tcols apart (tcols = ceil(columns / 4)), so that the threads of a warp read
// consecutive 16-byte entries of the staged rows (no shared-memory bank conflicts) and of the
// matrix (coalesced).
#pragma once

#include <cuda_runtime.h>

#include "gbsbin_df.cuh"

namespace gbsbin {

constexpr int kGjTile = 4;
constexpr int kGjMaxNb = 16;

// W (m x m, row stride ld) <- W^{-1}.  Per step of nb pivots B = [K, K + bs): the bs x bs
// block W_BB is inverted in shared memory (one element per thread per pivot: the scalar rule
// w'_kk = 1/p, w'_kj = w_kj/p, w'_ik = -w_ik/p, w'_ij = w_ij - w_ik w_kj/p), the block's rows
// become inv(W_BB) W_BJ, and the rest takes W_IJ - W_IB inv(W_BB) W_BJ with W_IB <- -W_IB inv(W_BB).
// The pivots are those of the unpivoted LU of W.  nb <= kGjMaxNb, nb^2 <= blockDim.x.  Rn (nb x m,
// may be null) takes inv(W_BB) W_BJ one entry per thread; without it a thread forms a column.
template <class Ar>
__device__ void gj_invert(typename Ar::E* W, int m, int ld, int nbm, typename Ar::E* Pc, typename Ar::E* Rx,
                          typename Ar::E* Dg, typename Ar::E* Rn) {
  using E = typename Ar::E;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int tcols = (m + kGjTile - 1) / kGjTile, ntiles = tcols * tcols;
  for (int K = 0; K < m; K += nbm) {
    const int bs = min(nbm, m - K);
    for (int t = tid; t < m * bs; t += NT) {
      const int i = t / bs, c = t - (t / bs) * bs;
      Pc[i * nbm + c] = (i >= K && i < K + bs) ? Ar::zero() : W[(size_t)i * ld + K + c];
    }
    for (int t = tid; t < bs * m; t += NT) {
      const int r = t / m, j = t - (t / m) * m;
      Rx[r * m + j] = W[(size_t)(K + r) * ld + j];
    }
    if (tid < bs * bs) Dg[tid] = W[(size_t)(K + tid / bs) * ld + K + tid % bs];
    __syncthreads();
    for (int k = 0; k < bs; ++k) {
      E nv = Ar::zero();
      if (tid < bs * bs) {
        const int i = tid / bs, j = tid - (tid / bs) * bs;
        const E p = Ar::recip(Dg[k * bs + k]);
        if (i == k && j == k) nv = p;
        else if (i == k) nv = Ar::mul(Dg[k * bs + j], p);
        else if (j == k) nv = Ar::neg(Ar::mul(Dg[i * bs + k], p));
        else nv = Ar::fms(Dg[tid], Ar::mul(Dg[i * bs + k], p), Dg[k * bs + j]);
      }
      __syncthreads();
      if (tid < bs * bs) Dg[tid] = nv;
      __syncthreads();
    }
    // the block's rows: inv(W_BB) W[B, :] outside the block's columns, inv(W_BB) on them
    E* Rb = Rx;
    if (Rn) {                                          // one entry per thread into Rn
      for (int t = tid; t < bs * m; t += NT) {
        const int r = t / m, j = t - (t / m) * m;
        if (j >= K && j < K + bs) {
          Rn[t] = Dg[r * bs + (j - K)];
          continue;
        }
        E acc = Ar::zero();
        for (int c = 0; c < bs; ++c) acc = Ar::fma(Dg[r * bs + c], Rx[c * m + j], acc);
        Rn[t] = acc;
      }
      Rb = Rn;
    } else {                                           // a column per thread, in place
      for (int j = tid; j < m; j += NT) {
        if (j >= K && j < K + bs) {
          for (int r = 0; r < bs; ++r) Rx[r * m + j] = Dg[r * bs + (j - K)];
          continue;
        }
        E col[kGjMaxNb];
#pragma unroll
        for (int c = 0; c < kGjMaxNb; ++c)
          if (c < bs) col[c] = Rx[c * m + j];
        for (int r = 0; r < bs; ++r) {
          E acc = Ar::zero();
#pragma unroll
          for (int c = 0; c < kGjMaxNb; ++c)
            if (c < bs) acc = Ar::fma(Dg[r * bs + c], col[c], acc);
          Rx[r * m + j] = acc;
        }
      }
    }
    __syncthreads();
    for (int tt = tid; tt < ntiles; tt += NT) {
      const int i0 = (tt / tcols) * kGjTile, jt = tt - (tt / tcols) * tcols;
      E acc[kGjTile][kGjTile];
#pragma unroll
      for (int r = 0; r < kGjTile; ++r)
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) {
          const int i = i0 + r, j = jt + q * tcols;
          acc[r][q] = (i < m && j < m && (j < K || j >= K + bs)) ? W[(size_t)i * ld + j] : Ar::zero();
        }
      for (int c = 0; c < bs; ++c) {
        E pv[kGjTile], rv[kGjTile];
#pragma unroll
        for (int r = 0; r < kGjTile; ++r) pv[r] = i0 + r < m ? Pc[(i0 + r) * nbm + c] : Ar::zero();
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) rv[q] = jt + q * tcols < m ? Rb[c * m + jt + q * tcols] : Ar::zero();
#pragma unroll
        for (int r = 0; r < kGjTile; ++r)
#pragma unroll
          for (int q = 0; q < kGjTile; ++q) acc[r][q] = Ar::fms(acc[r][q], pv[r], rv[q]);
      }
#pragma unroll
      for (int r = 0; r < kGjTile; ++r)
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) {
          const int i = i0 + r, j = jt + q * tcols;
          if (i >= m || j >= m) continue;
          W[(size_t)i * ld + j] = (i >= K && i < K + bs) ? Rb[(i - K) * m + j] : acc[r][q];
        }
    }
    __syncthreads();
  }
}

// C (m x n, row stride ldc) <- (acc ? C : 0) + sgn sum_k A(i, k) B(k, j), sgn = -1 if neg, with
// A(i, k) = A[i ars + k acs] and B(k, j) = B[k brs + j bcs] (strides give transposes).  k in
// blocks of kb: A's panel (m x kb) in As, B's (kb x n) in Bs; C read and written once per block.
// As holds m * kb entries, Bs kb * n.
template <class Ar>
__device__ void gemm_staged(typename Ar::E* C, int ldc, const typename Ar::E* A, long long ars, long long acs,
                            const typename Ar::E* B, long long brs, long long bcs, int m, int n, int k, bool acc,
                            bool neg, int kb, typename Ar::E* As, typename Ar::E* Bs) {
  using E = typename Ar::E;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int trows = (m + kGjTile - 1) / kGjTile, tcols = (n + kGjTile - 1) / kGjTile, ntiles = trows * tcols;
  if (k == 0 && !acc) {
    for (int t = tid; t < m * n; t += NT) C[(size_t)(t / n) * ldc + t % n] = Ar::zero();
    __syncthreads();
    return;
  }
  for (int K = 0; K < k; K += kb) {
    const int bs = min(kb, k - K);
    for (int t = tid; t < m * bs; t += NT) {
      const int i = t / bs, c = t - (t / bs) * bs;
      const E v = A[i * ars + (K + c) * acs];
      As[i * kb + c] = neg ? Ar::neg(v) : v;
    }
    for (int t = tid; t < bs * n; t += NT) {
      const int c = t / n, j = t - (t / n) * n;
      Bs[c * n + j] = B[(K + c) * brs + j * bcs];
    }
    __syncthreads();
    const bool first = K == 0 && !acc;
    for (int tt = tid; tt < ntiles; tt += NT) {
      const int i0 = (tt / tcols) * kGjTile, jt = tt - (tt / tcols) * tcols;
      E cv[kGjTile][kGjTile];
#pragma unroll
      for (int r = 0; r < kGjTile; ++r)
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) {
          const int i = i0 + r, j = jt + q * tcols;
          cv[r][q] = (!first && i < m && j < n) ? C[(size_t)i * ldc + j] : Ar::zero();
        }
      for (int c = 0; c < bs; ++c) {
        E av[kGjTile], bv[kGjTile];
#pragma unroll
        for (int r = 0; r < kGjTile; ++r) av[r] = i0 + r < m ? As[(i0 + r) * kb + c] : Ar::zero();
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) bv[q] = jt + q * tcols < n ? Bs[c * n + jt + q * tcols] : Ar::zero();
#pragma unroll
        for (int r = 0; r < kGjTile; ++r)
#pragma unroll
          for (int q = 0; q < kGjTile; ++q) cv[r][q] = Ar::fma(av[r], bv[q], cv[r][q]);
      }
#pragma unroll
      for (int r = 0; r < kGjTile; ++r)
#pragma unroll
        for (int q = 0; q < kGjTile; ++q) {
          const int i = i0 + r, j = jt + q * tcols;
          if (i < m && j < n) C[(size_t)i * ldc + j] = cv[r][q];
        }
    }
    __syncthreads();
  }
}

}  // namespace gbsbin
