// Reverse mode through the binned distribution: dL/dP(b) -> dL/dXA, dL/dgamma
// (the host then chains to Sigma^(1), z-bar and the physical parameters).  A shard's plan
// (a slice of the evaluated half grid) gives the gradient of its partial table: the slices'
// gradients sum to the whole one.
//
// Forward (per evaluated point k, arXiv:2412.17742 Sec. III Eq. q_d with the grouping of
// Sec. VI):  M_k = conj(D_k) - XA,  x_k = M_k^{-1} X gamma,
//            log q_k = 1/2 gamma^T x_k - 1/2 log det(D_k M_k),  G_k = exp(log q_k - log q_0),
//            P(b) = (1/N) sum_k G_k omega^{-k.b}.
// Reverse, with pbar(b) = dL/dP(b) real:
//   gbar_k  = (1/N) sum_b pbar(b) omega^{-k.b}          (adjoint of the inverse DFT)
//   a_k     = c_k gbar_k G_k, c_k = 2 for points whose conjugate partner is not evaluated,
//             1 for self-conjugate-axis points (k_{L-1} = 0 or R/2)
//   beta_k  = a_k for k != 0,  beta_0 = a_0 - sum_k a_k  (q_0 normalises every G_k)
//   dL      = Re sum_k beta_k d log q_k, and with y_k = M_k^{-T} gamma:
//   d log q = 1/2 sum_ij (y_i x_j + (M^{-1})_ji) dXA_ij + 1/2 (x + X y)^T dgamma
// so dL/dXA (bilinear) = 1/2 sum_k beta_k (y_k x_k^T + M_k^{-T}) and
//    dL/dgamma        = 1/2 sum_k beta_k (x_k + X y_k).
// Nothing of the forward is stored but log q: each point's M_k is rebuilt from -XA and the
// point's roots and inverted in place by a blocked Gauss-Jordan elimination without pivoting
// (its pivots are those of the forward's unpivoted LU), nb pivots per step: the nb x nb
// diagonal block inverted in shared memory, the block's rows multiplied by that inverse, and
// a rank-nb update of the rest streamed through registers in 4 x 4 tiles - n^3 complex
// multiply-adds per point, the same as LU plus inverse from stored factors, in the plan's
// arithmetic: FP64, or pairs of FP32 (~46 bits) on the FMA pipe for FP32-refine plans.  One
// CTA per SM, its matrix in an L2-resident slot, each accumulating its points into its own
// partials, reduced over CTAs in FP64 in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_backward_tree.h"
#include "gbsbin_gj.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// out[o, k, s] = sum_{b < nin} in[o, b, s] tw[(k b) mod R],  k < nout  (complex in, complex out)
__global__ void k_adj_axis(const double2* __restrict__ in, double2* __restrict__ out, long long outer, int nin,
                           int nout, long long inner, int R, const double2* __restrict__ tw) {
  const long long total = outer * nout * inner;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long s = t % inner;
    long long rest = t / inner;
    int k = (int)(rest % nout);
    long long o = rest / nout;
    const double2* src = in + o * nin * inner + s;
    double2 acc = make_double2(0.0, 0.0);
    int idx = 0;
    for (int b = 0; b < nin; ++b) {
      double2 v = src[(long long)b * inner], w = tw[idx];
      acc.x = fma(v.x, w.x, fma(-v.y, w.y, acc.x));
      acc.y = fma(v.x, w.y, fma(v.y, w.x, acc.y));
      idx += k;
      if (idx >= R) idx -= R;
    }
    out[t] = acc;
  }
}

__global__ void k_real_to_complex(const double* __restrict__ in, long long n, double2* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = make_double2(in[t], 0.0);
}

// a_k = c_k gbar_k G_k / N (gbar still unscaled, over the whole half grid), per evaluated
// point of this plan; a shard's point 0 outside its slice only normalises (a = 0 there, so
// beta_0 = -sum of the slice's a_k)
__global__ void k_adj_weights(const double2* __restrict__ gbar, const double2* __restrict__ logq, GridDesc g,
                              double2* __restrict__ a) {
  const double2 l0 = logq[0];
  const double scale = 1.0 / (double)g.npts;
  const int R = g.radix[g.L - 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.n_eval;
       e += (long long)gridDim.x * blockDim.x) {
    if (e == 0 && g.e_lo > 0) {
      a[e] = make_double2(0.0, 0.0);
      continue;
    }
    const long long t = global_point(e, g);
    const int klast = (int)(t % g.half);
    const double c = (klast == 0 || 2 * klast == R) ? 1.0 : 2.0;
    double2 v = logq[e];
    double m = exp(v.x - l0.x);
    double s, co;
    sincos(v.y - l0.y, &s, &co);
    double2 G = make_double2(m * co, m * s);
    double2 gb = gbar[t];
    a[e] = make_double2(c * scale * (gb.x * G.x - gb.y * G.y), c * scale * (gb.x * G.y + gb.y * G.x));
  }
}

// beta_0 = a_0 - sum_k a_k; one block, fixed order
__global__ void k_adj_beta0(double2* __restrict__ a, long long n) {
  __shared__ double sr[32], si[32];
  double r = 0.0, im = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    r += a[e].x;
    im += a[e].y;
  }
  r = warp_sum_d(r);
  im = warp_sum_d(im);
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = r;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += sr[w];
      ti += si[w];
    }
    a[0] = make_double2(a[0].x - tr, a[0].y - ti);
  }
}

// Per point: W = M^{-1} by blocked Gauss-Jordan; accumulate into this CTA's partials (S
// transposed: ST[j][i] = S[i][j], so that the term M^{-T} reads W row by row).
constexpr int kGjThreads = 256;

template <class Ar>
__global__ void __launch_bounds__(kGjThreads) k_backward_gj(BackwardArgs b) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = b.n, nbm = b.nb, tid = threadIdx.x, NT = kGjThreads;
  const GridDesc& g = b.grid;
  E* Pc = reinterpret_cast<E*>(smem);                 // n x nbm: W[:, B], rows of B zero
  E* Rx = Pc + (size_t)n * nbm;                       // nbm x n: inv(W_BB) W[B, :]
  E* Dg = Rx + (size_t)nbm * n;                       // bs x bs: W_BB, inverted in place
  E* gE = Dg + nbm * nbm;                             // n: gamma
  E* xgE = gE + n;                                    // n: X gamma
  E* xv = xgE + n;                                    // n: x = W X gamma
  E* yv = xv + n;                                     // n: y = W^T gamma
  double2* wr = reinterpret_cast<double2*>(yv + n);   // L: this point's roots
  E* Rn = b.rn ? reinterpret_cast<E*>(wr + GBSBIN_MAX_L) : nullptr;   // nb x n, if it fits
  E* W = reinterpret_cast<E*>(reinterpret_cast<char*>(b.ws) + (size_t)blockIdx.x * (size_t)b.ws_slot_bytes);
  E* ST = reinterpret_cast<E*>(b.partS) + (size_t)blockIdx.x * n * n;
  E* sg = reinterpret_cast<E*>(b.partg) + (size_t)blockIdx.x * n;
  for (int t = tid; t < n * n; t += NT) ST[t] = Ar::zero();
  for (int t = tid; t < n; t += NT) {
    sg[t] = Ar::zero();
    gE[t] = Ar::from(b.gamma[t]);
    xgE[t] = Ar::from(b.Xgamma[t]);
  }

  for (long long e = blockIdx.x; e < b.n_eval; e += gridDim.x) {
    const double2 beta = b.beta[e];
    if (beta.x == 0.0 && beta.y == 0.0) continue;  // no contribution
    if (tid < g.L) wr[tid] = grid_root(b.tw, g, tid, point_digit(e, g, tid));
    __syncthreads();
    for (int t = tid; t < n * n; t += NT) {          // M = conj(D) - XA
      const int i = t / n;
      double2 v = b.NXA[t];
      if (i * n + i == t) {
        const double2 d = wr[b.label[i]];
        v.x += d.x;
        v.y -= d.y;
      }
      W[t] = Ar::from(v);
    }
    __syncthreads();
    gj_invert<Ar>(W, n, n, nbm, Pc, Rx, Dg, Rn);
    // x = W X gamma (a warp per row), y = W^T gamma (a thread per column)
    {
      const int lane = tid & 31, warp = tid >> 5;
      for (int i = warp; i < n; i += NT / 32) {
        E acc = Ar::zero();
        for (int j = lane; j < n; j += 32) acc = Ar::fma(W[(size_t)i * n + j], xgE[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = Ar::add(acc, shfl_xor(acc, o));
        if (lane == 0) xv[i] = acc;
      }
      for (int j = tid; j < n; j += NT) {
        E acc = Ar::zero();
        for (int i = 0; i < n; ++i) acc = Ar::fma(W[(size_t)i * n + j], gE[i], acc);
        yv[j] = acc;
      }
    }
    __syncthreads();
    // ST[j][i] += beta/2 (y_i x_j + W[j][i]);  sg += beta/2 (x + X y)
    const E hb = Ar::from(make_double2(0.5 * beta.x, 0.5 * beta.y));
    for (int t = tid; t < n * n; t += NT) {
      const int j = t / n, i = t - (t / n) * n;
      ST[t] = Ar::fma(hb, Ar::fma(yv[i], xv[j], W[t]), ST[t]);
    }
    const int h = n / 2;
    for (int i = tid; i < n; i += NT) sg[i] = Ar::fma(hb, Ar::add(xv[i], yv[i < h ? i + h : i - h]), sg[i]);
    __syncthreads();
  }
}

// outS[i][j] = sum over CTAs c of ST_c[j][i], outg[i] = sum_c sg_c[i] (FP64, fixed order)
template <class Ar>
__global__ void k_backward_reduce(const void* __restrict__ partS, const void* __restrict__ partg, int nparts, int n,
                                  double2* __restrict__ outS, double2* __restrict__ outg) {
  using E = typename Ar::E;
  const E* pS = reinterpret_cast<const E*>(partS);
  const E* pg = reinterpret_cast<const E*>(partg);
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn + n;
       t += (long long)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    if (t < nn) {
      const long long i = t / n, j = t - (t / n) * n;
      for (int c = 0; c < nparts; ++c) s = cadd(s, Ar::to(pS[(size_t)c * nn + j * n + i]));
      outS[t] = s;
    } else {
      const long long i = t - nn;
      for (int c = 0; c < nparts; ++c) s = cadd(s, Ar::to(pg[(size_t)c * n + i]));
      outg[i] = s;
    }
  }
}

size_t backward_smem_bytes(int n, int nb) {
  return (size_t)16 * ((size_t)2 * n * nb + (size_t)nb * nb + 4 * (size_t)n) + sizeof(double2) * GBSBIN_MAX_L;
}

// The shared memory with the block-row buffer (nb x n) where it fits, else without; *rn says which.
static size_t backward_smem_choice(int n, int nb, int* rn) {
  const size_t base = backward_smem_bytes(n, nb), with = base + (size_t)16 * nb * n;
  *rn = with <= 226 * 1024 ? 1 : 0;
  return *rn ? with : base;
}

int backward_block(int n) { return n <= 320 ? GBSBIN_BWD_MAX_NB : GBSBIN_BWD_MAX_NB / 2; }

static unsigned nblk(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 16384) b = 16384;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_backward_weights(const BackwardArgs& b, const double* dLdP, cudaStream_t s,
                                    const double2** beta) {
  const GridDesc& g = b.grid;
  const int L = g.L;
  // gbar = adjoint DFT of dL/dP: table dims nout -> evaluated dims (radix..., half)
  long long table = 1;
  for (int l = 0; l < L; ++l) table *= g.nout[l];
  k_real_to_complex<<<nblk(table, 64), 64, 0, s>>>(dLdP, table, b.bufA);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // last axis first (nout -> half), so every intermediate fits max(table, n_eval)
  long long dims[GBSBIN_MAX_L];
  for (int l = 0; l < L; ++l) dims[l] = g.nout[l];
  double2* cur = b.bufA;
  double2* nxt = b.bufB;
  long long twoff[GBSBIN_MAX_L];
  long long off = 0;
  for (int l = 0; l < L; ++l) {
    twoff[l] = off;
    off += g.radix[l];
  }
  for (int step = 0; step < L; ++step) {
    const int l = step == 0 ? L - 1 : step - 1;
    long long outer = 1, inner = 1;
    for (int m = 0; m < l; ++m) outer *= dims[m];
    for (int m = l + 1; m < L; ++m) inner *= dims[m];
    const int nk = (l == L - 1) ? g.half : g.radix[l];
    k_adj_axis<<<nblk(outer * nk * inner, 64), 64, 0, s>>>(cur, nxt, outer, (int)dims[l], nk, inner, g.radix[l],
                                                            b.tw + twoff[l]);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    dims[l] = nk;
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  // weights a_k (into nxt), beta_0
  k_adj_weights<<<nblk(g.n_eval, 64), 64, 0, s>>>(cur, b.logq, g, nxt);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_adj_beta0<<<1, 1024, 0, s>>>(nxt, g.n_eval);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  *beta = nxt;
  return cudaSuccess;
}

cudaError_t launch_backward_reduce(const BackwardArgs& b, int nparts, cudaStream_t s) {
  const long long work = (long long)b.n * b.n + b.n;
  if (b.df)
    k_backward_reduce<ArDF><<<nblk(work, 256), 256, 0, s>>>(b.partS, b.partg, nparts, b.n, b.outS, b.outg);
  else
    k_backward_reduce<ArF64><<<nblk(work, 256), 256, 0, s>>>(b.partS, b.partg, nparts, b.n, b.outS, b.outg);
  return cudaGetLastError();
}

cudaError_t launch_backward_points(const BackwardArgs& b0, cudaStream_t s) {
  cudaError_t err;
  BackwardArgs b = b0;
  const size_t smem = backward_smem_choice(b.n, b.nb, &b.rn);
  if (b.ev0 && (err = cudaEventRecord(b.ev0, s)) != cudaSuccess) return err;
  if (b.df) {
    err = cudaFuncSetAttribute(k_backward_gj<ArDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_backward_gj<ArDF><<<b.nparts, kGjThreads, smem, s>>>(b);
  } else {
    err = cudaFuncSetAttribute(k_backward_gj<ArF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_backward_gj<ArF64><<<b.nparts, kGjThreads, smem, s>>>(b);
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (b.ev1 && (err = cudaEventRecord(b.ev1, s)) != cudaSuccess) return err;
  return launch_backward_reduce(b, b.nparts, s);
}

cudaError_t launch_backward(const BackwardArgs& b, const double* dLdP, cudaStream_t s) {
  const double2* beta = nullptr;
  cudaError_t err = launch_backward_weights(b, dLdP, s, &beta);
  if (err != cudaSuccess) return err;
  BackwardArgs bb = b;
  bb.beta = beta;
  return launch_backward_points(bb, s);
}

}  // namespace gbsbin
