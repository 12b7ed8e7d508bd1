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
// M_k^{-1} comes from the LU factors the FP64 forward stored: U^{-1} column by column,
// then X L = U^{-1} from the right.  All FP64; one CTA per SM, each accumulating its
// points into its own partial, reduced over CTAs in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "gbsbin_device.cuh"
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

// Per point: W = M^{-1} from the stored L\U; accumulate into this CTA's partials.
template <int NT>
__global__ void __launch_bounds__(NT) k_backward_points(BackwardArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = b.n, tid = threadIdx.x;
  double2* vec = (double2*)smem;
  double2* t_i = vec;          // n: scratch per row
  double2* lcol = vec + n;     // n: saved L column
  double2* y = vec + 2 * n;    // n
  double2* x = vec + 3 * n;    // n
  double2* W = (double2*)((char*)b.ws + (size_t)blockIdx.x * (size_t)b.ws_slot_bytes);
  double2* S = b.partS + (size_t)blockIdx.x * n * n;
  double2* sg = b.partg + (size_t)blockIdx.x * n;
  for (int t = tid; t < n * n; t += NT) S[t] = make_double2(0.0, 0.0);
  for (int t = tid; t < n; t += NT) sg[t] = make_double2(0.0, 0.0);
  __syncthreads();

  for (long long e = blockIdx.x; e < b.n_eval; e += gridDim.x) {
    const double2 beta = b.beta[e];
    if (beta.x == 0.0 && beta.y == 0.0) continue;  // no contribution
    const double2* F = b.lu_store + (size_t)e * n * n;
    for (int t = tid; t < n * n; t += NT) W[t] = F[t];
    for (int t = tid; t < n; t += NT) x[t] = b.x_store[(size_t)e * n + t];
    __syncthreads();
    // U^{-1} in place, column by column: Uinv[0:j, j] = -Uinv[0:j, 0:j] U[0:j, j] / u_jj
    for (int j = 0; j < n; ++j) {
      const double2 inv = crecip(W[(size_t)j * n + j]);
      for (int i = tid; i < j; i += NT) {
        double2 s = make_double2(0.0, 0.0);
        for (int k = i; k < j; ++k) {
          double2 a = W[(size_t)i * n + k], u = W[(size_t)k * n + j];
          s.x = fma(a.x, u.x, fma(-a.y, u.y, s.x));
          s.y = fma(a.x, u.y, fma(a.y, u.x, s.y));
        }
        t_i[i] = s;
      }
      __syncthreads();
      for (int i = tid; i < j; i += NT) {
        double2 s = cmul(t_i[i], inv);
        W[(size_t)i * n + j] = make_double2(-s.x, -s.y);
      }
      if (tid == 0) W[(size_t)j * n + j] = inv;
      __syncthreads();
    }
    // X L = Uinv, columns from the right: X[:, j] = Uinv[:, j] - sum_{k > j} X[:, k] L[k][j]
    for (int j = n - 2; j >= 0; --j) {
      for (int k = j + 1 + tid; k < n; k += NT) lcol[k] = W[(size_t)k * n + j];
      __syncthreads();
      for (int i = tid; i < n; i += NT) {
        double2 s = i <= j ? W[(size_t)i * n + j] : make_double2(0.0, 0.0);
        for (int k = j + 1; k < n; ++k) s = cfnma(s, W[(size_t)i * n + k], lcol[k]);
        W[(size_t)i * n + j] = s;
      }
      __syncthreads();
    }
    // y = M^{-T} gamma
    for (int i = tid; i < n; i += NT) {
      double2 s = make_double2(0.0, 0.0);
      for (int j = 0; j < n; ++j) {
        double2 m = W[(size_t)j * n + i], g = b.gamma[j];
        s.x = fma(m.x, g.x, fma(-m.y, g.y, s.x));
        s.y = fma(m.x, g.y, fma(m.y, g.x, s.y));
      }
      y[i] = s;
    }
    __syncthreads();
    // S += beta/2 (y x^T + M^{-T});  sg += beta/2 (x + X y)
    const double2 hb = cscale(beta, 0.5);
    for (int t = tid; t < n * n; t += NT) {
      const int i = t / n, j = t - i * n;
      double2 v = cadd(cmul(y[i], x[j]), W[(size_t)j * n + i]);
      S[t] = cadd(S[t], cmul(hb, v));
    }
    const int h = n / 2;
    for (int i = tid; i < n; i += NT) sg[i] = cadd(sg[i], cmul(hb, cadd(x[i], y[i < h ? i + h : i - h])));
    __syncthreads();
  }
}

// outS[t] = sum over CTAs c of partS[c][t] (fixed order)
__global__ void k_backward_reduce(const double2* __restrict__ part, int nparts, long long len, double2* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nparts; ++c) s = cadd(s, part[(size_t)c * len + t]);
    out[t] = s;
  }
}

static unsigned nblk(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 16384) b = 16384;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_backward(const BackwardArgs& b, const double* dLdP, cudaStream_t s) {
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
  BackwardArgs bb = b;
  bb.beta = nxt;
  const int NT = 256;
  size_t smem = (size_t)4 * b.n * sizeof(double2);
  err = cudaFuncSetAttribute(k_backward_points<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_backward_points<NT><<<b.nparts, NT, smem, s>>>(bb);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const long long nn = (long long)b.n * b.n;
  k_backward_reduce<<<nblk(nn, 256), 256, 0, s>>>(b.partS, b.nparts, nn, b.outS);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_backward_reduce<<<nblk(b.n, 256), 256, 0, s>>>(b.partg, b.nparts, b.n, b.outg);
  return cudaGetLastError();
}

}  // namespace gbsbin
