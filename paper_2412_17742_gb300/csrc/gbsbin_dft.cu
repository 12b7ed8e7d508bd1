// Inverse multidimensional DFT of the generating function on the roots-of-unity grid:
//
//   P~(b) = (1/N_pts) sum_k G(omega^k) prod_l omega_l^{-k_l b_l},   omega_l = exp(2 pi i / R_l)
//
// (the coefficient extraction that replaces the finite-difference sieve of
// arXiv:2412.17742, Sec. V/VI: on R_l-th roots of unity it returns the folded table
// sum_{b' = b mod R} P(b') exactly).  G(omega^k) = exp(log q_k - log q_0): point 0 is
// w = 1, so dividing by q(1) applies Pr(0) = 1/q(1) (Sec. III, Eq. sum_lhafs).
//
// Only half of the last axis was evaluated (G(omega^-k) = conj G(omega^k) since P is
// real).  The transform runs axis by axis in FP64: axes 0..L-2 as complex DFTs on the
// half array, keeping only the N_l + 1 outputs the table needs, then the last axis as a
// Hermitian (real-output) transform.  For any partial transform Y along the other axes
// Y(b', R - k) = conj Y(b', k), so the last axis needs only the stored half.  Small grids of
// three or more axes take a two-phase form with one grid barrier (k_dft_blocked).
#include <cuda_runtime.h>

#include <type_traits>

#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {

__device__ __forceinline__ double2 cfma2(double2 a, double2 b, double2 c) {  // c + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// log q from the warp kernel's unfinished form f = (P re, P im, A, r re, r im): P is the
// product of the factors d_i u'_ii of det K (each with Re > 0), A the FP32 sum of their
// arguments (within far less than pi of the exact sum), r the rest of log q.  Log det K =
// log|P| + i (Arg P + 2 pi m) with m the winding that brings Arg P to A.
__device__ __forceinline__ double2 finish_logq(const double* f) {
  const double TWO_PI = 6.283185307179586476925286766559;
  const double a0 = atan2(f[1], f[0]);
  const double re = 0.5 * log(fma(f[0], f[0], f[1] * f[1]));
  const double im = a0 + TWO_PI * rint((f[2] - a0) / TWO_PI);
  return make_double2(f[3] - 0.5 * re, f[4] - 0.5 * im);
}

// G = exp(log q - log q_0) on the whole evaluated half grid (finishing log q first when the
// point kernel left it unfinished).  A shard's plan evaluated point 0 and its slice
// [e_lo, e_hi) only: G is zero off the slice, so the transform gives the slice's partial
// table.  Items t0, t0 + stride, ... of the half grid; l0 = log q_0.
// G at half-grid point t (see stage_normalise); with ldfin, also stores the finished log q.
__device__ __forceinline__ double2 normalise_one(const double2* logq, const GridDesc& g, const double* __restrict__ ldfin,
                                                 double2* logq_fin, double2 l0, long long t) {
  const bool in_slice = t >= g.e_lo && t < g.e_hi;
  // this plan's index of half-grid point t (-1: not evaluated here)
  const long long loc = in_slice ? (g.e_lo > 0 ? t - g.e_lo + 1 : t) : (t == 0 ? 0 : -1);
  if (loc < 0) return make_double2(0.0, 0.0);
  double2 v;
  if (ldfin) {
    v = finish_logq(ldfin + 6 * loc);
    logq_fin[loc] = v;
  } else {
    v = logq[loc];
  }
  if (!in_slice) return make_double2(0.0, 0.0);     // point 0 of a later shard: normalisation only
  double m = exp(v.x - l0.x);
  double s, c;
  sincos(v.y - l0.y, &s, &c);
  return make_double2(m * c, m * s);
}

__device__ __forceinline__ void stage_normalise(const double2* logq, const GridDesc& g, double2* __restrict__ G,
                                                const double* __restrict__ ldfin, double2* logq_fin, double2 l0,
                                                long long t0, long long stride) {
  for (long long t = t0; t < g.n_full; t += stride) G[t] = normalise_one(logq, g, ldfin, logq_fin, l0, t);
}

// G given as partial sums over nparts ranges of some inner sum (Fock inputs: node ranges
// of the input-side extraction): G[t] = pscale sum_r parts[r n_full + t], r ascending.
__device__ __forceinline__ double2 sum_parts_one(const double2* __restrict__ parts, long long nparts, double pscale,
                                                 long long n_full, long long t) {
  double2 acc = make_double2(0.0, 0.0);
  for (long long r = 0; r < nparts; ++r) {
    const double2 v = parts[r * n_full + t];
    acc.x += v.x;
    acc.y += v.y;
  }
  return make_double2(acc.x * pscale, acc.y * pscale);
}

__device__ __forceinline__ void stage_sum_parts(const double2* __restrict__ parts, long long nparts, double pscale,
                                                const GridDesc& g, double2* __restrict__ G, long long t0,
                                                long long stride) {
  for (long long t = t0; t < g.n_full; t += stride) G[t] = sum_parts_one(parts, nparts, pscale, g.n_full, t);
}

__global__ void k_normalise(const double2* logq, GridDesc g, double2* __restrict__ G,
                            const double* __restrict__ ldfin, double2* logq_fin) {
  __shared__ double2 s_l0;
  if (threadIdx.x == 0) s_l0 = ldfin ? finish_logq(ldfin) : logq[0];
  __syncthreads();
  stage_normalise(logq, g, G, ldfin, logq_fin, s_l0, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x);
}

__global__ void k_sum_parts(const double2* parts, long long nparts, double pscale, GridDesc g,
                            double2* __restrict__ G) {
  stage_sum_parts(parts, nparts, pscale, g, G, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x);
}

// out[o, b, s] = sum_{k < R} in[o, k, s] tw[(k b) mod R],  b < nout
// Indices in 32 bits (every array here has at most GBSBIN_MAX_POINTS entries); the terms
// are loaded four at a time before their multiply-adds, which keep the order k = 0, 1, ...
__device__ __forceinline__ void stage_axis(const double2* __restrict__ in, double2* __restrict__ out, long long outer,
                                           int R, int nout, long long inner, const double2* __restrict__ tw,
                                           long long t0, long long stride) {
  const unsigned total = (unsigned)(outer * nout * inner), in32 = (unsigned)inner, nout32 = (unsigned)nout;
  const unsigned R32 = (unsigned)R;
  for (unsigned t = (unsigned)t0; t < total; t += (unsigned)stride) {
    const unsigned rest = t / in32, s = t - rest * in32;
    const unsigned o = rest / nout32, b = rest - o * nout32;
    const double2* src = in + (size_t)o * R32 * in32 + s;
    double2 acc = make_double2(0.0, 0.0);
    unsigned idx = 0;                                // (k b) mod R, b < R
    unsigned k = 0;
    for (; k + 4 <= R32; k += 4) {
      const unsigned i1 = idx + b >= R32 ? idx + b - R32 : idx + b;
      const unsigned i2 = i1 + b >= R32 ? i1 + b - R32 : i1 + b;
      const unsigned i3 = i2 + b >= R32 ? i2 + b - R32 : i2 + b;
      const double2 v0 = src[(size_t)k * in32], v1 = src[(size_t)(k + 1) * in32];
      const double2 v2 = src[(size_t)(k + 2) * in32], v3 = src[(size_t)(k + 3) * in32];
      const double2 w0 = tw[idx], w1 = tw[i1], w2 = tw[i2], w3 = tw[i3];
      acc = cfma2(v0, w0, acc);
      acc = cfma2(v1, w1, acc);
      acc = cfma2(v2, w2, acc);
      acc = cfma2(v3, w3, acc);
      idx = i3 + b >= R32 ? i3 + b - R32 : i3 + b;
    }
    for (; k < R32; ++k) {
      acc = cfma2(src[(size_t)k * in32], tw[idx], acc);
      idx += b;
      if (idx >= R32) idx -= R32;
    }
    out[t] = acc;
  }
}

__global__ void k_dft_axis(const double2* __restrict__ in, double2* __restrict__ out, long long outer,
                           int R, int nout, long long inner, const double2* __restrict__ tw) {
  stage_axis(in, out, outer, R, nout, inner, tw, blockIdx.x * (long long)blockDim.x + threadIdx.x,
             (long long)gridDim.x * blockDim.x);
}

// P[o, b] = scale (Re Y[o,0] + sum_{k=1}^{H-1} c_k Re(Y[o,k] tw[(k b) mod R])),
// c_k = 2, except c = 1 for the self-conjugate k = R/2 when R is even.
struct DiagAcc {
  double sum, im, mn, bad;
};

__device__ __forceinline__ void stage_last_real(const double2* __restrict__ Y, double* __restrict__ P,
                                                long long outer, int R, int H, int nout, double scale,
                                                const double2* __restrict__ tw, long long t0, long long stride,
                                                DiagAcc* acc_out = nullptr) {
  // 32-bit indices and four terms loaded ahead, the sum's order unchanged (as stage_axis)
  const unsigned total = (unsigned)(outer * nout), nout32 = (unsigned)nout, R32 = (unsigned)R;
  for (unsigned t = (unsigned)t0; t < total; t += (unsigned)stride) {
    const unsigned o = t / nout32, b = t - o * nout32;
    const double2* row = Y + (size_t)o * H;
    if (acc_out && b == 0) {                          // the row's self-conjugate entries
      acc_out->im = fmax(acc_out->im, fabs(row[0].y));
      if ((R & 1) == 0) acc_out->im = fmax(acc_out->im, fabs(row[H - 1].y));
    }
    double acc = row[0].x;
    unsigned idx = b >= R32 ? b - R32 : b;           // (k b) mod R at k = 1
    int k = 1;
    for (; k + 4 <= H; k += 4) {
      const unsigned i1 = idx + b >= R32 ? idx + b - R32 : idx + b;
      const unsigned i2 = i1 + b >= R32 ? i1 + b - R32 : i1 + b;
      const unsigned i3 = i2 + b >= R32 ? i2 + b - R32 : i2 + b;
      const double2 y0 = row[k], y1 = row[k + 1], y2 = row[k + 2], y3 = row[k + 3];
      const double2 w0 = tw[idx], w1 = tw[i1], w2 = tw[i2], w3 = tw[i3];
      acc += ((2 * k == R) ? 1.0 : 2.0) * fma(y0.x, w0.x, -y0.y * w0.y);
      acc += ((2 * (k + 1) == R) ? 1.0 : 2.0) * fma(y1.x, w1.x, -y1.y * w1.y);
      acc += ((2 * (k + 2) == R) ? 1.0 : 2.0) * fma(y2.x, w2.x, -y2.y * w2.y);
      acc += ((2 * (k + 3) == R) ? 1.0 : 2.0) * fma(y3.x, w3.x, -y3.y * w3.y);
      idx = i3 + b >= R32 ? i3 + b - R32 : i3 + b;
    }
    for (; k < H; ++k) {
      const double2 y = row[k], w = tw[idx];
      acc += ((2 * k == R) ? 1.0 : 2.0) * fma(y.x, w.x, -y.y * w.y);
      idx += b;
      if (idx >= R32) idx -= R32;
    }
    P[t] = acc * scale;
    if (acc_out) acc_out->sum += acc * scale;
  }
}

// Block reduction of the per-thread diagnostics into partial vb (the whole CTA calls it).
__device__ __forceinline__ void block_diag(DiagAcc a, double* __restrict__ part, int vb) {
  __shared__ double s_d[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    a.sum += __shfl_xor_sync(0xffffffffu, a.sum, o);
    a.im = fmax(a.im, __shfl_xor_sync(0xffffffffu, a.im, o));
    a.mn = fmin(a.mn, __shfl_xor_sync(0xffffffffu, a.mn, o));
    a.bad += __shfl_xor_sync(0xffffffffu, a.bad, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_d[0][w] = a.sum;
    s_d[1][w] = a.im;
    s_d[2][w] = a.mn;
    s_d[3][w] = a.bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      a.sum += s_d[0][i];
      a.im = fmax(a.im, s_d[1][i]);
      a.mn = fmin(a.mn, s_d[2][i]);
      a.bad += s_d[3][i];
    }
    part[4 * vb] = a.sum;
    part[4 * vb + 1] = a.im;
    part[4 * vb + 2] = a.mn;
    part[4 * vb + 3] = a.bad;
  }
}

__global__ void k_dft_last_real(const double2* __restrict__ Y, double* __restrict__ P, long long outer,
                                int R, int H, int nout, double scale, const double2* __restrict__ tw) {
  stage_last_real(Y, P, outer, R, H, nout, scale, tw, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x);
}

// Per-block partial diagnostics (the host finishes the reduction in a fixed order):
// part[4b + 0] = sum of P over the block's share, part[4b + 1] = max |Im| of the
// self-conjugate entries Y[o, 0] (and Y[o, R/2]), part[4b + 2] = min pivot Re,
// part[4b + 3] = number of bad points; part[4 nblocks] = Re log q_0.  Block vb of nvb
// blocks of blockDim.x threads; the whole CTA calls it.
__device__ __forceinline__ void stage_diag(const double* __restrict__ P, long long table, const double2* __restrict__ Y,
                                           long long outer, int H, int R, const double* __restrict__ minpiv,
                                           const double2* logq, long long n_eval, double* __restrict__ part,
                                           int vb, int nvb) {
  __shared__ double s_sum[32], s_im[32], s_min[32], s_bad[32];
  double sum = 0.0, im = 0.0, mn = 1.0e300, bad = 0.0;
  const long long stride = (long long)nvb * blockDim.x;
  const long long t0 = (long long)vb * blockDim.x + threadIdx.x;
  for (long long t = t0; t < table; t += stride) sum += P[t];
  for (long long o = t0; o < outer; o += stride) {
    im = fmax(im, fabs(Y[o * H].y));
    if ((R & 1) == 0) im = fmax(im, fabs(Y[o * H + H - 1].y));
  }
  for (long long e = t0; minpiv && e < n_eval; e += stride) {
    double m = minpiv[e];
    double2 l = logq ? logq[e] : make_double2(0.0, 0.0);
    bool ok = (m > 0.0) && isfinite(l.x) && isfinite(l.y);
    if (!ok) bad += 1.0;
    mn = fmin(mn, m);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    im = fmax(im, __shfl_xor_sync(0xffffffffu, im, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_sum[w] = sum;
    s_im[w] = im;
    s_min[w] = mn;
    s_bad[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int i = 1; i < nw; ++i) {
      sum += s_sum[i];
      im = fmax(im, s_im[i]);
      mn = fmin(mn, s_min[i]);
      bad += s_bad[i];
    }
    double* out = part + 4 * vb;
    out[0] = sum;
    out[1] = im;
    out[2] = mn;
    out[3] = bad;
    if (vb == 0) {
      part[4 * GBSBIN_DIAG_SLOTS] = logq ? logq[0].x : 0.0;
      part[4 * GBSBIN_DIAG_SLOTS + 2] = (double)nvb;
    }
  }
}

__global__ void k_diag(const double* __restrict__ P, long long table, const double2* __restrict__ Y,
                       long long outer, int H, int R, const double* __restrict__ minpiv,
                       const double2* __restrict__ logq, long long n_eval, double* __restrict__ part) {
  stage_diag(P, table, Y, outer, H, R, minpiv, logq, n_eval, part, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------- one cooperative launch, all stages
// The stages above run in sequence in one launch of co-resident CTAs (cooperative launch),
// separated by a grid barrier: bar[0] counts arrivals, bar[1] is the generation, bar[2]
// records a barrier that gave up waiting (after ~1 s), which the host reports as a CUDA
// error.  Items are dealt to the CTAs cyclically (item t to CTA t mod gridDim), and within
// a CTA across its warps, so the FP64 work of every stage spreads over all SMs and all
// their schedulers.  Every table entry is summed in the same order as in the multi-launch path, so
// the table is bit-identical to it (the diagnostics' partial sums are split differently).
struct DftStage {
  long long outer, inner, twoff;
  int R, nout;
};
struct DftFused {
  DftArgs a;
  int naxes;                         // complex axes 0 .. L-2
  DftStage ax[GBSBIN_MAX_L];
  long long last_outer, last_twoff;
  int last_R, H, last_nout;
  double scale;
  unsigned* bar;
};

__device__ __forceinline__ void grid_barrier(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g, old, cur;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    if (old == gridDim.x - 1) {
      bar[0] = 0;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      long long it = 0;
      do {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
        if (++it > (1ll << 23)) {          // ~1 s of L2 polls: give up, record it
          atomicExch(bar + 2, 1u);
          break;
        }
      } while (cur == g);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(128, 4) k_dft_fused(DftFused f) {
  const DftArgs& a = f.a;
  // the CTA's k-th item goes to lane k / 4 of warp k mod 4: a CTA's few items use all
  // four schedulers' FP64 units instead of one warp's
  const int tid = ((threadIdx.x & 31) << 2) | (threadIdx.x >> 5);
  const long long t0 = tid * (long long)gridDim.x + blockIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const bool first = !a.g_ready;
  if (a.g_ready) {
    // G already in bufA (written by the point kernel)
  } else if (a.parts) {
    stage_sum_parts(a.parts, a.nparts, a.pscale, a.grid, a.bufA, t0, stride);
  } else {
    __shared__ double2 s_l0;
    if (threadIdx.x == 0) s_l0 = a.ldfin ? finish_logq(a.ldfin) : a.logq[0];
    __syncthreads();
    stage_normalise(a.logq, a.grid, a.bufA, a.ldfin, a.logq_fin, s_l0, t0, stride);
  }
  double2* cur = a.bufA;
  double2* nxt = a.bufB;
  for (int l = 0; l < f.naxes; ++l) {
    if (l > 0 || first) grid_barrier(f.bar);
    const DftStage& st = f.ax[l];
    stage_axis(cur, nxt, st.outer, st.R, st.nout, st.inner, a.tw + st.twoff, t0, stride);
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (f.naxes > 0 || first) grid_barrier(f.bar);
  // the diagnostics ride along: every CTA reduces what its threads wrote or read into its
  // own partial (no barrier after the last stage)
  DiagAcc acc{0.0, 0.0, 1.0e300, 0.0};
  stage_last_real(cur, a.P, f.last_outer, f.last_R, f.H, f.last_nout, f.scale, a.tw + f.last_twoff, t0, stride,
                  a.diag ? &acc : nullptr);
  if (a.diag) {
    const double2* lq = a.g_ready ? nullptr : a.ldfin ? a.logq_fin : a.logq;
    for (long long e = t0; a.minpiv && e < a.grid.n_eval; e += stride) {
      const double m = a.minpiv[e];
      const double2 l = lq ? lq[e] : make_double2(0.0, 0.0);
      if (!((m > 0.0) && isfinite(l.x) && isfinite(l.y))) acc.bad += 1.0;
      acc.mn = fmin(acc.mn, m);
    }
    block_diag(acc, a.diag, blockIdx.x);
    if (t0 == 0) {
      a.diag[4 * GBSBIN_DIAG_SLOTS] = lq ? lq[0].x : 0.0;
      a.diag[4 * GBSBIN_DIAG_SLOTS + 1] = (double)*(volatile unsigned*)(f.bar + 2);
      a.diag[4 * GBSBIN_DIAG_SLOTS + 2] = (double)gridDim.x;
    }
  }
}

__global__ void k_finish_logq(const double* __restrict__ ldfin, double2* __restrict__ logq, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    logq[e] = finish_logq(ldfin + 6 * e);
}

// Small transforms use 64-thread blocks so the work spreads over many SMs (these kernels
// run on the FP64 pipe, which is narrow per SM).
constexpr int kDftThreads = 64;
static unsigned blocks_for(long long work) {
  long long b = (work + kDftThreads - 1) / kDftThreads;
  if (b > 16384) b = 16384;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_dft(const DftArgs& a, cudaStream_t s) {
  const GridDesc& g = a.grid;
  const int L = g.L;
  if (a.parts)
    k_sum_parts<<<blocks_for(g.n_full), kDftThreads, 0, s>>>(a.parts, a.nparts, a.pscale, g, a.bufA);
  else
    k_normalise<<<blocks_for(g.n_full), kDftThreads, 0, s>>>(a.logq, g, a.bufA, a.ldfin, a.logq_fin);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  long long dims[GBSBIN_MAX_L];
  for (int l = 0; l < L - 1; ++l) dims[l] = g.radix[l];
  dims[L - 1] = g.half;
  double2* cur = a.bufA;
  double2* nxt = a.bufB;
  long long twoff = 0;
  for (int l = 0; l < L - 1; ++l) {
    long long outer = 1, inner = 1;
    for (int m = 0; m < l; ++m) outer *= dims[m];
    for (int m = l + 1; m < L; ++m) inner *= dims[m];
    k_dft_axis<<<blocks_for(outer * g.nout[l] * inner), kDftThreads, 0, s>>>(cur, nxt, outer, g.radix[l], g.nout[l],
                                                                      inner, a.tw + twoff);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    dims[l] = g.nout[l];
    twoff += g.radix[l];
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  long long outer = 1;
  for (int m = 0; m < L - 1; ++m) outer *= dims[m];
  const double scale = 1.0 / (double)g.npts;
  k_dft_last_real<<<blocks_for(outer * g.nout[L - 1]), kDftThreads, 0, s>>>(cur, a.P, outer, g.radix[L - 1], g.half,
                                                                    g.nout[L - 1], scale, a.tw + twoff);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (a.diag) {
    k_diag<<<GBSBIN_DIAG_BLOCKS, 256, 0, s>>>(a.P, a.table_size, cur, outer, g.half, g.radix[L - 1],
                                              a.minpiv, a.logq, g.n_eval, a.diag);
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t launch_finish_logq(const double* ldfin, double2* logq, long long n, cudaStream_t s) {
  k_finish_logq<<<blocks_for(n), kDftThreads, 0, s>>>(ldfin, logq, n);
  return cudaGetLastError();
}

// ------------------------------------------- small grids: two phases, one grid barrier
// The separable transform needs a global exchange only between axis sets.  Phase 1: CTA per
// column c (one combination of the indices of axes h..L-1) gathers G[., c] (the prod_{l<h}
// R_l entries of the leading axes), runs axes 0..h-1 in shared memory and writes
// Y[b_0..b_{h-1}, c].  One grid barrier.  Phase 2: CTA per row (one combination of the
// leading outputs b_0..b_{h-1}) reads its contiguous Y row, runs axes h..L-2 and the
// Hermitian last axis in shared memory, and writes the table row.  Every entry is summed in
// the same order as by the axis-by-axis stages (the table is bit-identical to theirs); the
// grid barriers between the axes inside a phase become block barriers.
struct DftBlocked {
  DftArgs a;
  unsigned* bar;
  int L, h;
  int R[GBSBIN_MAX_L], nout[GBSBIN_MAX_L], twoff[GBSBIN_MAX_L];
  int outer[GBSBIN_MAX_L], inner[GBSBIN_MAX_L];   // per axis, within its phase's block
  int B1, C1, C2, O2;     // phase-1 block entries, columns; phase-2 rows, last-axis rows per row
  int H, last_R, last_nout, last_twoff, buf;      // buf: entries per shared buffer
  int ntw;                                          // twiddles of all axes (staged in shared memory)
  double scale;
};

// out[o, b, s] = sum_k in[o, k, s] tw[(k b) mod R] inside one CTA's shared block, in the
// arithmetic Ar (ArF64::fma is the FP64 complex multiply-add of the axis stages)
template <class Ar>
__device__ __forceinline__ void block_axis(const typename Ar::E* in, typename Ar::E* out, int outer, int R, int nout,
                                           int inner, const typename Ar::E* tw) {
  using E = typename Ar::E;
  const int total = outer * nout * inner;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int rest = t / inner, s = t - rest * inner;
    const int o = rest / nout, b = rest - o * nout;
    const E* src = in + o * R * inner + s;
    E acc = Ar::zero();
    int idx = 0;
    for (int k = 0; k < R; ++k) {
      acc = Ar::fma(src[k * inner], tw[idx], acc);
      idx += b;
      if (idx >= R) idx -= R;
    }
    out[t] = acc;
  }
}

// Order-preserving integer key of a double that is not NaN (negative values flipped).
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffll;
}
__device__ __forceinline__ double key_value(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffll);
}

// Per-warp diagnostics partial into slot vb: the sum in FP64, the maximum |Im| (non-negative)
// and the minimum pivot through their order-preserving integer keys, the count as an
// integer; no block barrier.
__device__ __forceinline__ void warp_diag(DiagAcc a, double* __restrict__ part, int vb) {
  double sum = a.sum;
  long long im = order_key(a.im), mn = order_key(a.mn);
  int bad = (int)a.bad;
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const long long io = __shfl_xor_sync(0xffffffffu, im, o), mo = __shfl_xor_sync(0xffffffffu, mn, o);
    im = io > im ? io : im;
    mn = mo < mn ? mo : mn;
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[4 * vb] = sum;
    part[4 * vb + 1] = key_value(im);
    part[4 * vb + 2] = key_value(mn);
    part[4 * vb + 3] = (double)bad;
  }
}

// Ar = ArF64: every entry summed as by the axis stages (bit-identical tables); Ar = ArDF:
// the transform in pairs of FP32 (about 46 bits) on the FMA pipe.
template <class Ar>
__global__ void __launch_bounds__(128) k_dft_blocked(DftBlocked f) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const DftArgs& a = f.a;
  E* S0 = reinterpret_cast<E*>(dsm_raw);
  E* S1 = S0 + f.buf;
  E* tws = S1 + f.buf;                               // all axes' twiddles
  E* Y = reinterpret_cast<E*>(a.bufB);               // 16-byte entries either way
  for (int j = threadIdx.x; j < f.ntw; j += blockDim.x) tws[j] = Ar::from(a.tw[j]);
  __shared__ double2 s_l0;
  if (!a.g_ready && !a.parts) {
    if (threadIdx.x == 0) s_l0 = a.ldfin ? finish_logq(a.ldfin) : a.logq[0];
    __syncthreads();
  }
  // the pivots' scan after phase 1 (log q may be finished there); its first pivot per
  // thread is loaded now, so that load's latency passes under phase 1
  DiagAcc acc{0.0, 0.0, 1.0e300, 0.0};
  const double2* lq = a.g_ready ? nullptr : a.ldfin ? a.logq_fin : a.logq;
  const long long e_first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool has_first = a.diag && a.minpiv && e_first < a.grid.n_eval;
  const double m_first = has_first ? a.minpiv[e_first] : 0.0;
  auto scan = [&]() {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = e_first; a.minpiv && e < a.grid.n_eval; e += stride) {
      const double m = e == e_first ? m_first : a.minpiv[e];
      const double2 l = lq ? lq[e] : make_double2(0.0, 0.0);
      if (!((m > 0.0) && isfinite(l.x) && isfinite(l.y))) acc.bad += 1.0;
      acc.mn = fmin(acc.mn, m);
    }
  };
  // phase 1: axes 0 .. h-1 per column
  for (int c = blockIdx.x; c < f.C1; c += gridDim.x) {
    for (int e = threadIdx.x; e < f.B1; e += blockDim.x) {
      const long long t = (long long)e * f.C1 + c;
      if (std::is_same<Ar, ArDF>::value && a.g_ready && a.g_df)
        S0[e] = reinterpret_cast<const E*>(a.bufA)[t];    // G written as a pair
      else
        S0[e] = Ar::from(a.g_ready ? a.bufA[t]
                         : a.parts ? sum_parts_one(a.parts, a.nparts, a.pscale, a.grid.n_full, t)
                                   : normalise_one(a.logq, a.grid, a.ldfin, a.logq_fin, s_l0, t));
    }
    __syncthreads();
    E* cur = S0;
    E* nxt = S1;
    for (int l = 0; l < f.h; ++l) {
      block_axis<Ar>(cur, nxt, f.outer[l], f.R[l], f.nout[l], f.inner[l], tws + f.twoff[l]);
      __syncthreads();
      E* t = cur;
      cur = nxt;
      nxt = t;
    }
    for (int e = threadIdx.x; e < f.C2; e += blockDim.x) Y[(long long)e * f.C1 + c] = cur[e];
    __syncthreads();
  }
  grid_barrier(f.bar);
  if (a.diag) scan();
  // phase 2: axes h .. L-2, then the last (Hermitian) axis, per row
  const int R = f.last_R, H = f.H, nout = f.last_nout;
  const E* tw = tws + f.last_twoff;
  for (int r = blockIdx.x; r < f.C2; r += gridDim.x) {
    for (int e = threadIdx.x; e < f.C1; e += blockDim.x) S0[e] = Y[(long long)r * f.C1 + e];
    __syncthreads();
    E* cur = S0;
    E* nxt = S1;
    for (int l = f.h; l < f.L - 1; ++l) {
      block_axis<Ar>(cur, nxt, f.outer[l], f.R[l], f.nout[l], f.inner[l], tws + f.twoff[l]);
      __syncthreads();
      E* t = cur;
      cur = nxt;
      nxt = t;
    }
    double* Prow = a.P + (long long)r * f.O2 * nout;
    for (int t = threadIdx.x; t < f.O2 * nout; t += blockDim.x) {
      const int o = t / nout, b = t - o * nout;
      const E* row = cur + o * H;
      if (b == 0) {                                   // the row's self-conjugate entries
        acc.im = fmax(acc.im, fabs((double)Ar::im(row[0])));
        if ((R & 1) == 0) acc.im = fmax(acc.im, fabs((double)Ar::im(row[H - 1])));
      }
      int idx = b >= R ? b - R : b;
      double v;
      if constexpr (std::is_same<Ar, ArF64>::value) {
        v = row[0].x;
        for (int k = 1; k < H; ++k) {
          const double2 y = row[k], w = tw[idx];
          v += ((2 * k == R) ? 1.0 : 2.0) * fma(y.x, w.x, -y.y * w.y);
          idx += b;
          if (idx >= R) idx -= R;
        }
      } else {                                        // Re(row[0] + sum_k c_k row[k] w), c_k = 2 or 1
        E acc2 = Ar::zero();
        for (int k = 1; k < H; ++k) {
          E yw = Ar::mul(row[k], tw[idx]);
          if (2 * k != R) yw = Ar::add(yw, yw);
          acc2 = Ar::add(acc2, yw);
          idx += b;
          if (idx >= R) idx -= R;
        }
        v = Ar::to(Ar::add(row[0], acc2)).x;
      }
      Prow[t] = v * f.scale;
      acc.sum += v * f.scale;
    }
    __syncthreads();
  }
  if (a.diag) {
    const int nw = blockDim.x >> 5;
    warp_diag(acc, a.diag, blockIdx.x * nw + (threadIdx.x >> 5));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.diag[4 * GBSBIN_DIAG_SLOTS] = lq ? lq[0].x : 0.0;
      a.diag[4 * GBSBIN_DIAG_SLOTS + 1] = (double)*(volatile unsigned*)(f.bar + 2);
      a.diag[4 * GBSBIN_DIAG_SLOTS + 2] = (double)(gridDim.x * nw);
    }
  }
}

// The blocked form where it suits: three or more axes, both phases' blocks and all axes'
// twiddles within kBlockedMaxEntries each (48 KB of shared memory at most), and at least
// kBlockedMinCtas columns and rows (the split h with the most of both); otherwise 0.
constexpr int kBlockedMaxEntries = 1024;
constexpr int kBlockedMinCtas = 32;
static int blocked_split(const GridDesc& g) {
  const int L = g.L;
  if (L < 3) return 0;
  long long ntw = 0;                                 // the twiddles go to shared memory too
  for (int l = 0; l < L; ++l) ntw += g.radix[l];
  if (ntw > kBlockedMaxEntries) return 0;
  long long d[GBSBIN_MAX_L];
  for (int l = 0; l < L - 1; ++l) d[l] = g.radix[l];
  d[L - 1] = g.half;
  int best = 0;
  long long best_min = 0;
  for (int h = 1; h < L; ++h) {
    long long B1 = 1, C1 = 1, C2 = 1;
    for (int l = 0; l < h; ++l) {
      B1 *= d[l];
      C2 *= g.nout[l];
    }
    for (int l = h; l < L; ++l) C1 *= d[l];
    if (B1 > kBlockedMaxEntries || C1 > kBlockedMaxEntries) continue;
    const long long mn = C1 < C2 ? C1 : C2;
    if (mn >= kBlockedMinCtas && mn > best_min) {
      best = h;
      best_min = mn;
    }
  }
  return best;
}

int dft_two_phase(const GridDesc& g) { return blocked_split(g) > 0 ? 1 : 0; }

template <class Ar>
static cudaError_t launch_dft_blocked(const DftArgs& a, int h, unsigned* bar, int num_sms, cudaStream_t s) {
  const GridDesc& g = a.grid;
  const int L = g.L;
  DftBlocked f{};
  f.a = a;
  f.bar = bar;
  f.L = L;
  f.h = h;
  int d[GBSBIN_MAX_L];
  for (int l = 0; l < L - 1; ++l) d[l] = g.radix[l];
  d[L - 1] = g.half;
  int twoff = 0;
  for (int l = 0; l < L; ++l) {
    f.R[l] = g.radix[l];
    f.nout[l] = g.nout[l];
    f.twoff[l] = twoff;
    twoff += g.radix[l];
  }
  // within phase 1 the block is [axes 0..h-1]; within phase 2 [axes h..L-1]; axes before l
  // in the block already hold outputs
  for (int l = 0; l < L - 1; ++l) {
    const int lo = l < h ? 0 : h, hi = l < h ? h : L;
    int outer = 1, inner = 1;
    for (int m = lo; m < l; ++m) outer *= g.nout[m];
    for (int m = l + 1; m < hi; ++m) inner *= d[m];
    f.outer[l] = outer;
    f.inner[l] = inner;
  }
  f.B1 = 1;
  f.C1 = 1;
  f.C2 = 1;
  f.O2 = 1;
  for (int l = 0; l < h; ++l) {
    f.B1 *= d[l];
    f.C2 *= g.nout[l];
  }
  for (int l = h; l < L; ++l) f.C1 *= d[l];
  for (int l = h; l < L - 1; ++l) f.O2 *= g.nout[l];
  f.H = g.half;
  f.last_R = g.radix[L - 1];
  f.last_nout = g.nout[L - 1];
  f.last_twoff = f.twoff[L - 1];
  f.buf = f.B1 > f.C1 ? f.B1 : f.C1;
  f.ntw = twoff;
  f.scale = 1.0 / (double)g.npts;
  const size_t smem = (2 * (size_t)f.buf + (size_t)f.ntw) * sizeof(double2);
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dft_blocked<Ar>, 128, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = f.C1 > f.C2 ? f.C1 : f.C2;     // one column or row per CTA
  if (blocks > (long long)per_sm * num_sms) blocks = (long long)per_sm * num_sms;
  if (blocks > GBSBIN_DIAG_SLOTS / 4) blocks = GBSBIN_DIAG_SLOTS / 4;   // a partial per warp
  void* params[] = {&f};
  return cudaLaunchCooperativeKernel((const void*)k_dft_blocked<Ar>, dim3((unsigned)blocks), dim3(128), params, smem,
                                     s);
}

cudaError_t launch_dft_fused(const DftArgs& a, unsigned* bar, int num_sms, cudaStream_t s) {
  const GridDesc& g = a.grid;
  const int L = g.L;
  const int h = blocked_split(g);
  if (h > 0) return a.df ? launch_dft_blocked<ArDF>(a, h, bar, num_sms, s)
                         : launch_dft_blocked<ArF64>(a, h, bar, num_sms, s);
  DftFused f{};
  f.a = a;
  f.bar = bar;
  f.naxes = L - 1;
  long long dims[GBSBIN_MAX_L];
  for (int l = 0; l < L - 1; ++l) dims[l] = g.radix[l];
  dims[L - 1] = g.half;
  long long twoff = 0;
  for (int l = 0; l < L - 1; ++l) {
    long long outer = 1, inner = 1;
    for (int m = 0; m < l; ++m) outer *= dims[m];
    for (int m = l + 1; m < L; ++m) inner *= dims[m];
    f.ax[l] = DftStage{outer, inner, twoff, g.radix[l], g.nout[l]};
    dims[l] = g.nout[l];
    twoff += g.radix[l];
  }
  long long outer = 1;
  for (int m = 0; m < L - 1; ++m) outer *= dims[m];
  f.last_outer = outer;
  f.last_twoff = twoff;
  f.last_R = g.radix[L - 1];
  f.H = g.half;
  f.last_nout = g.nout[L - 1];
  f.scale = 1.0 / (double)g.npts;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dft_fused, 128, 0);
  if (err != cudaSuccess) return err;
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one item per thread in the largest stage (the stages are FP64-latency-bound chains, so
  // more CTAs than that only add arrivals at every grid barrier); at least the diagnostics'
  // blocks
  const long long items = g.n_full > a.table_size ? g.n_full : a.table_size;
  long long blocks = (items + 127) / 128;
  if (blocks > (long long)per_sm * num_sms) blocks = (long long)per_sm * num_sms;
  if (blocks < GBSBIN_DIAG_BLOCKS) blocks = GBSBIN_DIAG_BLOCKS;
  if (blocks > GBSBIN_DIAG_SLOTS) blocks = GBSBIN_DIAG_SLOTS;
  if (blocks > (long long)per_sm * num_sms) return cudaErrorInvalidConfiguration;
  void* params[] = {&f};
  return cudaLaunchCooperativeKernel((const void*)k_dft_fused, dim3((unsigned)blocks), dim3(128), params, 0, s);
}

}  // namespace gbsbin
