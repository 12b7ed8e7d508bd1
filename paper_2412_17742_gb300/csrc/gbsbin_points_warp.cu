// Warp-per-point FP32 + refinement kernel for n <= 32 (arXiv:2412.17742, Sec. III
// Eq. q_d, Sec. VI Eq. Lamb_lhaf_master; same mathematics as k_points_fp32r).
//
// One warp evaluates one grid point with the whole matrix in registers.  The matrix
// M(w) = conj(D) - XA is padded to NP x NP (NP = 8, 16 or 32) with an identity block,
// which leaves its LU, pivots, residual and log det unchanged.  Lane (lr, lc) =
// (lane / 4, lane % 4) owns rows lr + 8 ra and columns lc + 4 cb (block-cyclic, so every
// lane keeps work until the last steps).  Each elimination step broadcasts column k of L
// and row k of U with warp shuffles.  Steps run in blocks of four: the block index is
// unrolled (so the owning register row/column is a compile-time constant), the step within
// the block is a runtime loop, which keeps the code small enough for the instruction
// cache.  The residual pass reads the digits of L\U from a per-warp shared tile in a
// runtime loop.
//
// Per point:
//   1. M^ = fl32(M) in registers; unpivoted LU in FP32.
//   2. Rounding of each row of L^ and column of U^ onto a 24-bit fixed-point grid (at most
//      the FP32 rounding of the row's / column's largest entry); int32 digits to the tile.
//   3. Log det from the rounded pivots: product of d_i u'_ii (each Re > 0) and the FP32 sum
//      of their arguments; the DFT's first kernel takes the Log (one point per thread).
//   4. Residual E = M - L^U^ exactly in int64 (Karatsuba digit products, M as fixed-point
//      -XA shifted to each entry's scale), rounded to FP32 once.
//   5. delta = tr(U^^{-1} L^^{-1} E): forward substitution on all columns, then back
//      substitution on the entries X[m][c], m >= c, that diag(X) needs.
//   6. If displaced: x^ = M^^{-1} X gamma, r = X gamma - M x^ by Dot2, x = x^ + M^^{-1} r.
//   7. log q = 1/2 gamma^T x - 1/2 (ld + delta), finished by the DFT's first kernel.
#include <cuda_runtime.h>

#include "gbsbin_device.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}

}  // namespace

template <int NP, int WARPS>
struct WarpShared {
  double2 w[WARPS][GBSBIN_MAX_L];
  float2 inv[WARPS][NP];
  float2 piv[WARPS][NP];
  float2 LU[WARPS][NP * (NP + 4)];
  float2 x[WARPS][NP];
  float2 r[WARPS][NP];
  int lab[NP];
};

// One grid point per warp: point e of problem a (e >= n_eval: idle warp).
template <int NP, int WARPS>
__device__ __forceinline__ void warp_point(const PointArgs& a, const long long e, WarpShared<NP, WARPS>& sh) {
  constexpr int RA = NP / 8;     // rows per lane
  constexpr int CB = NP / 4;     // columns per lane
  constexpr int NKB = NP / 4;    // 4-step blocks of the elimination
  constexpr int CH = CB / 2;     // columns per lane in one half of the residual pass
  constexpr int ES = NP + 4;     // row stride of the shared tile (bank stagger)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = lane >> 2, lc = lane & 3;
  const int n = a.n, L = a.grid.L;
  const int* s_lab = sh.lab;
  double2* w = sh.w[warp];
  float2* invk = sh.inv[warp];
  float2* pv = sh.piv[warp];
  float2* T = sh.LU[warp];
  float2* xs = sh.x[warp];
  float2* rs = sh.r[warp];
  const float2 zero = make_float2(0.0f, 0.0f);
  if (e < a.grid.n_eval) {
    if (lane < L) w[lane] = grid_root(a.tw, a.grid, lane, point_digit(e, a.grid, lane));
    __syncwarp();

    // ---- 1. M^ = fl32(conj(D) - XA), padded with the identity; LU in registers.
    // Steps run in blocks of four (k = 4 kb + kc): within a block the owning register
    // column kb and row ka = kb / 2 are compile-time constants, kc is a runtime loop.
    float2 A[RA][CB];
#pragma unroll
    for (int ra = 0; ra < RA; ++ra)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) {
        const int i = lr + 8 * ra, j = lc + 4 * cb;
        float2 v = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
        if (i < n && j < n) {
          if (i == j) {
            const double2 x = a.NXA[i * n + j], d = w[s_lab[i]];
            v = make_float2((float)(x.x + d.x), (float)(x.y - d.y));
          } else {
            v = a.NXA_hi[i * n + j];
          }
        }
        A[ra][cb] = v;
      }
#pragma unroll
    for (int kb = 0; kb < NKB; ++kb) {
      const int ka = kb >> 1;
#pragma unroll 1
      for (int kc = 0; kc < 4; ++kc) {
        const int k = 4 * kb + kc, kr = k & 7;
        const float2 inv = crecipf(shfl2(A[ka][kb], kr * 4 + kc));
        if (lane == 0) invk[k] = inv;
        if (k == NP - 1) break;
#pragma unroll
        for (int ra = 0; ra < RA; ++ra)
          if (8 * ra + 7 >= 4 * kb && lc == kc && lr + 8 * ra > k) A[ra][kb] = cmulf(A[ra][kb], inv);
        // the multipliers of rows <= k and the pivot-row entries of columns <= k are
        // broadcast as zero, which leaves those entries exactly unchanged (a - 0 u = a):
        // one select per broadcast value instead of one per updated entry
        float2 l[RA], u[CB];
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {
          const float2 v = (8 * ra + 7 < 4 * kb) ? zero : shfl2(A[ra][kb], lr * 4 + kc);
          l[ra] = lr + 8 * ra > k ? v : zero;
        }
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) {
          const float2 v = (cb < kb) ? zero : shfl2(A[ka][cb], kr * 4 + lc);
          u[cb] = lc + 4 * cb > k ? v : zero;
        }
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {
          if (8 * ra + 7 < 4 * kb) continue;
          if (8 * ra + 7 <= k) continue;        // warp-uniform
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            if (cb < kb) continue;
            A[ra][cb] = cfnmaf(A[ra][cb], l[ra], u[cb]);
          }
        }
      }
    }
    // ---- 2. rounding: row i of L^ onto the grid 2^(erow_i - 24), column j of U^ onto
    // 2^(fcol_j - 24), all entries below 2^erow_i (2^fcol_j); the rounded factors are used
    // from here on.  Their int32 digits go to the warp's tile, the exponents to sh.ex.
    int erow[RA], fcol[CB];
    bool bad = false;
#pragma unroll
    for (int ra = 0; ra < RA; ++ra) {
      const int i = lr + 8 * ra;
      float m = 0.0f;
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
        if (lc + 4 * cb < i) m = fmaxf(m, fmaxf(fabsf(A[ra][cb].x), fabsf(A[ra][cb].y)));
      m = fmaxf(m, __shfl_xor_sync(kFull, m, 1));
      m = fmaxf(m, __shfl_xor_sync(kFull, m, 2));
      const int ex = exponent_bound(m);
      bad |= ex > 20;
      erow[ra] = min(max(ex, 0), 20);
    }
#pragma unroll
    for (int cb = 0; cb < CB; ++cb) {
      const int j = lc + 4 * cb;
      float m = 0.0f;
#pragma unroll
      for (int ra = 0; ra < RA; ++ra)
        if (lr + 8 * ra <= j) m = fmaxf(m, fmaxf(fabsf(A[ra][cb].x), fabsf(A[ra][cb].y)));
      m = fmaxf(m, __shfl_xor_sync(kFull, m, 4));
      m = fmaxf(m, __shfl_xor_sync(kFull, m, 8));
      m = fmaxf(m, __shfl_xor_sync(kFull, m, 16));
      const int ex = exponent_bound(m);
      bad |= ex > 29;
      fcol[cb] = min(max(ex, -14), 29);
    }
    int2* Tq = reinterpret_cast<int2*>(T);
    __syncwarp();                       // the LU's writes of invk (lane 0) come first
#pragma unroll
    for (int ra = 0; ra < RA; ++ra)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) {
        const int i = lr + 8 * ra, j = lc + 4 * cb;
        const int sc = 24 - (i > j ? erow[ra] : fcol[cb]);
        const float qx = rintf(A[ra][cb].x * pow2f(sc)), qy = rintf(A[ra][cb].y * pow2f(sc));
        Tq[i * ES + j] = make_int2((int)qx, (int)qy);
        if (i == j) {
          const float2 u = make_float2(qx * pow2f(-sc), qy * pow2f(-sc));
          pv[i] = u;
          invk[i] = crecipf(u);
        }
      }
    __syncwarp();

    // ---- 3. log det = sum_i Log(d_i u'_ii) (each factor has Re > 0): the product of the
    // factors by a butterfly over the lanes in FP64 and the FP32 sum of their arguments
    // (each in (-pi/2, pi/2), so the sum is far closer to the exact one than pi, which
    // fixes the winding).  The Log of the product is taken by the DFT's first kernel,
    // one point per thread, off this kernel's FP64 pipe.
    double mn = 1.0e300;
    {
      double2 z = make_double2(1.0, 0.0);
      float arg = 0.0f;
      if (lane < n) {
        const float2 u = pv[lane];
        z = cmul(w[s_lab[lane]], make_double2(u.x, u.y));
        mn = z.x;
        if (!(z.x == z.x) || !(z.y == z.y)) mn = -1.0e300;
        arg = atan2f((float)z.y, (float)z.x);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double2 y = make_double2(__shfl_xor_sync(kFull, z.x, o), __shfl_xor_sync(kFull, z.y, o));
        z = cmul(z, y);
        arg += __shfl_xor_sync(kFull, arg, o);
      }
      if (lane == 0) {
        double* f = a.ldfin + 6 * e;
        f[0] = z.x;
        f[1] = z.y;
        f[2] = (double)arg;
        f[5] = 0.0;
      }
    }
    mn = warp_min_d(mn);
    if (__any_sync(kFull, bad)) mn = -1.0e300;

    // ---- 4. residual E = M - L^U^ exactly: digit products summed in int64 (Karatsuba,
    // three 32 x 32 -> 64-bit multiply-adds per complex term), M from the fixed-point
    // -XA shifted to the entry's scale 2^(erow_i + fcol_j - 48), one rounding to FP32.
    // Two columns per pass; terms outside k < min(i, j + 1) get a zero digit.
    float2 Z[RA][CB];
#pragma unroll
    for (int h = 0; h < CB / 2; ++h) {
      long long sa[RA][2], sb[RA][2], sc[RA][2];
#pragma unroll
      for (int ra = 0; ra < RA; ++ra)
#pragma unroll
        for (int q = 0; q < 2; ++q) sa[ra][q] = sb[ra][q] = sc[ra][q] = 0;
      const int kend = 4 * (2 * h + 1) + 3;   // largest column of this pass
#pragma unroll 4
      for (int k = 0; k < NP - 1 && k <= kend; ++k) {
        int ux[2], uy[2], us[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = lc + 4 * (2 * h + q);
          const int2 u = Tq[k * ES + j];
          ux[q] = k <= j ? u.x : 0;
          uy[q] = k <= j ? u.y : 0;
          us[q] = ux[q] + uy[q];
        }
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {
          if (8 * ra + 7 <= k) continue;        // warp-uniform: all rows of the group <= k
          const int i = lr + 8 * ra;
          const int2 l = Tq[i * ES + k];
          const int lx = k < i ? l.x : 0, ly = k < i ? l.y : 0, ls = lx + ly;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            sa[ra][q] += (long long)lx * ux[q];
            sb[ra][q] += (long long)ly * uy[q];
            sc[ra][q] += (long long)ls * us[q];
          }
        }
      }
#pragma unroll
      for (int ra = 0; ra < RA; ++ra)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int cb = 2 * h + q, i = lr + 8 * ra, j = lc + 4 * cb;
          const int sh = GBSBIN_FIX_BITS - 48 + erow[ra] + fcol[cb];
          longlong2 mf = make_longlong2(i == j ? (1ll << GBSBIN_FIX_BITS) : 0ll, 0ll);   // identity padding
          if (i < n && j < n) mf = a.NXA_fix[i * n + j];
          long long er = (mf.x >> sh) - (sa[ra][q] - sb[ra][q]);
          long long ei = (mf.y >> sh) - (sc[ra][q] - sa[ra][q] - sb[ra][q]);
          if (i <= j) {                  // L_ii U_ij = U_ij
            const int2 u = Tq[i * ES + j];
            er -= (long long)u.x << (24 - erow[ra]);
            ei -= (long long)u.y << (24 - erow[ra]);
          }
          if (i == j && i < n) {
            const longlong2 dc = conj_fix(w[s_lab[i]]);
            er += dc.x >> sh;
            ei += dc.y >> sh;
          }
          const float s = pow2f(erow[ra] + fcol[cb] - 48);
          Z[ra][cb] = make_float2(ll2f(er) * s, ll2f(ei) * s);
        }
    }
    // the rounded L\U back into registers (from the digits) and, as FP32, into the tile
    // for the exponent's substitutions
#pragma unroll
    for (int ra = 0; ra < RA; ++ra)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) {
        const int i = lr + 8 * ra, j = lc + 4 * cb;
        const int sc = (i > j ? erow[ra] : fcol[cb]) - 24;
        const int2 q = Tq[i * ES + j];
        A[ra][cb] = make_float2((float)q.x * pow2f(sc), (float)q.y * pow2f(sc));
      }
    __syncwarp();
#pragma unroll
    for (int ra = 0; ra < RA; ++ra)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) T[(lr + 8 * ra) * ES + lc + 4 * cb] = A[ra][cb];
    __syncwarp();

    // ---- 5. delta = tr(U^^{-1} L^^{-1} E): Z = L^^{-1} E, then X = U^^{-1} Z on m >= c
#pragma unroll
    for (int kb = 0; kb < NKB; ++kb) {
      const int ka = kb >> 1;
#pragma unroll 1
      for (int kc = 0; kc < 4; ++kc) {
        const int k = 4 * kb + kc, kr = k & 7;
        if (k == NP - 1) break;
        float2 l[RA], z[CB];
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {       // zero multiplier for rows <= k
          const float2 v = (8 * ra + 7 < 4 * kb) ? zero : shfl2(A[ra][kb], lr * 4 + kc);
          l[ra] = lr + 8 * ra > k ? v : zero;
        }
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) z[cb] = shfl2(Z[ka][cb], kr * 4 + lc);
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {
          if (8 * ra + 7 < 4 * kb) continue;
          if (8 * ra + 7 <= k) continue;
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) Z[ra][cb] = cfnmaf(Z[ra][cb], l[ra], z[cb]);
        }
      }
    }
#pragma unroll
    for (int kb = NKB - 1; kb >= 0; --kb) {
      const int ka = kb >> 1;
#pragma unroll 1
      for (int kc = 3; kc >= 0; --kc) {
        const int k = 4 * kb + kc, kr = k & 7;
        const float2 ik = invk[k];
        if (lr == kr) {
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) Z[ka][cb] = cmulf(Z[ka][cb], ik);
        }
        if (k == 0) break;
        float2 uk[RA], x[CB];
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {       // zero U entry for rows >= k
          const float2 v = (8 * ra > 4 * kb + 3) ? zero : shfl2(A[ra][kb], lr * 4 + kc);
          uk[ra] = lr + 8 * ra < k ? v : zero;
        }
#pragma unroll
        for (int cb = 0; cb < CB; ++cb) x[cb] = (cb > kb) ? zero : shfl2(Z[ka][cb], kr * 4 + lc);
#pragma unroll
        for (int ra = 0; ra < RA; ++ra) {
          if (8 * ra > 4 * kb + 3) continue;
          if (8 * ra >= k) continue;
#pragma unroll
          for (int cb = 0; cb < CB; ++cb) {
            if (cb > kb) continue;
            Z[ra][cb] = cfnmaf(Z[ra][cb], uk[ra], x[cb]);
          }
        }
      }
    }
    double dre = 0.0, dim = 0.0;
#pragma unroll
    for (int ra = 0; ra < RA; ++ra)
#pragma unroll
      for (int cb = 0; cb < CB; ++cb)
        if (lr + 8 * ra == lc + 4 * cb && lr + 8 * ra < n) {
          dre += (double)Z[ra][cb].x;
          dim += (double)Z[ra][cb].y;
        }
    dre = warp_sum_d(dre);
    dim = warp_sum_d(dim);

    // ---- 6. exponent with one refinement step (triangular solves read the tile)
    double ex_re = 0.0, ex_im = 0.0;
    if (a.has_gamma) {
      for (int pass = 0; pass < 2; ++pass) {
        float2* v = pass == 0 ? xs : rs;
        if (pass == 0) {
          if (lane < NP) v[lane] = lane < n ? a.Xg_hi[lane] : zero;
          __syncwarp();
        }
        for (int k = 0; k < NP - 1; ++k) {      // v_i -= L_ik v_k, i > k
          const float2 vk = v[k];
          __syncwarp();
          for (int i = k + 1 + lane; i < NP; i += 32) v[i] = cfnmaf(v[i], T[i * ES + k], vk);
          __syncwarp();
        }
        for (int k = NP - 1; k >= 0; --k) {     // v_k /= u_kk; v_i -= U_ik v_k, i < k
          const float2 vk = cmulf(v[k], invk[k]);
          __syncwarp();
          if (lane == 0) v[k] = vk;
          for (int i = lane; i < k; i += 32) v[i] = cfnmaf(v[i], T[i * ES + k], vk);
          __syncwarp();
        }
        if (pass == 0) {
          // r = X gamma - M x^ = X gamma - conj(d) x^ - NXA x^, Dot2 per row (lane = row)
          float2 rr = zero;
          if (lane < n) {
            const int i = lane;
            Acc2 sr = {0.0f, 0.0f}, si = {0.0f, 0.0f};
            const float2 gh = a.Xg_hi[i], gl = a.Xg_lo[i];
            acc2_add(sr, gh.x);
            acc2_add(sr, gl.x);
            acc2_add(si, gh.y);
            acc2_add(si, gl.y);
            for (int j = 0; j < n; ++j) {
              const float2 xh = a.NXA_hi[i * n + j], xl = a.NXA_lo[i * n + j], y = xs[j];
              acc2_add_prod(sr, -xh.x, y.x);
              acc2_add_prod(sr, xh.y, y.y);
              acc2_add_prod(sr, -xl.x, y.x);
              acc2_add_prod(sr, xl.y, y.y);
              acc2_add_prod(si, -xh.x, y.y);
              acc2_add_prod(si, -xh.y, y.x);
              acc2_add_prod(si, -xl.x, y.y);
              acc2_add_prod(si, -xl.y, y.x);
            }
            const double2 d = w[s_lab[i]];
            const float dhx = (float)d.x, dhy = (float)d.y;
            const float dlx = (float)(d.x - (double)dhx), dly = (float)(d.y - (double)dhy);
            const float2 y = xs[i];
            acc2_add_prod(sr, -dhx, y.x);
            acc2_add_prod(sr, -dhy, y.y);
            acc2_add_prod(si, -dhx, y.y);
            acc2_add_prod(si, dhy, y.x);
            acc2_add_prod(sr, -dlx, y.x);
            acc2_add_prod(sr, -dly, y.y);
            acc2_add_prod(si, -dlx, y.y);
            acc2_add_prod(si, dly, y.x);
            rr = make_float2(acc2_value(sr), acc2_value(si));
          }
          __syncwarp();
          if (lane < NP) rs[lane] = rr;
          __syncwarp();
        }
      }
      if (lane < n) {
        const double xr = (double)xs[lane].x + (double)rs[lane].x, xi = (double)xs[lane].y + (double)rs[lane].y;
        const double gr = (double)a.g_hi[lane].x + (double)a.g_lo[lane].x;
        const double gi = (double)a.g_hi[lane].y + (double)a.g_lo[lane].y;
        ex_re = gr * xr - gi * xi;
        ex_im = gr * xi + gi * xr;
      }
      ex_re = warp_sum_d(ex_re);
      ex_im = warp_sum_d(ex_im);
    }

    if (lane == 0) {
      // unfinished log q: log det is completed from (product, argument sum) by the DFT
      double* f = a.ldfin + 6 * e;
      f[3] = 0.5 * ex_re - 0.5 * dre;
      f[4] = 0.5 * ex_im - 0.5 * dim;
      a.minpiv[e] = mn;
    }
    __syncwarp();
  }
}

template <int NP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 3) k_points_fp32r_warp(PointArgs a0, PointBatch batch) {
  __shared__ __align__(16) WarpShared<NP, WARPS> sh;
  const int warp = threadIdx.x >> 5;
  if (!batch.probs) {
    for (int i = threadIdx.x; i < NP; i += WARPS * 32) sh.lab[i] = i < a0.n ? a0.label[i] : 0;
    __syncthreads();
    for (long long e = (long long)blockIdx.x * WARPS + warp; e < a0.grid.n_eval; e += (long long)gridDim.x * WARPS)
      warp_point<NP, WARPS>(a0, e, sh);
    return;
  }
  __shared__ PointArgs sa;
  __shared__ long long sj;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long j = atomicAdd(batch.queue, 1ull);
      sj = (long long)j;
      if ((long long)j < batch.njobs) sa = batch.probs[batch.jobs[j].prob];
    }
    __syncthreads();
    const long long j = sj;
    if (j >= batch.njobs) break;
    for (int i = threadIdx.x; i < NP; i += WARPS * 32) sh.lab[i] = i < sa.n ? sa.label[i] : 0;
    __syncthreads();
    warp_point<NP, WARPS>(sa, batch.jobs[j].e0 + warp, sh);
    __syncthreads();
  }
}

template <int NP>
static cudaError_t launch_warp_np(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  constexpr int WARPS = 4;
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_points_fp32r_warp<NP, WARPS>,
                                                                  WARPS * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  long long groups = batch.probs ? batch.njobs : (a.grid.n_eval + WARPS - 1) / WARPS;
  long long grid = (long long)per_sm * num_sms;
  if (grid > groups) grid = groups;
  if (grid < 1) grid = 1;
  k_points_fp32r_warp<NP, WARPS><<<(unsigned)grid, WARPS * 32, 0, s>>>(a, batch);
  return cudaGetLastError();
}

cudaError_t launch_points_warp(const PointArgs& a, int num_sms, cudaStream_t s) {
  PointBatch none{};
  if (a.n <= 8) return launch_warp_np<8>(a, none, num_sms, s);
  if (a.n <= 16) return launch_warp_np<16>(a, none, num_sms, s);
  if (a.n <= 32) return launch_warp_np<32>(a, none, num_sms, s);
  return cudaErrorInvalidValue;
}

// Batch: jobs of WARPS consecutive points of one problem; np is the padded size class.
cudaError_t launch_points_warp_batch(const PointBatch& batch, int np, int num_sms, cudaStream_t s) {
  PointArgs dummy{};
  dummy.grid.n_eval = 1;
  if (np == 8) return launch_warp_np<8>(dummy, batch, num_sms, s);
  if (np == 16) return launch_warp_np<16>(dummy, batch, num_sms, s);
  if (np == 32) return launch_warp_np<32>(dummy, batch, num_sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace gbsbin
