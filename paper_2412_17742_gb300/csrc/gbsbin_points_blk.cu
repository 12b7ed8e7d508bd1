// Blocked FP32 + refinement kernel for large n (arXiv:2412.17742, Sec. III Eq. q_d with the
// grouping of Sec. VI; the same mathematics as k_points_fp32r).
//
// One CTA of 256 threads per grid point (persistent over points / batch jobs).  The
// per-point matrix M = conj(D) - XA and the residual E live in the CTA's slot of an
// L2-resident global workspace; every O(n^3) phase runs blocked with NB = 32 columns so
// the inner loops are register-tiled (4 x 4 complex per thread) against panels staged in
// shared memory:
//   LU        right-looking: panel LU in shared memory, U12 = L11^{-1} A12 column by
//             column, A22 -= L21 U12 as a tiled rank-32 update;
//   rounding  each row of L^ and each column of U^ is rounded onto a 24-bit fixed-point
//             grid (scale 2^(24 - e) with |entries| < 2^e), which moves an entry by at most
//             the FP32 rounding of the largest one; the LU in use from here on is the rounded
//             one, exactly representable both as FP32 and as int32 digits;
//   residual  E = M - L^U^ exactly: the products of digits are summed in int64 (three
//             32 x 32 -> 64-bit multiply-adds per complex term, Karatsuba), M enters as a
//             fixed-point copy of -XA (2^62 scale) shifted to the entry's scale, and the
//             difference is rounded to FP32 once; 64 x 64 output blocks, digit chunks staged;
//   trace     Z = L^^{-1} E (blocked forward substitution on all columns) and the entries
//             X[m][c], m >= c, of X = U^^{-1} Z (blocked back substitution), delta =
//             sum_c X[c][c];
// then the FP64 epilogue: log det = sum Log(d_i u'_ii) + delta and the refined exponent.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbsbin_device.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int NT = 256;
constexpr int NB = 32;                  // panel width
constexpr int LDP = NB + 1;             // leading dimension of staged panels (bank stagger)
constexpr int EB = 64;                  // residual output block rows
constexpr int EBJ = 32;                 // residual output block columns
constexpr int CTAS_PER_SM = GBSBIN_BLK_CTAS_PER_SM;   // resident CTAs per SM where shared memory allows

// shared-memory plan (float2 units): panel [n x LDP], row block [NB x (n + 1)], vectors
struct BlkSmem {
  float2* panel;   // rows x LDP
  float2* rowb;    // NB x ldr
  int ldr;
  double2* w;      // L twiddles
  float2* pinv;    // n
  float2* xv;      // n
  float2* rv;      // n
  double2* red;    // NT / 32
  double2* red2;   // NT / 32
  int* lab;        // n
  int* erow;       // n: exponent bound of row i of L^ (|L^_ik| < 2^erow[i])
  int* fcol;       // n: exponent bound of column j of U^
  int* bad;        // 1: a factor fell outside the fixed-point range
};

__device__ __forceinline__ BlkSmem carve(unsigned char* smem, int n, int L) {
  BlkSmem s;
  const int R = n > EB ? n : EB;        // the residual pass stages EB-row chunks
  float2* f = (float2*)smem;
  s.panel = f;
  f += (size_t)R * LDP;
  s.ldr = R + 1;
  s.rowb = f;
  f += (size_t)NB * s.ldr;
  s.pinv = f;
  f += n;
  s.xv = f;
  f += n;
  s.rv = f;
  f += n;
  uintptr_t p = ((uintptr_t)f + 15) & ~(uintptr_t)15;
  s.w = (double2*)p;
  s.red = s.w + GBSBIN_MAX_L;
  s.red2 = s.red + NT / 32;
  s.lab = (int*)(s.red2 + NT / 32);
  s.erow = s.lab + n;
  s.fcol = s.erow + n;
  s.bad = s.fcol + n;
  return s;
}

// C[r0 + i][c0 + j] -= sum_{k < kd} Ls[i * LDP + k] Us[k * ldu + j]  for i < nr, j < nc,
// optionally only for entries with mask(i, j).  C is global with leading dimension ldc.
template <typename Mask>
__device__ __forceinline__ void tile_update(float2* C, int ldc, int r0, int c0, int nr, int nc, const float2* Ls,
                                            const float2* Us, int ldu, int kd, Mask mask) {
  // thread tile: rows ti .. ti+3, columns tj + b tc (b < 4), so that consecutive threads
  // read consecutive columns of the staged U rows and write consecutive entries of C
  const int tr = (nr + 3) >> 2, tc = (nc + 3) >> 2;
  for (int t = threadIdx.x; t < tr * tc; t += NT) {
    const int ti = (t / tc) * 4, tj = t - (t / tc) * tc;
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
    for (int k = 0; k < kd; ++k) {
      float2 l[4], u[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) l[a] = ti + a < nr ? Ls[(ti + a) * LDP + k] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int b = 0; b < 4; ++b) u[b] = tj + b * tc < nc ? Us[k * ldu + tj + b * tc] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x = fmaf(l[a].x, u[b].x, fmaf(-l[a].y, u[b].y, acc[a][b].x));
          acc[a][b].y = fmaf(l[a].x, u[b].y, fmaf(l[a].y, u[b].x, acc[a][b].y));
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ti + a, j = tj + b * tc;
        if (i < nr && j < nc && mask(i, j)) {
          float2* c = C + (size_t)(r0 + i) * ldc + (c0 + j);
          float2 v = *c;
          *c = make_float2(v.x - acc[a][b].x, v.y - acc[a][b].y);
        }
      }
  }
}

struct NoMask {
  __device__ bool operator()(int, int) const { return true; }
};


// v <- U^^{-1} L^^{-1} v for one right-hand side v (shared memory, n entries), with L\U
// in global memory (unit lower L) and pinv[k] = 1 / u_kk, by the whole CTA: per 32-row
// block, warp 0 solves the diagonal block with shuffles and all threads apply the
// off-diagonal rows.  Ends with __syncthreads().
__device__ __forceinline__ void cta_solve_lu(const float2* A, int n, const float2* pinv, float2* v) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k0 = 0; k0 < n; k0 += NB) {           // forward: L y = v
    const int nb = min(NB, n - k0);
    if (tid < 32) {
      float2 row[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        row[q] = (lane < nb && q < lane) ? A[(size_t)(k0 + lane) * n + k0 + q] : make_float2(0.f, 0.f);
      float2 vr = lane < nb ? v[k0 + lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < NB - 1; ++q) {
        const float2 vq = make_float2(__shfl_sync(0xffffffffu, vr.x, q), __shfl_sync(0xffffffffu, vr.y, q));
        if (lane > q) vr = cfnmaf(vr, row[q], vq);
      }
      if (lane < nb) v[k0 + lane] = vr;
    }
    __syncthreads();
    for (int i = k0 + nb + tid; i < n; i += NT) {
      float2 acc = v[i];
      for (int q = 0; q < nb; ++q) acc = cfnmaf(acc, A[(size_t)i * n + k0 + q], v[k0 + q]);
      v[i] = acc;
    }
    __syncthreads();
  }
  for (int k0 = ((n - 1) / NB) * NB; k0 >= 0; k0 -= NB) {   // backward: U x = y
    const int nb = min(NB, n - k0);
    if (tid < 32) {
      float2 row[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q)
        row[q] = (lane < nb && q > lane && q < nb) ? A[(size_t)(k0 + lane) * n + k0 + q] : make_float2(0.f, 0.f);
      float2 vr = lane < nb ? v[k0 + lane] : make_float2(0.f, 0.f);
      const float2 ip = lane < nb ? pinv[k0 + lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = NB - 1; q >= 0; --q) {
        if (lane == q) vr = cmulf(vr, ip);
        const float2 xq = make_float2(__shfl_sync(0xffffffffu, vr.x, q), __shfl_sync(0xffffffffu, vr.y, q));
        if (lane < q) vr = cfnmaf(vr, row[q], xq);
      }
      if (lane < nb) v[k0 + lane] = vr;
    }
    __syncthreads();
    for (int i = tid; i < k0; i += NT) {
      float2 acc = v[i];
      for (int q = 0; q < nb; ++q) acc = cfnmaf(acc, A[(size_t)i * n + k0 + q], v[k0 + q]);
      v[i] = acc;
    }
    __syncthreads();
  }
}

}  // namespace

__device__ void group_fp32r_blk(const PointArgs& a, const long long e, unsigned char* smem) {
  const int n = a.n, L = a.grid.L, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  BlkSmem sm = carve(smem, n, L);
  float2* A = (float2*)((char*)a.gws + (size_t)blockIdx.x * (size_t)a.gws_slot_bytes);
  float2* E = A + (size_t)n * n;
  for (int i = tid; i < n; i += NT) sm.lab[i] = a.label[i];
  if (tid < L) sm.w[tid] = root_of_unity(point_digit(e, a.grid, tid), a.grid.radix[tid]);
  __syncthreads();

  // M^ = fl32(conj(D) - XA)
  for (int t = tid; t < n * n; t += NT) {
    const int i = t / n, j = t - i * n;
    float2 v = a.NXA_hi[t];
    if (i == j) {
      const double2 d = sm.w[sm.lab[i]], x = a.NXA[t];
      v = make_float2((float)(x.x + d.x), (float)(x.y - d.y));
    }
    A[t] = v;
  }
  __syncthreads();

  // ---------------------------------------------------------------- blocked LU
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0), rows = n - k0, m = n - k0 - nb;
    for (int t = tid; t < rows * nb; t += NT) {
      const int i = t / nb, c = t - i * nb;
      sm.panel[i * LDP + c] = A[(size_t)(k0 + i) * n + k0 + c];
    }
    __syncthreads();
    for (int kk = 0; kk < nb; ++kk) {          // unblocked LU of the panel
      const float2 inv = crecipf(sm.panel[kk * LDP + kk]);
      if (tid == 0) sm.pinv[k0 + kk] = inv;
      for (int i = kk + 1 + tid; i < rows; i += NT) sm.panel[i * LDP + kk] = cmulf(sm.panel[i * LDP + kk], inv);
      __syncthreads();
      const int cols = nb - kk - 1;
      if (cols > 0)
        for (int t = tid; t < (rows - kk - 1) * cols; t += NT) {
          const int i = kk + 1 + t / cols, c = kk + 1 + (t - (t / cols) * cols);
          sm.panel[i * LDP + c] = cfnmaf(sm.panel[i * LDP + c], sm.panel[i * LDP + kk], sm.panel[kk * LDP + c]);
        }
      __syncthreads();
    }
    for (int t = tid; t < rows * nb; t += NT) {
      const int i = t / nb, c = t - i * nb;
      A[(size_t)(k0 + i) * n + k0 + c] = sm.panel[i * LDP + c];
    }
    if (m > 0) {
      // U12 = L11^{-1} A12: one column per thread, then stage it in rowb
      for (int j = tid; j < m; j += NT) {
        float2 col[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) col[r] = r < nb ? A[(size_t)(k0 + r) * n + k0 + nb + j] : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r < NB; ++r)
#pragma unroll
          for (int q = 0; q < r; ++q)
            if (r < nb) col[r] = cfnmaf(col[r], sm.panel[r * LDP + q], col[q]);
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < nb) {
            A[(size_t)(k0 + r) * n + k0 + nb + j] = col[r];
            sm.rowb[r * sm.ldr + j] = col[r];
          }
      }
      __syncthreads();
      tile_update(A, n, k0 + nb, k0 + nb, m, m, sm.panel + nb * LDP, sm.rowb, sm.ldr, nb, NoMask());
    }
    __syncthreads();
  }

  // --------------------------------------- rounding of L^ and U^ onto fixed-point grids
  // The integer digits share memory with E: the residual pass below visits its output
  // blocks in reverse order, and every digit of block (bi, bj) is read only by blocks
  // (bi, bj' >= bj) (an L digit) or (bi' >= bi, bj) (a U digit), which come earlier.
  int2* Q = (int2*)E;
  if (tid == 0) *sm.bad = 0;
  for (int i = warp; i < n; i += NT / 32) {      // row bound of L^ (k < i), warp per row
    float m = 0.0f;
    for (int k = lane; k < i; k += 32) {
      const float2 v = A[(size_t)i * n + k];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      int ex = exponent_bound(m);
      if (ex < 0) ex = 0;
      if (ex > 20) {                              // L^ entries this large: not a physical state
        ex = 20;
        *sm.bad = 1;
      }
      sm.erow[i] = ex;
    }
  }
  for (int j = tid; j < n; j += NT) {             // column bound of U^ (k <= j), thread per column
    float m = 0.0f;
    for (int k = 0; k <= j; ++k) {
      const float2 v = A[(size_t)k * n + j];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    int ex = exponent_bound(m);
    if (ex < -14) ex = -14;
    if (ex > 29) {                                // keeps the shift below 64
      ex = 29;
      *sm.bad = 1;
    }
    sm.fcol[j] = ex;
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += NT) {
    const int i = t / n, j = t - i * n;
    const int sc = 24 - (i > j ? sm.erow[i] : sm.fcol[j]);
    const float2 v = A[t];
    const float qx = rintf(v.x * pow2f(sc)), qy = rintf(v.y * pow2f(sc));
    A[t] = make_float2(qx * pow2f(-sc), qy * pow2f(-sc));
    Q[t] = make_int2((int)qx, (int)qy);
  }
  __syncthreads();
  for (int k = tid; k < n; k += NT) sm.pinv[k] = crecipf(A[(size_t)k * n + k]);

  // ------------------------------------------- residual E = M - L^U^, exact in int64
  // (panel / rowb stage the digits: L chunk EB x NB, U chunk NB x EBJ, int2)
  {
    int2* Ls = (int2*)sm.panel;
    int2* Us = (int2*)sm.rowb;
    const int nbi = (n + EB - 1) / EB, nbj = (n + EBJ - 1) / EBJ;
    // this thread's 4 x 2 entries of a 64 x 32 block: rows ti .. ti+3, columns tj, tj + 16
    const int ti = (tid >> 4) * 4, tj = tid & 15;
    for (int bi = nbi - 1; bi >= 0; --bi)
      for (int bj = nbj - 1; bj >= 0; --bj) {
        const int i0 = bi * EB, j0 = bj * EBJ;
        const int ni = min(EB, n - i0), nj = min(EBJ, n - j0);
        long long sa[4][2], sb[4][2], sc[4][2];   // sum lr ur, sum li ui, sum (lr+li)(ur+ui)
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 2; ++q) sa[p][q] = sb[p][q] = sc[p][q] = 0;
        const int kmax = min(i0 + ni, j0 + nj);   // terms need k < i and k <= j
        for (int kc = 0; kc < kmax; kc += NB) {
          const int kd = min(NB, kmax - kc);
          __syncthreads();
          for (int t = tid; t < EB * NB; t += NT) {
            const int r = t / NB, c = t - r * NB;
            Ls[r * LDP + c] = (r < ni && c < kd) ? Q[(size_t)(i0 + r) * n + kc + c] : make_int2(0, 0);
          }
          for (int t = tid; t < NB * EBJ; t += NT) {
            const int rr = t / EBJ, cc = t - rr * EBJ;
            Us[rr * sm.ldr + cc] = (rr < kd && cc < nj) ? Q[(size_t)(kc + rr) * n + j0 + cc] : make_int2(0, 0);
          }
          __syncthreads();
#pragma unroll 2
          for (int k = 0; k < kd; ++k) {
            const int kg = kc + k;
            int lx[4], ly[4], ls[4], ux[2], uy[2], us[2];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int2 v = Ls[(ti + p) * LDP + k];
              const bool ok = kg < i0 + ti + p;    // k < i: L_ik is a multiplier
              lx[p] = ok ? v.x : 0;
              ly[p] = ok ? v.y : 0;
              ls[p] = lx[p] + ly[p];
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int2 v = Us[k * sm.ldr + tj + 16 * q];
              const bool ok = kg <= j0 + tj + 16 * q;   // k <= j: U_kj is in the upper factor
              ux[q] = ok ? v.x : 0;
              uy[q] = ok ? v.y : 0;
              us[q] = ux[q] + uy[q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                sa[p][q] += (long long)lx[p] * ux[q];
                sb[p][q] += (long long)ly[p] * uy[q];
                sc[p][q] += (long long)ls[p] * us[q];
              }
          }
        }
        // every read of this block's digits by other threads happened in the staging above
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int i = i0 + ti + p, j = j0 + tj + 16 * q;
            if (ti + p >= ni || tj + 16 * q >= nj) continue;
            const size_t ij = (size_t)i * n + j;
            const int ei = sm.erow[i], fj = sm.fcol[j];
            const int sh = GBSBIN_FIX_BITS - 48 + ei + fj;   // 2^62 scale -> 2^(48 - ei - fj)
            const longlong2 mf = a.NXA_fix[ij];
            long long er = (mf.x >> sh) - (sa[p][q] - sb[p][q]);
            long long eim = (mf.y >> sh) - (sc[p][q] - sa[p][q] - sb[p][q]);
            if (i <= j) {                      // L_ii U_ij = U_ij (this thread's own digit)
              const int2 u = Q[ij];
              er -= (long long)u.x << (24 - ei);
              eim -= (long long)u.y << (24 - ei);
            }
            if (i == j) {                      // conj(d_i) on the diagonal of M
              const longlong2 dc = conj_fix(sm.w[sm.lab[i]]);
              er += dc.x >> sh;
              eim += dc.y >> sh;
            }
            const float s = pow2f(ei + fj - 48);     // value of one unit of the products
            E[ij] = make_float2(ll2f(er) * s, ll2f(eim) * s);
          }
      }
  }
  __syncthreads();

  // ------------------------------------------- Z = L^^{-1} E, all columns, blocked
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0), m = n - k0 - nb;
    for (int t = tid; t < nb * nb; t += NT) {      // L11 into the panel stage
      const int r = t / nb, c = t - r * nb;
      sm.panel[r * LDP + c] = A[(size_t)(k0 + r) * n + k0 + c];
    }
    __syncthreads();
    for (int j = tid; j < n; j += NT) {            // Z[k0 block, j] = L11^{-1} E[k0 block, j]
      float2 col[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) col[r] = r < nb ? E[(size_t)(k0 + r) * n + j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 1; r < NB; ++r)
#pragma unroll
        for (int q = 0; q < r; ++q)
          if (r < nb) col[r] = cfnmaf(col[r], sm.panel[r * LDP + q], col[q]);
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) {
          E[(size_t)(k0 + r) * n + j] = col[r];
          sm.rowb[r * sm.ldr + j] = col[r];
        }
    }
    __syncthreads();
    if (m > 0) {
      for (int t = tid; t < m * nb; t += NT) {     // L21 into the panel stage
        const int r = t / nb, c = t - r * nb;
        sm.panel[r * LDP + c] = A[(size_t)(k0 + nb + r) * n + k0 + c];
      }
      __syncthreads();
      tile_update(E, n, k0 + nb, 0, m, n, sm.panel, sm.rowb, sm.ldr, nb, NoMask());
    }
    __syncthreads();
  }
  // ------------------------- X = U^^{-1} Z on the entries X[m][c], m >= c, blocked
  const int last0 = ((n - 1) / NB) * NB;
  for (int k0 = last0; k0 >= 0; k0 -= NB) {
    const int nb = min(NB, n - k0);
    const int ncol = k0 + nb;                       // columns c <= block's last row
    for (int t = tid; t < nb * nb; t += NT) {       // U11 into the panel stage
      const int r = t / nb, c = t - r * nb;
      sm.panel[r * LDP + c] = A[(size_t)(k0 + r) * n + k0 + c];
    }
    __syncthreads();
    for (int j = tid; j < ncol; j += NT) {          // X[k0 block, j] = U11^{-1} Z[k0 block, j]
      float2 col[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) col[r] = r < nb ? E[(size_t)(k0 + r) * n + j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int r = NB - 1; r >= 0; --r) {
        if (r >= nb) continue;
#pragma unroll
        for (int q = r + 1; q < NB; ++q)
          if (q < nb) col[r] = cfnmaf(col[r], sm.panel[r * LDP + q], col[q]);
        col[r] = cmulf(col[r], sm.pinv[k0 + r]);
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) {
          E[(size_t)(k0 + r) * n + j] = col[r];
          sm.rowb[r * sm.ldr + j] = col[r];
        }
    }
    __syncthreads();
    if (k0 > 0) {
      for (int t = tid; t < k0 * nb; t += NT) {     // U01 (rows above the block) into the stage
        const int r = t / nb, c = t - r * nb;
        sm.panel[r * LDP + c] = A[(size_t)r * n + k0 + c];
      }
      __syncthreads();
      // rows i < k0 need columns c <= i only
      tile_update(E, n, 0, 0, k0, k0, sm.panel, sm.rowb, sm.ldr, nb, [](int i, int j) { return j <= i; });
    }
    __syncthreads();
  }
  double dr = 0.0, di = 0.0;
  for (int c = tid; c < n; c += NT) {
    const float2 v = E[(size_t)c * n + c];
    dr += v.x;
    di += v.y;
  }
  dr = warp_sum_d(dr);
  di = warp_sum_d(di);
  if (lane == 0) sm.red[warp] = make_double2(dr, di);
  __syncthreads();

  // ------------------------------------------------------------- FP64 epilogue
  double2 expo = make_double2(0.0, 0.0);
  if (a.has_gamma) {                  // x = M^{-1} X gamma with one refinement step
    float2* x = sm.xv;
    float2* rr = sm.rv;
    for (int i = tid; i < n; i += NT) x[i] = a.Xg_hi[i];
    __syncthreads();
    cta_solve_lu(A, n, sm.pinv, x);
    // r = X gamma - M x^ by Dot2, a thread per row
    for (int i = tid; i < n; i += NT) {
      Acc2 sr = {0.0f, 0.0f}, si = {0.0f, 0.0f};
      const float2 gh = a.Xg_hi[i], gl = a.Xg_lo[i];
      acc2_add(sr, gh.x);
      acc2_add(sr, gl.x);
      acc2_add(si, gh.y);
      acc2_add(si, gl.y);
      for (int j = 0; j < n; ++j) {
        const float2 xh = a.NXA_hi[(size_t)i * n + j], xl = a.NXA_lo[(size_t)i * n + j], y = x[j];
        acc2_add_prod(sr, -xh.x, y.x);
        acc2_add_prod(sr, xh.y, y.y);
        acc2_add_prod(sr, -xl.x, y.x);
        acc2_add_prod(sr, xl.y, y.y);
        acc2_add_prod(si, -xh.x, y.y);
        acc2_add_prod(si, -xh.y, y.x);
        acc2_add_prod(si, -xl.x, y.y);
        acc2_add_prod(si, -xl.y, y.x);
      }
      const double2 d = sm.w[sm.lab[i]];
      const float dhx = (float)d.x, dhy = (float)d.y;
      const float dlx = (float)(d.x - (double)dhx), dly = (float)(d.y - (double)dhy);
      const float2 y = x[i];
      acc2_add_prod(sr, -dhx, y.x);
      acc2_add_prod(sr, -dhy, y.y);
      acc2_add_prod(si, -dhx, y.y);
      acc2_add_prod(si, dhy, y.x);
      acc2_add_prod(sr, -dlx, y.x);
      acc2_add_prod(sr, -dly, y.y);
      acc2_add_prod(si, -dlx, y.y);
      acc2_add_prod(si, dly, y.x);
      rr[i] = make_float2(acc2_value(sr), acc2_value(si));
    }
    __syncthreads();
    cta_solve_lu(A, n, sm.pinv, rr);
    double sr = 0.0, si = 0.0;
    for (int i = tid; i < n; i += NT) {
      const double xr = (double)x[i].x + (double)rr[i].x, xi = (double)x[i].y + (double)rr[i].y;
      const double gr = (double)a.g_hi[i].x + (double)a.g_lo[i].x, gi = (double)a.g_hi[i].y + (double)a.g_lo[i].y;
      sr += gr * xr - gi * xi;
      si += gr * xi + gi * xr;
    }
    sr = warp_sum_d(sr);
    si = warp_sum_d(si);
    if (lane == 0) sm.red2[warp] = make_double2(sr, si);
    __syncthreads();
    if (tid == 0)
      for (int q = 0; q < NT / 32; ++q) {
        expo.x += sm.red2[q].x;
        expo.y += sm.red2[q].y;
      }
  }
  if (warp == 0) {
    double2 ld;
    double mn;
    warp_logdet(n, sm.w, sm.lab, [&](int i) { float2 u = A[(size_t)i * n + i]; return make_double2(u.x, u.y); },
                &ld, &mn);
    if (lane == 0) {
      double2 delta = make_double2(0.0, 0.0);
      for (int q = 0; q < NT / 32; ++q) {
        delta.x += sm.red[q].x;
        delta.y += sm.red[q].y;
      }
      a.logq[e] = make_double2(0.5 * expo.x - 0.5 * (ld.x + delta.x), 0.5 * expo.y - 0.5 * (ld.y + delta.y));
      a.minpiv[e] = *sm.bad ? -1.0e300 : mn;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, CTAS_PER_SM) k_points_fp32r_blk(PointArgs a0, PointBatch batch) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (!batch.probs) {
    for (long long e = blockIdx.x; e < a0.grid.n_eval; e += gridDim.x) group_fp32r_blk(a0, e, smem);
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
    group_fp32r_blk(sa, batch.jobs[j].e0, smem);
    __syncthreads();
  }
}

size_t points_blk_smem_bytes(int n) {
  const size_t R = n > EB ? n : EB;
  return R * LDP * 8 + (size_t)NB * (R + 1) * 8 + (size_t)3 * n * 8 + 16 + (size_t)GBSBIN_MAX_L * 16 +
         (size_t)(NT / 32) * 32 + (size_t)3 * n * 4 + 16;
}

// One CTA's workspace slot: L\U (float2) and the residual (float2; the integer digits of
// the rounded factors before it), n x n each.  The workspace holds
// GBSBIN_BLK_CTAS_PER_SM slots per SM.
int points_blk_ctas_per_sm(int n) {
  // 228 KB of shared memory per SM, 1 KB of it reserved per resident CTA
  return 2 * (points_blk_smem_bytes(n) + 1024) <= 228 * 1024 ? GBSBIN_BLK_CTAS_PER_SM : 1;
}

size_t points_blk_slot_bytes(int n) { return ((size_t)16 * n * n + 255) / 256 * 256; }

cudaError_t launch_points_blk(const PointArgs& a, const PointBatch& batch, size_t smem_batch, int num_sms,
                              cudaStream_t s) {
  const size_t smem = batch.probs ? smem_batch : points_blk_smem_bytes(a.n);
  cudaError_t err = cudaFuncSetAttribute(k_points_fp32r_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_points_fp32r_blk, NT, smem);
  if (err != cudaSuccess) return err;
  per_sm = per_sm < 1 ? 1 : per_sm > GBSBIN_BLK_CTAS_PER_SM ? GBSBIN_BLK_CTAS_PER_SM : per_sm;
  long long grid = (long long)num_sms * per_sm;  // one workspace slot per CTA
  const long long work = batch.probs ? batch.njobs : a.grid.n_eval;
  if (grid > work) grid = work;
  if (grid < 1) grid = 1;
  k_points_fp32r_blk<<<(unsigned)grid, NT, smem, s>>>(a, batch);
  return cudaGetLastError();
}

}  // namespace gbsbin
