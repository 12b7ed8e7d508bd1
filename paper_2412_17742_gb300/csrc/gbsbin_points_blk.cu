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
//             sum_c X[c][c]; the rank-32 updates of both substitutions run either on the
//             CUDA cores (register tiles, the default) or, in the tensor-core variant, on
//             the tensor cores (tcgen05, 3 x TF32, TMEM accumulator): they only feed the
//             correction delta, which needs ~1e-6 relative accuracy, while the LU's own
//             updates stay in exact FP32 on the CUDA cores (its rounding sets the
//             refinement's remainder);
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

// Bytes of the tensor-core operand stage (A hi/lo 128 x 64 and B hi/lo 64 x 64, FP32) and
// of the region at the start of shared memory that holds either it or panel + rowb.
constexpr int TC_STAGE_BYTES = (2 * 128 * 64 + 2 * 64 * 64) * 4;
__host__ __device__ __forceinline__ size_t region0_bytes(int n) {
  const size_t R = n > EB ? n : EB;
  const size_t pr = R * LDP * 8 + (size_t)NB * (R + 1) * 8;
  const size_t tc = (size_t)TC_STAGE_BYTES + 128;
  return pr > tc ? pr : tc;
}

__device__ __forceinline__ BlkSmem carve(unsigned char* smem, int n, int L) {
  BlkSmem s;
  const int R = n > EB ? n : EB;        // the residual pass stages EB-row chunks
  float2* f = (float2*)smem;
  s.panel = f;
  f += (size_t)R * LDP;
  s.ldr = R + 1;
  s.rowb = f;
  f = (float2*)(smem + region0_bytes(n));
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


// ------------------------------------------------------------ tensor cores (tcgen05)
// C -= A B for complex A (nr x kd), B (kd x nc), kd <= 32, on the 5th-generation tensor
// cores: realified to a real GEMM with K = 64 (A row i = [Re A_i., Im A_i.]; output column
// 2c from B column [Re B_.c, -Im B_.c], 2c + 1 from [Im B_.c, Re B_.c]), each operand split
// into hi + lo TF32 parts and the three products hi.hi + hi.lo + lo.hi accumulated in FP32 in
// tensor memory (about 2^-21 relative).  Tiles: 128 rows x 64 real columns, operands staged
// in shared memory in the K-major no-swizzle layout (8-row x 16-byte core matrices; 128 B
// between cores along K, 2048 B between 8-row groups), one thread issues the MMAs and
// commits them to an mbarrier that all threads wait on (bounded), tcgen05.ld brings the tile
// back (warp w reads TMEM lanes 32 (w mod 4) .. + 31, column half w / 4).
struct TcCtx {
  uint32_t tmem;        // base of this CTA's 64 TMEM columns
  uint32_t mbar;        // shared address of the completion mbarrier
  uint32_t phase;       // parity of the next completion
  float* stage;         // TC_STAGE_BYTES of shared memory, 128-byte aligned
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr) {   // LBO 128 B, SBO 2048 B, no swizzle
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
  hi = __uint_as_float(h);
  lo = v - hi;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
    if (done) return true;
  }
  return false;
}

// C[i * ldc + j] -= sum_k Ag[i * lda + k] Bg[k * ldb + j], i < nr, j < nc, k < kd <= 32.
// Called by the whole CTA; returns false if a completion wait gave up.
__device__ bool tc_sub_gemm(float2* C, int ldc, int nr, int nc, const float2* Ag, int lda, const float2* Bg, int ldb,
                            int kd, TcCtx& tc) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* Ahi = tc.stage;
  float* Alo = Ahi + 128 * 64;
  float* Bhi = Alo + 128 * 64;
  float* Blo = Bhi + 64 * 64;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  bool ok = true;
  for (int i0 = 0; i0 < nr; i0 += 128) {
    // A tile: complex element (r, k) -> real (r, k) = Re, (r, k + 32) = Im.  A warp takes one
    // 8 x 4 block of complex elements (eight 32-byte row segments), so its stores fill whole
    // 128-byte core matrices; every thread issues its 16 loads before any store.
    {
      float2 v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + NT * q, cc = e >> 5, w = e & 31;
        const int r = (cc >> 3) * 8 + (w >> 2), k = (cc & 7) * 4 + (w & 3);
        v[q] = (i0 + r < nr && k < kd) ? Ag[(size_t)(i0 + r) * lda + k] : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + NT * q, cc = e >> 5, w = e & 31;
        const int fre = (((cc >> 3) * 16 + (cc & 7)) << 5) + w;   // float index of (r, k)
        tf32_split(v[q].x, Ahi[fre], Alo[fre]);
        tf32_split(v[q].y, Ahi[fre + 8 * 32], Alo[fre + 8 * 32]);  // (r, k + 32): 8 cores on
      }
    }
    for (int j0 = 0; j0 < 2 * nc; j0 += 64) {
      // B tile (real rows jr = 2c' + part of the 32 complex columns c' of this tile):
      // B(k, c) -> (2c', k) = Re, (2c', k + 32) = -Im, (2c' + 1, k) = Im, (2c' + 1, k + 32) = Re.
      // A warp takes 8 k x 4 columns; loads first, then stores.
      {
        float2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + NT * q, grp = e >> 5, w = e & 31;
          const int cp = (grp & 7) * 4 + (w >> 3), k = (grp >> 3) * 8 + (w & 7), c = (j0 >> 1) + cp;
          v[q] = (c < nc && k < kd) ? Bg[(size_t)k * ldb + c] : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + NT * q, grp = e >> 5, w = e & 31;
          const int cp = (grp & 7) * 4 + (w >> 3), k = (grp >> 3) * 8 + (w & 7);
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const int jr = 2 * cp + part;
            const int f0 = (((jr >> 3) * 16 + (k >> 2)) << 5) + ((jr & 7) << 2) + (k & 3);   // (jr, k)
            const float lo_k = part ? v[q].y : v[q].x;        // K index k
            const float hi_k = part ? v[q].x : -v[q].y;       // K index k + 32
            tf32_split(lo_k, Bhi[f0], Blo[f0]);
            tf32_split(hi_k, Bhi[f0 + 8 * 32], Blo[f0 + 8 * 32]);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        const float* As[3] = {Ahi, Ahi, Alo};
        const float* Bs[3] = {Bhi, Blo, Bhi};
        uint32_t acc = 0;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int ks = 0; ks < 8; ++ks) {        // K = 8 per instruction: two cores along K
            const uint64_t da = kmajor_desc(smem_u32(As[p]) + ks * 256);
            const uint64_t db = kmajor_desc(smem_u32(Bs[p]) + ks * 256);
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tc.tmem),
                         "l"(da), "l"(db), "r"(idesc), "r"(acc));
            acc = 1;
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc.mbar)
                     : "memory");
      }
      ok &= mbar_wait(tc.mbar, tc.phase);
      tc.phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = i0 + 32 * (warp & 3) + lane;
      const int cbase = (j0 >> 1) + (warp >> 2) * 16;   // complex column of this warp's half
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r[16];
        const uint32_t ta = tc.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 32 + 16 * h);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                       "=r"(r[15])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < nr) {
          float2* crow = C + (size_t)row * ldc + cbase + 8 * h;
          const int nv = min(8, nc - (cbase + 8 * h));
          float2 cv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) cv[q] = q < nv ? crow[q] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < nv) crow[q] = make_float2(cv[q].x - __uint_as_float(r[2 * q]), cv[q].y - __uint_as_float(r[2 * q + 1]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  return ok;
}

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

template <bool TC>
__device__ void group_fp32r_blk(const PointArgs& a, const long long e, unsigned char* smem, TcCtx& tc) {
  const int n = a.n, L = a.grid.L, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  BlkSmem sm = carve(smem, n, L);
  float2* A = (float2*)((char*)a.gws + (size_t)blockIdx.x * (size_t)a.gws_slot_bytes);
  float2* E = A + (size_t)n * n;
  for (int i = tid; i < n; i += NT) sm.lab[i] = a.label[i];
  if (tid < L) sm.w[tid] = grid_root(a.tw, a.grid, tid, point_digit(e, a.grid, tid));
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
    // panel LU in two steps with two CTA barriers instead of two per column: warp 0
    // factorizes the nb x nb diagonal block (lane i owns row i, warp syncs only), then each
    // thread takes one row i below it and solves l_ik = (a_ik - sum_{q<k} l_iq u_qk) / u_kk
    // in registers against U11 (the same elimination, left-looking for L21)
    if (warp == 0) {
      for (int kk = 0; kk < nb; ++kk) {
        const float2 inv = crecipf(sm.panel[kk * LDP + kk]);
        if (lane == 0) sm.pinv[k0 + kk] = inv;
        if (lane > kk && lane < nb) {
          const float2 l = cmulf(sm.panel[lane * LDP + kk], inv);
          sm.panel[lane * LDP + kk] = l;
          for (int c = kk + 1; c < nb; ++c)
            sm.panel[lane * LDP + c] = cfnmaf(sm.panel[lane * LDP + c], l, sm.panel[kk * LDP + c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = nb + tid; i < rows; i += NT) {
      float2 row[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) row[c] = c < nb ? sm.panel[i * LDP + c] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k >= nb) continue;
        float2 acc = row[k];
#pragma unroll
        for (int q = 0; q < k; ++q) acc = cfnmaf(acc, row[q], sm.panel[q * LDP + k]);
        row[k] = cmulf(acc, sm.pinv[k0 + k]);
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nb) sm.panel[i * LDP + c] = row[c];
    }
    __syncthreads();
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
          // the stages hold zero digits off the factors' triangles (L_ik needs k < i, U_kj
          // needs k <= j), so the multiply-add loop below needs no masks
          for (int t = tid; t < EB * NB; t += NT) {
            const int r = t / NB, c = t - r * NB;
            Ls[r * LDP + c] = (r < ni && c < kd && kc + c < i0 + r) ? Q[(size_t)(i0 + r) * n + kc + c] : make_int2(0, 0);
          }
          for (int t = tid; t < NB * EBJ; t += NT) {
            const int rr = t / EBJ, cc = t - rr * EBJ;
            Us[rr * sm.ldr + cc] =
                (rr < kd && cc < nj && kc + rr <= j0 + cc) ? Q[(size_t)(kc + rr) * n + j0 + cc] : make_int2(0, 0);
          }
          __syncthreads();
#pragma unroll 2
          for (int k = 0; k < kd; ++k) {
            int lx[4], ly[4], ls[4], ux[2], uy[2], us[2];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int2 v = Ls[(ti + p) * LDP + k];
              lx[p] = v.x;
              ly[p] = v.y;
              ls[p] = lx[p] + ly[p];
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int2 v = Us[k * sm.ldr + tj + 16 * q];
              ux[q] = v.x;
              uy[q] = v.y;
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
    if (m > 0) {                                   // E[rows below] -= L21 Z1
      if constexpr (TC) {
        const bool ok = tc_sub_gemm(E + (size_t)(k0 + nb) * n, n, m, n, A + (size_t)(k0 + nb) * n + k0, n,
                                    E + (size_t)k0 * n, n, nb, tc);
        if (!ok) *sm.bad = 1;
      } else {
        for (int t = tid; t < m * nb; t += NT) {   // L21 into the panel stage
          const int r = t / nb, c = t - r * nb;
          sm.panel[r * LDP + c] = A[(size_t)(k0 + nb + r) * n + k0 + c];
        }
        __syncthreads();
        tile_update(E, n, k0 + nb, 0, m, n, sm.panel, sm.rowb, sm.ldr, nb, NoMask());
      }
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
        // q descending: the terms of the longest-finished unknowns first, so the chain of
        // col[r] does not start on col[r + 1], which was finished just before
#pragma unroll
        for (int q = NB - 1; q > r; --q)
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
    if (k0 > 0) {                                   // E[rows above][c < k0] -= U01 X1
      if constexpr (TC) {
        // only the entries c <= row are needed (the others are never read): the tensor
        // cores update the whole square
        const bool ok = tc_sub_gemm(E, n, k0, k0, A + k0, n, E + (size_t)k0 * n, n, nb, tc);
        if (!ok) *sm.bad = 1;
      } else {
        for (int t = tid; t < k0 * nb; t += NT) {   // U01 (rows above the block) into the stage
          const int r = t / nb, c = t - r * nb;
          sm.panel[r * LDP + c] = A[(size_t)r * n + k0 + c];
        }
        __syncthreads();
        tile_update(E, n, 0, 0, k0, k0, sm.panel, sm.rowb, sm.ldr, nb, [](int i, int j) { return j <= i; });
      }
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
    // r = X gamma - M x^ by Dot2, a thread per row; four independent accumulator pairs over
    // interleaved j keep the dependent chains a quarter as long
    for (int i = tid; i < n; i += NT) {
      Acc2 ar[4], ai[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ar[u] = ai[u] = Acc2{0.0f, 0.0f};
      for (int j0 = 0; j0 < n; j0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          if (j < n) {
            const float2 xh = a.NXA_hi[(size_t)i * n + j], xl = a.NXA_lo[(size_t)i * n + j], y = x[j];
            acc2_add_prod(ar[u], -xh.x, y.x);
            acc2_add_prod(ar[u], xh.y, y.y);
            acc2_add_prod(ar[u], -xl.x, y.x);
            acc2_add_prod(ar[u], xl.y, y.y);
            acc2_add_prod(ai[u], -xh.x, y.y);
            acc2_add_prod(ai[u], -xh.y, y.x);
            acc2_add_prod(ai[u], -xl.x, y.y);
            acc2_add_prod(ai[u], -xl.y, y.x);
          }
        }
      }
      // combine the pairs (each partial sum s + c exactly as accumulated)
      Acc2 sr = ar[0], si = ai[0];
#pragma unroll
      for (int u = 1; u < 4; ++u) {
        acc2_add(sr, ar[u].s);
        sr.c += ar[u].c;
        acc2_add(si, ai[u].s);
        si.c += ai[u].c;
      }
      const float2 gh = a.Xg_hi[i], gl = a.Xg_lo[i];
      acc2_add(sr, gh.x);
      acc2_add(sr, gl.x);
      acc2_add(si, gh.y);
      acc2_add(si, gl.y);
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

template <bool TC>
__global__ void __launch_bounds__(NT, CTAS_PER_SM) k_points_fp32r_blk(PointArgs a0, PointBatch batch) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  TcCtx tc{0u, 0u, 0u, nullptr};
  if constexpr (TC) {
    // 64 columns of tensor memory for the accumulator and the completion mbarrier, per CTA;
    // the allocation permit is given up at once so that the SM's other CTA can allocate too
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&s_tmem)));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc = TcCtx{s_tmem, smem_u32(&s_mbar), 0u, (float*)(((uintptr_t)smem + 127) & ~(uintptr_t)127)};
  }
  if (!batch.probs) {
    for (long long e = blockIdx.x; e < a0.grid.n_eval; e += gridDim.x) group_fp32r_blk<TC>(a0, e, smem, tc);
  } else {
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
      group_fp32r_blk<TC>(sa, batch.jobs[j].e0, smem, tc);
      __syncthreads();
    }
  }
  if constexpr (TC) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(s_tmem));
  }
}

size_t points_blk_smem_bytes(int n) {
  return region0_bytes(n) + (size_t)3 * n * 8 + 16 + (size_t)GBSBIN_MAX_L * 16 + (size_t)(NT / 32) * 32 +
         (size_t)3 * n * 4 + 16;
}

// One CTA's workspace slot: L\U (float2) and the residual (float2; the integer digits of
// the rounded factors before it), n x n each.  The workspace holds
// GBSBIN_BLK_CTAS_PER_SM slots per SM.
// Resident CTAs per SM for a dynamic shared-memory size: 228 KB per SM, 1 KB reserved per
// CTA, ~1 KB of static shared memory; registers allow two (__launch_bounds__(256, 2)), and
// two CTAs hold 2 x 64 of the 512 TMEM columns.  (The occupancy calculator answers 1 for
// any kernel with tcgen05 instructions, so it is not used here; measured on GB300: two such
// CTAs per SM, each holding TMEM after relinquishing the allocation permit, run together.)
static int blk_ctas_for_smem(size_t smem) {
  return 2 * (smem + 2048) <= 228 * 1024 ? GBSBIN_BLK_CTAS_PER_SM : 1;
}

int points_blk_ctas_per_sm(int n) { return blk_ctas_for_smem(points_blk_smem_bytes(n)); }

size_t points_blk_slot_bytes(int n) { return ((size_t)16 * n * n + 255) / 256 * 256; }

cudaError_t launch_points_blk(const PointArgs& a, const PointBatch& batch, size_t smem_batch, int num_sms,
                              cudaStream_t s, bool tensor_cores) {
  const size_t smem = batch.probs ? smem_batch : points_blk_smem_bytes(a.n);
  const void* fn = tensor_cores ? (const void*)k_points_fp32r_blk<true> : (const void*)k_points_fp32r_blk<false>;
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int per_sm = blk_ctas_for_smem(smem);
  long long grid = (long long)num_sms * per_sm;  // one workspace slot per CTA
  const long long work = batch.probs ? batch.njobs : a.grid.n_eval;
  if (grid > work) grid = work;
  if (grid < 1) grid = 1;
  if (tensor_cores)
    k_points_fp32r_blk<true><<<(unsigned)grid, NT, smem, s>>>(a, batch);
  else
    k_points_fp32r_blk<false><<<(unsigned)grid, NT, smem, s>>>(a, batch);
  return cudaGetLastError();
}

}  // namespace gbsbin
