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
//   residual  E = M - L^U^ by Dot2 over 64 x 64 output blocks, L/U chunks staged;
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
constexpr int EB = 64;                  // residual output block

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
  int* lab;        // n
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
  s.lab = (int*)(s.red + NT / 32);
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

  // ------------------------------------------- residual E = M - L^U^ by Dot2
  // (uses panel / rowb as the L and U chunk stages: L chunk EB x NB, U chunk NB x EB)
  const int nblk = (n + EB - 1) / EB;
  for (int bi = 0; bi < nblk; ++bi)
    for (int bj = 0; bj < nblk; ++bj) {
      const int i0 = bi * EB, j0 = bj * EB;
      const int ni = min(EB, n - i0), nj = min(EB, n - j0);
      // this thread's 4 x 4 entries of the 64 x 64 block: rows ti .. ti+3, columns tj + 16 q
      const int ti = (tid >> 4) * 4, tj = tid & 15;
      Acc2 er[4][4], ei[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          er[p][q] = Acc2{0.0f, 0.0f};
          ei[p][q] = Acc2{0.0f, 0.0f};
        }
      const int kmax = min(i0 + ni, j0 + nj);   // terms need k < i and k <= j
      for (int kc = 0; kc < kmax; kc += NB) {
        const int kd = min(NB, kmax - kc);
        __syncthreads();
        for (int t = tid; t < EB * NB; t += NT) {
          const int r = t / NB, c = t - r * NB;
          sm.panel[r * LDP + c] = (r < ni && c < kd) ? A[(size_t)(i0 + r) * n + kc + c] : make_float2(0.f, 0.f);
          const int rr = t / EB, cc = t - rr * EB;
          sm.rowb[rr * sm.ldr + cc] = (rr < kd && cc < nj) ? A[(size_t)(kc + rr) * n + j0 + cc] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int k = 0; k < kd; ++k) {
          const int kg = kc + k;
          float2 l[4], u[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float2 v = sm.panel[(ti + p) * LDP + k];
            const bool ok = kg < i0 + ti + p;    // k < i: L_ik is a multiplier
            l[p] = ok ? make_float2(-v.x, v.y) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 v = sm.rowb[k * sm.ldr + tj + 16 * q];
            const bool ok = kg <= j0 + tj + 16 * q;   // k <= j: U_kj is in the upper factor
            u[q] = ok ? v : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc2_add_prod(er[p][q], l[p].x, u[q].x);
              acc2_add_prod(er[p][q], l[p].y, u[q].y);
              acc2_add_prod(ei[p][q], l[p].x, u[q].y);
              acc2_add_prod(ei[p][q], -l[p].y, u[q].x);
            }
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + ti + p, j = j0 + tj + 16 * q;
          if (ti + p >= ni || tj + 16 * q >= nj) continue;
          const size_t ij = (size_t)i * n + j;
          if (i <= j) {                      // L_ii U_ij = U_ij
            const float2 u = A[ij];
            acc2_add(er[p][q], -u.x);
            acc2_add(ei[p][q], -u.y);
          }
          const float2 xh = a.NXA_hi[ij], xl = a.NXA_lo[ij];
          acc2_add(er[p][q], xh.x);
          acc2_add(er[p][q], xl.x);
          acc2_add(ei[p][q], xh.y);
          acc2_add(ei[p][q], xl.y);
          if (i == j) {
            const double2 d = sm.w[sm.lab[i]];
            const float dhx = (float)d.x, dhy = (float)d.y;
            acc2_add(er[p][q], dhx);
            acc2_add(er[p][q], (float)(d.x - (double)dhx));
            acc2_add(ei[p][q], -dhy);
            acc2_add(ei[p][q], -(float)(d.y - (double)dhy));
          }
          E[ij] = make_float2(acc2_value(er[p][q]), acc2_value(ei[p][q]));
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
  if (warp == 0) {
    double2 ld;
    double mn;
    warp_logdet(n, sm.w, sm.lab, [&](int i) { float2 u = A[(size_t)i * n + i]; return make_double2(u.x, u.y); },
                &ld, &mn);
    double2 expo = make_double2(0.0, 0.0);
    if (a.has_gamma) {
      float2* x = sm.xv;
      float2* rr = sm.rv;
      for (int i = lane; i < n; i += 32) x[i] = a.Xg_hi[i];
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        float2* v = pass == 0 ? x : rr;
        for (int k = 0; k < n - 1; ++k) {
          const float2 yk = v[k];
          __syncwarp();
          for (int i = k + 1 + lane; i < n; i += 32) v[i] = cfnmaf(v[i], A[(size_t)i * n + k], yk);
          __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
          const float2 xk = cmulf(v[k], sm.pinv[k]);
          __syncwarp();
          if (lane == 0) v[k] = xk;
          for (int i = lane; i < k; i += 32) v[i] = cfnmaf(v[i], A[(size_t)i * n + k], xk);
          __syncwarp();
        }
        if (pass == 0) {
          for (int i = lane; i < n; i += 32) {
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
          __syncwarp();
        }
      }
      double sr = 0.0, si = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double xr = (double)x[i].x + (double)rr[i].x, xi = (double)x[i].y + (double)rr[i].y;
        const double gr = (double)a.g_hi[i].x + (double)a.g_lo[i].x, gi = (double)a.g_hi[i].y + (double)a.g_lo[i].y;
        sr += gr * xr - gi * xi;
        si += gr * xi + gi * xr;
      }
      expo = make_double2(warp_sum_d(sr), warp_sum_d(si));
    }
    if (lane == 0) {
      double2 delta = make_double2(0.0, 0.0);
      for (int q = 0; q < NT / 32; ++q) {
        delta.x += sm.red[q].x;
        delta.y += sm.red[q].y;
      }
      a.logq[e] = make_double2(0.5 * expo.x - 0.5 * (ld.x + delta.x), 0.5 * expo.y - 0.5 * (ld.y + delta.y));
      a.minpiv[e] = mn;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) k_points_fp32r_blk(PointArgs a0, PointBatch batch) {
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
         (size_t)(NT / 32) * 16 + (size_t)n * 4 + 16;
}

cudaError_t launch_points_blk(const PointArgs& a, const PointBatch& batch, size_t smem_batch, int num_sms,
                              cudaStream_t s) {
  const size_t smem = batch.probs ? smem_batch : points_blk_smem_bytes(a.n);
  cudaError_t err = cudaFuncSetAttribute(k_points_fp32r_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  long long grid = num_sms;  // one workspace slot per CTA
  const long long work = batch.probs ? batch.njobs : a.grid.n_eval;
  if (grid > work) grid = work;
  if (grid < 1) grid = 1;
  k_points_fp32r_blk<<<(unsigned)grid, NT, smem, s>>>(a, batch);
  return cudaGetLastError();
}

}  // namespace gbsbin
