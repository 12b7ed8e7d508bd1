// Fock inputs through a lossy linear circuit (arXiv:2412.17742, App. C), binned outputs.
//
// p_j photons enter input port j of T (row = output port).  The generating function of
// the binned output counts is
//
//   G(z) = sum_b P(b) z^b = perm(B(z)[p, p]) / prod_j p_j!,   B(z) = I - T^dag (I - Z) T,
//
// Z = diag(z_label(i)): the generating function, over the output patterns, of the
// diagonal elements of App. C, Eq. probs_fock_circuit.  The permanent is the coefficient
// of x^p in Q(x) = prod_j (B(z) x)_j^{p_j}.  Q is homogeneous of degree N, so with one
// occupied input of smallest p held at x = 1 that coefficient is the mean over the nodes
// x_k = exp(2 pi i g_k / (p_k + 1)) of w(x) Q(x), w = prod_k x_k (= x^-p on the nodes):
// the finite differences of Sec. IV with their nodes on roots of unity, like the inverse
// DFT over the output groups that follows (Sec. VI).
//
// (B(z) x)_j = a_j + sum_l z_l v_j^(l), a = (I - T^dag T) x, v^(l) = T_l^dag T_l x (T_l:
// the rows of group l).  Per node the CTA tabulates v_j^(l) z_l for every root z_l of
// every group (nin x sum_l R_l entries), so at each of its output-group points a factor
// costs L additions.  The nodes are walked in reflected mixed-radix Gray order: from one
// node to the next a single coordinate moves by one root, so a and v change by one column
// of the coefficient matrices; every `chunk` nodes the state is recomputed directly.
//
// CTA = (tile of output-group points, node range): 128 threads with ZT points each (1 or 2
// for FP64, 2 or 4 for FP32 pairs, by how well the grid fills the tiles: independent
// product chains, one shared-memory read of a_j per photon); node
// restarts c = blockIdx.y, blockIdx.y + gridDim.y, ...; each point's sum over the CTA's
// nodes goes to parts[blockIdx.y][point], summed in order by the inverse DFT's first stage.
//
// Two arithmetics.  FP64 throughout (DFMA pipe).  Or pairs of FP32 (hi + lo, about 46
// bits) on the FMA pipe, which on this GPU issues ~70x more operations than the FP64 one:
// table entries are split as hi on the 2^-18 grid plus lo, so the L additions of a
// factor are exact in hi (every |partial sum| < 64) and plain FP32 in lo; products use
// Dekker's and Knuth's error-free transformations (TwoProduct by FMA, TwoSum, FastTwoSum);
// each point's running sum goes to FP64 every 32 nodes.
#include <cuda_runtime.h>

#include <type_traits>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int FT = GBSBIN_FOCK_THREADS;
constexpr int FLUSH = 32;

// ------------------------------------------------------------------ FP64 complex
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {   // c + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// (hi, lo) with hi = a rounded to a multiple of 2^-18 (|a| < 16: x + 48 lies in [32, 64),
// whose FP32 spacing is 2^-18) and lo = a - hi
__device__ __forceinline__ float4 df_split(float4 a) {
  const float C = 48.0f;
  const float hr = __fsub_rn(__fadd_rn(a.x, C), C), hi = __fsub_rn(__fadd_rn(a.y, C), C);
  return make_float4(hr, hi, __fadd_rn(__fsub_rn(a.x, hr), a.z), __fadd_rn(__fsub_rn(a.y, hi), a.w));
}
// running sum: hi by TwoSum, its errors and the lo parts gathered in lo (renormalised at
// the FP64 flush)
__device__ __forceinline__ void df_acc(float4& acc, float4 v) {
  float s, e;
  two_sum(acc.x, v.x, s, e);
  acc.x = s;
  acc.z = __fadd_rn(acc.z, __fadd_rn(e, v.z));
  two_sum(acc.y, v.y, s, e);
  acc.y = s;
  acc.w = __fadd_rn(acc.w, __fadd_rn(e, v.w));
}

template <bool DF, int ZT>
__global__ void __launch_bounds__(FT) k_fock(const FockArgs a) {
  using E = typename std::conditional<DF, float4, double2>::type;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int nin = a.nin, L = a.L, nd = a.nd, rsum = a.rsum;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nst = (L + 1) * nin;
  E* st = reinterpret_cast<E*>(fsm);             // [m * nin + j]: a (m = 0), v^(l) (m = 1 + l)
  E* ta = st + nst;                              // nin: a, as the points read it
  E* tab = ta + nin;                             // [j * rsum + roff[l] + c]: v_j^(l) z_l^c
  double2* xs = reinterpret_cast<double2*>(tab + (size_t)nin * rsum);   // nin: node at a restart
  E* ws = reinterpret_cast<E*>(xs + nin);        // weight w(x) of the current node
  const long long nfull = a.grid.n_full;

  // this thread's output-group points: their table row per group, two 16-bit rows per word
  // (rsum < 2^16: the table fits in shared memory)
  unsigned zrow[ZT][GBSBIN_FOCK_MAX_L / 2];
  bool zok[ZT];
#pragma unroll
  for (int zt = 0; zt < ZT; ++zt) {
    const long long e = ((long long)blockIdx.x * ZT + zt) * FT + tid;
    zok[zt] = e < nfull;
#pragma unroll
    for (int l2 = 0; l2 < GBSBIN_FOCK_MAX_L / 2; ++l2) {
      const int l0 = 2 * l2, l1 = 2 * l2 + 1;
      const unsigned r0 = (zok[zt] && l0 < L) ? (unsigned)(a.roff[l0] + point_digit(e, a.grid, l0)) : 0u;
      const unsigned r1 = (zok[zt] && l1 < L) ? (unsigned)(a.roff[l1] + point_digit(e, a.grid, l1)) : 0u;
      zrow[zt][l2] = r0 | (r1 << 16);
    }
  }
  double2 acc[ZT];
  float4 accd[ZT];
#pragma unroll
  for (int zt = 0; zt < ZT; ++zt) {
    acc[zt] = make_double2(0.0, 0.0);
    accd[zt] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  E w;                                           // thread 0's copy of the node weight
  int since_flush = 0;

  for (long long c = blockIdx.y; c < a.nchunks; c += gridDim.y) {
    const long long i0 = a.x_lo + c * a.chunk;
    const long long i1 = i0 + a.chunk < a.x_hi ? i0 + a.chunk : a.x_hi;
    // digit lane d (< nd) of every warp: ordinary digit n, Gray digit g, direction
    int R = 1, n = 0, g = 0, dir = 1;
    if (lane < nd) {
      R = a.drad[lane];
      const long long q = i0 / a.dstride[lane];
      n = (int)(q % R);
      dir = ((q / R) & 1) ? -1 : 1;
      g = dir > 0 ? n : R - 1 - n;
    }
    if (tid < 32) {                              // node coordinates: position k <- digit k - 1
      const int gk = __shfl_sync(0xffffffffu, g, (lane + 31) & 31);
      if (lane < nin) xs[lane] = lane == 0 ? make_double2(1.0, 0.0) : a.xtw[a.doff[lane - 1] + gk];
    }
    __syncthreads();
    for (int idx = tid; idx < nst; idx += FT) {  // direct state, FP64
      const int m = idx / nin, j = idx - m * nin;
      const double2* col = a.coef + (size_t)m * nin * nin + j;
      double2 s = make_double2(0.0, 0.0);
      for (int k = 0; k < nin; ++k) s = zfma(col[(size_t)k * nin], xs[k], s);
      if constexpr (DF) st[idx] = df_from(s);
      else st[idx] = s;
    }
    if (tid == 0) {
      double2 w64 = make_double2(1.0, 0.0);
      for (int k = 1; k < nin; ++k) w64 = zmul(w64, xs[k]);
      if constexpr (DF) w = df_from(w64);
      else w = w64;
    }

    for (long long i = i0; i < i1; ++i) {
      __syncthreads();                           // state of node i written; tab free
      for (int idx = tid; idx < nin * (rsum + 1); idx += FT) {
        const int j = idx / (rsum + 1), r = idx - j * (rsum + 1);
        if (r == rsum) {
          if constexpr (DF) ta[j] = df_split(st[j]);
          else ta[j] = st[j];
        } else {
          int l = 0;
          while (r >= a.roff[l + 1]) ++l;
          if constexpr (DF) tab[j * rsum + r] = df_split(df_mul(st[(1 + l) * nin + j], a.zr_df[r]));
          else tab[j * rsum + r] = zmul(st[(1 + l) * nin + j], a.zr[r]);
        }
      }
      if (tid == 0) *ws = w;
      __syncthreads();                           // table of node i complete

      // points: photon by photon, the thread's ZT products side by side (independent
      // chains); a point off the grid computes on row 0 and is not accumulated
      E F[ZT];
#pragma unroll
      for (int zt = 0; zt < ZT; ++zt) F[zt] = *ws;
      for (int j = 0; j < nin; ++j) {
        const E* row = tab + j * rsum;
        const E aj = ta[j];
        E s[ZT];
#pragma unroll
        for (int zt = 0; zt < ZT; ++zt) {
          s[zt] = aj;
#pragma unroll
          for (int l = 0; l < GBSBIN_FOCK_MAX_L; ++l) {
            if (l >= L) break;
            const E t = row[(zrow[zt][l >> 1] >> ((l & 1) * 16)) & 0xffffu];
            if constexpr (DF) {                  // hi parts exact, lo parts plain
              s[zt].x = __fadd_rn(s[zt].x, t.x);
              s[zt].y = __fadd_rn(s[zt].y, t.y);
              s[zt].z = __fadd_rn(s[zt].z, t.z);
              s[zt].w = __fadd_rn(s[zt].w, t.w);
            } else {
              s[zt] = zadd(s[zt], t);
            }
          }
          if constexpr (DF) {                    // renormalise (TwoSum: lo may exceed hi)
            float4 u;
            two_sum(s[zt].x, s[zt].z, u.x, u.z);
            two_sum(s[zt].y, s[zt].w, u.y, u.w);
            s[zt] = u;
          }
        }
        const int pj = a.pw[j];
        for (int rep = 0; rep < pj; ++rep) {
#pragma unroll
          for (int zt = 0; zt < ZT; ++zt) {
            if constexpr (DF) F[zt] = df_mul(F[zt], s[zt]);
            else F[zt] = zmul(F[zt], s[zt]);
          }
        }
      }
#pragma unroll
      for (int zt = 0; zt < ZT; ++zt) {
        if (!zok[zt]) continue;
        if constexpr (DF) df_acc(accd[zt], F[zt]);
        else acc[zt] = zadd(acc[zt], F[zt]);
      }
      if constexpr (DF) {
        if (++since_flush == FLUSH) {
          since_flush = 0;
#pragma unroll
          for (int zt = 0; zt < ZT; ++zt) {
            acc[zt] = zadd(acc[zt], df_to(accd[zt]));
            accd[zt] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }

      if (i + 1 < i1) {                          // next node: the lowest digit not at its end moves
        const unsigned adv = __ballot_sync(0xffffffffu, lane < nd && n != R - 1);
        const int ds = __ffs(adv) - 1;
        int gnew = g;
        const int gold = g;
        if (lane < ds) {
          n = 0;
          dir = -dir;
        } else if (lane == ds) {
          ++n;
          gnew = g + dir;
          g = gnew;
        }
        const int go = __shfl_sync(0xffffffffu, gold, ds);
        const int gn = __shfl_sync(0xffffffffu, gnew, ds);
        const int k = ds + 1;                    // position of the moved input
        if constexpr (DF) {
          const float4 xo = a.xtw_df[a.doff[ds] + go], xn = a.xtw_df[a.doff[ds] + gn];
          const float4 dx = df_add(xn, make_float4(-xo.x, -xo.y, -xo.z, -xo.w));
          for (int idx = tid; idx < nst; idx += FT) {
            const int m = idx / nin, j = idx - m * nin;
            st[idx] = df_add(st[idx], df_mul(a.coef_df[((size_t)m * nin + k) * nin + j], dx));
          }
          if (tid == 0) w = df_mul(w, df_mul(xn, df_conj(xo)));
        } else {
          const double2 xo = a.xtw[a.doff[ds] + go], xn = a.xtw[a.doff[ds] + gn];
          const double2 dx = make_double2(xn.x - xo.x, xn.y - xo.y);
          for (int idx = tid; idx < nst; idx += FT) {
            const int m = idx / nin, j = idx - m * nin;
            st[idx] = zfma(a.coef[((size_t)m * nin + k) * nin + j], dx, st[idx]);
          }
          if (tid == 0) w = zmul(w, zmul(xn, make_double2(xo.x, -xo.y)));
        }
      }
    }
    __syncthreads();                             // the last node's points are done with xs/st
  }
#pragma unroll
  for (int zt = 0; zt < ZT; ++zt) {
    if (!zok[zt]) continue;
    double2 v = acc[zt];
    if constexpr (DF) v = zadd(v, df_to(accd[zt]));
    const long long e = ((long long)blockIdx.x * ZT + zt) * FT + tid;
    a.parts[(long long)blockIdx.y * nfull + e] = v;
  }
}

template <bool DF, int ZT>
cudaError_t launch_one(const FockArgs& a, size_t smem, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(k_fock<DF, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const long long per = (long long)FT * ZT;
  const long long tiles = (a.grid.n_full + per - 1) / per;
  k_fock<DF, ZT><<<dim3((unsigned)tiles, (unsigned)a.xr), FT, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool DF, int ZT>
int ctas_one(size_t smem) {
  if (cudaFuncSetAttribute(k_fock<DF, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fock<DF, ZT>, FT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

}  // namespace

int fock_points_per_thread(bool df, long long n_full) {
  // the larger count gives more independent chains and shares each node's table among more
  // points; the smaller one wastes fewer slots of a CTA's last tile on small grids
  const int small = df ? 2 : 1, big = 2 * small;
  const double per = (double)FT;
  const double eff_small = (double)n_full / (per * small * (double)((n_full + FT * small - 1) / (FT * small)));
  const double eff_big = (double)n_full / (per * big * (double)((n_full + FT * big - 1) / (FT * big)));
  return eff_big >= 0.9 * eff_small ? big : small;
}

size_t fock_smem_bytes(int nin, int L, int rsum) {
  return 16 * ((size_t)(L + 3) * nin + (size_t)nin * rsum + 1);
}

int fock_ctas_per_sm(bool df, int zt, size_t smem) {
  if (df) return zt == 4 ? ctas_one<true, 4>(smem) : ctas_one<true, 2>(smem);
  return zt == 2 ? ctas_one<false, 2>(smem) : ctas_one<false, 1>(smem);
}

cudaError_t launch_fock(const FockArgs& a, bool df, int zt, cudaStream_t s) {
  const size_t smem = fock_smem_bytes(a.nin, a.L, a.rsum);
  if (df) return zt == 4 ? launch_one<true, 4>(a, smem, s) : launch_one<true, 2>(a, smem, s);
  return zt == 2 ? launch_one<false, 2>(a, smem, s) : launch_one<false, 1>(a, smem, s);
}

}  // namespace gbsbin
