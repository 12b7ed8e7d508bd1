// One detector group (arXiv:2412.17742, Sec. VIII, total photon-number distribution;
// Sec. III Eq. q_d with a single group): D(w) = w I, so
//
//   K(w) = I - w XA = Q (I - w H) Q^H,   XA = Q H Q^H with H upper Hessenberg,
//
// and det K(w) = det(I - w H).  The host reduces XA once per state; per grid point the
// unpivoted LU of the Hessenberg matrix B = I - w H costs O(n^2): each elimination step
// subtracts a multiple of the current pivot row from the next row only.  Since
// B = -w (H - conj(w) I), the steps run on H - conj(w) I (no multiplication per entry) and
// the pivots of B are -w times its pivots; every pivot of B has Re > 0 (||w H|| =
// ||XA|| < 1, so B has a positive-definite Hermitian part, as do its Schur complements), so
// sum_i Log p_i is the branch of log det K continuous from w = 0.
//
// Displacement: the exponent gamma^T (conj(w) - XA)^{-1} X gamma = -a^T N^{-1} c with
// N = H - conj(w) I, a = Q^T gamma, c = Q^H X gamma (reflectors applied on the host).  With
// N = L_N U_N from the same sweep, y = L_N^{-1} c is a scalar recurrence (L_N is bidiagonal:
// y_{i+1} = c_{i+1} - l_i y_i) and z^T = a^T U_N^{-1} follows row by row as the rows of U_N
// appear (z_i = (a_i - s_i) / u_ii, then s_j += z_i u_ij for j > i), so a^T N^{-1} c =
// sum_i z_i y_i needs no stored factors.
//
// One warp per point: lane t holds entries j = lane + 32 s of the current pivot row (and of
// the running sums s) in registers (s < 16, n <= 512); row i + 1 of H - conj(w) I is read
// from the L2-resident H.  log q = 1/2 gamma^T x - 1/2 log det K is left unfinished as
// (product of pivots with its power of two, FP32 sum of their arguments, the rest), finished
// one point per thread by the DFT's first stage.  The arithmetic class Ar is FP64 (kernel 8)
// or pairs of FP32 on the FMA pipe (kernel 16, with H, a and c stored as pairs; the pivot
// product renormalised every four pivots to stay in FP32's exponent range).
#include <cuda_runtime.h>

#include <type_traits>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int HW = 4;                         // warps (points) per CTA
constexpr int SMAX = GBSBIN_MAX_N / 32;       // row slots per lane

template <class Ar, bool DISP>
__device__ void hess_point(const PointArgs& a, long long e) {
  using E = typename Ar::E;
  const int n = a.n, lane = threadIdx.x & 31;
  const int S = (n + 31) >> 5;
  const double2 wd = grid_root(a.tw, a.grid, 0, point_digit(e, a.grid, 0));
  const E sg = Ar::from(make_double2(wd.x, -wd.y));             // conj(w)
  const E mw = Ar::from(make_double2(-wd.x, -wd.y));            // pivots of B = -w x pivots here
  const E* H = reinterpret_cast<const E*>(a.H);
  const E* av = H + (size_t)n * n;              // a = Q^T gamma
  const E* cv = av + n;                         // c = Q^H X gamma
  // row 0 of H - conj(w) I (the running sums only for displaced states)
  E r[SMAX], sacc[DISP ? SMAX : 1];
#pragma unroll
  for (int s = 0; s < SMAX; ++s) {
    const int j = lane + 32 * s;
    E v = Ar::zero();
    if (s < S && j < n) {
      v = H[j];
      if (j == 0) v = Ar::add(v, Ar::neg(sg));
    }
    r[s] = v;
    if constexpr (DISP) sacc[s] = Ar::zero();
  }
  E y = DISP ? cv[0] : Ar::zero();
  E zy = Ar::zero();                            // sum_i z_i y_i
  E prod = Ar::one();
  int e2 = 0;
  float args = 0.0f;
  constexpr bool f64 = std::is_same<Ar, ArF64>::value;
  using MinT = typename std::conditional<f64, double, float>::type;
  MinT mn = f64 ? (MinT)1.0e300 : (MinT)3.0e38f;   // FP64 plans: the exact pivot; pairs: its hi part
  bool bad = false;
#pragma unroll
  for (int sb = 0; sb < SMAX; ++sb) {           // pivot i = 32 sb + il sits in slot sb of lane il
    if (sb >= S) break;
    for (int il = 0; il < 32; ++il) {
      const int i = 32 * sb + il;
      if (i >= n) break;
      const E q = shfl(r[sb], il);              // pivot of H - conj(w) I
      const E p = Ar::mul(mw, q);               // pivot of B = I - w H
      const E iq = Ar::recip(q);
      if constexpr (DISP) {                     // z_i, then the running sums of later columns
        const E si = shfl(sacc[sb], il);
        const E zi = Ar::mul(Ar::add(av[i], Ar::neg(si)), iq);
        zy = Ar::fma(zi, y, zy);
#pragma unroll
        for (int s = 0; s < SMAX; ++s) {
          const int j = lane + 32 * s;
          if (s < S && j > i && j < n) sacc[s] = Ar::fma(zi, r[s], sacc[s]);
        }
      }
      const float pr = Ar::re(p), pi = Ar::im(p);
      if constexpr (f64) mn = fmin(mn, (double)Ar::to(p).x);
      else mn = fminf(mn, pr);
      if (!(pr == pr) || !(pi == pi)) bad = true;
      args += atan2f(pi, pr);
      prod = Ar::mul(prod, p);
      if ((i & 3) == 3) e2 += Ar::normalise(prod);   // |prod| stays in range
      if (i == n - 1) break;
      // row i + 1: its only entry left of the diagonal is H[i+1][i]; l = that / q
      const E* hrow = H + (size_t)(i + 1) * n;
      const E l = Ar::mul(hrow[i], iq);
      if constexpr (DISP) y = Ar::fms(cv[i + 1], l, y);   // y_{i+1} = c_{i+1} - l_i y_i
#pragma unroll
      for (int s = 0; s < SMAX; ++s) {
        const int j = lane + 32 * s;
        if (s < S && j > i && j < n) {
          E h = hrow[j];
          if (j == i + 1) h = Ar::add(h, Ar::neg(sg));
          r[s] = Ar::fms(h, l, r[s]);
        }
      }
    }
  }
  e2 += Ar::normalise(prod);
  if (lane == 0) {
    const double LN2 = 0.693147180559945309417232121458;
    const double2 pd = Ar::to(prod), zd = Ar::to(zy);
    double* f = a.ldfin + 6 * e;
    f[0] = pd.x;
    f[1] = pd.y;
    f[2] = (double)args;
    // log q = 1/2 gamma^T x - 1/2 log det K, gamma^T x = -sum_i z_i y_i
    f[3] = -0.5 * (double)e2 * LN2 - 0.5 * zd.x;
    f[4] = -0.5 * zd.y;
    f[5] = 0.0;
    a.minpiv[e] = bad ? -1.0e300 : (double)mn;
  }
}

// MODE 0 / 1: one problem, undisplaced / displaced (each with its own register budget);
// MODE 2: a batch job queue, displacement decided per problem.
template <class Ar, int MODE>
__global__ void __launch_bounds__(HW * 32) k_points_hess(PointArgs a0, PointBatch batch) {
  const int warp = threadIdx.x >> 5;
  if constexpr (MODE < 2) {
    for (long long e = (long long)blockIdx.x * HW + warp; e < a0.grid.n_eval; e += (long long)gridDim.x * HW)
      hess_point<Ar, MODE == 1>(a0, e);
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
      const long long e = batch.jobs[j].e0 + warp;
      if (e < sa.grid.n_eval) sa.has_gamma ? hess_point<Ar, true>(sa, e) : hess_point<Ar, false>(sa, e);
      __syncthreads();
    }
  }
}

template <class Ar, int MODE>
cudaError_t launch_hess_mode(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_points_hess<Ar, MODE>, HW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const long long groups = batch.probs ? batch.njobs : (a.grid.n_eval + HW - 1) / HW;
  long long grid = (long long)per_sm * num_sms;
  if (grid > groups) grid = groups;
  if (grid < 1) grid = 1;
  k_points_hess<Ar, MODE><<<(unsigned)grid, HW * 32, 0, s>>>(a, batch);
  return cudaGetLastError();
}

template <class Ar>
cudaError_t launch_hess_ar(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  if (batch.probs) return launch_hess_mode<Ar, 2>(a, batch, num_sms, s);
  return a.has_gamma ? launch_hess_mode<Ar, 1>(a, batch, num_sms, s) : launch_hess_mode<Ar, 0>(a, batch, num_sms, s);
}

}  // namespace

cudaError_t launch_points_hess(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s, bool df) {
  return df ? launch_hess_ar<ArDF>(a, batch, num_sms, s) : launch_hess_ar<ArF64>(a, batch, num_sms, s);
}

}  // namespace gbsbin
