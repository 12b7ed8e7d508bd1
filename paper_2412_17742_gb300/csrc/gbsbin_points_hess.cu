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
// One warp per point, FP64: lane t holds entries j = lane + 32 s of the current pivot row
// (and of the running sums s) in registers (s < 16, n <= 512); row i + 1 of H - conj(w) I is
// read from the L2-resident H.  log q = 1/2 gamma^T x - 1/2 log det K is left unfinished as
// (product of pivots with its power of two, FP32 sum of their arguments, the rest), finished
// one point per thread by the DFT's first stage.
#include <cuda_runtime.h>

#include "gbsbin_device.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int HW = 4;                         // warps (points) per CTA
constexpr int SMAX = GBSBIN_MAX_N / 32;       // row slots per lane

__device__ __forceinline__ double2 shfl_d2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// 2^-ex scaling of z with ex the binary exponent of max(|re|, |im|); returns ex.
__device__ __forceinline__ int renormalise(double2& z) {
  const double m = fmax(fabs(z.x), fabs(z.y));
  if (!(m > 0.0) || !(m < 1.0e300)) return 0;
  const int ex = ((__double2hiint(m) >> 20) & 0x7ff) - 1022;   // m in [2^(ex-1), 2^ex)
  const double sc = __hiloint2double((1023 - ex) << 20, 0);    // 2^-ex
  z.x *= sc;
  z.y *= sc;
  return ex;
}

template <bool DISP>
__device__ void hess_point(const PointArgs& a, long long e) {
  const int n = a.n, lane = threadIdx.x & 31;
  const int S = (n + 31) >> 5;
  const double2 w = grid_root(a.tw, a.grid, 0, point_digit(e, a.grid, 0));
  const double2 sg = make_double2(w.x, -w.y);                  // conj(w)
  const double2 mw = make_double2(-w.x, -w.y);                 // pivots of B = -w x pivots here
  const double2* H = a.H;
  const double2* av = H + (size_t)n * n;        // a = Q^T gamma
  const double2* cv = av + n;                   // c = Q^H X gamma
  constexpr bool disp = DISP;
  // row 0 of H - conj(w) I (the running sums only for displaced states)
  double2 r[SMAX], sacc[DISP ? SMAX : 1];
#pragma unroll
  for (int s = 0; s < SMAX; ++s) {
    const int j = lane + 32 * s;
    double2 v = make_double2(0.0, 0.0);
    if (s < S && j < n) {
      v = H[j];
      if (j == 0) v = make_double2(v.x - sg.x, v.y - sg.y);
    }
    r[s] = v;
    if constexpr (DISP) sacc[s] = make_double2(0.0, 0.0);
  }
  double2 y = disp ? cv[0] : make_double2(0.0, 0.0);
  double2 zy = make_double2(0.0, 0.0);          // sum_i z_i y_i
  double2 prod = make_double2(1.0, 0.0);
  int e2 = 0;
  float args = 0.0f;
  double mn = 1.0e300;
#pragma unroll
  for (int sb = 0; sb < SMAX; ++sb) {           // pivot i = 32 sb + il sits in slot sb of lane il
    if (sb >= S) break;
    for (int il = 0; il < 32; ++il) {
      const int i = 32 * sb + il;
      if (i >= n) break;
      const double2 q = shfl_d2(r[sb], il);     // pivot of H - conj(w) I
      const double2 p = cmul(mw, q);            // pivot of B = I - w H
      const double2 iq = crecip(q);
      if constexpr (DISP) {                     // z_i, then the running sums of later columns
        const double2 si = shfl_d2(sacc[sb], il);
        const double2 ai = av[i];
        const double2 zi = cmul(make_double2(ai.x - si.x, ai.y - si.y), iq);
        zy = make_double2(zy.x + (zi.x * y.x - zi.y * y.y), zy.y + (zi.x * y.y + zi.y * y.x));
#pragma unroll
        for (int s = 0; s < SMAX; ++s) {
          const int j = lane + 32 * s;
          if (s < S && j > i && j < n) sacc[s] = make_double2(sacc[s].x + (zi.x * r[s].x - zi.y * r[s].y),
                                                              sacc[s].y + (zi.x * r[s].y + zi.y * r[s].x));
        }
      }
      mn = fmin(mn, p.x);
      if (!(p.x == p.x) || !(p.y == p.y)) mn = -1.0e300;
      args += atan2f((float)p.y, (float)p.x);
      prod = cmul(prod, p);
      if (i == n - 1) break;
      // row i + 1: its only entry left of the diagonal is H[i+1][i]; l = that / q
      const double2* hrow = H + (size_t)(i + 1) * n;
      const double2 l = cmul(hrow[i], iq);
      if constexpr (DISP) y = cfnma(cv[i + 1], l, y);   // y_{i+1} = c_{i+1} - l_i y_i
#pragma unroll
      for (int s = 0; s < SMAX; ++s) {
        const int j = lane + 32 * s;
        if (s < S && j > i && j < n) {
          double2 h = hrow[j];
          if (j == i + 1) h = make_double2(h.x - sg.x, h.y - sg.y);
          r[s] = cfnma(h, l, r[s]);
        }
      }
    }
    e2 += renormalise(prod);                    // every 32 pivots: |prod| stays in range
  }
  if (lane == 0) {
    const double LN2 = 0.693147180559945309417232121458;
    double* f = a.ldfin + 6 * e;
    f[0] = prod.x;
    f[1] = prod.y;
    f[2] = (double)args;
    // log q = 1/2 gamma^T x - 1/2 log det K, gamma^T x = -sum_i z_i y_i
    f[3] = -0.5 * (double)e2 * LN2 - 0.5 * zy.x;
    f[4] = -0.5 * zy.y;
    f[5] = 0.0;
    a.minpiv[e] = mn;
  }
}

// MODE 0 / 1: one problem, undisplaced / displaced (each with its own register budget);
// MODE 2: a batch job queue, displacement decided per problem.
template <int MODE>
__global__ void __launch_bounds__(HW * 32) k_points_hess(PointArgs a0, PointBatch batch) {
  const int warp = threadIdx.x >> 5;
  if constexpr (MODE < 2) {
    for (long long e = (long long)blockIdx.x * HW + warp; e < a0.grid.n_eval; e += (long long)gridDim.x * HW)
      hess_point<MODE == 1>(a0, e);
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
      if (e < sa.grid.n_eval) sa.has_gamma ? hess_point<true>(sa, e) : hess_point<false>(sa, e);
      __syncthreads();
    }
  }
}

template <int MODE>
cudaError_t launch_hess_mode(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_points_hess<MODE>, HW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const long long groups = batch.probs ? batch.njobs : (a.grid.n_eval + HW - 1) / HW;
  long long grid = (long long)per_sm * num_sms;
  if (grid > groups) grid = groups;
  if (grid < 1) grid = 1;
  k_points_hess<MODE><<<(unsigned)grid, HW * 32, 0, s>>>(a, batch);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_points_hess(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  if (batch.probs) return launch_hess_mode<2>(a, batch, num_sms, s);
  return a.has_gamma ? launch_hess_mode<1>(a, batch, num_sms, s) : launch_hess_mode<0>(a, batch, num_sms, s);
}

}  // namespace gbsbin
