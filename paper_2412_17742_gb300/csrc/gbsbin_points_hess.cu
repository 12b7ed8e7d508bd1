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
// the running sums s) in registers (s < SMX <= 16, n <= 512; the kernel is instantiated for 4,
// 8, 12 and 16 slots and chosen by n); the next rows of H - conj(w) I are read from the
// L2-resident H ahead of their use.  log q = 1/2 gamma^T x - 1/2 log det K is left unfinished as
// (product of pivots with its power of two, FP32 sum of their arguments, the rest), finished
// one point per thread by the DFT's first stage.  The arithmetic class Ar is FP64 (kernel 8)
// or pairs of FP32 on the FMA pipe (kernel 16, with H, a and c stored as pairs; the pivot
// product renormalised every four pivots to stay in FP32's exponent range).
#include <cuda_runtime.h>

#include <algorithm>

#include <type_traits>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int HW = 4;                         // warps (points) per CTA

// Row slots per lane for n rows: 4, 8, 12 or 16 (n <= 512).
__host__ __device__ constexpr int hess_slots_for(int n) { return n <= 128 ? 4 : n <= 256 ? 8 : n <= 384 ? 12 : 16; }

// One point.  SMX row slots per lane (n <= 32 SMX).  With PF (prefetch, SMX <= 8) row i + 2 of H, its
// subdiagonal entry and c_{i+2} are loaded during step i, a full step ahead of their use (two
// register copies of a row); with 12 slots (two copies do not fit the registers) row i + 1 is
// loaded at the top of step i, ahead of the pivot's own work; with 16, where it is used.  The
// pivots' arguments are summed as arg(prod) + 2 pi (windings of prod around 0): each pivot of
// B has Re > 0, so it turns the running product by less than pi / 2, and a crossing of the
// negative real axis shows as a sign change of Im prod with both ends in the left half-plane.
template <class Ar, bool DISP, int SMX>
__device__ void hess_point(const PointArgs& a, long long e) {
  using E = typename Ar::E;
  constexpr bool PF = SMX <= 8, AHEAD = SMX <= 12;   // 16 slots: row i + 1 read where it is used
  const int n = a.n, lane = threadIdx.x & 31;
  const int S = (n + 31) >> 5;
  const double2 wd = grid_root(a.tw, a.grid, 0, point_digit(e, a.grid, 0));
  const E sg = Ar::from(make_double2(wd.x, -wd.y));             // conj(w)
  const E mw = Ar::from(make_double2(-wd.x, -wd.y));            // pivots of B = -w x pivots here
  const E* H = reinterpret_cast<const E*>(a.H);
  const E* av = H + (size_t)n * n;              // a = Q^T gamma
  const E* cv = av + n;                         // c = Q^H X gamma
  // row 0 of H - conj(w) I (the running sums only for displaced states); with PF also row 1
  E r[SMX], nx[AHEAD ? SMX : 1], sacc[DISP ? SMX : 1];
#pragma unroll
  for (int s = 0; s < SMX; ++s) {
    const int j = lane + 32 * s;
    E v = Ar::zero(), v1 = Ar::zero();
    if (s < S && j < n) {
      v = H[j];
      if (j == 0) v = Ar::add(v, Ar::neg(sg));
      if (PF && n > 1) v1 = H[(size_t)n + j];
    }
    r[s] = v;
    if constexpr (AHEAD) nx[s] = v1;
    if constexpr (DISP) sacc[s] = Ar::zero();
  }
  E hsub = (PF && n > 1) ? H[n] : Ar::zero();  // H[1][0]
  E cnext = (PF && DISP && n > 1) ? cv[1] : Ar::zero();
  E y = DISP ? cv[0] : Ar::zero();
  E zy = Ar::zero();                            // sum_i z_i y_i
  E prod = Ar::one();
  int e2 = 0, wind = 0;
  constexpr bool f64 = std::is_same<Ar, ArF64>::value;
  using MinT = typename std::conditional<f64, double, float>::type;
  MinT mn = f64 ? (MinT)1.0e300 : (MinT)3.0e38f;   // FP64 plans: the exact pivot; pairs: its hi part
  bool bad = false;
#pragma unroll
  for (int sb = 0; sb < SMX; ++sb) {            // pivot i = 32 sb + il sits in slot sb of lane il
    if (sb >= S) break;
    for (int il = 0; il < 32; ++il) {
      const int i = 32 * sb + il;
      if (i >= n) break;
      const bool more = i + 1 < n;
      E nx2[PF ? SMX : 1], hsub2 = Ar::zero(), cnext2 = Ar::zero();
      if constexpr (PF) {                       // row i + 2, a step ahead
        const bool more2 = i + 2 < n;
        const E* hrow2 = H + (size_t)(i + 2) * n;
#pragma unroll
        for (int s = 0; s < SMX; ++s) {
          const int j = lane + 32 * s;
          nx2[s] = (more2 && s >= sb && s < S && j > i + 1 && j < n) ? hrow2[j] : Ar::zero();
        }
        if (more2) {
          hsub2 = hrow2[i + 1];
          if constexpr (DISP) cnext2 = cv[i + 2];
        }
      } else if (AHEAD && more) {               // row i + 1, ahead of the pivot's work
        const E* hrow = H + (size_t)(i + 1) * n;
#pragma unroll
        for (int s = 0; s < SMX; ++s) {
          const int j = lane + 32 * s;
          nx[s] = (s >= sb && s < S && j > i && j < n) ? hrow[j] : Ar::zero();
        }
        hsub = hrow[i];
        if constexpr (DISP) cnext = cv[i + 1];
      }
      const E q = shfl(r[sb], il);              // pivot of H - conj(w) I
      const E p = Ar::mul(mw, q);               // pivot of B = I - w H
      const E iq = Ar::recip(q);
      if constexpr (DISP) {                     // z_i, then the running sums of later columns
        const E si = shfl(sacc[sb], il);
        const E zi = Ar::mul(Ar::add(av[i], Ar::neg(si)), iq);
        zy = Ar::fma(zi, y, zy);
#pragma unroll
        for (int s = 0; s < SMX; ++s) {
          const int j = lane + 32 * s;
          if (s >= sb && s < S && j > i && j < n) sacc[s] = Ar::fma(zi, r[s], sacc[s]);
        }
      }
      const float pr = Ar::re(p), pi = Ar::im(p);
      if constexpr (f64) mn = fmin(mn, (double)Ar::to(p).x);
      else mn = fminf(mn, pr);
      if (!(pr == pr) || !(pi == pi)) bad = true;
      const float x0 = Ar::re(prod), y0 = Ar::im(prod);
      prod = Ar::mul(prod, p);
      const float x1 = Ar::re(prod), y1 = Ar::im(prod);
      if (x0 < 0.f && x1 < 0.f) wind += (y0 >= 0.f && y1 < 0.f) ? 1 : (y0 < 0.f && y1 >= 0.f) ? -1 : 0;
      if ((i & 3) == 3) e2 += Ar::normalise(prod);   // |prod| stays in range
      if (!more) break;
      // row i + 1: its only entry left of the diagonal is H[i+1][i]; l = that / q
      const E* hrow1 = H + (size_t)(i + 1) * n;
      if constexpr (!AHEAD) {
        hsub = hrow1[i];
        if constexpr (DISP) cnext = cv[i + 1];
      }
      const E l = Ar::mul(hsub, iq);
      if constexpr (DISP) y = Ar::fms(cnext, l, y);   // y_{i+1} = c_{i+1} - l_i y_i
#pragma unroll
      for (int s = 0; s < SMX; ++s) {
        const int j = lane + 32 * s;
        if (s >= sb && s < S && j > i && j < n) {
          E h;
          if constexpr (AHEAD) h = nx[s];
          else h = hrow1[j];
          if (j == i + 1) h = Ar::add(h, Ar::neg(sg));
          r[s] = Ar::fms(h, l, r[s]);
        }
      }
      if constexpr (PF) {
#pragma unroll
        for (int s = 0; s < SMX; ++s) nx[s] = nx2[s];
        hsub = hsub2;
        cnext = cnext2;
      }
    }
  }
  e2 += Ar::normalise(prod);
  if (lane == 0) {
    const double LN2 = 0.693147180559945309417232121458;
    const double TWO_PI = 6.28318530717958647692;
    const double2 pd = Ar::to(prod), zd = Ar::to(zy);
    double* f = a.ldfin + 6 * e;
    f[0] = pd.x;
    f[1] = pd.y;
    f[2] = (double)atan2f(Ar::im(prod), Ar::re(prod)) + TWO_PI * (double)wind;
    // log q = 1/2 gamma^T x - 1/2 log det K, gamma^T x = -sum_i z_i y_i
    f[3] = -0.5 * (double)e2 * LN2 - 0.5 * zd.x;
    f[4] = -0.5 * zd.y;
    f[5] = 0.0;
    a.minpiv[e] = bad ? -1.0e300 : (double)mn;
  }
}

// MODE 0 / 1: one problem, undisplaced / displaced (each with its own register budget);
// MODE 2: a batch job queue (problems of at most 32 SMX rows), displacement decided per problem.
template <class Ar, int MODE, int SMX>
__global__ void __launch_bounds__(HW * 32) k_points_hess(PointArgs a0, PointBatch batch) {
  const int warp = threadIdx.x >> 5;
  if constexpr (MODE < 2) {
    for (long long e = (long long)blockIdx.x * HW + warp; e < a0.grid.n_eval; e += (long long)gridDim.x * HW)
      hess_point<Ar, MODE == 1, SMX>(a0, e);
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
      if (e < sa.grid.n_eval) sa.has_gamma ? hess_point<Ar, true, SMX>(sa, e) : hess_point<Ar, false, SMX>(sa, e);
      __syncthreads();
    }
  }
}

template <class Ar, int MODE, int SMX>
cudaError_t launch_hess_mode(const PointArgs& a, const PointBatch& batch, int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_points_hess<Ar, MODE, SMX>, HW * 32, 0);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  const long long groups = batch.probs ? batch.njobs : (a.grid.n_eval + HW - 1) / HW;
  long long grid = (long long)per_sm * num_sms;
  if (grid > groups) grid = groups;
  if (grid < 1) grid = 1;
  k_points_hess<Ar, MODE, SMX><<<(unsigned)grid, HW * 32, 0, s>>>(a, batch);
  return cudaGetLastError();
}

template <class Ar, int MODE>
cudaError_t launch_hess_slots(const PointArgs& a, const PointBatch& batch, int slots, int num_sms, cudaStream_t s) {
  switch (slots) {
    case 4: return launch_hess_mode<Ar, MODE, 4>(a, batch, num_sms, s);
    case 8: return launch_hess_mode<Ar, MODE, 8>(a, batch, num_sms, s);
    case 12: return launch_hess_mode<Ar, MODE, 12>(a, batch, num_sms, s);
    default: return launch_hess_mode<Ar, MODE, 16>(a, batch, num_sms, s);
  }
}

// A CTA per point, for grids with too few points to fill the GPU with a warp each (the
// warp kernel then runs one warp per SM at most and waits on every step's L2 reads): thread t
// holds entries j = t + HC_T s of the current pivot row (and of the running sums s_j).  Step i
// reads the pivot's broadcast (q_i, l_i = H[i+1][i] / q_i, z_i = (a_i - s_i) / q_i), updates
// the thread's entries j > i (s_j += z_i r_j, then r_j = N[i+1][j] - l_i r_j), and the owner of
// entry i + 1 forms the next broadcast, with H[i+2][i+1] and a_{i+1} loaded at the start of the
// step; one barrier per step, the broadcast double-buffered.  Row i + 2 is loaded during step
// i into the register set the step after it reads (two sets alternating).  Thread 0 keeps the
// scalar recurrences (the pivot product and its windings, y, z^T y).  256 threads (two entries
// each at n = 512): measured faster than 128 in both arithmetics and than 512 in FP64.
constexpr int HC_T = 256;
constexpr int HC_S = GBSBIN_MAX_N / HC_T;

template <class Ar, bool DISP>
__global__ void __launch_bounds__(HC_T) k_points_hess_cta(PointArgs a) {
  using E = typename Ar::E;
  __shared__ E bc[2][3];                        // q, l, z of the step (by parity)
  const int n = a.n, t = threadIdx.x;
  const E* H = reinterpret_cast<const E*>(a.H);
  const E* av = H + (size_t)n * n;
  const E* cv = av + n;
  constexpr bool f64 = std::is_same<Ar, ArF64>::value;
  using MinT = typename std::conditional<f64, double, float>::type;
  for (long long e = blockIdx.x; e < a.grid.n_eval; e += gridDim.x) {
    const double2 wd = grid_root(a.tw, a.grid, 0, point_digit(e, a.grid, 0));
    const E sg = Ar::from(make_double2(wd.x, -wd.y));   // conj(w)
    const E mw = Ar::from(make_double2(-wd.x, -wd.y));
    E r[HC_S], nx[HC_S], sacc[DISP ? HC_S : 1];
#pragma unroll
    for (int s = 0; s < HC_S; ++s) {
      const int j = t + HC_T * s;
      E v = Ar::zero(), v1 = Ar::zero();
      if (j < n) {
        v = H[j];
        if (j == 0) v = Ar::add(v, Ar::neg(sg));
        if (n > 1 && j >= 1) v1 = H[(size_t)n + j];
      }
      r[s] = v;
      nx[s] = v1;
      if constexpr (DISP) sacc[s] = Ar::zero();
    }
    if (t == 0) {                               // step 0's broadcast
      const E iq = Ar::recip(r[0]);
      bc[0][0] = r[0];
      bc[0][1] = n > 1 ? Ar::mul(H[n], iq) : Ar::zero();
      bc[0][2] = DISP ? Ar::mul(av[0], iq) : Ar::zero();
    }
    __syncthreads();
    E y = DISP ? cv[0] : Ar::zero(), zy = Ar::zero(), prod = Ar::one();
    int e2 = 0, wind = 0;
    MinT mn = f64 ? (MinT)1.0e300 : (MinT)3.0e38f;
    bool bad = false;
    // step i: row i + 1 in cur, row i + 2 loaded into nxt (two register sets alternating, so a
    // row's loads are waited for a whole step later); returns true after the last pivot
    auto step = [&](int i, E (&cur)[HC_S], E (&nxt)[HC_S]) -> bool {
      const int b = i & 1;
      const E q = bc[b][0], l = bc[b][1], z = bc[b][2];
      const int o = (i + 1) % HC_T, os = (i + 1) / HC_T;
      E hs = Ar::zero(), an = Ar::zero();
      if (t == o && i + 2 < n) hs = H[(size_t)(i + 2) * n + i + 1];
      if (DISP && t == o && i + 1 < n) an = av[i + 1];
      if (t == 0) {                             // the scalar recurrences
        const E p = Ar::mul(mw, q);
        const float pr = Ar::re(p), pi = Ar::im(p);
        if constexpr (f64) mn = fmin(mn, (double)Ar::to(p).x);
        else mn = fminf(mn, pr);
        if (!(pr == pr) || !(pi == pi)) bad = true;
        const float x0 = Ar::re(prod), y0 = Ar::im(prod);
        prod = Ar::mul(prod, p);
        const float x1 = Ar::re(prod), y1 = Ar::im(prod);
        if (x0 < 0.f && x1 < 0.f) wind += (y0 >= 0.f && y1 < 0.f) ? 1 : (y0 < 0.f && y1 >= 0.f) ? -1 : 0;
        if ((i & 3) == 3) e2 += Ar::normalise(prod);
        if constexpr (DISP) {
          zy = Ar::fma(z, y, zy);
          if (i + 1 < n) y = Ar::fms(cv[i + 1], l, y);   // y_{i+1} = c_{i+1} - l_i y_i
        }
      }
      if (i == n - 1) return true;
      // row i + 2, for the next step
      const E* hrow2 = H + (size_t)(i + 2) * n;
#pragma unroll
      for (int s = 0; s < HC_S; ++s) {
        const int j = t + HC_T * s;
        nxt[s] = (i + 2 < n && j > i + 1 && j < n) ? hrow2[j] : Ar::zero();
      }
#pragma unroll
      for (int s = 0; s < HC_S; ++s) {
        const int j = t + HC_T * s;
        if (j > i && j < n) {
          if constexpr (DISP) sacc[s] = Ar::fma(z, r[s], sacc[s]);
          E h = cur[s];
          if (j == i + 1) h = Ar::add(h, Ar::neg(sg));
          r[s] = Ar::fms(h, l, r[s]);
        }
      }
      if (t == o) {                             // the next step's broadcast
        E q1 = r[0], s1 = Ar::zero();
#pragma unroll
        for (int s = 0; s < HC_S; ++s)
          if (s == os) {
            q1 = r[s];
            if constexpr (DISP) s1 = sacc[s];
          }
        const E iq = Ar::recip(q1);
        bc[b ^ 1][0] = q1;
        bc[b ^ 1][1] = Ar::mul(hs, iq);
        bc[b ^ 1][2] = DISP ? Ar::mul(Ar::add(an, Ar::neg(s1)), iq) : Ar::zero();
      }
      __syncthreads();
      return false;
    };
    E nxb[HC_S];
    for (int i = 0; i < n; i += 2) {
      if (step(i, nx, nxb)) break;
      if (step(i + 1, nxb, nx)) break;
    }
    if (t == 0) {
      e2 += Ar::normalise(prod);
      const double LN2 = 0.693147180559945309417232121458;
      const double TWO_PI = 6.28318530717958647692;
      const double2 pd = Ar::to(prod), zd = Ar::to(zy);
      double* f = a.ldfin + 6 * e;
      f[0] = pd.x;
      f[1] = pd.y;
      f[2] = (double)atan2f(Ar::im(prod), Ar::re(prod)) + TWO_PI * (double)wind;
      f[3] = -0.5 * (double)e2 * LN2 - 0.5 * zd.x;
      f[4] = -0.5 * zd.y;
      f[5] = 0.0;
      a.minpiv[e] = bad ? -1.0e300 : (double)mn;
    }
    __syncthreads();                            // the broadcast buffer is reused by the next point
  }
}

template <class Ar>
cudaError_t launch_hess_cta(const PointArgs& a, int num_sms, cudaStream_t s) {
  const long long grid = std::min<long long>(a.grid.n_eval, 4LL * num_sms);
  if (a.has_gamma) k_points_hess_cta<Ar, true><<<(unsigned)grid, HC_T, 0, s>>>(a);
  else k_points_hess_cta<Ar, false><<<(unsigned)grid, HC_T, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Ar>
cudaError_t launch_hess_ar(const PointArgs& a, const PointBatch& batch, int slots, int num_sms, cudaStream_t s) {
  if (batch.probs) return launch_hess_slots<Ar, 2>(a, batch, slots, num_sms, s);
  if (a.n >= 128 && a.grid.n_eval < 4LL * num_sms) return launch_hess_cta<Ar>(a, num_sms, s);
  return a.has_gamma ? launch_hess_slots<Ar, 1>(a, batch, slots, num_sms, s)
                     : launch_hess_slots<Ar, 0>(a, batch, slots, num_sms, s);
}

}  // namespace

int hess_slots(int n) { return hess_slots_for(n); }

cudaError_t launch_points_hess(const PointArgs& a, const PointBatch& batch, int slots, int num_sms, cudaStream_t s,
                               bool df) {
  if (slots <= 0) slots = hess_slots_for(a.n);
  return df ? launch_hess_ar<ArDF>(a, batch, slots, num_sms, s) : launch_hess_ar<ArF64>(a, batch, slots, num_sms, s);
}

}  // namespace gbsbin
