// Exact cumulants of orders 1-4 of the binned counts on the GPU (Sec. VI, coarse-grained
// moments and cumulants), FP64 throughout.  With the moment generating function G(e^t) and
// e_l = e^{t_l} - 1,
//   log G = sum_r sum_{g_1..g_r} C_r[g_1..g_r] e_{g_1} ... e_{g_r},
//   C_r[g_1..g_r] = 1/(2r) tr(W_{g1 g2} W_{g2 g3} ... W_{gr g1}) + 1/2 v_{g1}^T W_{g1 g2} ... W_{g(r-1) gr} u_{gr},
// from -1/2 log det(I - E XA) and the exponent's Neumann series, with R = (I - XA)^{-1},
// W = XA R, u = R X gamma, v = R^T gamma and W_ab the block of rows of group a and columns of
// group b.  Since XA = I - Sigma^{-1}, R = Sigma and W = Sigma - I = Sigma^(1): the caller
// passes W itself (Hermitian), and u = X gamma + W X gamma, v = gamma + W^T gamma.  The rows
// arrive sorted by group (group l holds rows goff[l] .. goff[l+1] - 1), so every block is a
// contiguous sub-matrix.  Launches:
//   1. u and v (a warp per row; W^T gamma read as conj(W) gamma);
//   2. for order >= 3, Y_b = W_{:,b} W_{b,:} = W_{:,b} W_{:,b}^H per group b (Hermitian, so that
//      W_ab W_bc = Y_b[a rows, c columns]): the 32 x 32 tiles on and above the diagonal, each
//      written with its conjugate transpose below, the depth split into slices (summed in order
//      afterwards) where the tiles alone would leave SMs idle;
//   3. p_aL = v_a^T W_{a,:} and, for order >= 3, p_ab = v_a^T Y_b[a rows, :]; for order 4,
//      q_d = W_{:,d} u_d;
//   4. the coefficients, one CTA each, fixed-order sums over a block's entries:
//        C1[a]       = 1/2 sum_{i in a} (W_ii + v_i u_i)
//        C2[a,b]     = 1/4 sum_{i in a, j in b} |W_ij|^2 + 1/2 sum_{j in b} p_aL[j] u_j
//        C3[a,b,c]   = 1/6 sum_{i in a, k in c} Y_b[i,k] conj(W_ik) + 1/2 sum_{k in c} p_ab[k] u_k
//        C4[a,b,c,d] = 1/8 T_abcd + 1/2 sum_{k in c} p_ab[k] q_d[k],
//                      T_abcd = sum_{i in a, k in c} Y_b[i,k] conj(Y_d[i,k]) = conj(T_adcb),
//      so one CTA serves (a, b, c, d) and (a, d, c, b);
//   5. the chain rule of e(t) (each e_l depends on t_l alone and every derivative of e^t is 1
//      at t = 0): kappa(slots) = sum over the set partitions of the slots whose blocks each
//      carry a single group of F_{#blocks}(the blocks' groups), F_r the sum of C_r over all r!
//      orders of its indices; a warp per entry of every order, one launch.
// Work: ~n^3/2 complex multiply-adds for the Y_b and ~L^2 n^2/2 for the T, on this GPU's FP64
// pipe (2 FMAs per SM per clock); the launches are sized to occupy every SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "gbsbin_df.cuh"
#include "gbsbin_moments.h"

namespace gbsbin {
namespace {

constexpr int kMomThreads = 256;
constexpr int kGemmTile = 32;         // C tile of the products (2 x 2 entries per thread)
constexpr int kGemmK = 16;

// The kernels run in an arithmetic class Ar (gbsbin_df.cuh): ArF64, or ArDF (pairs of FP32 on
// the FMA pipe, ~46 bits); the coefficients leave them as FP64 for the chain rule.
template <class Ar>
__device__ __forceinline__ typename Ar::E scale(typename Ar::E a, double s) {
  return Ar::mul(a, Ar::from(make_double2(s, 0.0)));
}

template <class Ar>
__device__ __forceinline__ typename Ar::E warp_sum(typename Ar::E v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = Ar::add(v, shfl_xor(v, o));
  return v;
}

// Fixed-order CTA sum; every thread returns the total.
template <class Ar, class E>
__device__ E block_sum(E v, E* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kMomThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = Ar::add(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const E t = red[0];
  __syncthreads();
  return t;
}

// u_i = Xg_i + sum_k W_ik Xg_k, v_i = g_i + sum_k W_ki g_k = g_i + sum_k conj(W_ik) g_k
template <class Ar, class E = typename Ar::E>
__global__ void __launch_bounds__(kMomThreads) k_mom_uv(const E* W, const E* Xg, const E* g, E* u, E* v, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * (kMomThreads / 32) + warp;
  if (i >= n) return;
  E au = Ar::zero(), av = Ar::zero();
  for (int k = lane; k < n; k += 32) {
    const E w = W[(size_t)i * n + k];
    au = Ar::fma(w, Xg[k], au);
    av = Ar::fma(Ar::conj(w), g[k], av);
  }
  au = warp_sum<Ar>(au);
  av = warp_sum<Ar>(av);
  if (lane == 0) {
    u[i] = Ar::add(Xg[i], au);
    v[i] = Ar::add(g[i], av);
  }
}

// Slices of Y_b = W_{:,b} W_{:,b}^H over the s-th of S slices of group b's columns, one 32 x 32
// tile on or above the diagonal per CTA (blockIdx.z = b S + s): P_{b,s}(i, j) = sum_k W[i, k]
// conj(W[j, k]), k in the slice.  A thread owns rows 2 tr, 2 tr + 1 and columns tc, tc + 16 of
// the tile.  With S = 1 the tile goes straight to Y_b and, off the diagonal, its conjugate
// transpose below it.
template <class E>
struct YArgs {
  E* P;                    // Y (S = 1) or the slices, n^2 apart
  const E* W;
  const int* goff;
  int n, S;
};

template <class Ar>
__global__ void __launch_bounds__(kMomThreads) k_mom_gram(YArgs<typename Ar::E> g) {
  using E = typename Ar::E;
  if (blockIdx.x < blockIdx.y) return;
  __shared__ E As[kGemmTile * kGemmK];
  __shared__ E Bs[kGemmK * kGemmTile];
  const int n = g.n;
  const int b = blockIdx.z / g.S, sl = blockIdx.z - b * g.S;
  const int off = g.goff[b], kz = g.goff[b + 1] - off;
  const int chunk = (kz + g.S - 1) / g.S;
  const int k0 = off + min(kz, sl * chunk), k1 = off + min(kz, (sl + 1) * chunk);
  const int i0 = blockIdx.y * kGemmTile, j0 = blockIdx.x * kGemmTile;
  const int t = threadIdx.x, tr = t / 16, tc = t % 16;
  E acc[2][2] = {{Ar::zero(), Ar::zero()}, {Ar::zero(), Ar::zero()}};
  for (int kk = k0; kk < k1; kk += kGemmK) {
    const int kc = min(kGemmK, k1 - kk);
    for (int e = t; e < kGemmTile * kGemmK; e += kMomThreads) {
      const int r = e / kGemmK, c = e % kGemmK;
      As[e] = (i0 + r < n && c < kc) ? g.W[(size_t)(i0 + r) * n + kk + c] : Ar::zero();
      // Bs[c][r] = conj(W[j0 + r, kk + c])
      Bs[c * kGemmTile + r] = (j0 + r < n && c < kc) ? Ar::conj(g.W[(size_t)(j0 + r) * n + kk + c]) : Ar::zero();
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < kc; ++q) {
      const E a0 = As[(2 * tr) * kGemmK + q], a1 = As[(2 * tr + 1) * kGemmK + q];
      const E b0 = Bs[q * kGemmTile + tc], b1 = Bs[q * kGemmTile + tc + 16];
      acc[0][0] = Ar::fma(a0, b0, acc[0][0]);
      acc[0][1] = Ar::fma(a0, b1, acc[0][1]);
      acc[1][0] = Ar::fma(a1, b0, acc[1][0]);
      acc[1][1] = Ar::fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  E* P = g.P + (long long)blockIdx.z * n * n;
  const bool mirror = g.S == 1 && blockIdx.x > blockIdx.y;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int i = i0 + 2 * tr + x, j = j0 + tc + 16 * y;
      if (i < n && j < n) {
        P[(size_t)i * n + j] = acc[x][y];
        if (mirror) P[(size_t)j * n + i] = Ar::conj(acc[x][y]);
      }
    }
}

// Y_b(i, j) = sum_s P_{b,s}(i, j) in order s = 0 .. S-1 for tiles on or above the diagonal,
// conj(Y_b(j, i)) below it
template <class Ar, class E = typename Ar::E>
__global__ void __launch_bounds__(kMomThreads) k_mom_sum_slices(E* Y, const E* P, int S, int n, int L) {
  const long long nn = (long long)n * n, total = nn * L;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / nn, x = e - b * nn;
    const int i = (int)(x / n), j = (int)(x - (long long)i * n);
    const bool upper = j / kGemmTile >= i / kGemmTile;
    const long long src = upper ? x : (long long)j * n + i;
    E acc = Ar::zero();
    for (int sl = 0; sl < S; ++sl) acc = Ar::add(acc, P[(b * S + sl) * nn + src]);
    Y[b * nn + x] = upper ? acc : Ar::conj(acc);
  }
}

// In place: the FP64 values uploaded into a buffer of Ar::E (16 bytes either way) in Ar.
template <class Ar>
__global__ void __launch_bounds__(kMomThreads) k_mom_from_f64(typename Ar::E* buf, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    buf[e] = Ar::from(reinterpret_cast<const double2*>(buf)[e]);
}

// Slices of the depth so that the launch has about one CTA per SM at least (each slice >= 32 deep).
int gemm_slices(long long ctas, int kmin, int sms) {
  int S = 1;
  while (S < 8 && ctas * S < sms && kmin / (2 * S) >= 32) S *= 2;
  return S;
}

// q_d[k] = sum_{j in d} W_kj u_j (a warp per (d, k))
template <class Ar, class E = typename Ar::E>
__global__ void __launch_bounds__(kMomThreads) k_mom_q(const E* W, const E* u, E* q, const int* goff, int n, int L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long t = (long long)blockIdx.x * (kMomThreads / 32) + warp;
  if (t >= (long long)L * n) return;
  const int d = (int)(t / n), k = (int)(t - (long long)d * n);
  E acc = Ar::zero();
  for (int j = goff[d] + lane; j < goff[d + 1]; j += 32) acc = Ar::fma(W[(size_t)k * n + j], u[j], acc);
  acc = warp_sum<Ar>(acc);
  if (lane == 0) q[t] = acc;
}

// p_ab[k] = sum_{i in a} v_i Y_b[i, k] for b < L and p_aL[k] = sum_{i in a} v_i W_ik, at
// p + (a (L + 1) + b) n: blockIdx.y = a (L + 1) + b when Y was formed, else blockIdx.y = a and
// b = L only.  A lane per k, the CTA's eight warps over the rows of a, their partials added in
// order.
template <class Ar, class E = typename Ar::E>
__global__ void __launch_bounds__(kMomThreads) k_mom_p(const E* Y, const E* W, const E* v, E* p, const int* goff, int n,
                                                       int L) {
  __shared__ E red[kMomThreads];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + lane;
  const int a = Y ? blockIdx.y / (L + 1) : blockIdx.y;
  const int b = Y ? blockIdx.y - a * (L + 1) : L;
  const E* X = b < L ? Y + (size_t)b * n * n : W;
  E acc = Ar::zero();
  if (k < n)
    for (int i = goff[a] + warp; i < goff[a + 1]; i += kMomThreads / 32) acc = Ar::fma(v[i], X[(size_t)i * n + k], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  if (warp == 0 && k < n) {
    E t = red[lane];
    for (int w = 1; w < kMomThreads / 32; ++w) t = Ar::add(t, red[w * 32 + lane]);
    p[((size_t)a * (L + 1) + b) * n + k] = t;
  }
}

template <class E>
struct CoefArgs {
  int n, L, order;
  const int* goff;
  const E* W;
  const E* Y;              // Y_b at Y + b n^2
  const E* u;
  const E* v;
  const E* q;              // q_d at q + d n
  const E* p;              // p_ab at p + (a (L + 1) + b) n; b = L: v_a^T W_{a,:}
  E* out;                  // L^order coefficients, row-major in (g_1 .. g_order)
};

// Orders 1-3: one CTA per coefficient C_order[g_1..g_order]:
//   C1[a]     = 1/2 sum_{i in a} (W_ii + v_i u_i)
//   C2[a,b]   = 1/4 sum_{i in a, j in b} |W_ij|^2 + 1/2 sum_{j in b} p_aL[j] u_j
//   C3[a,b,c] = 1/6 sum_{i in a, k in c} Y_b[i,k] conj(W_ik) + 1/2 sum_{k in c} p_ab[k] u_k
template <class Ar>
__global__ void __launch_bounds__(kMomThreads) k_mom_coef(CoefArgs<typename Ar::E> a) {
  using E = typename Ar::E;
  __shared__ E red[kMomThreads];
  const int n = a.n, L = a.L;
  int g0 = 0, g1 = 0, g2 = 0;
  long long t = blockIdx.x;
  if (a.order == 1) {
    g0 = (int)t;
  } else if (a.order == 2) {
    g0 = (int)(t / L);
    g1 = (int)(t % L);
  } else {
    g2 = (int)(t % L);
    t /= L;
    g1 = (int)(t % L);
    g0 = (int)(t / L);
  }
  const int ga = a.goff[g0], na = a.goff[g0 + 1] - ga;
  if (a.order == 1) {
    E acc = Ar::zero();
    for (int i = ga + threadIdx.x; i < ga + na; i += kMomThreads)
      acc = Ar::add(acc, Ar::add(a.W[(size_t)i * n + i], Ar::mul(a.v[i], a.u[i])));
    acc = block_sum<Ar>(acc, red);
    if (threadIdx.x == 0) a.out[blockIdx.x] = scale<Ar>(acc, 0.5);
    return;
  }
  const int hc = a.order == 2 ? g1 : g2;
  const int gc = a.goff[hc], nc = a.goff[hc + 1] - gc;
  const long long cnt = (long long)na * nc;
  const E* Yb = a.order == 3 ? a.Y + (size_t)g1 * n * n : nullptr;
  E tr = Ar::zero(), vec = Ar::zero();
  for (long long e = threadIdx.x; e < cnt; e += kMomThreads) {
    const size_t x = (size_t)(ga + (int)(e / nc)) * n + gc + (int)(e - (e / nc) * nc);
    const E w = a.W[x];
    if (a.order == 2) tr = Ar::fma(w, Ar::conj(w), tr);   // |W_ij|^2
    else tr = Ar::fma(Yb[x], Ar::conj(w), tr);
  }
  const E* pv = a.p + ((size_t)g0 * (L + 1) + (a.order == 2 ? L : g1)) * n;
  for (int k = gc + threadIdx.x; k < gc + nc; k += kMomThreads) vec = Ar::fma(pv[k], a.u[k], vec);
  tr = block_sum<Ar>(tr, red);
  vec = block_sum<Ar>(vec, red);
  if (threadIdx.x == 0) a.out[blockIdx.x] = Ar::add(scale<Ar>(tr, a.order == 2 ? 0.25 : 1.0 / 6.0), scale<Ar>(vec, 0.5));
}

// Order 4: one CTA per (a, c, b <= d) writes C4[a,b,c,d] and C4[a,d,c,b].
template <class Ar>
__global__ void __launch_bounds__(kMomThreads) k_mom_coef4(CoefArgs<typename Ar::E> a) {
  using E = typename Ar::E;
  __shared__ E red[kMomThreads];
  const int n = a.n, L = a.L, npair = L * (L + 1) / 2;
  const int ac = blockIdx.x / npair;
  int pi = blockIdx.x - ac * npair;
  const int ga0 = ac / L, gc0 = ac - ga0 * L;
  int b = 0;
  while (pi >= L - b) {                              // pairs (b, d), b <= d, row by row
    pi -= L - b;
    ++b;
  }
  const int d = b + pi;
  const int ga = a.goff[ga0], na = a.goff[ga0 + 1] - ga;
  const int gc = a.goff[gc0], nc = a.goff[gc0 + 1] - gc;
  const E* Yb = a.Y + (size_t)b * n * n;
  const E* Yd = a.Y + (size_t)d * n * n;
  E tr = Ar::zero(), s1 = Ar::zero(), s2 = Ar::zero();
  const long long cnt = (long long)na * nc;
  for (long long e = threadIdx.x; e < cnt; e += kMomThreads) {
    const size_t x = (size_t)(ga + (int)(e / nc)) * n + gc + (int)(e - (e / nc) * nc);
    tr = Ar::fma(Yb[x], Ar::conj(Yd[x]), tr);
  }
  // the vector terms: sum_{k in c} p_ab[k] q_d[k] and sum_{k in c} p_ad[k] q_b[k]
  const E* pab = a.p + ((size_t)ga0 * (L + 1) + b) * n;
  const E* pad = a.p + ((size_t)ga0 * (L + 1) + d) * n;
  for (int k = gc + threadIdx.x; k < gc + nc; k += kMomThreads) {
    s1 = Ar::fma(pab[k], a.q[(size_t)d * n + k], s1);
    s2 = Ar::fma(pad[k], a.q[(size_t)b * n + k], s2);
  }
  tr = block_sum<Ar>(tr, red);
  s1 = block_sum<Ar>(s1, red);
  s2 = block_sum<Ar>(s2, red);
  if (threadIdx.x == 0) {
    const long long base = (long long)ga0 * L * L * L + (long long)gc0 * L;
    a.out[base + (long long)b * L * L + d] = Ar::add(scale<Ar>(tr, 0.125), scale<Ar>(s1, 0.5));
    if (b != d) a.out[base + (long long)d * L * L + b] = Ar::add(scale<Ar>(Ar::conj(tr), 0.125), scale<Ar>(s2, 0.5));
  }
}

template <class E>
struct KappaArgs {
  int L, order;
  const E* C[5];           // C[r]: L^r coefficients (C[0] unused)
  double* kappa;           // orders 1 .. order: L + L^2 + ... entries
};

// F_r(h_1..h_r): C_r summed over all r! orders of its indices (Heap's algorithm)
template <class Ar>
__device__ double2 F_sym(const KappaArgs<typename Ar::E>& a, int r, const int* h) {
  const int L = a.L;
  if (r == 1) return Ar::to(a.C[1][h[0]]);
  int o[4] = {0, 1, 2, 3};
  int c[4] = {0, 0, 0, 0};
  auto term = [&]() {
    long long idx = 0;
    for (int x = 0; x < r; ++x) idx = idx * L + h[o[x]];
    return Ar::to(a.C[r][idx]);
  };
  double2 s = term();
  int i = 1;
  while (i < r) {
    if (c[i] < i) {
      const int sw = (i % 2 == 0) ? 0 : c[i];
      const int tmp = o[sw];
      o[sw] = o[i];
      o[i] = tmp;
      s = ArF64::add(s, term());
      ++c[i];
      i = 1;
    } else {
      c[i] = 0;
      ++i;
    }
  }
  return s;
}

// kappa over the set partitions of the slots (orders <= 4: 1, 2, 5 and 15 partitions, as
// restricted growth strings: a block label per slot) whose blocks carry one group each.  A warp
// per entry: every lane walks the partitions, lane p evaluates those with index = p (mod 32),
// and the lanes' terms are added by a fixed butterfly.
template <class Ar>
__global__ void k_mom_kappa(KappaArgs<typename Ar::E> a) {
  const int L = a.L, lane = threadIdx.x & 31;
  long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  double* out = a.kappa;
  int r = 1;
  long long span = L;
  while (r <= a.order && t >= span) {
    t -= span;
    out += span;
    ++r;
    span *= L;
  }
  if (r > a.order) return;                          // the whole warp
  int g[4];
  long long x = t;
  for (int s = r - 1; s >= 0; --s) {
    g[s] = (int)(x % L);
    x /= L;
  }
  double2 kap = ArF64::zero();
  int lab[4] = {0, 0, 0, 0};
  for (int idx = 0;; ++idx) {
    if ((idx & 31) == lane) {
      int nblk = 0;
      for (int s = 0; s < r; ++s) nblk = max(nblk, lab[s] + 1);
      int bg[4] = {-1, -1, -1, -1};
      bool ok = true;
      for (int s = 0; s < r && ok; ++s) {
        if (bg[lab[s]] < 0) bg[lab[s]] = g[s];
        else if (bg[lab[s]] != g[s]) ok = false;
      }
      if (ok) kap = ArF64::add(kap, F_sym<Ar>(a, nblk, bg));
    }
    // next restricted growth string: lab[0] = 0, lab[s] <= 1 + max(lab[0..s-1])
    int s = r - 1;
    for (; s >= 1; --s) {
      int mx = 0;
      for (int y = 0; y < s; ++y) mx = max(mx, lab[y]);
      if (lab[s] <= mx) {
        ++lab[s];
        for (int y = s + 1; y < r; ++y) lab[y] = 0;
        break;
      }
    }
    if (s < 1) break;
  }
  kap = warp_sum<ArF64>(kap);
  if (lane == 0) out[t] = kap.x;
}

template <class Ar>
int cumulants_run(int n, int L, const int* goff, const double* W, const double* gamma, const double* Xgamma, int order,
                  double* const* kappa, cudaStream_t s, float* ms) {
  using E = typename Ar::E;
  static_assert(sizeof(E) == sizeof(double2), "the FP64 uploads share the buffers");
  const size_t nn = (size_t)n * n;
  long long Lp[5] = {1, L, (long long)L * L, (long long)L * L * L, (long long)L * L * L * L};
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  const int gt = (n + kGemmTile - 1) / kGemmTile;
  int kmin = n;
  for (int l = 0; l < L; ++l) kmin = std::min(kmin, goff[l + 1] - goff[l]);
  const int SY = order >= 3 ? gemm_slices((long long)gt * (gt + 1) / 2 * L, kmin, sms) : 1;
  const size_t ywords = order >= 3 ? (size_t)L * nn : 0, pwords = SY > 1 ? (size_t)SY * L * nn : 0;
  // device workspace: W, Y (order >= 3), the products' slices, gamma, X gamma, u, v, q, p,
  // C_1..C_order
  size_t words = nn + ywords + pwords + 4 * (size_t)n + (size_t)L * n + (size_t)L * (L + 1) * n;
  size_t kwords = 0;
  for (int r = 1; r <= order; ++r) {
    words += (size_t)Lp[r];
    kwords += (size_t)Lp[r];
  }
  E* ws = nullptr;
  double* dk = nullptr;
  int* dgoff = nullptr;
  if (cudaMalloc(&ws, words * sizeof(E)) != cudaSuccess || cudaMalloc(&dk, kwords * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dgoff, (L + 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (ws) cudaFree(ws);
    if (dk) cudaFree(dk);
    if (dgoff) cudaFree(dgoff);
    return GBSBIN_ERR_NOMEM;
  }
  E* dW = ws;
  E* Y = dW + nn;
  E* Pb = Y + ywords;
  E* dg = Pb + pwords;
  E* dXg = dg + n;
  E* du = dXg + n;
  E* dv = du + n;
  E* dq = dv + n;
  E* dp = dq + (size_t)L * n;
  E* dC[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  dC[1] = dp + (size_t)L * (L + 1) * n;
  for (int r = 2; r <= order; ++r) dC[r] = dC[r - 1] + Lp[r - 1];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaSuccess;
  if (ms) {
    err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(dW, W, nn * sizeof(E), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(dg, gamma, n * sizeof(E), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(dXg, Xgamma, n * sizeof(E), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(dgoff, goff, (L + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && ms) err = cudaEventRecord(e0, s);
  if (err == cudaSuccess) {
    const int wpb = kMomThreads / 32;
    if (!std::is_same<Ar, ArF64>::value) {           // the uploads into the arithmetic's format
      k_mom_from_f64<Ar><<<(unsigned)std::min<size_t>((nn + kMomThreads - 1) / kMomThreads, 4096), kMomThreads, 0, s>>>(
          dW, (long long)nn);
      k_mom_from_f64<Ar><<<1, kMomThreads, 0, s>>>(dg, 2LL * n);   // gamma and X gamma (adjacent)
    }
    k_mom_uv<Ar><<<(n + wpb - 1) / wpb, kMomThreads, 0, s>>>(dW, dXg, dg, du, dv, n);
    if (order >= 3) {
      YArgs<E> ya{SY > 1 ? Pb : Y, dW, dgoff, n, SY};
      k_mom_gram<Ar><<<dim3(gt, gt, L * SY), kMomThreads, 0, s>>>(ya);
      if (SY > 1)
        k_mom_sum_slices<Ar><<<(unsigned)std::min<size_t>((nn * L + kMomThreads - 1) / kMomThreads, 8 * (size_t)sms),
                           kMomThreads, 0, s>>>(Y, Pb, SY, n, L);
    }
    if (order >= 4) k_mom_q<Ar><<<(unsigned)(((long long)L * n + wpb - 1) / wpb), kMomThreads, 0, s>>>(dW, du, dq, dgoff, n, L);
    if (order >= 2)
      k_mom_p<Ar><<<dim3((n + 31) / 32, order >= 3 ? L * (L + 1) : L), kMomThreads, 0, s>>>(order >= 3 ? Y : nullptr, dW, dv,
                                                                                           dp, dgoff, n, L);
    for (int r = 1; r <= std::min(order, 3); ++r) {
      CoefArgs<E> ca{n, L, r, dgoff, dW, Y, du, dv, dq, dp, dC[r]};
      k_mom_coef<Ar><<<(unsigned)Lp[r], kMomThreads, 0, s>>>(ca);
    }
    if (order >= 4) {
      CoefArgs<E> ca{n, L, 4, dgoff, dW, Y, du, dv, dq, dp, dC[4]};
      k_mom_coef4<Ar><<<(unsigned)(Lp[2] * (L * (L + 1) / 2)), kMomThreads, 0, s>>>(ca);
    }
    KappaArgs<E> ka{L, order, {nullptr, dC[1], dC[2], dC[3], dC[4]}, dk};
    k_mom_kappa<Ar><<<(unsigned)((kwords + 3) / 4), 128, 0, s>>>(ka);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess && ms) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) {
    double* dko = dk;
    for (int r = 1; r <= order && err == cudaSuccess; ++r) {
      if (kappa[r - 1]) err = cudaMemcpyAsync(kappa[r - 1], dko, Lp[r] * sizeof(double), cudaMemcpyDeviceToHost, s);
      dko += Lp[r];
    }
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err == cudaSuccess && ms) err = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ws);
  cudaFree(dk);
  cudaFree(dgoff);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  return GBSBIN_OK;
}

}  // namespace

int cumulants_device(int n, int L, const int* goff, const double* W, const double* gamma, const double* Xgamma,
                     int order, bool pairs, double* const* kappa, cudaStream_t s, float* ms) {
  if (order < 1 || order > 4 || L < 1 || L > GBSBIN_MOM_MAX_L || n < 1) return GBSBIN_ERR_ARG;
  return pairs ? cumulants_run<ArDF>(n, L, goff, W, gamma, Xgamma, order, kappa, s, ms)
               : cumulants_run<ArF64>(n, L, goff, W, gamma, Xgamma, order, kappa, s, ms);
}

}  // namespace gbsbin
