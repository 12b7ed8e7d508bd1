// Grid points by a tree of block eliminations (arXiv:2412.17742, Sec. III Eq. q_d on the
// roots-of-unity grid of Sec. VI), in pairs of FP32 or in FP64.
//
// Order the rows and columns of K(w) = I - D(w) A (A = XA) by detector group, group 0
// first (a symmetric permutation: det and the bilinear form below are unchanged, and
// every unpivoted pivot keeps Re > 0, so the branch of log det is the one of the
// per-point LU).  The leading block of group 0 is B = I - w_0 A_00, and eliminating it
// leaves the Schur complement
//
//   K_rr - K_r0 B^-1 K_0r = I - D_r (A_rr + A_r0 W),   W = w_0 B^-1 A_0r,
//
// again of the form I - D' A' with A' depending on w_0 only.  So every point with the same
// phases w_0..w_l shares the first l + 1 eliminations: depth l of the tree holds one
// reduced matrix per combination of the first l axes' roots, and a grid point is a leaf
// (the last group's block, last axis halved by conjugate symmetry).  The displacement term
// u^T K^-1 v, u = gamma, v = D X gamma, splits the same way: each elimination adds
// u_0^T y with y = w_0 B^-1 c_0 (v = D c), and leaves c' = c_r + A_r0 y, u' = u_r + W^T u_0.
//
// A level CTA runs one Gauss-Jordan sweep over the first nb columns of
//
//   [ B      | w A_0r | w c_0 ]        ->   [ I | W  | y  ]
//   [ -A_r0  | A_rr   | c_r   ]             [ . | A' | c' ],
//
// whose pivots are those of B's unpivoted LU.  log q = 1/2 sum(u_0^T y) - 1/2 sum Log(pivots).
// Each node carries a path record - the pivot product (scaled by a power of two), the FP32
// sum of the pivots' arguments, the exponent sum and the smallest pivot real part - and
// leaves write the unfinished form that the inverse DFT's first stage finishes in FP64.
//
// Arithmetic: every kernel is written once over an arithmetic (gbsbin_df.cuh): pairs of
// FP32 (about 46 bits) on the FMA pipe, or FP64.  The chains here are short and dependent;
// the FP64 pipe of this GPU issues one 32-lane instruction per ~64 cycles per scheduler,
// the FMA pipe one per cycle, so the pairs are the fast form and FP64 the exact-type one.
// Both store 16-byte elements (float4 hi/lo pairs or double2), so the tree's buffers and
// its launch shapes are the same.
#include <cuda_runtime.h>

#include <type_traits>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int LT_MAX = 512;      // threads of a level CTA (at most)
constexpr int SPAN_MAX = 4;      // groups one level launch may eliminate

// Path record of a node (48 bytes in both arithmetics): the pivot product scaled by a power
// of two; (FP32 argument sum, power of two, smallest pivot real part, -); the exponent sum.
template <class E>
struct PathRec {
  E prod;
  float4 meta;
  E ex;
};
static_assert(sizeof(PathRec<float4>) == 3 * sizeof(float4) && sizeof(PathRec<double2>) == 3 * sizeof(float4),
              "path records are three 16-byte slots");

template <class Ar>
__device__ __forceinline__ PathRec<typename Ar::E>* path_at(float4* base, long long node) {
  return reinterpret_cast<PathRec<typename Ar::E>*>(base + 3 * node);
}
template <class Ar>
__device__ __forceinline__ typename Ar::E* elem(float4* p) {
  return reinterpret_cast<typename Ar::E*>(p);
}

// w = exp(2 pi i k / R_l): from the pairs-of-FP32 table for ArDF (no FP64 conversion), else
// from the FP64 twiddles
template <class Ar>
__device__ __forceinline__ typename Ar::E root_at(const TreeArgs& a, int l, int k) {
  if constexpr (std::is_same<Ar, ArDF>::value) {
    int off = 0;
    for (int q = 0; q < l; ++q) off += a.grid.radix[q];
    return a.twdf[off + k];
  } else {
    return Ar::from(grid_root(a.tw, a.grid, l, k));
  }
}

// The path record after a set of pivots, by one full warp: lane t holds pivot t of the set
// (count <= span, a power of two <= 32; lanes beyond hold 1).  Product by a butterfly of
// pair products over aligned groups of span lanes (each level rescaled by a power of two),
// argument sum and smallest real part by butterflies too.  pr: the parent's record on
// input, the child's on output (every lane of the first group; all lanes when span = 32).
template <class Ar>
__device__ __forceinline__ void path_warp(PathRec<typename Ar::E>& pr, typename Ar::E piv, bool real, int span) {
  using E = typename Ar::E;
  E p = real ? piv : Ar::one();
  const float pre = Ar::re(piv), pim = Ar::im(piv);
  float arg = real ? atan2f(pim, pre) : 0.f;
  float mn = real ? pre : 3.0e38f;
  if (real && (!(pre == pre) || !(pim == pim))) mn = -3.0e38f;
  float e2 = 0.f;
  for (int o = span >> 1; o > 0; o >>= 1) {
    p = Ar::mul(p, shfl_xor(p, o));
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    e2 += (float)Ar::normalise(p);
    arg = __fadd_rn(arg, __shfl_xor_sync(0xffffffffu, arg, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  // every lane now holds the same product, exponent, sum and minimum; fold in the parent
  E q = Ar::mul(pr.prod, p);
  const float e = pr.meta.y + e2 + (float)Ar::normalise(q);
  pr.prod = q;
  pr.meta = make_float4(__fadd_rn(pr.meta.x, arg), e, fminf(pr.meta.z, mn), 0.f);
}

// Level l: one CTA per child (parent, k) of depth l.  Forward elimination of the nb pivot
// columns of the (m + 1) x (m + 1) augmented matrix
//
//   [ B      | w A_0r | w c_0 ]
//   [ -A_r0  | A_rr   | c_r   ]
//   [ -u_0^T | u_r^T  | 0     ]
//
// leaves the child's A' and c' in the middle rows and (u'^T | u_0^T y) in the last row:
// eliminating block 0 from a row [a_0 | a_r] gives a_r - a_0 B^-1 [w A_0r | w c_0].  Rows
// are never scaled (only the Schur complement is needed): step kk subtracts
// (G[i][kk] / G[kk][kk]) row kk from every row i > kk, each entry one fused multiply-subtract
// with its row's multiplier.  The multipliers run one step ahead: in step kk warp 0 updates
// column kk + 1 and then forms pivot kk + 1's reciprocal (every lane) and step kk + 1's
// multipliers, while warps 1.. update the columns right of it - one barrier per step, the
// hand-off off the critical path.  After the sweep warp 0 forms the child's path record
// while the other warps copy out the child's matrix and vectors.
//
// A launch may eliminate span consecutive groups l .. l + span - 1 at once (a node of depth
// l + span from its ancestor at depth l): the leading block is then those groups' rows, each
// pivot row scaled by its own group's root, and the Schur complement of that block is the
// same A'' as after span single-group sweeps (eliminating block 0 and then block 1 of the
// first Schur complement is eliminating [0 1] at once), with the same pivots.
// (48 registers: five 256-thread CTAs per SM, so a 729-CTA level runs in one wave)
template <class Ar>
__global__ void __maxnreg__(48) k_tree_level(TreeArgs a, int l, int span) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  // the child's roots, last merged axis fastest in its index, and the pivot-row bounds
  E wg[SPAN_MAX];
  int bound[SPAN_MAX];
  long long rest = blockIdx.x;
  int nb = 0;
#pragma unroll
  for (int g = SPAN_MAX - 1; g >= 0; --g) {
    if (g < span) {
      const int R = a.grid.radix[l + g];
      const long long up = rest / R;
      wg[g] = root_at<Ar>(a, l + g, (int)(rest - up * R));
      rest = up;
    }
  }
#pragma unroll
  for (int g = 0; g < SPAN_MAX; ++g) {
    if (g < span) nb += a.nb[l + g];
    bound[g] = nb;
  }
  const long long child = blockIdx.x, parent = rest;
  const int m = a.m[l], mc = m - nb, cols = m + 1;
  const int rows = a.has_gamma ? m + 1 : m;
  E* G = reinterpret_cast<E*>(gsm_raw);              // rows x cols
  E* pv = G + (size_t)rows * cols;                   // nb pivots
  E* Lm = pv + nb;                                   // 2 x rows: multipliers, this step and next
  const E* Ap = elem<Ar>(a.A[l]) + parent * (long long)m * m;
  const E* cp = elem<Ar>(a.c[l]) + parent * (long long)m;
  const E* up = elem<Ar>(a.u[l]) + parent * (long long)m;
  const int tid = threadIdx.x, LT = blockDim.x;
  const E zero = Ar::zero();
  for (int idx = tid; idx < rows * cols; idx += LT) {
    const int i = idx / cols, s = idx - (idx / cols) * cols;
    E g;
    if (i == m) {                                   // the u row
      g = s < nb ? Ar::neg(up[s]) : s < m ? up[s] : zero;
    } else {
      const E v = s < m ? Ap[(long long)i * m + s] : (a.has_gamma ? cp[i] : zero);
      if (i < nb) {
        E w = wg[0];                                 // the root of row i's group
#pragma unroll
        for (int q = 1; q < SPAN_MAX; ++q)
          if (q < span && i >= bound[q - 1]) w = wg[q];
        g = Ar::mul(w, v);
        if (s < nb) {
          g = Ar::neg(g);
          if (s == i) g = Ar::add(g, Ar::one());
        }
      } else {
        g = s < nb ? Ar::neg(v) : v;
      }
    }
    G[idx] = g;
  }
  // one step of look-ahead: warp 0 updates column kk + 1 and at once forms pivot kk + 1's
  // reciprocal and the next multipliers (into the other buffer) while warps 1.. update the
  // columns right of it; one barrier per step
  __syncthreads();                                   // the matrix is filled
  if (tid < 32) {                                    // pivot 0 and its multipliers
    const E piv = G[0];
    if (tid == 0) pv[0] = piv;
    const E r = Ar::recip(piv);
    for (int i = 1 + tid; i < rows; i += 32) Lm[i] = Ar::mul(G[i * cols], r);
  }
  __syncthreads();
  for (int kk = 0; kk < nb; ++kk) {
    const E* Lc = Lm + (kk & 1) * rows;              // this step's multipliers
    if (tid < 32) {
      E* Ln = Lm + ((kk + 1) & 1) * rows;
      const int s1 = kk + 1;
      for (int i = kk + 1 + tid; i < rows; i += 32)
        G[i * cols + s1] = Ar::fms(G[i * cols + s1], Lc[i], G[kk * cols + s1]);
      if (kk + 1 < nb) {
        __syncwarp();
        const E piv = G[s1 * cols + s1];
        if (tid == 0) pv[s1] = piv;
        const E r = Ar::recip(piv);
        for (int i = s1 + 1 + tid; i < rows; i += 32) Ln[i] = Ar::mul(G[i * cols + s1], r);
      }
    } else {
      // entries (i, s), i in (kk, rows), s in (kk + 1, cols), over threads 32..; two
      // independent entries per pass.  floor(idx / w_) from a float reciprocal: idx < 2^14
      // and w_ <= 65, so (idx + 1/2) / w_ stays more than 1/(2 w_) from an integer
      const int t = tid - 32, LO = LT - 32;
      const int w_ = cols - kk - 2, total = (rows - kk - 1) * w_;
      const float rw = 1.0f / (float)(w_ > 0 ? w_ : 1);
      for (int idx = t; idx < total; idx += 2 * LO) {
        const int idx2 = idx + LO;
        const int i = kk + 1 + (int)(((float)idx + 0.5f) * rw);
        const int sc = kk + 2 + (idx - (i - kk - 1) * w_);
        const E g1 = Ar::fms(G[i * cols + sc], Lc[i], G[kk * cols + sc]);
        if (idx2 < total) {
          const int i2 = kk + 1 + (int)(((float)idx2 + 0.5f) * rw);
          const int s2 = kk + 2 + (idx2 - (i2 - kk - 1) * w_);
          G[i2 * cols + s2] = Ar::fms(G[i2 * cols + s2], Lc[i2], G[kk * cols + s2]);
        }
        G[i * cols + sc] = g1;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid >= 32) {                                   // the child's A', c', u' (warps 1..)
    const int t = tid - 32, LO = LT - 32;
    E* Ac = elem<Ar>(a.A[l + span]) + child * (long long)mc * mc;
    for (int idx = t; idx < mc * mc; idx += LO) {
      const int i = idx / mc, j = idx - (idx / mc) * mc;
      Ac[idx] = G[(nb + i) * cols + nb + j];
    }
    if (a.has_gamma) {
      E* cc = elem<Ar>(a.c[l + span]) + child * (long long)mc;
      E* uc = elem<Ar>(a.u[l + span]) + child * (long long)mc;
      for (int j = t; j < mc; j += LO) {
        cc[j] = G[(nb + j) * cols + m];
        uc[j] = G[m * cols + nb + j];
      }
    }
  } else {                                           // the child's path record (warp 0)
    PathRec<E> pr = *path_at<Ar>(a.path[l], parent);
    int width = 1;                                   // butterfly over the pivots' lanes only
    while (width < nb && width < 32) width <<= 1;
    for (int t0 = 0; t0 < nb; t0 += 32) {
      const int t = t0 + tid;
      path_warp<Ar>(pr, t < nb ? pv[t] : zero, t < nb, width);
    }
    if (a.has_gamma) pr.ex = Ar::add(pr.ex, G[m * cols + m]);
    if (tid == 0) *path_at<Ar>(a.path[l + span], child) = pr;
  }
}


// Leaves: a team of NL lanes per evaluated point (32 / NL teams per warp), lane r holding
// row r of B = I - w A_leaf and of the right-hand side w c in registers.  Step kk
// broadcasts row kk from its lane; the rows below subtract their multiple of it (the
// right-hand side with them), so U and L^-1 (w c) come out together; the back substitution
// then broadcasts one solution entry per step.  Lane r keeps pivot r; the team reduces the
// path record into its first lane, which writes the point.
template <class Ar, int NL>
__global__ void __launch_bounds__(128) k_tree_leaf(TreeArgs a) {
  using E = typename Ar::E;
  constexpr int TEAMS = 32 / NL;
  const int lane = threadIdx.x & 31;
  const int team = lane / NL, r = lane - team * NL;
  const int base = team * NL;
  const long long leaf = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * TEAMS + team;
  const bool live = team < TEAMS && leaf < a.grid.n_eval;
  const int l = a.grid.L - 1;
  const int H = a.grid.half;
  const long long parent = live ? leaf / H : 0;
  const int k = live ? (int)(leaf - parent * H) : 0;
  const E w = root_at<Ar>(a, l, k);
  const E* Ap = elem<Ar>(a.A[l]) + parent * (long long)NL * NL + (long long)(live ? r : 0) * NL;
  const E one = Ar::one(), zero = Ar::zero();
  E b[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    b[j] = Ar::neg(Ar::mul(w, Ap[j]));
    if (j == r) b[j] = Ar::add(b[j], one);
  }
  E y = zero, u = zero;
  if (a.has_gamma) {
    y = Ar::mul(w, elem<Ar>(a.c[l])[parent * NL + (live ? r : 0)]);
    u = elem<Ar>(a.u[l])[parent * NL + (live ? r : 0)];
  }
  E myinv = one, mypiv = one;
  // the step loop stays rolled (an unrolled copy per step overflows the instruction
  // cache); the row stays in registers, entries left of the step skipped by a uniform test
#pragma unroll 1
  for (int kk = 0; kk < NL; ++kk) {
    const int src = base + kk;
    E bk = b[0];
#pragma unroll
    for (int j = 1; j < NL; ++j)
      if (j == kk) bk = b[j];
    const E piv = shfl(bk, src);
    const E ykk = shfl(y, src);
    const E inv = Ar::recip(piv);
    if (r == kk) {
      myinv = inv;
      mypiv = piv;
    }
    const bool below = r > kk;
    const E li = Ar::mul(bk, inv);                   // used by the rows below only
#pragma unroll
    for (int j = 1; j < NL; ++j) {
      if (j <= kk) continue;
      const E rj = shfl(b[j], src);
      if (below) b[j] = Ar::fms(b[j], li, rj);
    }
    if (below) y = Ar::fms(y, li, ykk);
  }
  // the path record: lane r holds pivot r; a tree over the team (partner r + o, o = 8, 4,
  // 2, 1) leaves the product (rescaled by powers of two), the argument sum and the smallest
  // real part in lane 0, which folds in the parent's record
  PathRec<E> pr = *path_at<Ar>(a.path[l], parent);
  {
    E p = mypiv;
    const float pre = Ar::re(p), pim = Ar::im(p);
    float arg = atan2f(pim, pre), mn = pre, e2 = 0.f;
    if (!(pre == pre) || !(pim == pim)) mn = -3.0e38f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      if (o >= NL) continue;
      const int partner = (lane + o) & 31;
      const E q = shfl(p, partner);
      const float qa = __shfl_sync(0xffffffffu, arg, partner), qm = __shfl_sync(0xffffffffu, mn, partner);
      const float qe = __shfl_sync(0xffffffffu, e2, partner);
      if (r + o < NL) {
        p = Ar::mul(p, q);
        e2 += qe + (float)Ar::normalise(p);
        arg = __fadd_rn(arg, qa);
        mn = fminf(mn, qm);
      }
    }
    E prod = Ar::mul(pr.prod, p);
    const float e = pr.meta.y + e2 + (float)Ar::normalise(prod);
    pr.prod = prod;
    pr.meta = make_float4(__fadd_rn(pr.meta.x, arg), e, fminf(pr.meta.z, mn), 0.f);
  }
  E ex = pr.ex;
  if (a.has_gamma) {                                  // x = U^-1 y, ex += u^T x
    E acc = y, x = zero;
#pragma unroll
    for (int t = NL - 1; t >= 0; --t) {
      if (r == t) x = Ar::mul(acc, myinv);
      const E xt = shfl(x, base + t);
      if (r < t) acc = Ar::fms(acc, b[t], xt);
    }
    E part = Ar::mul(u, x);
#pragma unroll
    for (int t = 0; t < NL; ++t) ex = Ar::add(ex, shfl(part, base + t));
  }
  if (!live || r != 0) return;
  const double LN2 = 0.693147180559945309417232121458;
  const double2 P = Ar::to(pr.prod), X = Ar::to(ex);
  double* f = a.ldfin + 6 * leaf;
  f[0] = P.x;
  f[1] = P.y;
  f[2] = (double)pr.meta.x;
  f[3] = -0.5 * (double)pr.meta.y * LN2 + 0.5 * X.x;
  f[4] = 0.5 * X.y;
  f[5] = 0.0;
  a.minpiv[leaf] = (double)pr.meta.z;
  if (a.gout) {                                      // G = q / q(1) = (P0 / P)^(1/2) 2^((e0 - e)/2) (-1)^w
    const float TWO_PI = 6.28318530717958647692f;
    const float argP = atan2f(Ar::im(pr.prod), Ar::re(pr.prod));
    const float m = rintf((pr.meta.x - argP) / TWO_PI);         // winding of log det at this point
    E p0;
    if constexpr (std::is_same<Ar, ArDF>::value) p0 = a.p0df;
    else p0 = Ar::from(make_double2(a.p0re, a.p0im));
    const E Z = Ar::mul(p0, Ar::recip(pr.prod));
    const float kz = rintf((atan2f(Ar::im(Z), Ar::re(Z)) - (a.p0arg - argP)) / TWO_PI);
    const int wind = (int)(kz + m - a.m0);
    const int d = (int)(a.e0 - pr.meta.y);
    const int hexp = (d - (d & 1)) / 2;
    if constexpr (std::is_same<Ar, ArDF>::value) {
      // sqrt(2) and 2^hexp applied to the pair (exact power-of-two scaling), one conversion
      E g = Ar::csqrt(Z);
      if (d & 1) {
        constexpr double SQ2 = 1.41421356237309504880;
        constexpr float SQ2_HI = (float)SQ2;
        constexpr float SQ2_LO = (float)(SQ2 - (double)SQ2_HI);
        g = Ar::mul(g, make_float4(SQ2_HI, 0.f, SQ2_LO, 0.f));
      }
      if (hexp >= -126 && hexp <= 127) {
        const float sc = __uint_as_float((unsigned)(127 + hexp) << 23) * ((wind & 1) ? -1.f : 1.f);
        g = make_float4(g.x * sc, g.y * sc, g.z * sc, g.w * sc);
        if (a.gout_df) reinterpret_cast<float4*>(a.gout)[leaf] = g;   // the DFT reads pairs
        else a.gout[leaf] = Ar::to(g);
      } else {
        const double2 gd = Ar::to(g);
        const double sg = (wind & 1) ? -1.0 : 1.0;
        const double2 gv = make_double2(sg * ldexp(gd.x, hexp), sg * ldexp(gd.y, hexp));
        if (a.gout_df) reinterpret_cast<float4*>(a.gout)[leaf] = Ar::from(gv);
        else a.gout[leaf] = gv;
      }
    } else {
      double2 g = Ar::to(Ar::csqrt(Z));
      if (d & 1) {
        g.x *= 1.41421356237309504880;
        g.y *= 1.41421356237309504880;
      }
      const double sg = (wind & 1) ? -1.0 : 1.0;
      a.gout[leaf] = make_double2(sg * ldexp(g.x, hexp), sg * ldexp(g.y, hexp));
    }
  }
}

template <class Ar, int NL>
cudaError_t launch_leaf(const TreeArgs& a, cudaStream_t s) {
  constexpr int TEAMS = 32 / NL;
  const long long warps = (a.grid.n_eval + TEAMS - 1) / TEAMS;
  const long long blocks = (warps + 1) / 2;           // two warps per CTA: spread evenly over SMs
  k_tree_leaf<Ar, NL><<<(unsigned)blocks, 64, 0, s>>>(a);
  return cudaGetLastError();
}

// Levels whose children would fill fewer than half the SMs take the next level into the
// same launch (a level's fixed costs - launch, fill from the parent, copy-out, path record -
// are then paid once), up to SPAN_MAX groups and while a level remains before the leaves.
template <class Ar>
cudaError_t launch_tree(const TreeArgs& a, int num_sms, cudaStream_t s, int* launches) {
  cudaError_t err = cudaSuccess;
  *launches = 1;                                      // the leaves
  long long nodes = 1;
  for (int l = 0; l + 1 < a.grid.L;) {
    long long children = nodes * a.grid.radix[l];
    int span = 1, nb = a.nb[l];
    while (span < SPAN_MAX && l + span + 1 < a.grid.L && 2 * children < num_sms) {
      children *= a.grid.radix[l + span];
      nb += a.nb[l + span];
      ++span;
    }
    const size_t smem = tree_level_smem_bytes(nb, a.m[l]);
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(k_tree_level<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    const int m = a.m[l], width = m * m;              // entries of the first elimination step
    const int threads = width >= 1024 ? 512 : width >= 256 ? 256 : 128;
    k_tree_level<Ar><<<(unsigned)children, threads, smem, s>>>(a, l, span);
    ++*launches;
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    nodes = children;
    l += span;
  }
  switch (a.m[a.grid.L - 1]) {
    case 2: return launch_leaf<Ar, 2>(a, s);
    case 4: return launch_leaf<Ar, 4>(a, s);
    case 6: return launch_leaf<Ar, 6>(a, s);
    case 8: return launch_leaf<Ar, 8>(a, s);
    case 10: return launch_leaf<Ar, 10>(a, s);
    case 12: return launch_leaf<Ar, 12>(a, s);
    case 14: return launch_leaf<Ar, 14>(a, s);
    case 16: return launch_leaf<Ar, 16>(a, s);
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace

size_t tree_level_smem_bytes(int nb, int m) { return sizeof(float4) * ((size_t)(m + 1) * (m + 1) + nb + 2 * (m + 1)); }

// Leaf blocks of 2, 4, ..., 16 rows have a kernel instance (0: not supported).
int tree_leaf_threads(int n) { return (n >= 2 && n <= 16 && n % 2 == 0) ? n : 0; }

cudaError_t launch_points_tree(const TreeArgs& a, bool fp64, int num_sms, cudaStream_t s, int* launches) {
  return fp64 ? launch_tree<ArF64>(a, num_sms, s, launches) : launch_tree<ArDF>(a, num_sms, s, launches);
}

}  // namespace gbsbin
