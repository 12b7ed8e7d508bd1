// Grid points of large matrices by a tree of block eliminations with Hessenberg leaves
// (arXiv:2412.17742, Sec. III Eq. q_d on the roots-of-unity grid of Sec. VI), in pairs of
// FP32 or in FP64.
//
// Rows and columns of K(w) = I - D(w) A are ordered by detector group (a symmetric
// permutation: det, the exponent's bilinear form and the pivots' Re > 0 are unchanged).
// Eliminating group 0's block leaves a matrix of the same form whose A' depends on w_0 only,
// so depth l of the tree holds one reduced matrix per combination of the first l axes'
// roots.  Each node stores the augmented matrix
//
//   [ A    c  ]      A: m x m,  c: the right-hand side's coefficients (v = D c),
//   [ u^T  ex ]      u: the exponent's left vector, ex: the exponent collected so far,
//
// and a level turns it, for the child's root w of the group's axis, into
//
//   [ I - w A_00   w A_0r   w c_0 ]
//   [   -A_r0       A_rr     c_r  ]        (the "G form")
//   [   -u_0^T      u_r^T    ex   ]
//
// whose forward elimination over the group's nb pivot columns leaves exactly the child's
// augmented matrix [[A', c'], [u'^T, ex + u_0^T y]] (A' = A_rr + A_r0 W, W = w B^-1 A_0r,
// y = w B^-1 c_0): the exponent rides along in the corner.  The pivots are those of the
// per-point unpivoted LU of the permuted K(w), each with Re > 0.
//
// A level runs in sub-steps of nbs pivots (as many as fit in shared memory), each in two
// launches:
//   top:    one CTA per child eliminates the nbs pivot rows among themselves in shared
//           memory (one barrier per step) and writes them with their reciprocal pivots; one
//           warp folds the pivots into the child's path record;
//   bottom: several CTAs per child stage those pivot rows in shared memory and stream the
//           other rows through registers (a warp per row: lane t holds columns t + 32 s),
//           each eliminated against the pivot rows, and write the trailing block - the next
//           sub-step's input, or the child's augmented matrix after the level's last one.
//
// Leaves.  The last group's block is I - w A_L for every root w of the last axis, so one
// Householder reduction A_L = Q H Q^H per leaf parent (a CTA per node, the matrix in shared
// memory, or for last groups above GBSBIN_BT_MAX_HESS rows in the node's slot of the Hessenberg
// buffer through L2) serves all of them: det(I - w A_L) = det(I - w H), and with N = H - conj(w) I =
// -conj(w) (I - w H) the pivots of I - w H are -w times those of N.  The exponent's leaf term
// u^T (I - w A_L)^-1 w c = -a^T N^-1 b with a = Q^T u, b = Q^H c (reflectors applied to c and
// to conj(u) as extra columns).  A warp per evaluated point runs the O(m^2) unpivoted
// elimination of the Hessenberg matrix N (each step updates the next row only), with the
// exponent by the recurrences y_{i+1} = b_{i+1} - l_i y_i and z_i = (a_i - s_i) / n_ii,
// s_j += z_i n_ij, a^T N^-1 b = sum z_i y_i, and writes the point's unfinished log q.  Every
// pivot of I - w H has Re > 0 (a unitary similarity of the Schur complement I - w A_L, which
// has a positive-definite Hermitian part), and Sum Log over any unpivoted elimination of a
// matrix of that class is the branch of log det continuous along (1 - t) I + t K, so the
// branch is the per-point LU's.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int TOP_THREADS = 512;
constexpr int BOT_WARPS = 16;
constexpr int HESS_THREADS = 256;
constexpr int LEAF_WARPS = 4;
constexpr int LEAF_SMAX = (GBSBIN_BT_MAX_HESS + 31) / 32;       // leaves of last groups <= 128 rows
constexpr int LEAF_SMAX_BIG = (GBSBIN_BT_MAX_LAST + 31) / 32;   // and above

template <class Ar>
__device__ __forceinline__ typename Ar::E* elem(float4* p) {
  return reinterpret_cast<typename Ar::E*>(p);
}
template <class Ar>
__device__ __forceinline__ const typename Ar::E* elem(const float4* p) {
  return reinterpret_cast<const typename Ar::E*>(p);
}

// w = exp(2 pi i k / R_l) (k counted from k0_lo on axis 0 of a shard)
template <class Ar>
__device__ __forceinline__ typename Ar::E bt_root(const BTreeArgs& a, int l, int k) {
  if (l == 0) k += a.k0_lo;
  if constexpr (std::is_same<Ar, ArDF>::value) {
    int off = 0;
    for (int q = 0; q < l; ++q) off += a.grid.radix[q];
    return a.twdf[off + k];
  } else {
    return Ar::from(grid_root(a.tw, a.grid, l, k));
  }
}

// Entry (i, s) of a level's G form from the parent's augmented entry v (see the top of the
// file): the group's rows (i < nbg) are scaled by the root and their group columns become
// I - w A_00; the other rows have their group columns negated.
template <class Ar>
__device__ __forceinline__ typename Ar::E g_form(typename Ar::E v, int i, int s, int nbg, typename Ar::E w) {
  if (i < nbg) {
    v = Ar::mul(w, v);
    if (s < nbg) {
      v = Ar::neg(v);
      if (s == i) v = Ar::add(v, Ar::one());
    }
  } else if (s < nbg) {
    v = Ar::neg(v);
  }
  return v;
}

// Path record: the pivot product scaled by a power of two, then (FP32 sum of the pivots'
// arguments, the power of two, the smallest pivot real part, -).
template <class E>
struct BRec {
  E prod;
  float4 meta;
};
static_assert(sizeof(BRec<float4>) == 2 * sizeof(float4) && sizeof(BRec<double2>) == 2 * sizeof(float4),
              "path records are two 16-byte slots");

// Fold count pivots (read through piv(k)) into the record rec, by one full warp: each lane
// multiplies its share, a butterfly combines them.  Every lane returns the new record.
template <class Ar, class PivFn>
__device__ __forceinline__ BRec<typename Ar::E> fold_pivots(BRec<typename Ar::E> rec, int count, PivFn piv) {
  using E = typename Ar::E;
  const int lane = threadIdx.x & 31;
  E p = Ar::one();
  float arg = 0.f, mn = 3.0e38f, e2 = 0.f;
  int since = 0;
  for (int k = lane; k < count; k += 32) {
    const E q = piv(k);
    const float qr = Ar::re(q), qi = Ar::im(q);
    arg = __fadd_rn(arg, atan2f(qi, qr));
    mn = fminf(mn, qr);
    if (!(qr == qr) || !(qi == qi)) mn = -3.0e38f;
    p = Ar::mul(p, q);
    if (++since == 8) {                              // |pivot| <= 2: rescale every 8
      e2 += (float)Ar::normalise(p);
      since = 0;
    }
  }
  e2 += (float)Ar::normalise(p);
  for (int o = 16; o > 0; o >>= 1) {
    p = Ar::mul(p, shfl_xor(p, o));
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    e2 += (float)Ar::normalise(p);
    arg = __fadd_rn(arg, __shfl_xor_sync(0xffffffffu, arg, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  BRec<E> out;
  out.prod = Ar::mul(rec.prod, p);
  const float e = rec.meta.y + e2 + (float)Ar::normalise(out.prod);
  out.meta = make_float4(__fadd_rn(rec.meta.x, arg), e, fminf(rec.meta.z, mn), 0.f);
  return out;
}

template <class Ar>
__device__ __forceinline__ BRec<typename Ar::E>* rec_at(float4* base, long long node) {
  return reinterpret_cast<BRec<typename Ar::E>*>(base + 2 * node);
}

// Input matrix of a sub-step for a child: the parent's augmented matrix (first sub-step of
// a level, roots applied on load) or the child's own trailing block.
template <class Ar>
__device__ __forceinline__ const typename Ar::E* step_input(const BTreeArgs& a, const BTreeStep& st, long long child,
                                                            long long parent) {
  const long long DD = (long long)st.D * st.D;
  return st.first ? elem<Ar>(a.mat[st.l]) + parent * DD : elem<Ar>(st.in) + child * DD;
}

// ---------------------------------------------------------------------------- top
// CTA (child, part): the nbs pivot rows in shared memory - their first nbs columns (the pivot
// block) and the part's share of the columns right of it (every column when parts = 1; the
// parts split the right-hand columns when a level has few children, each redoing the pivot
// block) - and their forward elimination among themselves.  Step kk: every warp forms
// 1 / u_kk and the multipliers of its own rows (column kk and row kk are not written in step
// kk), then updates its rows right of kk; one barrier per step.  Part 0 also writes the pivot
// block, the reciprocal pivots and the child's path record.
template <class Ar>
__global__ void __launch_bounds__(TOP_THREADS) k_bt_top(BTreeArgs a, BTreeStep st, int parts, int W) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int D = st.D, nbs = st.nbs;                  // W: right-hand columns per part, (parts - 1) W < D - nbs
  const long long child = blockIdx.x / parts;
  const int part = (int)(blockIdx.x - child * parts);
  const int c0 = nbs + part * W, c1 = min(D, c0 + W);  // this part's right-hand columns
  const int Dl = nbs + (c1 - c0);                    // local columns: pivot block, then the share
  E* U = reinterpret_cast<E*>(sm_raw);               // nbs x Dl
  E* pinv = U + (size_t)nbs * Dl;                    // nbs
  const int R = a.cnt[st.l];
  const long long parent = child / R;
  const E w = bt_root<Ar>(a, st.l, (int)(child - parent * R));
  const E* src = step_input<Ar>(a, st, child, parent);
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = T >> 5;
  for (int idx = tid; idx < nbs * Dl; idx += T) {
    const int i = idx / Dl, c = idx - i * Dl;
    const int g = c < nbs ? c : c0 + (c - nbs);
    E v = src[(long long)i * D + g];
    if (st.first) v = g_form<Ar>(v, i, g, st.nbg, w);
    U[idx] = v;
  }
  __syncthreads();
  for (int kk = 0; kk < nbs; ++kk) {
    const E* Uk = U + (size_t)kk * Dl;
    const E r = Ar::recip(Uk[kk]);
    if (tid == 0) pinv[kk] = r;
    for (int i = kk + 1 + warp; i < nbs; i += NW) {
      E* Ui = U + (size_t)i * Dl;
      const E li = Ar::mul(Ui[kk], r);
      for (int j = kk + 1 + lane; j < Dl; j += 32) Ui[j] = Ar::fms(Ui[j], li, Uk[j]);
    }
    __syncthreads();
  }
  E* Ug = elem<Ar>(a.U) + child * (long long)nbs * D;
  for (int idx = tid; idx < nbs * Dl; idx += T) {
    const int i = idx / Dl, c = idx - i * Dl;
    if (c >= nbs) Ug[(long long)i * D + c0 + (c - nbs)] = U[idx];
    else if (part == 0) Ug[(long long)i * D + c] = U[idx];
  }
  if (part != 0) return;
  E* pg = elem<Ar>(a.inv) + child * (long long)nbs;
  for (int k = tid; k < nbs; k += T) pg[k] = pinv[k];
  if (warp == 0) {
    const BRec<E> in = st.first ? *rec_at<Ar>(a.path[st.l], parent) : *rec_at<Ar>(a.path[st.l + 1], child);
    const BRec<E> out = fold_pivots<Ar>(in, nbs, [&](int k) { return U[(size_t)k * Dl + k]; });
    if (lane == 0) *rec_at<Ar>(a.path[st.l + 1], child) = out;
  }
}

// ---------------------------------------------------------------------------- bottom
// The other rows of every child, D - nbs per child, taken as one sequence (child-major) and
// split evenly over the CTAs (one per resident slot): a CTA walks its share child by child,
// staging each child's nbs pivot rows and reciprocals in shared memory.  A warp per row: the
// row's first Dm columns in registers (lane t: columns t + 32 s), eliminated against pivot
// rows 0 .. nbs - 1 in order (the multiplier is the row's current entry kk, broadcast from
// its lane; lane kk mod 32 keeps it), then the trailing part (columns nbs ..) written as row
// - nbs of the output.  Columns Dm .. D - 1 (a short tail, such as the augmented column when
// D = 32 s + 1) need no register slot: each is its initial value minus the dot product of the
// kept multipliers with the pivot rows' entries, summed over the lanes by a fixed butterfly.
template <class Ar, int SMAX>
__global__ void __launch_bounds__(BOT_WARPS * 32) k_bt_bottom(BTreeArgs a, BTreeStep st, int Dm, long long rows_total) {
  using E = typename Ar::E;
  constexpr int LMS = GBSBIN_BT_MAX_NBS / 32;          // register slots of the multipliers
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int D = st.D, nbs = st.nbs, Do = D - nbs, S = (Dm + 31) >> 5;
  E* U = reinterpret_cast<E*>(sm_raw);
  E* pinv = U + (size_t)nbs * D;
  const int R = a.cnt[st.l];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long g0 = rows_total * blockIdx.x / gridDim.x, g1 = rows_total * (blockIdx.x + 1) / gridDim.x;
  for (long long gs = g0; gs < g1;) {
    const long long child = gs / Do;
    const long long ge = min(g1, (child + 1) * Do);  // this child's rows in the share
    const long long parent = child / R;
    const E w = bt_root<Ar>(a, st.l, (int)(child - parent * R));
    const E* src = step_input<Ar>(a, st, child, parent);
    E* dst = elem<Ar>(st.out) + child * (long long)Do * Do;
    const E* Ug = elem<Ar>(a.U) + child * (long long)nbs * D;
    const E* pg = elem<Ar>(a.inv) + child * (long long)nbs;
    __syncthreads();                                 // the previous child's rows are done
    for (int idx = tid; idx < nbs * D; idx += blockDim.x) U[idx] = Ug[idx];
    for (int k = tid; k < nbs; k += blockDim.x) pinv[k] = pg[k];
    __syncthreads();
    for (long long gr = gs + warp; gr < ge; gr += BOT_WARPS) {
      const int i = nbs + (int)(gr - child * Do);
      const E* srow = src + (long long)i * D;
      E r[SMAX], lm[LMS];
#pragma unroll
      for (int s = 0; s < SMAX; ++s) {
        const int j = lane + 32 * s;
        E v = Ar::zero();
        if (s < S && j < Dm) {
          v = srow[j];
          if (st.first) v = g_form<Ar>(v, i, j, st.nbg, w);
        }
        r[s] = v;
      }
#pragma unroll
      for (int s = 0; s < LMS; ++s) lm[s] = Ar::zero();
#pragma unroll
      for (int sb = 0; sb < SMAX; ++sb) {            // pivot kk = 32 sb + il sits in slot sb of lane il
        if (32 * sb >= nbs) break;
        const int kend = min(32, nbs - 32 * sb);
        for (int il = 0; il < kend; ++il) {
          const int kk = 32 * sb + il;
          const E x = shfl(r[sb], il);
          const E li = Ar::mul(x, pinv[kk]);
          if (sb < LMS && lane == il) lm[sb < LMS ? sb : 0] = li;
          const E* Uk = U + (size_t)kk * D;
#pragma unroll
          for (int s = sb; s < SMAX; ++s) {
            const int j = lane + 32 * s;
            if (s < S && j > kk && j < Dm) r[s] = Ar::fms(r[s], li, Uk[j]);
          }
        }
      }
      E* drow = dst + (long long)(i - nbs) * Do;
#pragma unroll
      for (int s = 0; s < SMAX; ++s) {
        const int j = lane + 32 * s;
        if (s < S && j >= nbs && j < Dm) drow[j - nbs] = r[s];
      }
      for (int t = Dm; t < D; ++t) {                 // the tail: initial value - sum_kk l_kk U[kk][t]
        E acc = Ar::zero();
#pragma unroll
        for (int s = 0; s < LMS; ++s) {
          const int kk = lane + 32 * s;
          if (kk < nbs) acc = Ar::fma(lm[s], U[(size_t)kk * D + t], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc = Ar::add(acc, shfl_xor(acc, o));
        if (lane == 0) {
          E v = srow[t];
          if (st.first) v = g_form<Ar>(v, i, t, st.nbg, w);
          drow[t - nbs] = Ar::add(v, Ar::neg(acc));
        }
      }
    }
    gs = ge;
  }
}

// ------------------------------------------------------------------------- Hessenberg
// One CTA per leaf parent: the m x m block A_L with c and conj(u) as two extra columns in
// shared memory (row stride m + 3, odd in 16-byte units), or, for GM (m above
// GBSBIN_BT_MAX_HESS), A_L in the node's slot of the Hessenberg buffer H (row stride m, read and
// written through L2) with the two columns in shared memory, reduced to upper Hessenberg form
// by Householder reflectors H_k = I - beta v v^H on rows/columns k + 1 .. m - 1
// (v = x - alpha e_1, alpha = -e^{i arg x_0} ||x||, beta = 2 / ||v||^2), applied from the left
// to A and the two columns and from the right to A.  Each product vector (v^H A per column,
// A v per row) is formed by g threads per column or row over interleaved index sets, then
// summed in a fixed order, so the dependent chains are m / g long.  Writes H (m x m),
// a = Q^T u, b = Q^H c and the exponent collected so far (the augmented corner).
template <class Ar, bool GM>
__global__ void __launch_bounds__(HESS_THREADS) k_bt_hess(BTreeArgs a) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int m = a.mL, ld = GM ? m : m + 3, D = m + 1;
  const long long node = blockIdx.x;
  E* const Hn = elem<Ar>(a.H) + node * (long long)m * m;
  E* A = GM ? Hn : reinterpret_cast<E*>(sm_raw);     // m x ld (+ the two columns in shared memory)
  E* v = GM ? reinterpret_cast<E*>(sm_raw) : A + (size_t)m * ld;   // m
  E* sv = v + m;                                     // m + 2 (left products per column)
  E* tv = sv + m + 2;                                // m (right products per row)
  E* sc = tv + m;                                    // alpha, beta
  E* part = sc + 2;                                  // HESS_THREADS partial sums
  E* X = part + HESS_THREADS;                        // GM: c and conj(u), m x 2
  // entry (i, j) of the augmented block, j < m + 2
  auto at = [&](int i, int j) -> E& {
    if constexpr (GM) {
      if (j >= m) return X[2 * i + (j - m)];
    }
    return A[(size_t)i * ld + j];
  };
  const E* src = elem<Ar>(a.mat[a.L - 1]) + node * (long long)D * D;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < m * (m + 2); idx += T) {
    const int i = idx / (m + 2), j = idx - i * (m + 2);
    E val;
    if (j < m) val = src[(long long)i * D + j];
    else if (j == m) val = src[(long long)i * D + m];                 // c
    else val = Ar::conj(src[(long long)m * D + i]);                    // conj(u)
    at(i, j) = val;
  }
  __syncthreads();
  for (int k = 0; k + 2 < m; ++k) {
    if (warp == 0) {                                 // the reflector of column k
      E nrm2 = Ar::zero();
      for (int i = k + 1 + lane; i < m; i += 32) nrm2 = Ar::add(nrm2, Ar::norm2(at(i, k)));
      for (int o = 16; o > 0; o >>= 1) nrm2 = Ar::add(nrm2, shfl_xor(nrm2, o));
      const E x0 = at(k + 1, k);
      E alpha = Ar::zero(), beta = Ar::zero();
      if (Ar::re(nrm2) > 0.f) {
        const E nrm = Ar::rsqrt_real(nrm2);
        const E ax0 = Ar::rsqrt_real(Ar::norm2(x0));
        alpha = Ar::re(ax0) > 0.f ? Ar::neg(Ar::mul(x0, Ar::mul(nrm, Ar::rrecip(ax0)))) : Ar::neg(nrm);
        // ||v||^2 = ||x||^2 - 2 Re(conj(alpha) x0) + |alpha|^2 = 2 (||x||^2 + ||x|| |x0|)
        const E vn2 = Ar::add(Ar::add(nrm2, nrm2), Ar::add(Ar::mul(nrm, ax0), Ar::mul(nrm, ax0)));
        beta = Ar::add(Ar::rrecip(vn2), Ar::rrecip(vn2));
      }
      for (int i = k + 1 + lane; i < m; i += 32) {
        E vi = at(i, k);
        if (i == k + 1) vi = Ar::add(vi, Ar::neg(alpha));
        v[i] = vi;
      }
      if (lane == 0) {
        sc[0] = alpha;
        sc[1] = beta;
      }
    }
    __syncthreads();
    const E beta = sc[1];
    if (Ar::re(beta) > 0.f) {
      // left: s_j = beta sum_{i > k} conj(v_i) A_ij, columns j > k and the two extra columns
      const int nc = m + 1 - k, gl = max(1, min(8, T / nc));
      {
        const int c = tid / gl, g = tid - c * gl;
        if (c < nc) {
          const int j = k + 1 + c;
          E s = Ar::zero();
          for (int i = k + 1 + g; i < m; i += gl) s = Ar::fma(Ar::conj(v[i]), at(i, j), s);
          part[tid] = s;
        }
      }
      __syncthreads();
      for (int c = tid; c < nc; c += T) {
        E s = part[c * gl];
        for (int g = 1; g < gl; ++g) s = Ar::add(s, part[c * gl + g]);
        sv[k + 1 + c] = Ar::mul(beta, s);
      }
      __syncthreads();
      const int wl = m + 2 - (k + 1);
      for (int idx = tid; idx < (m - k - 1) * wl; idx += T) {
        const int i = k + 1 + idx / wl, j = k + 1 + idx % wl;
        at(i, j) = Ar::fms(at(i, j), v[i], sv[j]);
      }
      __syncthreads();
      // right: t_i = beta sum_{j > k} A_ij v_j, every row
      const int gr = max(1, min(8, T / m));
      {
        const int i = tid / gr, g = tid - i * gr;
        if (i < m) {
          E t = Ar::zero();
          for (int j = k + 1 + g; j < m; j += gr) t = Ar::fma(at(i, j), v[j], t);
          part[tid] = t;
        }
      }
      __syncthreads();
      for (int i = tid; i < m; i += T) {
        E t = part[i * gr];
        for (int g = 1; g < gr; ++g) t = Ar::add(t, part[i * gr + g]);
        tv[i] = Ar::mul(beta, t);
      }
      __syncthreads();
      const int wr = m - (k + 1);
      for (int idx = tid; idx < m * wr; idx += T) {
        const int i = idx / wr, j = k + 1 + idx % wr;
        at(i, j) = Ar::fms(at(i, j), tv[i], Ar::conj(v[j]));
      }
      if (tid == 0) at(k + 1, k) = sc[0];
    }
    __syncthreads();
  }
  E* hv = elem<Ar>(a.hv) + node * (long long)(2 * m + 1);
  if constexpr (!GM)                                 // (GM: the reduction ran in place)
    for (int idx = tid; idx < m * m; idx += T) {
      const int i = idx / m, j = idx - i * m;
      Hn[idx] = at(i, j);
    }
  for (int i = tid; i < m; i += T) {
    hv[i] = Ar::conj(at(i, m + 1));     // a = Q^T u = conj(Q^H conj(u))
    hv[m + i] = at(i, m);               // b = Q^H c
  }
  if (tid == 0) hv[2 * m] = src[(long long)m * D + m];   // the exponent so far
}

// ----------------------------------------------------------------------------- leaves
// Unfinished log q record of evaluated point e (see the inverse DFT's first stage), or of its
// conjugate point: log q(-k) = conj log q(k), so the record becomes (conj P, -arguments,
// Re part, -Im part).
__device__ __forceinline__ void write_record(const BTreeArgs& a, long long e, double2 P, double args, double r3,
                                             double r4, double mn, bool conj) {
  double* f = a.ldfin + 6 * e;
  f[0] = P.x;
  f[1] = conj ? -P.y : P.y;
  f[2] = conj ? -args : args;
  f[3] = r3;
  f[4] = conj ? -r4 : r4;
  f[5] = 0.0;
  a.minpiv[e] = mn;
}

// A warp per leaf: the Hessenberg elimination of N = H - conj(w) I with the exponent
// recurrences (see the top of the file).  Lane t holds entries t + 32 s of the current pivot
// row (and of the running sums s_j); row i + 1 of H, the subdiagonal entry and b_{i+1} are read
// from L2 one step ahead of their use.
template <class Ar, bool DISP, int SMX>
__global__ void __launch_bounds__(LEAF_WARPS * 32, SMX <= LEAF_SMAX ? (DISP ? 3 : 4) : 2) k_bt_leaf(BTreeArgs a) {
  using E = typename Ar::E;
  const int lane = threadIdx.x & 31;
  const long long leaf = (long long)blockIdx.x * LEAF_WARPS + (threadIdx.x >> 5);
  if (leaf >= a.n_leaves) return;
  const int m = a.mL, S = (m + 31) >> 5, l = a.grid.L - 1;
  const int kl = a.cnt[l];
  const long long parent = leaf / kl;
  const int klast = (int)(leaf - parent * kl);
  const E w = bt_root<Ar>(a, l, klast);
  const E sg = Ar::conj(w), mw = Ar::neg(w);
  const E* H = elem<Ar>(a.H) + parent * (long long)m * m;
  const E* hv = elem<Ar>(a.hv) + parent * (long long)(2 * m + 1);
  const E* av = hv;
  const E* bv = hv + m;
  E r[SMX], nx[SMX], sacc[DISP ? SMX : 1];
#pragma unroll
  for (int s = 0; s < SMX; ++s) {
    const int j = lane + 32 * s;
    E x = Ar::zero(), y1 = Ar::zero();
    if (s < S && j < m) {
      x = H[j];
      if (j == 0) x = Ar::add(x, Ar::neg(sg));
      if (m > 1) y1 = H[(long long)m + j];           // row 1, used in step 0
    }
    r[s] = x;
    nx[s] = y1;
    if constexpr (DISP) sacc[s] = Ar::zero();
  }
  E hsub = m > 1 ? H[m] : Ar::zero();                // H[1][0]
  E bnext = (DISP && m > 1) ? bv[1] : Ar::zero();
  E y = DISP ? bv[0] : Ar::zero();
  E zy = Ar::zero();
  const BRec<E> rec = *rec_at<Ar>(a.path[l], parent);
  // the leaf's own pivot product lp (scaled by powers of two) and its windings around 0: each
  // pivot turns lp by less than pi/2 (Re > 0), so a turn across the negative real axis has
  // both ends in the left half-plane and shows as a sign change of Im lp there
  E lp = Ar::one();
  int wind = 0;
  float e2 = rec.meta.y, mn = rec.meta.z;
#pragma unroll
  for (int sb = 0; sb < SMX; ++sb) {
    if (sb >= S) break;
    for (int il = 0; il < 32; ++il) {
      const int i = 32 * sb + il;
      if (i >= m) break;
      // the next step's row, subdiagonal entry and right-hand side, loaded ahead
      E nx2[SMX], hsub2 = Ar::zero(), bnext2 = Ar::zero();
      const bool more = i + 2 < m;
      const E* hrow2 = H + (long long)(i + 2) * m;
#pragma unroll
      for (int s = 0; s < SMX; ++s) {
        const int j = lane + 32 * s;
        nx2[s] = (more && s >= sb && s < S && j > i + 1 && j < m) ? hrow2[j] : Ar::zero();
      }
      if (more) {
        hsub2 = hrow2[i + 1];
        if constexpr (DISP) bnext2 = bv[i + 2];
      }
      const E q = shfl(r[sb], il);                   // pivot of N
      const E p = Ar::mul(mw, q);                    // pivot of I - w H
      const E iq = Ar::recip(q);
      if constexpr (DISP) {
        const E si = shfl(sacc[sb], il);
        const E zi = Ar::mul(Ar::add(av[i], Ar::neg(si)), iq);
        zy = Ar::fma(zi, y, zy);
#pragma unroll
        for (int s = sb; s < SMX; ++s) {
          const int j = lane + 32 * s;
          if (s < S && j > i && j < m) sacc[s] = Ar::fma(zi, r[s], sacc[s]);
        }
      }
      const float pr = Ar::re(p), pi = Ar::im(p);
      mn = fminf(mn, pr);
      if (!(pr == pr) || !(pi == pi)) mn = -3.0e38f;
      const float x0 = Ar::re(lp), y0 = Ar::im(lp);
      lp = Ar::mul(lp, p);
      const float x1 = Ar::re(lp), y1 = Ar::im(lp);
      if (x0 < 0.f && x1 < 0.f) wind += (y0 >= 0.f && y1 < 0.f) ? 1 : (y0 < 0.f && y1 >= 0.f) ? -1 : 0;
      if ((il & 7) == 7) e2 += (float)Ar::normalise(lp);
      if (i == m - 1) break;
      const E li = Ar::mul(hsub, iq);
      if constexpr (DISP) y = Ar::fms(bnext, li, y);
#pragma unroll
      for (int s = sb; s < SMX; ++s) {
        const int j = lane + 32 * s;
        if (s < S && j > i && j < m) {
          E h = nx[s];
          if (j == i + 1) h = Ar::add(h, Ar::neg(sg));
          r[s] = Ar::fms(h, li, r[s]);
        }
      }
#pragma unroll
      for (int s = 0; s < SMX; ++s) nx[s] = nx2[s];
      hsub = hsub2;
      bnext = bnext2;
    }
  }
  e2 += (float)Ar::normalise(lp);
  if (lane != 0) return;
  const float TWO_PI = 6.28318530717958647692f;
  const float args = __fadd_rn(rec.meta.x, atan2f(Ar::im(lp), Ar::re(lp)) + TWO_PI * (float)wind);
  E prod = Ar::mul(rec.prod, lp);
  e2 += (float)Ar::normalise(prod);
  // ex = exponent so far + the leaf's term -a^T N^-1 b
  const E ex = DISP ? Ar::add(hv[2 * m], Ar::neg(zy)) : Ar::zero();
  const double LN2 = 0.693147180559945309417232121458;
  const double2 P = Ar::to(prod), X = Ar::to(ex);
  const double r3 = -0.5 * (double)e2 * LN2 + 0.5 * X.x, r4 = 0.5 * X.y;
  if (!a.halve_first) {
    const GridDesc& g = a.grid;
    if (g.e_lo == 0 && g.e_hi == g.n_full) {
      write_record(a, leaf, P, (double)args, r3, r4, (double)mn, false);
    } else {                                         // a shard: its slice only, local indices
      long long inner = 1;                           // evaluated points per level-0 root
      for (int q = 1; q + 1 < g.L; ++q) inner *= g.radix[q];
      const long long e = leaf + (long long)a.k0_lo * inner * g.half;
      if (e >= g.e_lo && e < g.e_hi)
        write_record(a, e - g.e_lo + (g.e_lo > 0 ? 1 : 0), P, (double)args, r3, r4, (double)mn, false);
      if (leaf == 0 && g.e_lo > 0)                   // point 0 (w = 1), for the normalisation
        write_record(a, 0, make_double2(1.0, 0.0), 0.0, a.q1re, a.q1im, a.q1minpiv, false);
    }
    return;
  }
  // the leaf's digits (cnt radices) -> its evaluated point and, where it is the source, the
  // conjugate evaluated point
  const GridDesc& g = a.grid;
  int dig[GBSBIN_MAX_L];
  long long rest = leaf;
  for (int q = g.L - 1; q >= 0; --q) {
    const long long up = rest / a.cnt[q];
    dig[q] = (int)(rest - up * a.cnt[q]);
    rest = up;
  }
  const int RL = g.radix[g.L - 1];
  if (2 * dig[g.L - 1] <= RL) {
    long long e = 0;
    for (int q = 0; q + 1 < g.L; ++q) e = e * g.radix[q] + dig[q];
    write_record(a, e * g.half + dig[g.L - 1], P, (double)args, r3, r4, (double)mn, false);
  }
  if (dig[0] >= 1 && 2 * dig[0] < g.radix[0] && (dig[g.L - 1] == 0 || 2 * dig[g.L - 1] >= RL)) {
    long long e = 0;
    for (int q = 0; q + 1 < g.L; ++q) e = e * g.radix[q] + (dig[q] == 0 ? 0 : g.radix[q] - dig[q]);
    const int cl = dig[g.L - 1] == 0 ? 0 : RL - dig[g.L - 1];
    write_record(a, e * g.half + cl, P, (double)args, r3, r4, (double)mn, true);
  }
}

// ---------------------------------------------------------------------------- launch
size_t top_smem(const BTreeStep& st) { return sizeof(float4) * ((size_t)st.nbs * st.D + st.nbs); }

// Columns of the bottom rows kept in registers: all D, or D rounded down to a multiple of 32
// when the rest (the tail) is cheaper as dot products of the kept multipliers (~280 pair
// operations per tail column against 64 per pivot for a register slot).
int bottom_main_columns(int D, int nbs) {
  const int tail = D % 32;
  if (tail == 0 || D - tail <= nbs || tail * 280 >= nbs * 64) return D;
  return D - tail;
}

template <class Ar, int SMAX>
cudaError_t launch_bottom(const BTreeArgs& a, const BTreeStep& st, long long children, int Dm, int num_sms,
                          cudaStream_t s) {
  const size_t smem = top_smem(st);
  cudaError_t err = cudaSuccess;
  if (smem > 48 * 1024) {
    err = cudaFuncSetAttribute(k_bt_bottom<Ar, SMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bt_bottom<Ar, SMAX>, BOT_WARPS * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  // one CTA per resident slot, each with an even share of all children's rows
  const long long rows = children * (long long)(st.D - st.nbs);
  const long long grid = std::min<long long>((long long)per_sm * num_sms, rows);
  k_bt_bottom<Ar, SMAX><<<(unsigned)grid, BOT_WARPS * 32, smem, s>>>(a, st, Dm, rows);
  return cudaGetLastError();
}

template <class Ar>
cudaError_t launch_btree_ar(const BTreeArgs& a, const BTreeStep* steps, int nsteps, int num_sms, cudaStream_t s,
                            int* launches) {
  cudaError_t err = cudaSuccess;
  *launches = 0;
  for (int q = 0; q < nsteps; ++q) {
    const BTreeStep& st = steps[q];
    long long children = 1;
    for (int l = 0; l <= st.l; ++l) children *= a.cnt[l];
    // few children: split the pivot rows' right-hand columns over several CTAs per child
    const int X = st.D - st.nbs;
    int parts = 1;
    if (2 * children < num_sms) {
      const long long want = (num_sms + children - 1) / children;
      parts = (int)std::max<long long>(1, std::min<long long>(want, (X + 15) / 16));
    }
    const int Wp = (X + parts - 1) / parts;
    parts = (X + Wp - 1) / Wp;                        // no empty part: (parts - 1) Wp < X
    const size_t smem = btree_step_smem_bytes(st.nbs, st.nbs + Wp);
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(k_bt_top<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    k_bt_top<Ar><<<(unsigned)(children * parts), TOP_THREADS, smem, s>>>(a, st, parts, Wp);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int Dm = bottom_main_columns(st.D, st.nbs);
    const int S = (Dm + 31) / 32;
    err = S <= 4    ? launch_bottom<Ar, 4>(a, st, children, Dm, num_sms, s)
          : S <= 8  ? launch_bottom<Ar, 8>(a, st, children, Dm, num_sms, s)
          : S <= 12 ? launch_bottom<Ar, 12>(a, st, children, Dm, num_sms, s)
                    : launch_bottom<Ar, 17>(a, st, children, Dm, num_sms, s);
    if (err != cudaSuccess) return err;
    *launches += 2;
  }
  long long parents = 1;
  for (int l = 0; l + 1 < a.grid.L; ++l) parents *= a.cnt[l];
  const size_t hsmem = btree_hess_smem_bytes(a.mL);
  if (a.mL <= GBSBIN_BT_MAX_HESS) {
    if (hsmem > 48 * 1024) {
      err = cudaFuncSetAttribute(k_bt_hess<Ar, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
      if (err != cudaSuccess) return err;
    }
    k_bt_hess<Ar, false><<<(unsigned)parents, HESS_THREADS, hsmem, s>>>(a);
  } else {
    k_bt_hess<Ar, true><<<(unsigned)parents, HESS_THREADS, hsmem, s>>>(a);
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const long long blocks = (a.n_leaves + LEAF_WARPS - 1) / LEAF_WARPS;
  if (a.mL <= 32 * LEAF_SMAX) {
    if (a.has_gamma) k_bt_leaf<Ar, true, LEAF_SMAX><<<(unsigned)blocks, LEAF_WARPS * 32, 0, s>>>(a);
    else k_bt_leaf<Ar, false, LEAF_SMAX><<<(unsigned)blocks, LEAF_WARPS * 32, 0, s>>>(a);
  } else {
    if (a.has_gamma) k_bt_leaf<Ar, true, LEAF_SMAX_BIG><<<(unsigned)blocks, LEAF_WARPS * 32, 0, s>>>(a);
    else k_bt_leaf<Ar, false, LEAF_SMAX_BIG><<<(unsigned)blocks, LEAF_WARPS * 32, 0, s>>>(a);
  }
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace

size_t btree_step_smem_bytes(int nbs, int D) { return sizeof(float4) * ((size_t)nbs * D + nbs); }
size_t btree_hess_smem_bytes(int m) {
  const size_t vecs = (size_t)m + (m + 2) + m + 2 + HESS_THREADS;
  if (m > GBSBIN_BT_MAX_HESS) return sizeof(float4) * (vecs + 2 * (size_t)m);   // the block in H
  return sizeof(float4) * ((size_t)m * (m + 3) + vecs);
}

cudaError_t launch_points_btree(const BTreeArgs& a, const BTreeStep* steps, int nsteps, bool fp64, int num_sms,
                                cudaStream_t s, int* launches) {
  return fp64 ? launch_btree_ar<ArF64>(a, steps, nsteps, num_sms, s, launches)
              : launch_btree_ar<ArDF>(a, steps, nsteps, num_sms, s, launches);
}

}  // namespace gbsbin
