// The reverse pass along the tree of block eliminations (arXiv:2412.17742, Sec. III Eq. q_d on
// the product grid of Sec. VI; the adjoint follows from d log det A = tr(A^{-1} dA)).
//
// With rows ordered by group, E the rows of groups 0 .. L-2 and F the last group's, the
// per-point matrix M = conj(D) - XA of a grid point splits as [[M_EE, M_EF], [M_FE, M_FF]],
// and only M_FF = conj(w) I - XA_FF depends on the last axis's root w.  For a parent (a
// combination of the first L-1 axes' roots) let A = inv(M_EE), U = A M_EF, V = M_FE A; each
// leaf's Schur complement is S(w) = conj(w) I - C with C = XA_FF - XA_FE U, and
//   inv(M) = [[A + U inv(S) V, -U inv(S)], [-inv(S) V, inv(S)]],
//   x = inv(M) X gamma:  x_F = s = inv(S) c_F,  x_E = a_E - U s   (c_F = b_F - V b_E, a_E = A b_E),
//   y = inv(M)^T gamma:  y_F = t = inv(S)^T d_F,  y_E = e_E - V^T t (d_F = g_F - U^T g_E, e_E = A^T g_E).
// Summed over the parent's leaves with the weights beta, the adjoint 1/2 sum beta (y x^T + inv(M)^T)
// needs only R = sum beta inv(S), Q = sum beta t s^T, sigma_s = sum beta s, sigma_t = sum beta t and
// the beta sum b: with Z = Q + R^T,
//   EE = b (e_E a_E^T + A^T) - e_E (U sigma_s)^T - (V^T sigma_t) a_E^T + V^T Z U^T,
//   EF = e_E sigma_s^T - V^T Z,   FE = sigma_t a_E^T - Z U^T,   FF = Z,
// and 1/2 sum beta (x + X y) from sum beta x = (b a_E - U sigma_s, sigma_s), sum beta y =
// (b e_E - V^T sigma_t, sigma_t).  So a leaf inverts an mF x mF matrix instead of n x n, and the
// parent's O(n^3) products are shared by its leaves.  Three launches per wave of parents: the
// parents' inverse and products, the leaves (each CTA a contiguous run of leaves, its sums per
// parent in its own slots), the parents' assembly into per-CTA partials (in the original row
// order, transposed as the per-point kernel keeps them), reduced once at the end in FP64.
#include <cuda_runtime.h>

#include "gbsbin_backward_tree.h"
#include "gbsbin_device.cuh"
#include "gbsbin_df.cuh"
#include "gbsbin_gj.cuh"

namespace gbsbin {
namespace {

constexpr int kBtThreads = 256;

// The block-row buffer (nb x n) after the kernels' other shared arrays.
__host__ __device__ __forceinline__ size_t backward_tree_rn_offset(int n, int nb) {
  return (size_t)16 * ((size_t)2 * n * nb + (size_t)nb * nb + 4 * (size_t)n + 1) + sizeof(double2) * GBSBIN_MAX_L;
}

struct Parent {                    // the parent's slot in pbuf
  template <class E>
  __device__ static void map(E* P, int mE, int mF, E** A, E** U, E** V, E** C, E** aE, E** eE, E** cF, E** dF) {
    *A = P;
    *U = *A + mE * mE;
    *V = *U + mE * mF;
    *C = *V + mF * mE;
    *aE = *C + mF * mF;
    *eE = *aE + mE;
    *cF = *eE + mE;
    *dF = *cF + mF;
  }
};

__device__ __forceinline__ int group_of(const BwdTree& t, int a) {
  int l = 0;
  while (l + 1 < t.L && a >= t.goff[l + 1]) ++l;
  return l;
}

// Per parent: A = inv(M_EE), U = -A XA_EF, V = -XA_FE A, C = XA_FF - XA_FE U and the vectors.
template <class Ar>
__global__ void __launch_bounds__(kBtThreads) k_bwdt_parent(BackwardArgs b, BwdTree t) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = b.n, nb = b.nb, mE = t.mE, mF = t.mF, D = t.D, tid = threadIdx.x, NT = kBtThreads;
  E* Pc = reinterpret_cast<E*>(smem);
  E* Rx = Pc + (size_t)n * nb;
  E* Dg = Rx + (size_t)nb * n;
  double2* wr = reinterpret_cast<double2*>(Dg + nb * nb);
  const E* A0 = reinterpret_cast<const E*>(t.A0);
  for (long long p = t.p0 + blockIdx.x; p < t.p1; p += gridDim.x) {
    E *A, *U, *V, *C, *aE, *eE, *cF, *dF;
    Parent::map(reinterpret_cast<E*>(t.pbuf) + (size_t)(p - t.p0) * t.pstride, mE, mF, &A, &U, &V, &C, &aE, &eE,
                &cF, &dF);
    if (tid < t.L - 1) wr[tid] = grid_root(b.tw, b.grid, tid, point_digit(p * t.half, b.grid, tid));
    __syncthreads();
    for (int q = tid; q < mE * mE; q += NT) {        // M_EE = conj(D_E) - XA_EE
      const int i = q / mE, j = q - (q / mE) * mE;
      E v = Ar::neg(A0[(size_t)i * D + j]);
      if (i == j) {
        const double2 w = wr[group_of(t, i)];
        v = Ar::add(v, Ar::from(make_double2(w.x, -w.y)));
      }
      A[q] = v;
    }
    __syncthreads();
    gj_invert<Ar>(A, mE, mE, nb, Pc, Rx, Dg, t.rn ? reinterpret_cast<E*>(smem + backward_tree_rn_offset(n, nb)) : nullptr);
    // U = -A XA_EF, V = -XA_FE A, C = XA_FF - XA_FE U
    gemm_staged<Ar>(U, mF, A, mE, 1, A0 + mE, D, 1, mE, mF, mE, false, true, nb, Pc, Rx);
    gemm_staged<Ar>(V, mE, A0 + (size_t)mE * D, D, 1, A, mE, 1, mF, mE, mE, false, true, nb, Pc, Rx);
    for (int q = tid; q < mF * mF; q += NT) C[q] = A0[(size_t)(mE + q / mF) * D + mE + q % mF];
    __syncthreads();
    gemm_staged<Ar>(C, mF, A0 + (size_t)mE * D, D, 1, U, mF, 1, mF, mF, mE, true, true, nb, Pc, Rx);
    // a_E = A b_E, e_E = A^T g_E (b = X gamma: column n; g = gamma: row n)
    for (int i = tid; i < mE; i += NT) {
      E sa = Ar::zero(), se = Ar::zero();
      for (int k = 0; k < mE; ++k) {
        sa = Ar::fma(A[(size_t)i * mE + k], A0[(size_t)k * D + n], sa);
        se = Ar::fma(A[(size_t)k * mE + i], A0[(size_t)n * D + k], se);
      }
      aE[i] = sa;
      eE[i] = se;
    }
    // c_F = b_F - V b_E, d_F = g_F - U^T g_E
    for (int f = tid; f < mF; f += NT) {
      E sc = A0[(size_t)(mE + f) * D + n], sd = A0[(size_t)n * D + mE + f];
      for (int k = 0; k < mE; ++k) {
        sc = Ar::fms(sc, V[(size_t)f * mE + k], A0[(size_t)k * D + n]);
        sd = Ar::fms(sd, U[(size_t)k * mF + f], A0[(size_t)n * D + k]);
      }
      cF[f] = sc;
      dF[f] = sd;
    }
    __syncthreads();
  }
}

// Leaves: CTA c takes leaves [c per, (c + 1) per) of the wave (parent-major); per leaf
// inv(S(w)), s, t and the sums into the slot of (c, parent).
template <class Ar>
__global__ void __launch_bounds__(kBwdLeafThreads, 2) k_bwdt_leaf(BackwardArgs b, BwdTree t) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char smem[];
  // shared memory sized by mF (backward_leaf_smem_bytes): two CTAs of four warps per SM, so
  // that one leaf's barriers overlap another's arithmetic
  const int mE = t.mE, mF = t.mF, nb = kBwdLeafNb, tid = threadIdx.x, NT = kBwdLeafThreads;
  E* Pc = reinterpret_cast<E*>(smem);
  E* Rx = Pc + (size_t)mF * nb;
  E* Rnb = Rx + (size_t)nb * mF;
  E* Dg = Rnb + (size_t)nb * mF;
  E* cFs = Dg + nb * nb;
  E* dFs = cFs + mF;
  E* sv = dFs + mF;
  E* tv = sv + mF;
  const int per_slot = t.leaf_ctas > b.nparts ? 2 : 1;   // leaf CTAs sharing one n x n slot
  E* W = reinterpret_cast<E*>(reinterpret_cast<char*>(b.ws) + (size_t)(blockIdx.x / per_slot) * (size_t)b.ws_slot_bytes) +
         (size_t)(blockIdx.x % per_slot) * mF * mF;
  const long long nleaves = (t.p1 - t.p0) * t.half;
  const long long l0 = (long long)blockIdx.x * t.per, l1 = min(l0 + t.per, nleaves);
  const long long pfirst = l0 / t.half;
  long long cur = -1;
  E* Cp = nullptr;
  for (long long l = l0; l < l1; ++l) {
    const long long pr = l / t.half, kl = l - pr * t.half;
    E* part = reinterpret_cast<E*>(t.part) + ((size_t)blockIdx.x * t.maxspan + (size_t)(pr - pfirst)) * t.lstride;
    E* R = part;
    E* Q = R + mF * mF;
    E* ss = Q + mF * mF;
    E* st = ss + mF;
    E* bb = st + mF;
    if (pr != cur) {                                   // a new parent: zero its sums, load c_F, d_F
      E *A, *U, *V, *aE, *eE, *cF, *dF;
      Parent::map(reinterpret_cast<E*>(t.pbuf) + (size_t)pr * t.pstride, mE, mF, &A, &U, &V, &Cp, &aE, &eE, &cF,
                  &dF);
      for (long long q = tid; q < t.lstride; q += NT) part[q] = Ar::zero();
      for (int f = tid; f < mF; f += NT) {
        cFs[f] = cF[f];
        dFs[f] = dF[f];
      }
      cur = pr;
      __syncthreads();
    }
    const long long e = (t.p0 + pr) * t.half + kl;
    const double2 beta = b.beta[e];
    if (beta.x == 0.0 && beta.y == 0.0) continue;
    const double2 w = grid_root(b.tw, b.grid, t.L - 1, (int)kl);
    for (int q = tid; q < mF * mF; q += NT) {        // S = conj(w) I - C
      const int i = q / mF, j = q - (q / mF) * mF;
      E v = Ar::neg(Cp[q]);
      if (i == j) v = Ar::add(v, Ar::from(make_double2(w.x, -w.y)));
      W[q] = v;
    }
    __syncthreads();
    gj_invert<Ar>(W, mF, mF, nb, Pc, Rx, Dg, Rnb);
    {                                                  // s = inv(S) c_F (warp per row), t = inv(S)^T d_F
      const int lane = tid & 31, warp = tid >> 5;
      for (int i = warp; i < mF; i += NT / 32) {
        E acc = Ar::zero();
        for (int j = lane; j < mF; j += 32) acc = Ar::fma(W[(size_t)i * mF + j], cFs[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = Ar::add(acc, shfl_xor(acc, o));
        if (lane == 0) sv[i] = acc;
      }
      for (int j = tid; j < mF; j += NT) {
        E acc = Ar::zero();
        for (int i = 0; i < mF; ++i) acc = Ar::fma(W[(size_t)i * mF + j], dFs[i], acc);
        tv[j] = acc;
      }
    }
    __syncthreads();
    const E be = Ar::from(beta);
    for (int q = tid; q < mF * mF; q += NT) {
      const int i = q / mF, j = q - (q / mF) * mF;
      R[q] = Ar::fma(be, W[q], R[q]);
      Q[q] = Ar::fma(be, Ar::mul(tv[i], sv[j]), Q[q]);
    }
    for (int f = tid; f < mF; f += NT) {
      ss[f] = Ar::fma(be, sv[f], ss[f]);
      st[f] = Ar::fma(be, tv[f], st[f]);
    }
    if (tid == 0) bb[0] = Ar::add(bb[0], be);
    __syncthreads();
  }
}

// Per parent: the leaves' sums, Z = Q + R^T, the three products, and 1/2 (Phi + Psi^T) into this
// CTA's partials in the original row order (ST[j][i] = S[i][j]).
template <class Ar>
__global__ void __launch_bounds__(kBtThreads) k_bwdt_assemble(BackwardArgs b, BwdTree t) {
  using E = typename Ar::E;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = b.n, nb = b.nb, mE = t.mE, mF = t.mF, tid = threadIdx.x, NT = kBtThreads;
  E* Pc = reinterpret_cast<E*>(smem);
  E* Rx = Pc + (size_t)n * nb;
  E* Dg = Rx + (size_t)nb * n;
  E* ss = Dg + nb * nb;
  E* st = ss + mF;
  E* uS = st + mF;
  E* vT = uS + mE;
  E* bbs = vT + mE;
  E* ST = reinterpret_cast<E*>(b.partS) + (size_t)blockIdx.x * n * n;
  E* sg = reinterpret_cast<E*>(b.partg) + (size_t)blockIdx.x * n;
  E* W = reinterpret_cast<E*>(reinterpret_cast<char*>(b.ws) + (size_t)blockIdx.x * (size_t)b.ws_slot_bytes);
  E* Z = W;
  E* X1 = Z + mF * mF;                                 // Z U^T (mF x mE)
  E* X2 = X1 + mF * mE;                                // V^T Z U^T (mE x mE)
  E* X3 = X2 + mE * mE;                                // V^T Z (mE x mF)
  if (t.zero_partials) {
    for (long long q = tid; q < (long long)n * n; q += NT) ST[q] = Ar::zero();
    for (int q = tid; q < n; q += NT) sg[q] = Ar::zero();
  }
  for (long long p = t.p0 + blockIdx.x; p < t.p1; p += gridDim.x) {
    const long long pr = p - t.p0;
    E *A, *U, *V, *C, *aE, *eE, *cF, *dF;
    Parent::map(reinterpret_cast<E*>(t.pbuf) + (size_t)pr * t.pstride, mE, mF, &A, &U, &V, &C, &aE, &eE, &cF, &dF);
    const long long c0 = (pr * t.half) / t.per, c1 = (pr * t.half + t.half - 1) / t.per;
    for (int q = tid; q < mF * mF; q += NT) {
      const int i = q / mF, j = q - (q / mF) * mF;
      E z = Ar::zero();
      for (long long c = c0; c <= c1; ++c) {
        const E* part = reinterpret_cast<const E*>(t.part) +
                        ((size_t)c * t.maxspan + (size_t)(pr - (c * t.per) / t.half)) * t.lstride;
        z = Ar::add(z, Ar::add(part[mF * mF + q], part[(size_t)j * mF + i]));   // Q + R^T
      }
      Z[q] = z;
    }
    for (int f = tid; f < 2 * mF + 1; f += NT) {
      E v = Ar::zero();
      for (long long c = c0; c <= c1; ++c) {
        const E* part = reinterpret_cast<const E*>(t.part) +
                        ((size_t)c * t.maxspan + (size_t)(pr - (c * t.per) / t.half)) * t.lstride;
        v = Ar::add(v, part[2 * mF * mF + f]);
      }
      if (f < mF) ss[f] = v;
      else if (f < 2 * mF) st[f - mF] = v;
      else bbs[0] = v;
    }
    __syncthreads();
    gemm_staged<Ar>(X1, mE, Z, mF, 1, U, 1, mF, mF, mE, mF, false, false, nb, Pc, Rx);
    gemm_staged<Ar>(X2, mE, V, 1, mE, X1, mE, 1, mE, mE, mF, false, false, nb, Pc, Rx);
    gemm_staged<Ar>(X3, mF, V, 1, mE, Z, mF, 1, mE, mF, mF, false, false, nb, Pc, Rx);
    for (int i = tid; i < mE; i += NT) {             // U sigma_s, V^T sigma_t
      E su = Ar::zero(), sv = Ar::zero();
      for (int k = 0; k < mF; ++k) {
        su = Ar::fma(U[(size_t)i * mF + k], ss[k], su);
        sv = Ar::fma(V[(size_t)k * mE + i], st[k], sv);
      }
      uS[i] = su;
      vT[i] = sv;
    }
    __syncthreads();
    const E bsum = bbs[0];
    const E half = Ar::from(make_double2(0.5, 0.0));
    for (long long q = tid; q < (long long)n * n; q += NT) {
      const int jo = (int)(q / n), io = (int)(q - (q / n) * n);   // ST[jo][io] = S[io][jo]
      const int a = t.pinv[io], c = t.pinv[jo];
      E v;
      if (a < mE && c < mE)
        v = Ar::add(Ar::fma(bsum, Ar::add(Ar::mul(eE[a], aE[c]), A[(size_t)c * mE + a]),
                            Ar::neg(Ar::add(Ar::mul(eE[a], uS[c]), Ar::mul(vT[a], aE[c])))),
                    X2[(size_t)a * mE + c]);
      else if (a < mE)
        v = Ar::fms(Ar::mul(eE[a], ss[c - mE]), Ar::one(), X3[(size_t)a * mF + (c - mE)]);
      else if (c < mE)
        v = Ar::fms(Ar::mul(st[a - mE], aE[c]), Ar::one(), X1[(size_t)(a - mE) * mE + c]);
      else
        v = Z[(size_t)(a - mE) * mF + (c - mE)];
      ST[q] = Ar::fma(half, v, ST[q]);
    }
    for (int io = tid; io < n; io += NT) {           // 1/2 (sum beta x + X sum beta y)
      const int h = n / 2, po = io < h ? io + h : io - h;
      const int a = t.pinv[io], ap = t.pinv[po];
      const E xs = a < mE ? Ar::fms(Ar::mul(bsum, aE[a]), Ar::one(), uS[a]) : ss[a - mE];
      const E ys = ap < mE ? Ar::fms(Ar::mul(bsum, eE[ap]), Ar::one(), vT[ap]) : st[ap - mE];
      sg[io] = Ar::fma(half, Ar::add(xs, ys), sg[io]);
    }
    __syncthreads();
  }
}

template <class Ar>
cudaError_t tree_wave(const BackwardArgs& b, const BwdTree& t0, cudaStream_t s) {
  BwdTree t = t0;
  const size_t base = backward_tree_smem_bytes(b.n, b.nb), with = base + (size_t)16 * b.nb * b.n;
  t.rn = with <= 226 * 1024 ? 1 : 0;
  const size_t smem = t.rn ? with : base;
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(k_bwdt_parent<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess ||
      (err = cudaFuncSetAttribute(k_bwdt_assemble<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return err;
  const long long parents = t.p1 - t.p0;
  const long long gp = parents < b.nparts ? parents : b.nparts;
  k_bwdt_parent<Ar><<<(unsigned)gp, kBtThreads, smem, s>>>(b, t);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const long long nleaves = parents * t.half;
  const long long gl = (nleaves + t.per - 1) / t.per;
  const size_t lsmem = backward_leaf_smem_bytes(t.mF);
  if ((err = cudaFuncSetAttribute(k_bwdt_leaf<Ar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem)) !=
      cudaSuccess)
    return err;
  k_bwdt_leaf<Ar><<<(unsigned)gl, kBwdLeafThreads, lsmem, s>>>(b, t);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_bwdt_assemble<Ar><<<(unsigned)t.nparts, kBtThreads, smem, s>>>(b, t);
  return cudaGetLastError();
}

}  // namespace

size_t backward_leaf_smem_bytes(int mF) {
  return (size_t)16 * ((size_t)3 * mF * kBwdLeafNb + (size_t)kBwdLeafNb * kBwdLeafNb + 4 * (size_t)mF);
}

size_t backward_tree_smem_bytes(int n, int nb) {
  return (size_t)16 * ((size_t)2 * n * nb + (size_t)nb * nb + 4 * (size_t)n + 1) + sizeof(double2) * GBSBIN_MAX_L;
}

cudaError_t launch_backward_tree_wave(const BackwardArgs& b, const BwdTree& t, cudaStream_t s) {
  return b.df ? tree_wave<ArDF>(b, t, s) : tree_wave<ArF64>(b, t, s);
}

}  // namespace gbsbin
