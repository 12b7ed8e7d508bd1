// The reverse pass along the tree of block eliminations (gbsbin_backward_tree.cu) and the
// split of the per-point reverse pass (gbsbin_backward.cu) into its stages.  Not part of the
// public ABI.
#pragma once

#include "gbsbin_internal.h"

namespace gbsbin {

// Rows ordered by group (the large-matrix tree's permutation): E = the rows of groups
// 0 .. L-2 (mE), F = the last group's (mF).  A parent is a combination of the first L-1 axes'
// roots; its leaves are the evaluated roots of the last axis (half of them).
struct BwdTree {
  int L;
  int mE, mF;
  int D;                    // row stride of the permuted augmented state (n + 1)
  const void* A0;           // permuted state in the plan's arithmetic: XA (n x n, stride D),
                            // X gamma in column n, gamma in row n
  const int* pinv;          // [n] original row -> permuted row
  int goff[GBSBIN_MAX_L + 1];   // first permuted row of each group
  long long half;           // leaves per parent
  long long p0, p1;         // the parents of this wave
  void* pbuf;               // (p1 - p0) x pstride: inv(M_EE), U, V, C, a_E, e_E, c_F, d_F
  long long pstride;        // n^2 + 2 n
  void* part;               // leaf partials: leaf CTAs x maxspan x lstride
  long long lstride;        // 2 mF^2 + 2 mF + 1: R, Q, sigma_s, sigma_t, beta sum
  int per;                  // leaves per CTA of the leaf launch
  int maxspan;              // parents one leaf CTA can touch
  int nparts;               // CTAs of the assembly launch (its partials)
  int zero_partials;        // first wave: the assembly zeroes its partials
  int rn;                   // the kernels' shared memory holds the block-row buffer (nb x n)
  int leaf_ctas;            // CTAs of the leaf launch: two per SM (128 threads each) where two
                            // mF x mF slots fit in an SM's n x n workspace slot, else one
};
constexpr int kBwdLeafThreads = 128;
constexpr int kBwdLeafNb = 8;             // pivots per Gauss-Jordan step in the leaves (nb^2 <= 128)

// Adjoint of the inverse DFT and the per-point weights beta (into b.bufB); *beta receives it.
cudaError_t launch_backward_weights(const BackwardArgs& b, const double* dLdP, cudaStream_t s, const double2** beta);
// The per-point kernel and the reduce over its CTAs (b.beta set).
cudaError_t launch_backward_points(const BackwardArgs& b, cudaStream_t s);
// One wave of the tree's reverse pass: the parents' products, the leaves' inverses and sums,
// the parents' assembly into the partials (b.beta set).
cudaError_t launch_backward_tree_wave(const BackwardArgs& b, const BwdTree& t, cudaStream_t s);
// outS, outg from the first nparts partials.
cudaError_t launch_backward_reduce(const BackwardArgs& b, int nparts, cudaStream_t s);
size_t backward_tree_smem_bytes(int n, int nb);
size_t backward_leaf_smem_bytes(int mF);

}  // namespace gbsbin
