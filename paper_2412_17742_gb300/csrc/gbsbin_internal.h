// Internal interface between the host plan (gbsbin_host.cpp) and the kernels
// (gbsbin_points.cu, gbsbin_dft.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gbsbin.h"

#define GBSBIN_MAX_L 16
// Largest n whose n x n complex matrix (and, for the FP32 path, its residual) fits in
// one CTA's shared memory next to the small vectors.
#define GBSBIN_SMEM_MAX_N 112
// Blocks of the diagnostics reduction of the multi-launch DFT; the host finishes the sum
// over the partials.  The diagnostics array holds GBSBIN_DIAG_SLOTS partials of 4 doubles
// (sum of P, max |Im| of the self-conjugate entries, min pivot real part, bad points), then
// Re log q(1), the grid-barrier error flag and the number of partials written.
#define GBSBIN_DIAG_BLOCKS 64
#define GBSBIN_DIAG_SLOTS 1024
#define GBSBIN_DIAG_DOUBLES (4 * GBSBIN_DIAG_SLOTS + 4)
// Fixed-point scale of the integer copy of -XA used by the exact integer residual.
#define GBSBIN_FIX_BITS 62

namespace gbsbin {

// Roots-of-unity grid.  Axis l has radix[l] = oversample (N_l + 1) points; by conjugate
// symmetry G(omega^-k) = conj G(omega^k) only half = radix[L-1]/2 + 1 values of the
// last axis are evaluated (all values of the other axes).
struct GridDesc {
  int L;
  int radix[GBSBIN_MAX_L];
  int nout[GBSBIN_MAX_L];   // N_l + 1: table extent per axis
  int half;
  long long n_eval;         // points this plan evaluates: (npts / radix[L-1]) * half, or for a
                            // shard 1 + (e_hi - e_lo) (point 0 first, then the slice)
  long long npts;
  long long n_full;         // (npts / radix[L-1]) * half: the whole evaluated half grid
  long long e_lo, e_hi;     // the shard [e_lo, e_hi) of the half grid (0, n_full: no shard)
};

struct PointArgs {
  int n;
  int has_gamma;
  int P;                    // grid points per CTA (power of two)
  int logP;
  const double2* NXA;       // n*n FP64, row-major: -XA (the off-diagonal part of conj(D) - XA)
  const double2* Xgamma;    // n: X gamma = Sigma^{-1} z-bar
  const double2* gamma;     // n
  const float2* NXA_hi;     // n*n: -XA rounded to FP32
  const float2* NXA_lo;     // n*n: (-XA) - NXA_hi rounded to FP32
  const longlong2* NXA_fix; // n*n: -XA in fixed point, round(-XA * 2^GBSBIN_FIX_BITS) (|XA_ij| < 1)
  const float2* Xg_hi;      // n
  const float2* Xg_lo;      // n
  const float2* g_hi;       // n
  const float2* g_lo;       // n
  const int* label;         // n: detector group of each row
  const double2* tw;        // twiddles exp(-2 pi i m / radix[l]), m < radix[l], axis after axis
  const double2* H;         // one-group plans: Hessenberg form of XA, n*n FP64 (else nullptr)
  GridDesc grid;
  double2* logq;            // n_eval outputs: log q at each evaluated point
  double* minpiv;           // n_eval outputs: min_i Re u_ii
  void* gws;                // L2-resident workspace for the global-memory variants
  long long gws_slot_bytes; // bytes of one CTA's slot
  double* ldfin;            // warp kernel only: n_eval x 6 doubles (the product of the
                            // pivots d_i u'_ii re/im, the FP32 sum of their arguments, the
                            // rest of log q re/im, unused); log q is finished by the DFT
};

// A batch of problems for one point-kernel launch: jobs are (problem, first point) groups
// taken in order from an atomic counter (reset to 0 before every launch).
struct PointJob {
  int prob;
  int pad;
  long long e0;
};
struct PointBatch {
  const PointArgs* probs;   // device array of per-problem descriptors (nullptr: single problem)
  const PointJob* jobs;     // device array
  long long njobs;
  unsigned long long* queue;
};

#define GBSBIN_BWD_MAX_NB 16         // pivots per blocked Gauss-Jordan step (n <= 320; 8 above)
struct BackwardArgs {
  int n;
  int df;                   // nonzero: the per-point inverse in pairs of FP32, else FP64
  int nb;                   // pivots per Gauss-Jordan step (backward_block(n))
  int rn;                   // set by the launcher: shared memory holds the block-row buffer
  GridDesc grid;
  long long n_eval;
  const double2* NXA;       // n*n: -XA
  const double2* Xgamma;    // n
  const int* label;         // n: detector group of each row
  const double2* gamma;     // n
  const double2* logq;      // n_eval
  const double2* tw;        // twiddles, as for the DFT
  double2* bufA;            // max(table, n_eval) complex scratch
  double2* bufB;            // max(table, n_eval) complex scratch
  const double2* beta;      // set by the launcher
  void* ws;                 // nparts slots of n*n complex (16 bytes an entry)
  long long ws_slot_bytes;
  void* partS;              // nparts x n*n, 16 bytes an entry (FP64 or FP32 pairs), transposed
  void* partg;              // nparts x n, the same
  int nparts;
  double2* outS;            // n*n: dL/dXA (bilinear)
  double2* outg;            // n: dL/dgamma (bilinear)
  cudaEvent_t ev0, ev1;     // optional: recorded around the per-point kernel
};
size_t backward_smem_bytes(int n, int nb);
int backward_block(int n);

struct DftArgs {
  GridDesc grid;
  int g_ready;              // bufA already holds G on the evaluated half grid: no first stage
  const double2* parts;     // non-null: G is given as nparts partial sums per half-grid point
                            // (parts[r * n_full + t]); the transform uses pscale * their sum
                            // (summed in order r = 0, 1, ...) instead of exp(log q - log q_0)
  long long nparts;
  double pscale;
  const double2* logq;      // n_eval
  const double* ldfin;      // nullptr, or the warp kernel's unfinished log det (see PointArgs)
  double2* logq_fin;        // with ldfin: where the finished log q go (n_eval)
  const double2* tw;        // concatenated exp(-2 pi i m / radix[l]), m < radix[l]
  double2* bufA;            // n_eval complex scratch
  double2* bufB;            // n_eval complex scratch
  double* P;                // table out (prod nout doubles)
  double* diag;             // GBSBIN_DIAG_DOUBLES: partial reductions (see above), or nullptr
  const double* minpiv;     // n_eval
  long long table_size;
  int df;                   // nonzero: the two-phase transform (where it applies) in pairs of
                            // FP32 (plans whose points are computed in pairs of FP32)
  int g_df;                 // with g_ready and df: bufA holds G as pairs of FP32 (float4)
};

// Tree of block eliminations over the grid (gbsbin_points_tree.cu), in pairs of FP32
// (float4 = hi re, hi im, lo re, lo im) or in FP64 (double2 in the same 16-byte slots):
// rows ordered by group; depth l holds one reduced matrix A' per combination of the first
// l axes' roots (A[l]: nodes x m[l] x m[l], row-major; c, u: the displacement vectors;
// path: 3 slots per node - pivot product, (argument sum, power of two, smallest pivot
// real part, -) as FP32, exponent sum).  Depth 0 is the permuted state.  Leaves (depth L - 1, last axis halved) write the unfinished log q of
// every evaluated point to ldfin (FP64).
struct TreeArgs {
  int has_gamma;
  int nb[GBSBIN_MAX_L];     // rows of group l
  int m[GBSBIN_MAX_L];      // size of the reduced matrices at depth l (m[0] = n)
  float4* A[GBSBIN_MAX_L];
  float4* c[GBSBIN_MAX_L];
  float4* u[GBSBIN_MAX_L];
  float4* path[GBSBIN_MAX_L];
  const double2* tw;
  const float4* twdf;       // the same roots w = exp(2 pi i k / R_l) as pairs of FP32 (the pair
                            // kernels read these instead of converting FP64 twiddles)
  GridDesc grid;
  double* ldfin;
  double* minpiv;
  // undisplaced plans: the leaves also write G = q / q(1) per evaluated point to gout, from
  // the pivot product P0 = p0 2^e0 of I - XA (host FP64, same row order), its argument
  // p0arg and winding m0 (log det(I - XA) = log|P0| + e0 log 2 + i (p0arg + 2 pi m0))
  double2* gout;
  int gout_df;              // nonzero (pairs plans whose DFT runs in pairs): G stored as a pair
                            // of FP32 (float4) in the 16-byte slots of gout
  double p0re, p0im;
  float4 p0df;              // p0 as a pair of FP32
  float p0arg, e0, m0;
};
// Tree of block eliminations for large matrices with Hessenberg leaves
// (gbsbin_points_btree.cu), in pairs of FP32 or FP64 (16-byte elements either way).  Depth d
// holds one augmented matrix [[A, c], [u^T, ex]] ((m_d + 1)^2 elements) per combination of
// the first d axes' roots, and a path record (pivot product; FP32 argument sum, power of
// two, smallest pivot real part).  Level l runs as sub-steps of nbs pivots of its group,
// each a top launch (CTA per child) and a bottom launch (CTAs per row chunk); the last
// group's blocks are reduced to Hessenberg form (a CTA per leaf parent) and every evaluated
// point is an O(m^2) Hessenberg elimination (a warp per point) writing the unfinished log q.
#define GBSBIN_BT_MAX_HESS 116          // largest last group reduced in shared memory (225 KB at 116)
#define GBSBIN_BT_MAX_LAST 192          // largest last group (above 116 rows the reduction works
                                        // in the plan's Hessenberg buffer, through L2)
#define GBSBIN_BT_SMEM (200 * 1024)     // shared-memory budget of one sub-step's pivot rows
#define GBSBIN_BT_MAX_NBS 128           // pivots of one sub-step (at most)
struct BTreeStep {
  int l;                    // level: the grid axis whose roots this sub-step applies
  int first;                // first sub-step of the level: input is the parent's matrix at depth l
  int nbg;                  // rows of the level's group (the G form of the first sub-step)
  int nbs;                  // pivots eliminated by this sub-step
  int D;                    // dimension of the input matrix (augmented)
  const float4* in;         // later sub-steps: the previous trailing blocks, one per child
  float4* out;              // trailing blocks (D - nbs)^2 per child: depth l + 1 after the last sub-step
};
struct BTreeArgs {
  int L;
  int has_gamma;
  int mL;                   // rows of the last group
  int cnt[GBSBIN_MAX_L];    // roots of axis l the tree takes: child = parent * cnt[l] + k.  Either
                            // every axis in full but the last halved (leaf = evaluated point), or
                            // the first halved (cnt[0] = radix[0] / 2 + 1) and the rest in full,
                            // which halves every level's nodes: each leaf k then writes its
                            // evaluated point when k_{L-1} <= radix[L-1] / 2 and the conjugate
                            // point -k (conjugated record) when 1 <= k_0 < radix[0] / 2 and
                            // k_{L-1} = 0 or 2 k_{L-1} >= radix[L-1], so every evaluated point of
                            // the half grid is written exactly once
  int halve_first;
  long long n_leaves;       // leaves: prod cnt[l]
  // a shard (last axis halved): level 0 takes the roots k0_lo .. k0_lo + cnt[0] - 1, and the
  // leaves write only the evaluated points of the grid's slice [e_lo, e_hi) (grid), at their
  // local index; with e_lo > 0 the first leaf also writes point 0's record from log q(1),
  // computed on the host
  int k0_lo;
  double q1re, q1im, q1minpiv;
  GridDesc grid;
  const double2* tw;
  const float4* twdf;
  float4* mat[GBSBIN_MAX_L];
  float4* path[GBSBIN_MAX_L];
  float4* U;                // per child of the current sub-step: nbs x D pivot rows
  float4* inv;              // per child: nbs reciprocal pivots
  float4* H;                // per leaf parent: mL x mL Hessenberg form
  float4* hv;               // per leaf parent: a = Q^T u (mL), b = Q^H c (mL), the exponent so far
  double* ldfin;
  double* minpiv;
};
size_t btree_step_smem_bytes(int nbs, int D);
size_t btree_hess_smem_bytes(int m);
cudaError_t launch_points_btree(const BTreeArgs& a, const BTreeStep* steps, int nsteps, bool fp64, int num_sms,
                                cudaStream_t s, int* launches);
size_t tree_level_smem_bytes(int nb, int m);
int tree_leaf_threads(int n);   // lanes per leaf (0: no kernel for a last group of n rows)
cudaError_t launch_points_tree(const TreeArgs& a, bool fp64, int num_sms, cudaStream_t s, int* launches);

// Fock inputs through a lossy circuit (gbsbin_fock.cu).  nin occupied inputs in position
// order (position 0 is the held input, x = 1; positions 1..nd are the Gray digits); per
// node x of the roots-of-unity grid the state is st_m = coef_m x (m = 0: I - T^dag T,
// m = 1 + l: T_l^dag T_l, all restricted to the occupied inputs), and at output-group
// point z the node contributes w(x) prod_j (st_0 + sum_l z_l st_{1+l})_j^{p_j}.
#define GBSBIN_FOCK_MAX_IN 32
#define GBSBIN_FOCK_MAX_L 8
struct FockArgs {
  int nin, L, nd;
  int rsum;                          // sum of the group radices
  int pw[GBSBIN_FOCK_MAX_IN];        // photons per position
  int drad[GBSBIN_FOCK_MAX_IN];      // radix p + 1 of digit d (position d + 1)
  int doff[GBSBIN_FOCK_MAX_IN];      // offset of digit d's roots in xtw
  long long dstride[GBSBIN_FOCK_MAX_IN + 1];   // prod_{d' < d} drad[d']
  int roff[GBSBIN_FOCK_MAX_L + 1];   // offset of group l's rows in the table (sum of radices)
  long long S;                       // nodes: dstride[nd]
  long long x_lo, x_hi;              // the nodes this plan walks (a shard: a subrange of [0, S))
  long long chunk, nchunks;          // Gray steps per restart, restarts over [x_lo, x_hi)
  const double2* coef;               // (L + 1) x nin x nin, [m][k][j] (column k contiguous)
  const float4* coef_df;             // the same as (hi re, hi im, lo re, lo im)
  const double2* xtw;                // exp(2 pi i g / drad[d]), g < drad[d], digit after digit
  const float4* xtw_df;
  const float4* zr_df;               // exp(2 pi i c / radix[l]), c < radix[l], group after group
  const double2* zr;
  GridDesc grid;                     // output-group grid (half of the last axis)
  int xr;                            // CTAs along the nodes (restarts dealt cyclically)
  double2* parts;                    // xr x n_full partial sums
};
#define GBSBIN_FOCK_THREADS 128
int fock_points_per_thread(bool df, long long n_full);   // output-group points per thread
size_t fock_smem_bytes(int nin, int L, int rsum);
int fock_ctas_per_sm(bool df, int zt, size_t smem);      // 0: does not fit
cudaError_t launch_fock(const FockArgs& a, bool df, int zt, cudaStream_t s);

// Kernel launchers (return the launch error).
cudaError_t launch_points(const PointArgs& a, int kernel, int num_sms, cudaStream_t s);
cudaError_t launch_points_warp(const PointArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_points_batch(const PointBatch& batch, int kernel, int threads, size_t smem, int num_sms,
                                cudaStream_t s);
cudaError_t launch_points_warp_batch(const PointBatch& batch, int np, int num_sms, cudaStream_t s);
// Blocked large-n FP32 + refinement kernel (gbsbin_points_blk.cu); n <= GBSBIN_BLK_MAX_N.
#define GBSBIN_BLK_MAX_N 384
#define GBSBIN_BLK_CTAS_PER_SM 2
size_t points_blk_smem_bytes(int n);
size_t points_blk_slot_bytes(int n);
int points_blk_ctas_per_sm(int n);   // resident CTAs per SM that the shared memory allows (1 or 2)
cudaError_t launch_points_blk(const PointArgs& a, const PointBatch& batch, size_t smem_batch, int num_sms,
                              cudaStream_t s, bool tensor_cores);
// One-group (L = 1) undisplaced kernel (gbsbin_points_hess.cu): warp per point, four
// points per CTA; batch jobs are groups of four consecutive points of one problem.
// slots: row slots per lane of the instantiation (hess_slots(n) for the largest n it serves;
// 0: from a.n)
cudaError_t launch_points_hess(const PointArgs& a, const PointBatch& batch, int slots, int num_sms, cudaStream_t s,
                               bool df);
int hess_slots(int n);
size_t points_smem_bytes(int kernel, int n, int P, int L);
size_t points_matrix_bytes(int kernel, int n, int P);
int points_per_cta(int kernel, int n, int L);
int points_threads(int kernel, int n);
cudaError_t launch_dft(const DftArgs& a, cudaStream_t s);
// log q of n evaluated points from the unfinished form (ldfin) - for plans whose DFT took G
// directly and did not finish them.
cudaError_t launch_finish_logq(const double* ldfin, double2* logq, long long n, cudaStream_t s);
// All DFT stages and the diagnostics in one cooperative launch; bar: 4 zeroed unsigned ints
// of grid-barrier state owned by the caller; diag (if any) holds GBSBIN_DIAG_DOUBLES.
cudaError_t launch_dft_fused(const DftArgs& a, unsigned* bar, int num_sms, cudaStream_t s);
// Nonzero when launch_dft_fused takes the two-phase form for this grid.
int dft_two_phase(const GridDesc& g);

// App. D's sum over the evaluation points m <= pattern on the device (gbsbin_distinguishable.cu):
// d (K x M) and S (K x M x M) the rank-2 blocks' trace and Frobenius-norm coefficients; the
// signed, binomial-weighted sum of f_N(m) to *total (compensated) and the sum of the terms'
// magnitudes to *abs_total.  Launches of at most kDistChunkFlops estimated FP64 work each,
// synchronous on s; N <= kDistMaxN, M <= kDistMaxM and the whole sum at most kDistMaxFlops
// (else GBSBIN_ERR_UNSUPPORTED).
constexpr int kDistMaxN = 64;
constexpr int kDistMaxM = 64;
constexpr double kDistChunkFlops = 2e10;   // ~20 ms of FP64 work per launch on this GPU
constexpr double kDistMaxFlops = 3e13;     // ~30 s
int distinguishable_sum_device(int M, int K, int N, const int* pattern, const double* d, const double* S,
                               double* total, double* abs_total, cudaStream_t s);
cudaError_t launch_backward(const BackwardArgs& b, const double* dLdP, cudaStream_t s);
cudaError_t launch_alu_peak(int fp64, int blocks, float* out_sink, int iters, cudaStream_t s);

}  // namespace gbsbin
