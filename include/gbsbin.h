/*
 * gbsbin - binned photon-number distributions of Gaussian states on GB300 (sm_103a).
 *
 * C ABI of the library.  Plain C types only; no exceptions cross it; every call returns
 * a gbsbin_status (0 = GBSBIN_OK) unless stated otherwise.
 *
 * What it computes (arXiv:2412.17742):
 *   A Gaussian state on n' = M*K modes (M external ports x K internal modes) with
 *   normally ordered covariance Sigma^(1) and mean z-bar (Sec. II) has adjacency data
 *   XA = I - Sigma^{-1}, gamma = X Sigma^{-1} z-bar, Sigma = I + Sigma^(1)
 *   (Eqs. defA, defgamma, x_matrix_husimi_cov).  The detectors are grouped by a set
 *   partition Lambda_1..Lambda_L of the M ports (Sec. VI, Eq. coarse_grained_subset).
 *   The probability generating function of the binned counts b is
 *     G(w) = q(A, gamma, D(w)) / q(A, gamma, 1),   D(w) = diag(w_label(i)) (+) same,
 *     q = exp(1/2 gamma^T [I - D XA]^{-1} D X gamma) / sqrt(det[I - D XA])
 *   (Sec. III, Eq. q_d; Sec. VI, Eq. Lamb_lhaf_master).  On the grid of roots of unity
 *   w_l = exp(2 pi i k_l / (N_l + 1)) the library evaluates G at every point (one
 *   unpivoted LU of the complex n x n matrix I - D(w) XA per point, n = 2 M K) and
 *   returns the folded table
 *     P~(b) = (1/N_pts) sum_k G(omega^k) omega^{-k.b},  0 <= b_l <= N_l,
 *   which equals sum over b' = b mod (N+1) of the binned probability P(b')
 *   (Sec. VI, Eq. coarse_grained_prob).  With options.oversample = s > 1 the grid has
 *   s (N_l + 1) points per axis and the returned table is its first N_l + 1 entries per
 *   axis, i.e. P(b) itself up to the probability mass beyond s (N_l + 1) - 1.
 *
 * Memory: a plan owns its device workspaces.  Table buffers passed to *_execute are
 * owned by the caller; device pointers unless the function name says _host.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Thread safety: one plan per thread/stream; distinct plans are independent.
 */
#ifndef GBSBIN_H
#define GBSBIN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re, im;
} gbsbin_complex;

typedef enum {
  GBSBIN_OK = 0,
  GBSBIN_ERR_ARG = 1,          /* null pointer, M <= 0, K <= 0, L not in [1, M], bad option */
  GBSBIN_ERR_PARTITION = 2,    /* a detector group is empty or a label is out of [0, L)     */
  GBSBIN_ERR_CUTOFF = 3,       /* N_l < 0, or the grid exceeds GBSBIN_MAX_POINTS            */
  GBSBIN_ERR_NONPHYSICAL = 4,  /* Sigma not Hermitian, or Sigma - I/2 not positive definite
                                  (then ||XA||_2 >= 1 and the pivots lose Re > 0)           */
  GBSBIN_ERR_CUDA = 5,         /* a CUDA runtime call failed                                */
  GBSBIN_ERR_NOMEM = 6,        /* host or device allocation failed                          */
  GBSBIN_ERR_NUMERIC = 7,      /* a pivot with Re u_ii <= 0 or a non-finite value at some
                                  grid point (see gbsbin_diagnostics)                      */
  GBSBIN_ERR_UNSUPPORTED = 8,  /* size beyond what this build supports (n > GBSBIN_MAX_N)   */
  GBSBIN_ERR_TIMEOUT = 9,      /* a bounded device-side wait gave up                        */
  GBSBIN_ERR_PRECISION = 10    /* the result lost its significant digits to cancellation (its
                                  rounding-error estimate exceeds 1e-3 of it); the value is
                                  still written                                           */
} gbsbin_status;

#define GBSBIN_MAX_N 512                 /* largest matrix size n = 2 M K            */
#define GBSBIN_MAX_POINTS (1LL << 26)    /* largest grid prod(oversample (N_l + 1))   */

typedef enum {
  GBSBIN_FP64 = 0,          /* every step in FP64 (DFMA pipe)                               */
  GBSBIN_FP32_REFINE = 1    /* FP32 LU, one refinement step of log det and of the exponent
                               solve whose residual is formed with error-free FP32
                               transformations; FP64 epilogue and DFT.  Where the tree of
                               block eliminations applies (GBSBIN_KERNEL_TREE_DF32), pairs
                               of FP32 instead of the refinement, and the inverse DFT in
                               pairs of FP32 too where its two-phase form applies (three or
                               more groups on a small grid)                                 */
} gbsbin_precision;

typedef struct {
  int precision;          /* gbsbin_precision; default GBSBIN_FP64                          */
  int oversample;         /* >= 1; default 1 (folded table on the N_l + 1 grid)             */
  int want_diagnostics;   /* nonzero: gbsbin_execute also reduces sum/imag diagnostics     */
  int tile_override;      /* 0 = automatic kernel choice; otherwise a gbsbin_kernel id      */
  int want_timing;        /* nonzero: execute records CUDA events around the point kernel on
                             its stream; gbsbin_diagnostics reports the elapsed time         */
  int want_backward;      /* nonzero: allocate what gbsbin_backward needs (one n x n
                             workspace per SM; no per-point storage)                       */
  long long shard_begin;  /* shard_end > 0: this plan evaluates only the evaluated points    */
  long long shard_end;    /* e in [shard_begin, shard_end) of the half grid (plus point 0,
                             w = 1, for the normalisation) and returns the PARTIAL table of
                             their terms; the tables of shards that partition [0, n_evaluated)
                             sum to the whole table (the DFT is linear).  0, 0 = whole grid.
                             gbsbin_backward on a shard's plan gives the gradient of its
                             partial table: the shards' gradients sum to the whole gradient.
                             Not for batches (ERR_UNSUPPORTED).                             */
} gbsbin_options;

/*
 * One problem.  Give EITHER the physical description (r, T, optional alpha and V) OR the
 * state directly (sigma1, optional zbar); sigma1 != NULL selects the latter.
 *
 * Physical description (Sec. II; output covariance as in Sec. VIII,
 * Eq. output_cov_internal; internal modes as in Sec. VI and App. B):
 *   r[i*K + k]     real squeezing of internal mode k of input port i
 *   T[j*M + i]     M x M transfer matrix, output j <- input i, ||T||_2 <= 1 (loss allowed)
 *   alpha[i*K + k] displacement of internal mode k of input port i (NULL = none)
 *   V[(i*K + l)*K + k]  K x K unitary per input port: column k is the internal state of
 *                  squeezer k of port i in the detector's internal basis (NULL = identity)
 *   The full transfer on the M*K modes is T_full[(j,l),(i,k)] = T[j,i] V_i[l,k]; then
 *   Sigma^(1) = W Sigma^(1)_in W^dag with W = T_full (+) T_full^*, z-bar = (T_full alpha,
 *   conj), mode order zeta = (a_(0,0) .. a_(M-1,K-1), a^dag_(0,0) ..) (external-major).
 * Direct description:
 *   sigma1[p*n + q] n x n Hermitian, the s = 1 (normally ordered) covariance in the mode
 *   order above; zbar[n] the mean vector (NULL = zero), n = 2 M K.
 * Grouping:
 *   bin_of_mode[j] in [0, L): detector group of output port j (every group non-empty);
 *   cutoff[l] = N_l >= 0.
 * All arrays are host memory, read during the call only.
 */
typedef struct {
  int M;
  int K;
  const double* r;
  const gbsbin_complex* T;
  const gbsbin_complex* alpha;
  const gbsbin_complex* V;
  const gbsbin_complex* sigma1;
  const gbsbin_complex* zbar;
  const int* bin_of_mode;
  int L;
  const int* cutoff;
} gbsbin_problem;

typedef struct gbsbin_plan gbsbin_plan;

typedef struct {
  double sum_P;              /* sum of the returned table (1 up to rounding on the folded grid) */
  double max_imag;           /* max |Im P~| before the real part is taken (round-off probe)    */
  double min_pivot_re;       /* min over evaluated points of min_i Re u_ii (> 0 in theory)     */
  long long n_bad_points;    /* evaluated points with a pivot Re <= 0 or a non-finite value    */
  long long n_points;        /* grid points prod(oversample (N_l + 1))                         */
  long long n_evaluated;     /* points evaluated: conjugate symmetry halves the last axis      */
  long long table_size;      /* doubles written to P_out: prod(N_l + 1)                        */
  int n;                     /* matrix size 2 M K                                              */
  int kernel;                /* gbsbin_kernel id used by the last execute                      */
  double log_q1_re;          /* log q(A, gamma, 1) = -log Pr(0), from the w = 1 grid point    */
  double point_kernel_ms;    /* duration of the last point-kernel launch (want_timing), else 0 */
  long long state_upload_bytes; /* bytes one state upload (plan creation, gbsbin_plan_set_state or
                                   gbsbin_fock_plan_set_transfer) copies from host to device    */
  int launches;              /* kernel launches of the last execute (point stage, inverse DFT
                                with its diagnostics), 0 before the first                       */
  double backward_kernel_ms; /* duration of the last reverse pass's per-point (or per-tree)
                                kernels (plans with want_timing and want_backward), else 0      */
  int backward_path;         /* how the plan's reverse pass runs: 0 no reverse pass, 1 one
                                inverse per evaluated point, 2 along the large-matrix tree      */
} gbsbin_diag;

typedef enum {
  GBSBIN_KERNEL_AUTO = 0,
  GBSBIN_KERNEL_SMEM_FP64 = 1,     /* CTA per point, matrix in shared memory, FP64          */
  GBSBIN_KERNEL_SMEM_FP32R = 2,    /* CTA per point, shared memory, FP32 LU + refinement    */
  GBSBIN_KERNEL_GMEM_FP64 = 3,     /* CTA per point, matrix in an L2-resident workspace     */
  GBSBIN_KERNEL_GMEM_FP32R = 4,
  GBSBIN_KERNEL_WARP_FP32R = 5,    /* warp per point, matrix in registers (n <= 32)        */
  GBSBIN_KERNEL_BLK_FP32R = 6,     /* CTA per point, blocked (NB = 32) on an L2-resident
                                      slot, register-tiled updates (n <= 384)              */
  GBSBIN_KERNEL_BLK_TC_FP32R = 7,  /* as 6, the trace-correction updates on the tensor
                                      cores (tcgen05, 3 x TF32, TMEM accumulator)         */
  GBSBIN_KERNEL_HESS_FP64 = 8,     /* one detector group (L = 1, the total photon number of
                                      Sec. VIII): D(w) = w I, so one Hessenberg reduction
                                      XA = Q H Q^H per state (host) serves every point,
                                      O(n^2) per point (warp per point, FP64), displacement
                                      through Q^T gamma and Q^H X gamma; chosen
                                      automatically for GBSBIN_FP64 plans with L = 1       */
  GBSBIN_KERNEL_FOCK_FP64 = 9,     /* Fock inputs (gbsbin_fock_*): FP64 throughout           */
  GBSBIN_KERNEL_FOCK_DF32 = 10,    /* Fock inputs: pairs of FP32 (hi + lo, ~46 bits) on the
                                      FMA pipe, running sums flushed to FP64               */
  GBSBIN_KERNEL_TREE_DF32 = 11,    /* L >= 2: rows ordered by group, the grid evaluated as a
                                      tree of block eliminations - depth l holds one reduced
                                      matrix I - D'A' per combination of the first l axes'
                                      roots (the Schur complement after eliminating groups
                                      0..l-1 depends on their phases only), every grid point
                                      a leaf; the same pivots as the per-point unpivoted LU
                                      of the permuted matrix; pairs of FP32 (~46 bits) on
                                      the FMA pipe, FP64 results; chosen automatically for
                                      GBSBIN_FP32_REFINE plans with n <= 64, last group <= 16
                                      rows and no shard                                    */
  GBSBIN_KERNEL_TREE_FP64 = 12,    /* the same tree in FP64 (DFMA pipe); chosen automatically
                                      for GBSBIN_FP64 plans under the same conditions      */
  GBSBIN_KERNEL_BTREE_DF32 = 13,   /* L >= 2, large matrices: the same tree of block
                                      eliminations with the reduced matrices in HBM/L2 - a
                                      level's pivot rows factored by one CTA per child in
                                      shared memory, the other rows streamed through
                                      registers by many CTAs per child - and the last
                                      group's block I - w A_L of every leaf parent reduced
                                      once to Hessenberg form (A_L = Q H Q^H), so each grid
                                      point is an O(m^2) elimination of H - conj(w) I;
                                      pairs of FP32; chosen automatically for standalone
                                      GBSBIN_FP32_REFINE plans where kernel 11 does not
                                      apply and it needs under half the per-point LUs'
                                      work (last group <= 192 rows; above 116 the
                                      Hessenberg reduction works through L2); a shard runs the
                                      first-axis subtrees that cover its slice          */
  GBSBIN_KERNEL_BTREE_FP64 = 14,   /* the same in FP64; chosen for GBSBIN_FP64 plans under
                                      the same conditions                                   */
  GBSBIN_KERNEL_HERALD_FP64 = 15,  /* heralded states (gbsbin_herald_*): CTA per point, FP64;
                                      not a choice for gbsbin_plan_create                   */
  GBSBIN_KERNEL_HESS_DF32 = 16     /* as 8 in pairs of FP32 on the FMA pipe (H, a, c stored as
                                      pairs; FP64 results); chosen automatically for
                                      GBSBIN_FP32_REFINE plans with L = 1, also in batches   */
} gbsbin_kernel;

/* Fill *o with defaults: FP64, oversample 1, diagnostics on, automatic kernel. */
void gbsbin_default_options(gbsbin_options* o);

/*
 * Validate the problem, build Sigma^(1), z-bar, Sigma^{-1}, XA and gamma on the host in
 * FP64 (Sec. II), upload them and allocate device workspaces.  Synchronous.
 * Errors: ERR_ARG, ERR_PARTITION, ERR_CUTOFF, ERR_NONPHYSICAL, ERR_UNSUPPORTED,
 * ERR_NOMEM, ERR_CUDA.  On error *out is NULL.
 */
int gbsbin_plan_create(const gbsbin_problem* p, const gbsbin_options* o, gbsbin_plan** out);

/*
 * Replace the state of an existing plan (same M, K, L, cutoffs and grouping; new r, T,
 * alpha, V or sigma1/zbar): redo the host FP64 algebra and enqueue the upload on
 * `stream`, ordered after the work already enqueued there.  The plan stages uploads in two
 * pinned buffers used in turn, so the call waits only for the upload two calls back, not
 * for the stream: the host algebra of the next state overlaps the device work of the
 * current one.  Same errors as plan_create; ERR_ARG if a shape differs.
 */
int gbsbin_plan_set_state(gbsbin_plan* plan, const gbsbin_problem* p, void* stream);

/* Free the plan and its device workspaces (synchronises the device first). */
int gbsbin_plan_destroy(gbsbin_plan* plan);

/* Number of doubles in the output table, prod(N_l + 1); -1 if plan is NULL. */
long long gbsbin_plan_table_size(const gbsbin_plan* plan);

/*
 * Evaluate G on the grid and write the table to P_out (device, table_size doubles,
 * row-major over l = 0..L-1, last group fastest).  Asynchronous on `stream`.  Numeric
 * failures (ERR_NUMERIC) are reported by gbsbin_diagnostics, not here.
 */
int gbsbin_execute(gbsbin_plan* plan, double* P_out, void* stream);

/*
 * Same as gbsbin_execute but P_out is host memory; the device-to-host copy is enqueued
 * on `stream` and the call synchronises it before returning.
 */
int gbsbin_execute_host(gbsbin_plan* plan, double* P_out_host, void* stream);

/*
 * As gbsbin_execute_host without the final synchronisation: the execute and the
 * device-to-host copy are enqueued on `stream` and the call returns.  P_out_host (pinned
 * memory for an asynchronous copy) holds the table once the stream has reached the copy;
 * the caller synchronises before reading it and must not reuse it for a later call until
 * then.  Errors as gbsbin_execute, ERR_ARG for a null pointer.
 */
int gbsbin_execute_host_async(gbsbin_plan* plan, double* P_out_host, void* stream);

/*
 * Diagnostics of the last execute on this plan.  Synchronises `stream`.  Returns
 * GBSBIN_ERR_NUMERIC if any evaluated point had a non-positive or non-finite pivot.
 */
int gbsbin_diagnostics(gbsbin_plan* plan, gbsbin_diag* out, void* stream);

/*
 * Copy the per-point results of the last execute to host memory: logq_host receives
 * n_evaluated complex values log q(A, gamma, D(omega^k)) (interleaved re, im) and
 * minpiv_host (may be NULL) n_evaluated doubles min_i Re u_ii.  Evaluated point e has
 * digits k_{L-1} = e mod half, then the other axes in mixed radix (last fastest), where
 * half = radix_{L-1}/2 + 1 and radix_l = oversample (N_l + 1).  Synchronises `stream`.
 */
int gbsbin_read_points(gbsbin_plan* plan, double* logq_host, double* minpiv_host, void* stream);

/*
 * Binned table from per-point log q without allocating device memory.  The paper has no
 * counterpart: this is a library-level convenience for callers that must not call
 * cudaMalloc, such as code running under a device-memory budget owned by another
 * framework's pool allocator (where an extra allocation can fail or fragment the pool), or
 * latency-critical loops where cudaMalloc/cudaFree would synchronise the device and stall
 * work on other streams.
 *
 * It performs the inverse DFT stage of gbsbin_execute: logq (device, n_eval complex values,
 * interleaved re, im, in the evaluated-point order described at gbsbin_read_points, for
 * the grid radix_l = oversample (N_l + 1)) -> P_out (device, prod(N_l + 1) doubles).
 * The caller passes inputs and outputs; cutoff (L ints) is host memory.
 *
 * Scratch: one fixed array of GBSBIN_NOALLOC_MAX_TWIDDLES + 2 GBSBIN_NOALLOC_MAX_EVAL
 * complex doubles (about 4.25 MB) held by every GPU that loads the library until the
 * process exits.  Grids with n_eval > GBSBIN_NOALLOC_MAX_EVAL or sum of radices >
 * GBSBIN_NOALLOC_MAX_TWIDDLES are rejected with GBSBIN_ERR_UNSUPPORTED; other errors:
 * ERR_ARG, ERR_CUTOFF, ERR_CUDA.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the same array and leaves its
 * contents behind (nothing in it has to start at zero), so calls whose kernels overlap
 * on the GPU - on different streams or from different threads - race with each other;
 * serialise them.  Asynchronous on `stream`.
 */
#define GBSBIN_NOALLOC_MAX_EVAL (1LL << 17)
#define GBSBIN_NOALLOC_MAX_TWIDDLES (1LL << 14)
int gbsbin_table_from_logq_noalloc(int L, const int* cutoff, int oversample, const double* logq,
                                   double* P_out, void* stream);

/*
 * Gradients of a scalar loss L(P) with respect to the problem's inputs (reverse mode
 * through the inverse DFT, the per-point log det and exponent, and the FP64 state
 * algebra).  Complex parameters use the convention g = dL/dRe z + i dL/dIm z, entries
 * treated as independent.  d_sigma1 and d_zbar are exact along physical directions
 * (perturbations keeping Sigma^(1) = [[N^T, Mm], [Mm^*, N]] and z-bar = (m, conj m)), the
 * only ones under which the table stays real; the evaluation relies on that symmetry.  Every pointer may be NULL (not wanted); all are host memory
 * owned by the caller.  d_r, d_T, d_alpha, d_V need the physical description
 * (r, T, alpha, V) at plan creation / set_state; d_alpha and d_V are zero-filled when the
 * problem had no alpha / V.
 */
typedef struct {
  double* d_r;                /* [M*K]                                  */
  gbsbin_complex* d_T;        /* [M*M]                                  */
  gbsbin_complex* d_alpha;    /* [M*K]                                  */
  gbsbin_complex* d_V;        /* [M*K*K]                                */
  gbsbin_complex* d_sigma1;   /* [n*n] w.r.t. Sigma^(1)                 */
  gbsbin_complex* d_zbar;     /* [n]   w.r.t. z-bar                     */
} gbsbin_grads;

/*
 * Reverse pass for the plan's current state (no counterpart in the paper, which leaves
 * differentiability to future work; the adjoint follows from d log det A = tr(A^{-1} dA)).
 * dL_dP: device, table_size doubles, dL/dP(b) for the table of the last execute.  Needs a
 * plan created with want_backward.  Nothing of the forward is kept but log q at the
 * evaluated points: each point's matrix M = conj(D(w)) - XA is rebuilt and inverted in place
 * (blocked Gauss-Jordan without pivoting, n^3 complex multiply-adds per point, in a per-SM
 * workspace of n^2 entries) in FP64 for GBSBIN_FP64 plans and in pairs of FP32 (~46 bits)
 * for GBSBIN_FP32_REFINE plans.  Plans on the large-matrix tree (kernels 13, 14; no shard)
 * instead go along the tree where that needs under half the work: per combination of the
 * first L-1 axes' roots the inverse of the leading groups' block and its products with the
 * rest, per evaluated point only the inverse of the last group's Schur complement
 * (gbsbin_diag.backward_path says which).  If the state changed since the last execute, an
 * execute (into the plan's own table) runs first.  Synchronises `stream`.
 * Errors: ERR_ARG (NULL plan/dL_dP/g, plan without want_backward, physical gradients
 * requested for a direct-covariance problem), ERR_NUMERIC (a non-finite adjoint),
 * ERR_CUDA, ERR_NOMEM.
 */
int gbsbin_backward(gbsbin_plan* plan, const double* dL_dP, gbsbin_grads* g, void* stream);

/*
 * The same reverse pass up to the adjoints of the adjacency data, on the device and
 * asynchronous: S = dL_dXA (n*n, row-major) and s = dL_dgamma (n), device buffers, such that
 * dL = Re( sum_ij S_ij dXA_ij + sum_i s_i dgamma_i ) with the entries of XA = I - Sigma^{-1}
 * and gamma treated as independent (the gradient in the d/dRe + i d/dIm convention above is
 * conj(S), conj(s)); the caller chains them further.  Errors: ERR_ARG, ERR_CUDA.
 */
int gbsbin_backward_device(gbsbin_plan* plan, const double* dL_dP, gbsbin_complex* dL_dXA, gbsbin_complex* dL_dgamma,
                           void* stream);

/*
 * Measured autotuning of the point kernel (no counterpart in the paper): for matrix size
 * n (even, <= GBSBIN_MAX_N) and a precision, times the candidate kernels (warp per point
 * for FP32R n <= 32; shared-memory CTA kernel with 1, 2, 4 or 8 points per CTA where they
 * fit; L2-workspace kernel) on a synthetic state with ~1024 evaluated points and returns the
 * fastest as a gbsbin_kernel id, points per CTA and microseconds per evaluated point.
 * Results are cached per (n rounded up to a multiple of 16, precision) for the process.
 * Synchronous; uses the current device.
 */
int gbsbin_autotune(int n, int precision, int* kernel, int* points_per_cta, double* us_per_point);

/*
 * Batches of independent problems (uneven sizes, groupings and cutoffs) evaluated
 * together: one persistent point-kernel launch per kernel class takes (problem, point
 * group) jobs from a device work queue, largest first; the inverse DFT then runs per
 * problem.  Options apply to every problem (want_backward and want_timing are not
 * supported: ERR_ARG); autotune != 0 picks each size's kernel with gbsbin_autotune.
 * gbsbin_batch_capture_graph records one execute (into the given outputs) as a CUDA
 * graph on a non-default stream; gbsbin_batch_replay relaunches it.  P_out is a host
 * array of nprob device pointers, P_out[i] holding gbsbin_batch_table_size(b, i) doubles.
 */
typedef struct gbsbin_batch gbsbin_batch;
int gbsbin_batch_create(const gbsbin_problem* probs, int nprob, const gbsbin_options* o, int autotune,
                        gbsbin_batch** out);
int gbsbin_batch_execute(gbsbin_batch* b, double* const* P_out, void* stream);
int gbsbin_batch_capture_graph(gbsbin_batch* b, double* const* P_out, void* stream);
int gbsbin_batch_replay(gbsbin_batch* b, void* stream);
long long gbsbin_batch_table_size(const gbsbin_batch* b, int i);
int gbsbin_batch_diagnostics(gbsbin_batch* b, int i, gbsbin_diag* out, void* stream);
int gbsbin_batch_read_points(gbsbin_batch* b, int i, double* logq_host, double* minpiv_host, void* stream);
int gbsbin_batch_destroy(gbsbin_batch* b);

/*
 * Exact mean and covariance of the binned counts (Sec. VI, coarse-grained moments and
 * cumulants): with G(e^t) the moment generating function of b, they are the first and
 * second derivatives of log G(e^t) at t = 0, where log G = 1/2 gamma^T (I - D XA)^{-1} D X
 * gamma - 1/2 log det(I - D XA) + const and D = diag(e^{t_l(i)}).  Written out with
 * R = (I - XA)^{-1}, W = XA R, u = R X gamma, v = R^T gamma:
 *   mean_l   = 1/2 sum_{i in l} (v_i u_i + W_ii)
 *   cov_lm   = 1/2 [sum_{i in m, j in l} v_i W_ij u_j + sum_{i in l, j in m} v_i W_ij u_j
 *                   + d_lm sum_{i in l} v_i u_i + sum_{i in m, j in l} W_ij W_ji
 *                   + d_lm sum_{i in l} W_ii].
 * Unfolded (no cutoff enters: p->cutoff is validated but unused).  Host only, FP64, O(n^3);
 * no device is used.  mean: L doubles, cov: L x L doubles row-major, caller-owned host.
 * Errors: ERR_ARG / ERR_PARTITION / ERR_NONPHYSICAL as for gbsbin_plan_create.
 */
int gbsbin_moments(const gbsbin_problem* p, double* mean, double* cov);
/*
 * Exact third cumulants of the binned counts (Sec. VI, coarse-grained moments and
 * cumulants): kappa_lmn = third derivative of log G(e^t) at t = 0.  With e_l = e^{t_l} - 1,
 * log G = sum_l c_l e_l + sum_lm a_lm e_l e_m + sum_lmn b_lmn e_l e_m e_n + O(e^4), where
 * (R, W, u, v as for gbsbin_moments; i in l means row i belongs to group l)
 *   c_l   = 1/2 sum_{i in l} (W_ii + v_i u_i)
 *   a_lm  = sum_{i in l, j in m} (1/4 W_ij W_ji + 1/2 v_i W_ij u_j)
 *   b_lmn = sum_{i in l, j in m, k in n} (1/6 W_ij W_jk W_ki + 1/2 v_i W_ij W_jk u_k),
 * from -1/2 log det(I - D XA) = const + 1/2 sum_k tr((E W)^k) / k and the exponent's
 * Neumann series, E = diag(e_label(i)).  Then
 *   kappa_lmn = sum over the 6 orders of (l, m, n) of b
 *               + d_lm Q_ln + d_ln Q_lm + d_mn Q_ml + d_lm d_mn c_l,   Q = a + a^T.
 * Unfolded (no cutoff enters).  Host only, FP64, O(n^3); k3: L x L x L doubles, row-major,
 * caller-owned host memory.  Errors: as gbsbin_moments.
 */
int gbsbin_cumulants3(const gbsbin_problem* p, double* k3);

/*
 * Exact fourth cumulants of the binned counts (Sec. VI, coarse-grained moments and
 * cumulants): kappa_{l1 l2 l3 l4} = fourth derivative of log G(e^t) at t = 0.  In
 * e_l = e^{t_l} - 1, log G = sum_{r >= 1} sum_{m1..mr} C_r(m1..mr) e_m1 ... e_mr with
 *   C_r(m1..mr) = sum_{i_k in m_k} ( 1/(2r) W_i1i2 W_i2i3 ... W_iri1
 *                                    + 1/2 v_i1 W_i1i2 ... W_i(r-1)ir u_ir )
 * (W, u, v as for gbsbin_moments; r = 1..3 are the c, a, b of gbsbin_cumulants3).  Each e_l
 * depends on t_l alone and every derivative of e^t is 1 at 0, so kappa is the sum over the
 * set partitions of the four index slots whose blocks each carry a single group of F_r (the
 * blocks' groups), F_r(m1..mr) = sum over the orders of (m1..mr) of C_r.  Unfolded (no cutoff
 * enters).  Host only, FP64, O(n^3 + L^4 (n/L)^2); k4: L^4 doubles, row-major, caller-owned
 * host memory.  Errors: as gbsbin_moments.
 */
int gbsbin_cumulants4(const gbsbin_problem* p, double* k4);

/*
 * The cumulants of gbsbin_moments, gbsbin_cumulants3 and gbsbin_cumulants4 (Sec. VI,
 * coarse-grained moments and cumulants) computed on the GPU.  precision GBSBIN_FP64: every
 * device step in FP64; GBSBIN_FP32_REFINE: the products and block sums in pairs of FP32 on the
 * FMA pipe (~46 bits), the chain rule in FP64.  With
 * XA = I - Sigma^{-1}, R = (I - XA)^{-1} = Sigma, so W = XA R = Sigma^(1) (Hermitian),
 * u = R X gamma = X gamma + W X gamma and v = R^T gamma = gamma + W^T gamma: no inverse is
 * formed.  The host builds and validates the state as for gbsbin_plan_create and sorts the rows
 * by group; the device then forms (C_r as for gbsbin_cumulants4; W_ab the block of rows of
 * group a, columns of group b):
 *   u, v;
 *   for order >= 3, Y_b = W_{:,b} W_{:,b}^H per group b (Hermitian: the 32 x 32 tiles on and
 *     above the diagonal, the depth split into slices where the tiles alone leave SMs idle);
 *   for order 4, q_d = W_{:,d} u_d and p_ab = v_a^T Y_b[a rows, :];
 *   C_1 .. C_order, one CTA per coefficient, each a fixed-order sum over one block:
 *     C_3(a,b,c) = sum_{i in a, k in c} Y_b[i,k] (1/6 conj(W_ik) + 1/2 v_i u_k),
 *     C_4(a,b,c,d) = 1/8 sum_{i in a, k in c} Y_b[i,k] conj(Y_d[i,k]) + 1/2 sum_{k in c} p_ab[k] q_d[k]
 *     (one CTA for (a,b,c,d) and (a,d,c,b), whose traces are conjugate);
 *   kappa by the chain rule of e = e^t - 1 over the set partitions of the slots, a thread per
 *     entry.
 * The highest non-null output sets the order: mean (L doubles), cov (L x L), k3 (L^3), k4 (L^4),
 * row-major, caller-owned host memory; lower orders may be null.  Work ~n^3/2 complex
 * multiply-adds for the Y_b and ~L^2 n^2/2 for the C_4 traces; device memory up to
 * (1 + 2 L) n^2 x 16 bytes, allocated and freed per call.  Synchronous on `stream`.
 * *kernel_ms (may be NULL) receives the device time of the launches by CUDA events (uploads and
 * the final copies excluded).  Errors: ERR_ARG (p NULL, every output NULL, or another
 * precision), ERR_UNSUPPORTED (L > 16), then as gbsbin_moments, ERR_NOMEM, ERR_CUDA.
 */
int gbsbin_cumulants_device(const gbsbin_problem* p, int precision, double* mean, double* cov, double* k3, double* k4,
                            double* kernel_ms, void* stream);

/*
 * Total photon-number distribution Pr(N), N = 0..Nmax, over all detectors (grouping
 * ignored), by the power series of Sec. IV / App. A: with z = (eta, ..., eta),
 * log q(eta) = sum_k a_k eta^k, a_k = tr((XA)^k) / (2k) + 1/2 gamma^T (XA)^(k-1) X gamma,
 * and Pr(N) = Pr(0) [eta^N] exp(sum_k a_k eta^k), Pr(0) = 1 / q(1).  Unfolded (exact up to
 * rounding; no grid).  A second evaluator beside the roots-of-unity transform of the
 * one-group plans.  Host only, FP64, O(Nmax n^3) (the powers of XA by repeated
 * multiplication); P_out: Nmax + 1 doubles, caller-owned host memory.  Errors: ERR_ARG
 * (Nmax < 0, null pointers), ERR_UNSUPPORTED (Nmax > 2^20), then as gbsbin_moments.
 */
int gbsbin_total_photon_series(const gbsbin_problem* p, int Nmax, double* P_out);

/*
 * Joint cumulant <<n_S1 n_S2 ... n_Sr>> of the counts of r distinct groups (bit l of `mask`
 * selects group l): the coarse-grained loop Montrealer of Sec. VI.  With distinct groups only
 * the all-singleton set partition enters the chain rule from e = e^t - 1, so
 *   kappa_S = 1/2 sum over the directed Hamiltonian cycles a -> b -> ... -> a through S of
 *             tr(W_ab W_bc ... W_za)
 *           + 1/2 sum over the Hamiltonian paths a -> ... -> z through S of
 *             v_a^T W_ab ... W_yz u_z
 * (W, u, v as for gbsbin_moments; W_ab the block of rows of group a, columns of group b);
 * r = 1, 2, 3, 4 give the mean, the covariance and the distinct-index entries of
 * gbsbin_cumulants3/4.  Dynamic programming over the subsets of S, O(2^r r^2 (n/r)^3), host
 * FP64; *kappa: one double.  Errors: ERR_ARG (mask empty or naming a group >= L, null
 * pointers), ERR_UNSUPPORTED (more than 10 groups, or above ~1 GB of partial products),
 * then as gbsbin_moments.
 */
int gbsbin_cumulant_groups(const gbsbin_problem* p, unsigned mask, double* kappa);

/*
 * Fine-grained Pr(n) (pattern[k] photons in external mode k, k < M) of an undisplaced state
 * whose internal modes are fully distinguishable (App. D): XA block diagonal over the
 * internal modes (aligned internal bases, each internal mode carrying one source), every
 * block B_l of rank <= 2.  By the finite differences at integer points,
 *   Pr(n) = Pr(0) / prod n_k! sum_{m <= n} prod C(n_k, m_k) (-1)^(N - |m|) f_N(m),
 * f_N(m) = [eta^N] exp(sum_j p_j eta^j / (2j)), p_j = sum_l (lambda1^j + lambda2^j) with the two
 * eigenvalues of sqrt(D(m)) B_l sqrt(D(m)) from its trace T and Frobenius norm F,
 * lambda = T/2 +- sqrt(2F^2 - T^2)/2.  prod (n_k + 1) points, O(K M^2 + K N + N^2) each.  The
 * alternating sum cancels, more as N grows: it is summed with Neumaier compensation next to
 * the sum of the terms' magnitudes, and abs_err (may be NULL) receives the estimate
 * (N + 16) eps Pr(0) / prod n_k! x sum |terms| of the result's absolute rounding error.  Host
 * only.  Errors: ERR_ARG (null pointers, a negative count), ERR_UNSUPPORTED (displaced, not
 * block diagonal over internal modes, a block of rank above 2, or more than 2^40 evaluation
 * points), then as gbsbin_moments; ERR_PRECISION when that estimate exceeds 1e-3 of |Pr(n)|
 * (the value is still written: fewer than three significant digits are left).
 */
int gbsbin_prob_distinguishable(const gbsbin_problem* p, const int* pattern, double* prob, double* abs_err);

/*
 * The same Pr(n) with the sum over the prod (n_k + 1) evaluation points on the GPU: one thread
 * per point (its digits, the rank-2 blocks' eigenvalues, the power sums and the FP64 series),
 * compensated per thread and per CTA, the CTAs' partials added in a fixed order on the host;
 * host setup as above.  The points run in launches of at most ~2e10 estimated FP64 operations
 * (about 20 ms each on this GPU), so no launch runs long on a shared device.  Synchronous on
 * `stream`; device buffers are allocated and freed per call.  Errors: as
 * gbsbin_prob_distinguishable, ERR_UNSUPPORTED for N or M above 64 or more than ~3e13
 * estimated operations in all (about 30 s), ERR_NOMEM, ERR_CUDA.
 */
int gbsbin_prob_distinguishable_device(const gbsbin_problem* p, const int* pattern, double* prob, double* abs_err,
                                       void* stream);

/*
 * Fock inputs through a lossy linear circuit (App. C of the paper).  photons[j] >= 0
 * photons enter input port j of the M x M transfer matrix T (T[i*M + j]: output i <- input
 * j, ||T||_2 <= 1), the output ports are grouped as for Gaussian states, and the library
 * returns the binned output table.  The generating function of the binned counts is
 *   G(z) = perm(B(z)[p, p]) / prod_j p_j!,   B(z) = I - T^dag (I - Z) T,  Z = diag(z_label(i)),
 * the generating function of the diagonal elements of Eq. probs_fock_circuit over the
 * output patterns.  The permanent is taken as the coefficient of x^p in
 * prod_j (B(z) x)_j^{p_j} on roots-of-unity nodes x_k = exp(2 pi i g_k / (p_k + 1)) (exact:
 * the polynomial is homogeneous of degree N = sum p, so with one occupied input of
 * smallest p held at x = 1 nothing aliases), and the table is the inverse DFT of G over
 * the grid z_l = exp(2 pi i k_l / R_l), R_l = oversample (N_l + 1), exactly as for
 * gbsbin_execute: the folded table P~(b), 0 <= b_l <= N_l, which is P(b) itself when every
 * N_l >= N (no group sees more than N photons).
 * Work: prod over the other occupied inputs of (p_k + 1) nodes x (half the output grid)
 * points, each factor O(L).  Options: precision GBSBIN_FP64 (kernel 9) or
 * GBSBIN_FP32_REFINE, which here selects pairs of FP32 (kernel 10); oversample,
 * want_diagnostics, want_timing and tile_override (9 or 10) as for gbsbin_plan_create;
 * want_backward is not supported (ERR_UNSUPPORTED).  shard_begin/shard_end select a range
 * [begin, end) of the input nodes in the order the kernel walks them: node i has digits
 * g_d (one per occupied input other than the held one, which is the occupied input with the
 * fewest photons, lowest port on ties; the others in port order, the first the fastest)
 * given by the reflected mixed-radix Gray code: with n_d = floor(i / s_d) mod R_d,
 * s_d = prod_{d' < d} R_d', R_d = p + 1, g_d = n_d if floor(i / s_{d+1}) is even, else
 * R_d - 1 - n_d.  gbsbin_fock_plan_nodes gives the count.  The plan then returns the
 * PARTIAL table of those nodes' share G_p of G (normalised by the whole node count) in the
 * half-grid form every plan's inverse DFT takes - last axis k <= R/2 only, weight 1 at
 * k = 0 (and R/2 for even R) and 2 elsewhere, real part - exact for the whole G, whose
 * conjugate symmetry a share lacks: the tables of shards that partition [0, nodes) sum to
 * the whole table, and one shard's table alone is not a distribution.
 * Limits: at most GBSBIN_FOCK_MAX_INPUTS occupied inputs, GBSBIN_FOCK_MAX_PER_INPUT photons
 * in one input, GBSBIN_FOCK_MAX_GROUPS groups, GBSBIN_FOCK_MAX_NODES nodes, the output grid as for Gaussian states (ERR_UNSUPPORTED /
 * ERR_CUTOFF).  ERR_NONPHYSICAL if ||T||_2 > 1.  All arrays are host memory read during
 * the call.  gbsbin_fock_diagnostics fills sum_P and max_imag as gbsbin_diagnostics does,
 * n_points (output grid), n_evaluated (half-grid points), n = occupied inputs, kernel and
 * point_kernel_ms; min_pivot_re = 1, n_bad_points = 0 and log_q1_re = 0 do not apply.
 */
#define GBSBIN_FOCK_MAX_INPUTS 32
#define GBSBIN_FOCK_MAX_GROUPS 8
#define GBSBIN_FOCK_MAX_NODES (1LL << 40)
#define GBSBIN_FOCK_MAX_PER_INPUT (1 << 20)   /* photons in one input port */
typedef struct {
  int M;
  const gbsbin_complex* T;
  const int* photons;
  const int* bin_of_mode;
  int L;
  const int* cutoff;
} gbsbin_fock_problem;
typedef struct gbsbin_fock_plan gbsbin_fock_plan;
int gbsbin_fock_plan_create(const gbsbin_fock_problem* p, const gbsbin_options* o, gbsbin_fock_plan** out);
/* New transfer matrix T (same M, photons, grouping, cutoffs): host FP64 algebra, one
 * upload enqueued on `stream`.  ERR_ARG / ERR_NONPHYSICAL as for plan creation. */
int gbsbin_fock_plan_set_transfer(gbsbin_fock_plan* plan, const gbsbin_complex* T, void* stream);
long long gbsbin_fock_plan_table_size(const gbsbin_fock_plan* plan);
/* Input nodes of the whole problem, prod over the occupied inputs but the held one of
 * (p_k + 1); -1 if plan is NULL. */
long long gbsbin_fock_plan_nodes(const gbsbin_fock_plan* plan);
/* Table to P_out (device, table_size doubles, last group fastest); asynchronous. */
int gbsbin_fock_execute(gbsbin_fock_plan* plan, double* P_out, void* stream);
/* The same into host memory; synchronises `stream`. */
int gbsbin_fock_execute_host(gbsbin_fock_plan* plan, double* P_out_host, void* stream);
int gbsbin_fock_diagnostics(gbsbin_fock_plan* plan, gbsbin_diag* out, void* stream);
int gbsbin_fock_plan_destroy(gbsbin_fock_plan* plan);
/*
 * Heralded states (Sec. VII of the paper, Eqs. heralded_state_internal and
 * lhaf_heralded_offd_internal_1).  The M*K modes of a Gaussian state (state fields of
 * gbsbin_problem as for gbsbin_plan_create; its bin_of_mode, L and cutoff are ignored) take a
 * role each: role[m] = l in [0, L) - mode m belongs to heralding group l (a photon-number-
 * resolving detector, or a group of them whose counts are summed); GBSBIN_HERALD_TRACED - the
 * mode is discarded (traced out); GBSBIN_HERALD_KEPT - the mode carries the heralded state.
 * For every heralding outcome b (0 <= b_l <= cutoff[l]) the library returns the unnormalised
 * heralded state restricted to Fock indices <= fock_cutoff on each kept mode,
 *   rho(b) = sum over heralding patterns n with group counts b of Tr_traced <n| rho |n>,
 * and its trace over all kept
 * photon numbers, Pr(b) (the probability of outcome b; rho(b) / Pr(b) is the normalised
 * state).  Method: with A = X (I - Sigma^{-1}) and gamma as for the binned tables, the sum
 * over heralding and traced photon numbers weighted by w^n / n! is a complex-Gaussian
 * expectation, so that
 *   <v| rho(b) |u> = Pr(0) sqrt(u! v!) [w^b][x^u y^v] exp(xi^T M(w) xi / 2 + l(w)^T xi + e(w))
 *                  / sqrt(det(I - X D(w) A_DD)),
 * xi = (x, y) on the kept modes' two halves, M(w), l(w), e(w) from one solve with the
 * heralding and traced block I - X D(w) A_DD (w = 1 on traced modes), and the coefficient of
 * w^b by an inverse DFT over the grid w_l = exp(2 pi i k_l / R_l), R_l = oversample
 * (cutoff[l] + 1) (folded: photon numbers beyond R_l - 1 alias onto b, as for the binned
 * tables; oversample to unfold).  Pr(b) is the binned table of the heralding groups with
 * every other mode traced.  The Taylor coefficients of the kept modes follow from the
 * recurrence (p_i + 1) c_{p + e_i} = l_i c_p + sum_j M_ij c_{p - e_j} and are exact (no
 * folding) up to fock_cutoff.
 * Layout of rho_out: element [b_0 .. b_{L-1}][u_1 .. u_k][v_1 .. v_k] = <v| rho(b) |u> (the
 * conjugate of <u| rho(b) |v>), the last index fastest, u_i / v_i the ket / bra Fock index of
 * the i-th kept mode (in mode order), each of extent
 * fock_cutoff + 1: table_size = prod (cutoff[l] + 1) x (fock_cutoff + 1)^(2k) complex values;
 * prob_out: prod (cutoff[l] + 1) doubles.  FP64 throughout (kernel 15).
 * Limits: 2 x (modes not kept) and 2 M K at most GBSBIN_HERALD_MAX_MODES2, at most
 * GBSBIN_HERALD_MAX_KEPT kept modes (at least one), (fock_cutoff + 1)^(2k) at most
 * GBSBIN_HERALD_MAX_COEF (ERR_UNSUPPORTED); grid as for gbsbin_plan_create (ERR_CUTOFF).
 * Errors: ERR_ARG (null pointers, a role outside [-2, L), L < 1, fock_cutoff < 0, options
 * other than precision GBSBIN_FP64 / oversample / want_timing / want_diagnostics), ERR_PARTITION (a heralding group
 * without modes), ERR_NONPHYSICAL as for plan creation.  Options: oversample, want_timing
 * (point_kernel_ms of gbsbin_herald_diagnostics: all its launches).  All arrays host memory read
 * during the call.  gbsbin_herald_diagnostics: sum_P = sum of Pr(b) over the table,
 * min_pivot_re / n_bad_points over both eliminations of every point (n_bad_points > 0 makes
 * execute's results unreliable; the diagnostics call returns ERR_NUMERIC then), n_points =
 * n_evaluated = grid points, table_size as gbsbin_herald_table_size, n = 2 M K, kernel 15,
 * log_q1_re = -log Pr(0).
 */
#define GBSBIN_HERALD_TRACED (-1)
#define GBSBIN_HERALD_KEPT (-2)
#define GBSBIN_HERALD_MAX_MODES2 96
#define GBSBIN_HERALD_MAX_KEPT 4
#define GBSBIN_HERALD_MAX_COEF (1 << 20)
typedef struct {
  gbsbin_problem state;
  const int* role;     /* [M*K], external-major mode order (port i, internal k: i*K + k) */
  int L;
  const int* cutoff;   /* [L] */
  int fock_cutoff;
} gbsbin_herald_problem;
typedef struct gbsbin_herald_plan gbsbin_herald_plan;
int gbsbin_herald_plan_create(const gbsbin_herald_problem* p, const gbsbin_options* o, gbsbin_herald_plan** out);
/* Complex elements of rho_out (-1 if plan is NULL); prob_out has table_size / (fock_cutoff
 * + 1)^(2k) entries. */
long long gbsbin_herald_table_size(const gbsbin_herald_plan* plan);
long long gbsbin_herald_prob_size(const gbsbin_herald_plan* plan);
/* rho_out, prob_out device memory; asynchronous on `stream` (1 + L launches: the points, then the
 * inverse DFT one heralding axis at a time). */
int gbsbin_herald_execute(gbsbin_herald_plan* plan, gbsbin_complex* rho_out, double* prob_out, void* stream);
/* The same into host memory; synchronises `stream`. */
int gbsbin_herald_execute_host(gbsbin_herald_plan* plan, gbsbin_complex* rho_out_host, double* prob_out_host,
                               void* stream);
int gbsbin_herald_diagnostics(gbsbin_herald_plan* plan, gbsbin_diag* out, void* stream);
int gbsbin_herald_plan_destroy(gbsbin_herald_plan* plan);

/* Static description of a status code. */
const char* gbsbin_strerror(int status);

/*
 * Measurement utility (no counterpart in the paper): device throughput of dependent
 * multiply-add chains in FP64 (precision = GBSBIN_FP64), 32 x 32 -> 64-bit integer
 * (precision = GBSBIN_ALU_INT64, PTX mad.wide.s32) or FP32 (otherwise), in tera-ops/s
 * (2 per multiply-add), from one launch of `blocks` x 256 threads.  Synchronous.
 */
#define GBSBIN_ALU_INT64 2
int gbsbin_alu_peak(int precision, int blocks, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSBIN_H */
