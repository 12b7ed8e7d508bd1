// Host side of the library: validation, the FP64 Gaussian-state algebra of a problem
// (arXiv:2412.17742, Sec. II; output covariance as in Sec. VIII, Eq. output_cov_internal;
// internal modes as in Sec. VI and App. B), device workspaces and launch orchestration.
#include <algorithm>
#include <tuple>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gbsbin_backward_tree.h"
#include "gbsbin_host_state.h"
#include "gbsbin_internal.h"
#include "gbsbin_moments.h"

using cd = std::complex<double>;
using namespace gbsbin;

struct gbsbin_plan {
  int M = 0, K = 0, L = 0, n = 0;
  gbsbin_options opt{};
  std::vector<int> cutoff, bin_of_mode, label;
  GridDesc grid{};
  long long table_size = 0;
  int kernel = 0;
  int num_sms = 0;
  int device = 0;
  int has_gamma = 0;
  // host copies of the state (FP64)
  std::vector<cd> XA, gamma, Xgamma;
  // device buffers
  int P = 1;  // grid points per CTA of the point kernel
  // the state arrays below live in one device block laid out like the pinned staging
  // buffer, so an upload is a single copy
  unsigned char* d_state = nullptr;
  double2 *d_NXA = nullptr, *d_gamma = nullptr, *d_Xgamma = nullptr;
  float2 *d_NXA_hi = nullptr, *d_NXA_lo = nullptr, *d_Xg_hi = nullptr, *d_Xg_lo = nullptr;
  float2 *d_g_hi = nullptr, *d_g_lo = nullptr;
  longlong2* d_NXA_fix = nullptr;
  double* d_ldfin = nullptr;          // warp kernel: unfinished log det per evaluated point
  unsigned* d_bar = nullptr;          // grid-barrier state of the fused DFT launch
  double2* d_H = nullptr;             // Hessenberg form of XA (one-group, undisplaced plans)
  // tree plans: rows ordered by group (tree_perm[new] = old), depth-0 arrays in d_state,
  // depths 1 .. L-1 in d_tree
  std::vector<int> tree_perm;
  TreeArgs tree{};
  bool tree_g = false;                // undisplaced tree plan: leaves write G, the DFT skips a stage
  double tree_logq0 = 0.0;            // Re log q(1) from the host LU (diagnostics)
  unsigned char* d_tree = nullptr;
  // large-matrix tree plans (kernels 13, 14): the same row order, depth-0 augmented matrix in
  // d_state, the other depths, sub-step scratch and Hessenberg leaves in d_tree
  BTreeArgs btree{};
  std::vector<BTreeStep> btree_steps;
  size_t bt_scratch[3] = {0, 0, 0};   // 16-byte slots: each trailing-block buffer, pivot rows, reciprocals
  cd logq1 = 0.0;                     // sharded large-matrix tree plans: log q(1) of the state (host FP64)
  double logq1_minpiv = 1.0;          // and the smallest real part of its pivots
  int last_launches = 0;              // kernel launches of the last execute
  long long upload_bytes = 0;         // host-to-device bytes of one state upload
  int* d_label = nullptr;
  double2* d_logq = nullptr;
  double* d_minpiv = nullptr;
  double2 *d_bufA = nullptr, *d_bufB = nullptr;
  double2* d_tw = nullptr;
  float4* d_twdf = nullptr;           // tree plans: the roots w = conj(twiddle) as pairs of FP32
  double* d_diag = nullptr;
  double* d_table = nullptr;  // device copy of the table for execute_host
  void* d_gws = nullptr;
  long long gws_slot_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // reverse pass
  bool physical = false;              // state given as r, T (alpha, V)
  std::vector<double> r;
  std::vector<cd> T, alpha, V, zbar;
  bool has_alpha = false, has_V = false;
  double2 *d_adjA = nullptr, *d_adjB = nullptr, *d_bws = nullptr;
  double2 *d_partS = nullptr, *d_partg = nullptr, *d_outS = nullptr, *d_outg = nullptr;
  bool logq_valid = false;            // d_logq holds the current state's log q (an execute ran)
  bool dft_plain = false;             // tree plans inside a batch: the inverse DFT as ordinary
                                      // launches (several trees run at once on side streams, and
                                      // cooperative launches are not run concurrently)
  long long bws_slot_bytes = 0;       // per-SM slot of d_bws (the reverse pass's matrices)
  cudaEvent_t ev_b0 = nullptr, ev_b1 = nullptr;   // want_timing: around the reverse per-point kernel
  bool backward_ran = false;
  // reverse pass along the large-matrix tree (non-shard tree plans where it pays)
  bool bwd_tree = false;
  BwdTree bt{};
  long long bt_parents = 0, bt_wave = 0;
  unsigned char* d_bt = nullptr;      // parent buffers of one wave, leaf partials, pinv
  // pinned staging for uploads
  // two pinned staging buffers used in turn, each with the event recorded after the copy
  // that last read it: an upload waits only for the copy two uploads back
  void* h_stage[2] = {nullptr, nullptr};
  cudaEvent_t ev_stage[2] = {nullptr, nullptr};
  int stage_next = 0;
  size_t h_stage_bytes = 0;
};

namespace {

const double kHermTol = 1e-10;

int check_cuda(cudaError_t e) { return e == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA; }

// ---------------------------------------------------------------- validation
int validate_shape(const gbsbin_problem* p, const gbsbin_options* o) {
  if (!p || !o) return GBSBIN_ERR_ARG;
  if (p->M <= 0 || p->K <= 0) return GBSBIN_ERR_ARG;
  if (p->L < 1 || p->L > p->M || p->L > GBSBIN_MAX_L) return GBSBIN_ERR_ARG;
  if (!p->bin_of_mode || !p->cutoff) return GBSBIN_ERR_ARG;
  if (!p->sigma1 && (!p->r || !p->T)) return GBSBIN_ERR_ARG;
  if (o->precision != GBSBIN_FP64 && o->precision != GBSBIN_FP32_REFINE) return GBSBIN_ERR_ARG;
  if (o->oversample < 1) return GBSBIN_ERR_ARG;
  if (o->tile_override < 0 ||
      (o->tile_override > GBSBIN_KERNEL_HESS_FP64 && o->tile_override != GBSBIN_KERNEL_TREE_DF32 &&
       o->tile_override != GBSBIN_KERNEL_TREE_FP64 && o->tile_override != GBSBIN_KERNEL_BTREE_DF32 &&
       o->tile_override != GBSBIN_KERNEL_BTREE_FP64 && o->tile_override != GBSBIN_KERNEL_HESS_DF32))
    return GBSBIN_ERR_ARG;
  long long n = 2LL * p->M * p->K;
  if (n > GBSBIN_MAX_N) return GBSBIN_ERR_UNSUPPORTED;
  std::vector<int> count(p->L, 0);
  for (int j = 0; j < p->M; ++j) {
    int b = p->bin_of_mode[j];
    if (b < 0 || b >= p->L) return GBSBIN_ERR_PARTITION;
    count[b]++;
  }
  for (int l = 0; l < p->L; ++l)
    if (count[l] == 0) return GBSBIN_ERR_PARTITION;
  long long npts = 1;
  for (int l = 0; l < p->L; ++l) {
    if (p->cutoff[l] < 0) return GBSBIN_ERR_CUTOFF;
    long long R = (long long)o->oversample * (p->cutoff[l] + 1LL);
    if (R > (1LL << 26)) return GBSBIN_ERR_CUTOFF;
    npts *= R;
    if (npts > GBSBIN_MAX_POINTS) return GBSBIN_ERR_CUTOFF;
  }
  return GBSBIN_OK;
}

// ------------------------------------------------------- Gaussian-state algebra
// Normally ordered covariance Sigma^(1) (n x n) and mean z-bar of the output state.
// Sigma^(1)_in = [[N^T, Mm], [Mm^*, N]] with N = diag(sinh^2 r), Mm = diag(sinh r cosh r);
// Sigma^(1)_out = W Sigma^(1)_in W^dag, W = T_full (+) T_full^*.
int physical_state(const gbsbin_problem* p, std::vector<cd>& S1, std::vector<cd>& zbar) {
  const int M = p->M, K = p->K, MK = M * K, n = 2 * MK;
  for (int q = 0; q < MK; ++q)
    if (!std::isfinite(p->r[q])) return GBSBIN_ERR_ARG;
  std::vector<cd> Tf((size_t)MK * MK, 0.0);
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      cd t(p->T[j * M + i].re, p->T[j * M + i].im);
      if (!std::isfinite(t.real()) || !std::isfinite(t.imag())) return GBSBIN_ERR_ARG;
      for (int l = 0; l < K; ++l)
        for (int k = 0; k < K; ++k) {
          cd v = (l == k) ? cd(1.0) : cd(0.0);
          if (p->V) v = cd(p->V[(i * K + l) * K + k].re, p->V[(i * K + l) * K + k].im);
          Tf[(size_t)(j * K + l) * MK + (i * K + k)] = t * v;
        }
    }
  std::vector<double> nn(MK), mm(MK);
  for (int q = 0; q < MK; ++q) {
    double sh = std::sinh(p->r[q]), ch = std::cosh(p->r[q]);
    nn[q] = sh * sh;
    mm[q] = sh * ch;
  }
  // N_out[a][b] = sum_q conj(Tf[a][q]) n_q Tf[b][q] (Hermitian), Mm_out[a][b] = sum_q
  // Tf[a][q] m_q Tf[b][q] (symmetric): the b >= a half, on split real/imaginary rows
  std::vector<double> tr((size_t)MK * MK), ti((size_t)MK * MK), nr((size_t)MK * MK), ni((size_t)MK * MK),
      mr((size_t)MK * MK), mi((size_t)MK * MK);
  for (size_t q = 0; q < (size_t)MK * MK; ++q) {
    const double w_n = nn[q % MK], w_m = mm[q % MK];
    tr[q] = Tf[q].real();
    ti[q] = Tf[q].imag();
    nr[q] = tr[q] * w_n;                            // conj(Tf) n
    ni[q] = -ti[q] * w_n;
    mr[q] = tr[q] * w_m;                            // Tf m
    mi[q] = ti[q] * w_m;
  }
  S1.assign((size_t)n * n, 0.0);
  // every unordered pair {a, b} belongs to the thread of min(a, b): rows dealt cyclically
  parallel_run(MK >= 32 ? host_threads() : 1, [&](int t, int nt) {
  for (int a = t; a < MK; a += nt)
    for (int b = a; b < MK; ++b) {
      const double *ar = &nr[(size_t)a * MK], *ai = &ni[(size_t)a * MK], *br = &tr[(size_t)b * MK],
                   *bi = &ti[(size_t)b * MK], *cr = &mr[(size_t)a * MK], *ci = &mi[(size_t)a * MK];
      double Nr = 0.0, Ni = 0.0, Mr = 0.0, Mi = 0.0;
      for (int q = 0; q < MK; ++q) {
        Nr += ar[q] * br[q] - ai[q] * bi[q];
        Ni += ar[q] * bi[q] + ai[q] * br[q];
        Mr += cr[q] * br[q] - ci[q] * bi[q];
        Mi += cr[q] * bi[q] + ci[q] * br[q];
      }
      const cd N(Nr, Ni), Mo(Mr, Mi);
      S1[(size_t)b * n + a] = N;                     // top-left: N^T
      S1[(size_t)a * n + (MK + b)] = Mo;             // top-right: Mm
      S1[(size_t)(MK + a) * n + b] = std::conj(Mo);  // bottom-left: Mm^*
      S1[(size_t)(MK + a) * n + (MK + b)] = N;       // bottom-right: N
      if (b != a) {                                  // (b, a): conj(N), Mo
        S1[(size_t)a * n + b] = std::conj(N);
        S1[(size_t)b * n + (MK + a)] = Mo;
        S1[(size_t)(MK + b) * n + a] = std::conj(Mo);
        S1[(size_t)(MK + b) * n + (MK + a)] = std::conj(N);
      }
    }
  });
  zbar.assign(n, 0.0);
  if (p->alpha) {
    for (int a = 0; a < MK; ++a) {
      cd s = 0.0;
      for (int q = 0; q < MK; ++q) s += Tf[(size_t)a * MK + q] * cd(p->alpha[q].re, p->alpha[q].im);
      zbar[a] = s;
      zbar[MK + a] = std::conj(s);
    }
  }
  return GBSBIN_OK;
}

// Complex dot products over split real / imaginary rows: MODE 0: sum a_k b_k,
// 1: sum a_k conj(b_k), 2: sum conj(a_k) b_k.
template <int MODE>
inline void cdot(const double* __restrict__ ar, const double* __restrict__ ai, const double* __restrict__ br,
                 const double* __restrict__ bi, int len, double* re, double* im) {
  double r = 0.0, m = 0.0;
  for (int k = 0; k < len; ++k) {
    if (MODE == 0) {
      r += ar[k] * br[k] - ai[k] * bi[k];
      m += ar[k] * bi[k] + ai[k] * br[k];
    } else if (MODE == 1) {
      r += ar[k] * br[k] + ai[k] * bi[k];
      m += ai[k] * br[k] - ar[k] * bi[k];
    } else {
      r += ar[k] * br[k] + ai[k] * bi[k];
      m += ar[k] * bi[k] - ai[k] * br[k];
    }
  }
  *re = r;
  *im = m;
}

// In-place Cholesky of a Hermitian matrix (lower factor) held as split real / imaginary
// row-major arrays; false if not positive definite.  Blocked right-looking: per block of B
// columns the diagonal block is factored on one thread (L_jj = sqrt(A_jj - sum_k |L_jk|^2),
// L_ij = (A_ij - sum_k L_ik conj(L_jk)) / L_jj over the block's earlier columns), then the
// rows below are solved against it and the trailing matrix updated, A_ij -= sum over the
// block of L_ik conj(L_jk), both in parallel over rows (dealt cyclically).
bool cholesky(std::vector<double>& re, std::vector<double>& im, int n) {
  const int B = 48;
  const int nt = n >= 96 ? host_threads() : 1;
  for (int k0 = 0; k0 < n; k0 += B) {
    const int k1 = std::min(n, k0 + B);
    for (int j = k0; j < k1; ++j) {
      const double* rj = &re[(size_t)j * n];
      const double* ij = &im[(size_t)j * n];
      double d = rj[j];
      for (int k = k0; k < j; ++k) d -= rj[k] * rj[k] + ij[k] * ij[k];
      if (!(d > 0.0) || !std::isfinite(d)) return false;
      const double ljj = std::sqrt(d);
      re[(size_t)j * n + j] = ljj;
      im[(size_t)j * n + j] = 0.0;
      for (int i = j + 1; i < k1; ++i) {
        double* ri = &re[(size_t)i * n];
        double* ii = &im[(size_t)i * n];
        double sr = ri[j], si = ii[j];
        for (int k = k0; k < j; ++k) {
          sr -= ri[k] * rj[k] + ii[k] * ij[k];
          si -= ii[k] * rj[k] - ri[k] * ij[k];
        }
        ri[j] = sr / ljj;
        ii[j] = si / ljj;
      }
    }
    if (k1 == n) break;
    parallel_run(nt, [&](int t, int nth) {            // rows below the block: L_i,[k0,k1)
      for (int i = k1 + t; i < n; i += nth) {
        double* ri = &re[(size_t)i * n];
        double* ii = &im[(size_t)i * n];
        for (int j = k0; j < k1; ++j) {
          const double* rj = &re[(size_t)j * n];
          const double* ij = &im[(size_t)j * n];
          double sr, si;
          cdot<1>(ri + k0, ii + k0, rj + k0, ij + k0, j - k0, &sr, &si);
          ri[j] = (ri[j] - sr) / rj[j];
          ii[j] = (ii[j] - si) / rj[j];
        }
      }
    });
    parallel_run(nt, [&](int t, int nth) {            // trailing update of the lower triangle
      for (int i = k1 + t; i < n; i += nth) {
        double* ri = &re[(size_t)i * n];
        double* ii = &im[(size_t)i * n];
        for (int j = k1; j <= i; ++j) {
          const double* rj = &re[(size_t)j * n];
          const double* ij = &im[(size_t)j * n];
          double sr, si;
          cdot<1>(ri + k0, ii + k0, rj + k0, ij + k0, k1 - k0, &sr, &si);
          ri[j] -= sr;
          ii[j] -= si;
        }
      }
    });
  }
  return true;
}

// XA = I - Sigma^{-1}, Xgamma = Sigma^{-1} z-bar, gamma = X Xgamma, Sigma = I + Sigma^(1).
int adjacency(const std::vector<cd>& S1, const std::vector<cd>& zbar, int n, std::vector<cd>& XA,
              std::vector<cd>& gamma, std::vector<cd>& Xgamma) {
  double scale2 = 1.0;                               // running max of |a|^2 (squares compared)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cd a = S1[(size_t)i * n + j], b = S1[(size_t)j * n + i];
      if (!std::isfinite(a.real()) || !std::isfinite(a.imag())) return GBSBIN_ERR_ARG;
      scale2 = std::fmax(scale2, std::norm(a));
      if (std::norm(a - std::conj(b)) > kHermTol * kHermTol * scale2) return GBSBIN_ERR_NONPHYSICAL;
    }
  // physicality: Sigma - I/2 = Sigma^(1) + I/2 positive definite <=> ||I - Sigma^{-1}|| < 1
  const size_t nn = (size_t)n * n;
  std::vector<double> cr(nn), ci(nn);
  for (size_t q = 0; q < nn; ++q) {
    cr[q] = S1[q].real();
    ci[q] = S1[q].imag();
  }
  for (int i = 0; i < n; ++i) cr[(size_t)i * n + i] += 0.5;
  if (!cholesky(cr, ci, n)) return GBSBIN_ERR_NONPHYSICAL;
  // Sigma = C C^H; Sigma^{-1} = C^{-H} C^{-1}
  for (size_t q = 0; q < nn; ++q) {
    cr[q] = S1[q].real();
    ci[q] = S1[q].imag();
  }
  for (int i = 0; i < n; ++i) cr[(size_t)i * n + i] += 1.0;
  if (!cholesky(cr, ci, n)) return GBSBIN_ERR_NONPHYSICAL;
  // X = C^{-1} (lower triangular) column by column, stored transposed (xr, xi row j = column
  // j of X): X_jj = 1 / C_jj, X_ij = -(sum_{j <= k < i} C_ik X_kj) / C_ii; columns in parallel,
  // dealt cyclically from the longest
  const int nt = n >= 96 ? host_threads() : 1;
  std::vector<double> xr(nn, 0.0), xi(nn, 0.0);
  parallel_run(nt, [&](int t, int nth) {
    for (int j = t; j < n; j += nth) {
      double* xrj = &xr[(size_t)j * n];
      double* xij = &xi[(size_t)j * n];
      xrj[j] = 1.0 / cr[(size_t)j * n + j];
      for (int i = j + 1; i < n; ++i) {
        const double* ci_r = &cr[(size_t)i * n];
        const double* ci_i = &ci[(size_t)i * n];
        double sr, si;
        cdot<0>(ci_r + j, ci_i + j, xrj + j, xij + j, i - j, &sr, &si);
        const double cii = ci_r[i];
        xrj[i] = -sr / cii;
        xij[i] = -si / cii;
      }
    }
  });
  // S = X^H X (lower half): S_ij = sum_{k >= i} conj(X_ki) X_kj, j <= i - dot products of the
  // stored columns i and j over k >= i; rows in parallel
  std::vector<double> sr(nn, 0.0), si(nn, 0.0);
  parallel_run(nt, [&](int t, int nth) {
    for (int i = t; i < n; i += nth) {
      const double* ar = &xr[(size_t)i * n];
      const double* ai = &xi[(size_t)i * n];
      for (int j = 0; j <= i; ++j) {
        const double* br = &xr[(size_t)j * n];
        const double* bi = &xi[(size_t)j * n];
        double vr, vi;
        cdot<2>(ar + i, ai + i, br + i, bi + i, n - i, &vr, &vi);
        sr[(size_t)i * n + j] = vr;
        si[(size_t)i * n + j] = vi;
      }
    }
  });
  XA.assign(nn, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      const cd v(sr[(size_t)i * n + j], si[(size_t)i * n + j]);
      XA[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - v;
      if (i != j) XA[(size_t)j * n + i] = -std::conj(v);
    }
  Xgamma.assign(n, 0.0);
  gamma.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    cd s = 0.0;
    for (int j = 0; j < n; ++j) {
      cd sij = (i == j ? 1.0 : 0.0) - XA[(size_t)i * n + j];  // Sigma^{-1}
      s += sij * zbar[j];
    }
    Xgamma[i] = s;
  }
  const int h = n / 2;
  for (int i = 0; i < n; ++i) gamma[i] = Xgamma[i < h ? i + h : i - h];
  return GBSBIN_OK;
}

int build_state(const gbsbin_problem* p, int n, std::vector<cd>& XA, std::vector<cd>& gamma,
                std::vector<cd>& Xgamma, int* has_gamma, std::vector<cd>* zbar_out = nullptr,
                std::vector<cd>* s1_out = nullptr) {
  std::vector<cd> S1, zbar;
  if (p->sigma1) {
    S1.resize((size_t)n * n);
    for (size_t q = 0; q < S1.size(); ++q) S1[q] = cd(p->sigma1[q].re, p->sigma1[q].im);
    zbar.assign(n, 0.0);
    if (p->zbar)
      for (int q = 0; q < n; ++q) zbar[q] = cd(p->zbar[q].re, p->zbar[q].im);
  } else {
    int st = physical_state(p, S1, zbar);
    if (st) return st;
  }
  int st = adjacency(S1, zbar, n, XA, gamma, Xgamma);
  if (st) return st;
  if (zbar_out) *zbar_out = zbar;
  if (s1_out) s1_out->swap(S1);
  *has_gamma = 0;
  for (int i = 0; i < n; ++i)
    if (gamma[i] != cd(0.0)) *has_gamma = 1;
  return GBSBIN_OK;
}

void free_device(gbsbin_plan* P) {
  if (P->d_twdf) cudaFree(P->d_twdf);
  void* ptrs[] = {P->d_state, P->d_label, P->d_logq,  P->d_minpiv, P->d_bufA, P->d_bufB, P->d_tw,
                  P->d_diag,  P->d_gws,   P->d_table, P->d_ldfin,  P->d_bar,  P->d_H,    P->d_tree};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int b = 0; b < 2; ++b) {
    if (P->h_stage[b]) cudaFreeHost(P->h_stage[b]);
    if (P->ev_stage[b]) cudaEventDestroy(P->ev_stage[b]);
  }
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->ev_b0) cudaEventDestroy(P->ev_b0);
  if (P->ev_b1) cudaEventDestroy(P->ev_b1);
  void* bw[] = {P->d_adjA, P->d_adjB, P->d_bws, P->d_partS, P->d_partg, P->d_outS, P->d_outg, P->d_bt};
  for (void* q : bw)
    if (q) cudaFree(q);
}

template <typename T>
int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return GBSBIN_ERR_NOMEM;
  }
  return check_cuda(e);
}

// The tree of block eliminations, in pairs of FP32 or in FP64; and its large-matrix form.
inline bool is_tree(int kernel) { return kernel == GBSBIN_KERNEL_TREE_DF32 || kernel == GBSBIN_KERNEL_TREE_FP64; }
inline bool is_hess(int kernel) { return kernel == GBSBIN_KERNEL_HESS_FP64 || kernel == GBSBIN_KERNEL_HESS_DF32; }
inline bool is_btree(int kernel) { return kernel == GBSBIN_KERNEL_BTREE_DF32 || kernel == GBSBIN_KERNEL_BTREE_FP64; }
// 16-byte slots of a tree plan's depth-0 region in the state block
size_t tree_region_slots(int n, int kernel) {
  if (is_tree(kernel)) return (size_t)n * n + 2 * (size_t)n + 3;   // permuted XA, X gamma, gamma, path record
  if (is_btree(kernel)) return (size_t)(n + 1) * (n + 1) + 2;    // augmented matrix, path record
  return 0;
}

// Layout of the pinned staging buffer for one state upload.
struct Stage {
  size_t off_XA, off_g, off_Xg, off_XAhi, off_XAlo, off_Xghi, off_Xglo, off_ghi, off_glo, off_XAfix;
  size_t off_tree;   // tree plans: permuted XA (n x n), X gamma, gamma (FP32 pairs or FP64), root path record
  size_t total;
};
Stage stage_layout(int n, size_t tree_slots) {
  Stage s{};
  size_t nn = (size_t)n * n, o = 0;
  s.off_XA = o;   o += nn * sizeof(double2);
  s.off_g = o;    o += n * sizeof(double2);
  s.off_Xg = o;   o += n * sizeof(double2);
  s.off_XAhi = o; o += nn * sizeof(float2);
  s.off_XAlo = o; o += nn * sizeof(float2);
  s.off_Xghi = o; o += n * sizeof(float2);
  s.off_Xglo = o; o += n * sizeof(float2);
  s.off_ghi = o;  o += n * sizeof(float2);
  s.off_glo = o;  o += n * sizeof(float2);
  s.off_XAfix = o; o += nn * sizeof(longlong2);
  s.off_tree = o;
  o += tree_slots * sizeof(float4);
  s.total = o;
  return s;
}

// v as a pair of FP32 per component: (hi re, hi im, lo re, lo im)
float4 split4(cd v) {
  const float hr = (float)v.real(), hi = (float)v.imag();
  return make_float4(hr, hi, (float)(v.real() - (double)hr), (float)(v.imag() - (double)hi));
}

void split(cd v, float2* hi, float2* lo) {
  float hr = (float)v.real(), hi_ = (float)v.imag();
  *hi = make_float2(hr, hi_);
  *lo = make_float2((float)(v.real() - (double)hr), (float)(v.imag() - (double)hi_));
}

int upload_hessenberg(gbsbin_plan* P, cudaStream_t stream);

// Stage the state and enqueue its upload on `stream`.
int upload_state(gbsbin_plan* P, cudaStream_t stream) {
  const int n = P->n;
  const bool tree = is_tree(P->kernel) || is_btree(P->kernel);
  const bool per_point = !tree || P->opt.want_backward;   // the reverse pass reads -XA, gamma, X gamma
  Stage s = stage_layout(n, tree_region_slots(n, P->kernel));
  // the copy that last read this staging buffer (two uploads back) must have finished
  const int sb = P->stage_next;
  P->stage_next ^= 1;
  cudaError_t e = cudaEventSynchronize(P->ev_stage[sb]);
  if (e != cudaSuccess) return GBSBIN_ERR_CUDA;
  char* h = (char*)P->h_stage[sb];
  double2* XA = (double2*)(h + s.off_XA);
  double2* g = (double2*)(h + s.off_g);
  double2* Xg = (double2*)(h + s.off_Xg);
  float2* XAhi = (float2*)(h + s.off_XAhi);
  float2* XAlo = (float2*)(h + s.off_XAlo);
  float2* Xghi = (float2*)(h + s.off_Xghi);
  float2* Xglo = (float2*)(h + s.off_Xglo);
  float2* ghi = (float2*)(h + s.off_ghi);
  float2* glo = (float2*)(h + s.off_glo);
  longlong2* XAfix = (longlong2*)(h + s.off_XAfix);
  // the per-point kernels' copies of the state (tree plans read only their own region, and
  // their reverse pass the FP64 copies)
  const double fix_scale = std::ldexp(1.0, GBSBIN_FIX_BITS);
  for (size_t q = 0; per_point && q < (size_t)n * n; ++q) {  // the kernels use -XA
    XA[q] = make_double2(-P->XA[q].real(), -P->XA[q].imag());
    split(-P->XA[q], &XAhi[q], &XAlo[q]);
    // |XA_ij| <= ||XA||_2 < 1 for a physical state, so the scaled value fits in 63 bits
    XAfix[q] = make_longlong2(std::llrint(-P->XA[q].real() * fix_scale), std::llrint(-P->XA[q].imag() * fix_scale));
  }
  for (int i = 0; per_point && i < n; ++i) {
    g[i] = make_double2(P->gamma[i].real(), P->gamma[i].imag());
    Xg[i] = make_double2(P->Xgamma[i].real(), P->Xgamma[i].imag());
    split(P->Xgamma[i], &Xghi[i], &Xglo[i]);
    split(P->gamma[i], &ghi[i], &glo[i]);
  }
  if (is_btree(P->kernel) && P->grid.e_lo > 0)     // a shard without point 0: log q(1) on the host
    P->logq1 = host_logq1(P->XA, P->gamma, P->Xgamma, n, &P->logq1_minpiv);
  if (is_btree(P->kernel)) {                       // depth 0: the permuted augmented matrix
    float4* A0 = (float4*)(h + s.off_tree);
    const std::vector<int>& pm = P->tree_perm;
    const bool f64 = P->kernel == GBSBIN_KERNEL_BTREE_FP64;
    auto slot = [f64](cd v) {
      if (!f64) return split4(v);
      float4 o;
      const double2 d = make_double2(v.real(), v.imag());
      std::memcpy(&o, &d, sizeof(o));
      return o;
    };
    const size_t D = (size_t)n + 1;
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) A0[i * D + j] = slot(P->XA[(size_t)pm[i] * n + pm[j]]);
      A0[i * D + n] = slot(P->Xgamma[pm[i]]);             // c: v = D(w) c
      A0[n * D + i] = slot(P->gamma[pm[i]]);              // u
    }
    A0[n * D + n] = slot(cd(0.0, 0.0));                   // the exponent collected so far
    A0[D * D] = slot(cd(1.0, 0.0));                       // path record: pivot product
    A0[D * D + 1] = make_float4(0.f, 0.f, 3.0e38f, 0.f);  // argument sum, power of two, min Re pivot
  } else if (tree) {                               // depth 0 of the tree: the permuted state
    float4* A0 = (float4*)(h + s.off_tree);
    float4* c0 = A0 + (size_t)n * n;
    float4* u0 = c0 + n;
    float4* path = u0 + n;
    const std::vector<int>& pm = P->tree_perm;
    const bool f64 = P->kernel == GBSBIN_KERNEL_TREE_FP64;
    // one 16-byte slot per element: (hi re, hi im, lo re, lo im) FP32 pairs, or a double2
    auto slot = [f64](cd v) {
      if (!f64) return split4(v);
      float4 o;
      const double2 d = make_double2(v.real(), v.imag());
      std::memcpy(&o, &d, sizeof(o));
      return o;
    };
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) A0[(size_t)i * n + j] = slot(P->XA[(size_t)pm[i] * n + pm[j]]);
      c0[i] = slot(P->Xgamma[pm[i]]);
      u0[i] = slot(P->gamma[pm[i]]);
    }
    path[0] = slot(cd(1.0, 0.0));                       // pivot product
    path[1] = make_float4(0.f, 0.f, 3.0e38f, 0.f);    // argument sum, power of two, min Re pivot
    path[2] = slot(cd(0.0, 0.0));                       // exponent sum
    // the w = 1 point on the host: unpivoted LU of I - XA in the tree's row order, its pivot
    // product p0 2^e0, argument and winding (each pivot has Re > 0)
    P->tree_g = !P->has_gamma;
    if (P->tree_g) {
      // split real / imaginary rows; each pivot's reciprocal once, rows updated contiguously
      std::vector<double> kr((size_t)n * n), ki((size_t)n * n);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const cd v = (i == j ? 1.0 : 0.0) - P->XA[(size_t)pm[i] * n + pm[j]];
          kr[(size_t)i * n + j] = v.real();
          ki[(size_t)i * n + j] = v.imag();
        }
      cd prod = 1.0;
      int e0 = 0;
      double args = 0.0;
      for (int k = 0; k < n; ++k) {
        const cd piv(kr[(size_t)k * n + k], ki[(size_t)k * n + k]);
        prod *= piv;
        int ex;
        std::frexp(std::max(std::fabs(prod.real()), std::fabs(prod.imag())), &ex);
        prod = cd(std::ldexp(prod.real(), -ex), std::ldexp(prod.imag(), -ex));
        e0 += ex;
        args += std::atan2(piv.imag(), piv.real());
        const double d = std::norm(piv), pr = piv.real() / d, pi = -piv.imag() / d;   // 1 / piv
        const double* rk = &kr[(size_t)k * n];
        const double* ik = &ki[(size_t)k * n];
        for (int i = k + 1; i < n; ++i) {
          double* ri = &kr[(size_t)i * n];
          double* ii = &ki[(size_t)i * n];
          const double lr = ri[k] * pr - ii[k] * pi, lim = ri[k] * pi + ii[k] * pr;
          for (int j = k + 1; j < n; ++j) {
            ri[j] -= lr * rk[j] - lim * ik[j];
            ii[j] -= lr * ik[j] + lim * rk[j];
          }
        }
      }
      const double TWO_PI = 6.283185307179586476925286766559;
      const double arg0 = std::atan2(prod.imag(), prod.real());
      P->tree.p0re = prod.real();
      P->tree.p0im = prod.imag();
      P->tree.p0df = split4(prod);
      P->tree.p0arg = (float)arg0;
      P->tree.e0 = (float)e0;
      P->tree.m0 = (float)std::nearbyint((args - arg0) / TWO_PI);
      P->tree_logq0 = -0.5 * (std::log(std::abs(prod)) + e0 * 0.693147180559945309417232121458);
    }
  }
  // the device block has the staging layout: one copy (of the tree region alone for trees
  // without a reverse pass)
  const size_t off = per_point ? 0 : s.off_tree;
  P->upload_bytes = (long long)(s.total - off);
  e = cudaMemcpyAsync(P->d_state + off, h + off, s.total - off, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess || cudaEventRecord(P->ev_stage[sb], stream) != cudaSuccess) return GBSBIN_ERR_CUDA;
  if (is_hess(P->kernel)) return upload_hessenberg(P, stream);
  return GBSBIN_OK;
}

// In place: A (n x n, row-major) <- Q^H A Q upper Hessenberg, Q a product of Householder
// reflectors (FP64); each reflector is also applied to the vectors in `vecs` (which become
// Q^H vec).  Similar matrices share det(I - w A) for every w.
void hessenberg(std::vector<cd>& A, int n, std::vector<std::vector<cd>*> vecs = {}) {
  std::vector<cd> v(n), sv(n);
  for (int k = 0; k + 2 < n; ++k) {
    double nrm2 = 0.0;
    for (int i = k + 1; i < n; ++i) nrm2 += std::norm(A[(size_t)i * n + k]);
    if (nrm2 == 0.0) continue;
    const double nrm = std::sqrt(nrm2);
    const cd x0 = A[(size_t)(k + 1) * n + k];
    const double ax0 = std::abs(x0);
    const cd alpha = (ax0 > 0.0 ? -x0 / ax0 : cd(-1.0, 0.0)) * nrm;   // -e^{i arg x0} ||x||
    for (int i = k + 1; i < n; ++i) v[i] = A[(size_t)i * n + k];
    v[k + 1] -= alpha;
    double vn2 = 0.0;
    for (int i = k + 1; i < n; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;
    // rows k+1.. : A <- (I - beta v v^H) A
    for (int j = 0; j < n; ++j) sv[j] = 0.0;
    for (int i = k + 1; i < n; ++i) {
      const cd vc = std::conj(v[i]);
      const cd* row = &A[(size_t)i * n];
      for (int j = 0; j < n; ++j) sv[j] += vc * row[j];
    }
    for (int i = k + 1; i < n; ++i) {
      const cd vi = beta * v[i];
      cd* row = &A[(size_t)i * n];
      for (int j = 0; j < n; ++j) row[j] -= vi * sv[j];
    }
    // columns k+1.. : A <- A (I - beta v v^H)
    for (int i = 0; i < n; ++i) {
      cd* row = &A[(size_t)i * n];
      cd t = 0.0;
      for (int j = k + 1; j < n; ++j) t += row[j] * v[j];
      t *= beta;
      for (int j = k + 1; j < n; ++j) row[j] -= t * std::conj(v[j]);
    }
    for (std::vector<cd>* x : vecs) {           // x <- (I - beta v v^H) x
      cd t = 0.0;
      for (int i = k + 1; i < n; ++i) t += std::conj(v[i]) * (*x)[i];
      t *= beta;
      for (int i = k + 1; i < n; ++i) (*x)[i] -= t * v[i];
    }
    A[(size_t)(k + 1) * n + k] = alpha;
    for (int i = k + 2; i < n; ++i) A[(size_t)i * n + k] = 0.0;
  }
}

// The one-group plans' Hessenberg form of the current XA, followed by a = Q^T gamma and
// c = Q^H X gamma (the exponent gamma^T (conj(w) - XA)^{-1} X gamma = a^T (conj(w) - H)^{-1} c),
// uploaded on `stream`.
int upload_hessenberg(gbsbin_plan* P, cudaStream_t stream) {
  const int n = P->n;
  std::vector<cd> H(P->XA), ga(n), c(P->Xgamma);
  for (int i = 0; i < n; ++i) ga[i] = std::conj(P->gamma[i]);     // Q^T g = conj(Q^H conj(g))
  hessenberg(H, n, {&ga, &c});
  std::vector<double2> h((size_t)n * n + 2 * (size_t)n);
  for (size_t q = 0; q < (size_t)n * n; ++q) h[q] = make_double2(H[q].real(), H[q].imag());
  for (int i = 0; i < n; ++i) {
    h[(size_t)n * n + i] = make_double2(ga[i].real(), -ga[i].imag());
    h[(size_t)n * n + n + i] = make_double2(c[i].real(), c[i].imag());
  }
  if (P->kernel == GBSBIN_KERNEL_HESS_DF32)        // pairs of FP32 in the same 16-byte slots
    for (size_t q = 0; q < h.size(); ++q) {
      const float4 f = split4(cd(h[q].x, h[q].y));
      std::memcpy(&h[q], &f, sizeof(f));
    }
  // a pageable source: the call returns once the data are staged, so h may go out of scope
  if (cudaMemcpyAsync(P->d_H, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  P->upload_bytes += (long long)(h.size() * sizeof(double2));
  return GBSBIN_OK;
}

void record_inputs(gbsbin_plan* P, const gbsbin_problem* p) {
  const int M = p->M, K = p->K;
  P->physical = p->sigma1 == nullptr;
  if (!P->physical) return;
  P->r.assign(p->r, p->r + M * K);
  P->T.resize((size_t)M * M);
  for (int q = 0; q < M * M; ++q) P->T[q] = cd(p->T[q].re, p->T[q].im);
  P->has_alpha = p->alpha != nullptr;
  P->alpha.assign((size_t)M * K, 0.0);
  if (p->alpha)
    for (int q = 0; q < M * K; ++q) P->alpha[q] = cd(p->alpha[q].re, p->alpha[q].im);
  P->has_V = p->V != nullptr;
  P->V.assign((size_t)M * K * K, 0.0);
  for (int i = 0; i < M; ++i)
    for (int l = 0; l < K; ++l)
      for (int k = 0; k < K; ++k)
        P->V[((size_t)i * K + l) * K + k] = p->V ? cd(p->V[(i * K + l) * K + k].re, p->V[(i * K + l) * K + k].im)
                                                 : cd(l == k ? 1.0 : 0.0);
}


// ------------------------------------------------------------ reverse-pass helpers
// C = A B for n x n row-major complex matrices (i, k, j loop order).
// C = A B (n x n, complex, row-major): rows of C in parallel on the host threads, each row
// accumulated over k in order with the products written out in real arithmetic (the library's
// complex operator would guard every product against infinities).
void matmul(const std::vector<cd>& A, const std::vector<cd>& B, std::vector<cd>& C, int n) {
  C.assign((size_t)n * n, 0.0);
  const double* a = reinterpret_cast<const double*>(A.data());
  const double* b = reinterpret_cast<const double*>(B.data());
  double* c = reinterpret_cast<double*>(C.data());
  parallel_run(n >= 64 ? host_threads() : 1, [&](int t, int nt) {
    for (int i = t; i < n; i += nt) {
      double* ci = c + (size_t)2 * i * n;
      for (int k = 0; k < n; ++k) {
        const double ar = a[2 * ((size_t)i * n + k)], ai = a[2 * ((size_t)i * n + k) + 1];
        if (ar == 0.0 && ai == 0.0) continue;
        const double* bk = b + (size_t)2 * k * n;
        for (int j = 0; j < n; ++j) {
          const double br = bk[2 * j], bi = bk[2 * j + 1];
          ci[2 * j] += ar * br - ai * bi;
          ci[2 * j + 1] += ar * bi + ai * br;
        }
      }
    }
  });
}

std::vector<cd> transpose(const std::vector<cd>& A, int n) {
  std::vector<cd> T((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[(size_t)j * n + i] = A[(size_t)i * n + j];
  return T;
}

// The blocked FP32 + refinement kernel, with its trace updates on the CUDA cores or on the
// tensor cores.
inline bool is_blk(int kernel) { return kernel == GBSBIN_KERNEL_BLK_FP32R || kernel == GBSBIN_KERNEL_BLK_TC_FP32R; }


// Tree plans: rows ordered by group (stable within a group), the block sizes, and the
// reduced-matrix sizes and node counts per depth.  Returns the scratch bytes of depths
// 1 .. L-1, or 0 when the problem does not suit the tree (one group, a level block or the
// last group too large for the kernels' shared memory, scratch beyond 2 GB).
size_t tree_layout(gbsbin_plan* P) {
  const int L = P->L, n = P->n;
  if (L < 2 || n > 64) return 0;
  TreeArgs& t = P->tree;
  P->tree_perm.clear();
  for (int l = 0; l < L; ++l) {
    t.nb[l] = 0;
    for (int q = 0; q < n; ++q)
      if (P->label[q] == l) {
        P->tree_perm.push_back(q);
        ++t.nb[l];
      }
  }
  int rem = n;
  for (int l = 0; l < L; ++l) {
    t.m[l] = rem;
    rem -= t.nb[l];
  }
  if (tree_leaf_threads(t.m[L - 1]) == 0) return 0;
  size_t bytes = 0;
  long long nodes = 1;
  for (int l = 0; l + 1 < L; ++l) {
    if (tree_level_smem_bytes(t.nb[l], t.m[l]) > 200 * 1024) return 0;
    nodes *= P->grid.radix[l];
    const size_t mc = (size_t)t.m[l + 1];
    bytes += (size_t)nodes * (mc * mc + 2 * mc + 3) * sizeof(float4);
  }
  return bytes <= (2ull << 30) ? bytes : 0;
}

// Complex multiply-adds of the large-matrix tree for the plan's sub-step list and root
// counts (for choosing between its two halvings and against one LU per evaluated point).
double btree_macs(const gbsbin_plan* P) {
  const BTreeArgs& t = P->btree;
  double macs = 0.0;
  for (const BTreeStep& st : P->btree_steps) {
    double children = 1.0;
    for (int l = 0; l <= st.l; ++l) children *= t.cnt[l];
    double top = 0.0, row = 0.0;
    for (int kk = 0; kk < st.nbs; ++kk) {
      top += (double)(st.nbs - kk - 1) * (st.D - kk - 1);
      row += (double)(st.D - kk - 1);
    }
    macs += children * (top + (double)(st.D - st.nbs) * row);
  }
  double parents = 1.0;
  for (int l = 0; l + 1 < P->L; ++l) parents *= t.cnt[l];
  const double m = t.mL;
  double hess = 0.0;
  for (int k = 0; k + 2 < t.mL; ++k) hess += 2.0 * (m - k - 1) * (m - k + 1) + 2.0 * m * (m - k - 1);
  macs += parents * hess;
  macs += (double)t.n_leaves * (P->has_gamma ? 2.0 : 1.0) * m * m / 2.0;
  return macs;
}

// The sub-step list and scratch sizes of the large-matrix tree for one halving (the last
// axis, or the first); nb, m: rows of each group and reduced sizes.  Returns the 16-byte
// slots of device memory it needs.
size_t btree_configure(gbsbin_plan* P, int halve_first, const int* nb, const int* m) {
  const int L = P->L;
  BTreeArgs& t = P->btree;
  const GridDesc& g = P->grid;
  t.halve_first = halve_first;
  for (int l = 0; l < L; ++l) t.cnt[l] = g.radix[l];
  t.k0_lo = 0;
  if (halve_first) {
    t.cnt[0] = g.radix[0] / 2 + 1;
  } else {
    t.cnt[L - 1] = g.half;
    if (g.e_lo != 0 || g.e_hi != g.n_full) {        // a shard: the level-0 roots covering its slice
      const long long per_k0 = g.n_full / g.radix[0];
      t.k0_lo = (int)(g.e_lo / per_k0);
      t.cnt[0] = (int)((g.e_hi + per_k0 - 1) / per_k0) - t.k0_lo;
    }
  }
  t.n_leaves = 1;
  for (int l = 0; l < L; ++l) t.n_leaves *= t.cnt[l];
  P->btree_steps.clear();
  size_t bytes = 0, tmp_max = 0, u_max = 0, inv_max = 0;
  long long nodes = 1;
  for (int l = 0; l + 1 < L; ++l) {
    const long long children = nodes * t.cnt[l];
    int D = m[l] + 1;
    const int cap = std::min(GBSBIN_BT_MAX_NBS, (int)(GBSBIN_BT_SMEM / sizeof(float4)) / (D + 1));   // pivots per sub-step
    if (cap < 1) return 0;
    const int nsub = (nb[l] + cap - 1) / cap;
    const int per = (nb[l] + nsub - 1) / nsub;
    for (int p0 = 0; p0 < nb[l]; p0 += per) {
      BTreeStep st{};
      st.l = l;
      st.first = p0 == 0;
      st.nbg = nb[l];
      st.nbs = std::min(per, nb[l] - p0);
      st.D = D;
      P->btree_steps.push_back(st);
      u_max = std::max(u_max, (size_t)children * st.nbs * D);
      inv_max = std::max(inv_max, (size_t)children * st.nbs);
      D -= st.nbs;
      if (p0 + st.nbs < nb[l]) tmp_max = std::max(tmp_max, (size_t)children * D * D);
    }
    bytes += (size_t)children * (m[l + 1] + 1) * (m[l + 1] + 1) + 2 * (size_t)children;
    nodes = children;
  }
  const size_t hslots = (size_t)nodes * ((size_t)t.mL * t.mL + 2 * (size_t)t.mL + 1);
  P->bt_scratch[0] = tmp_max;
  P->bt_scratch[1] = u_max;
  P->bt_scratch[2] = inv_max;
  return bytes + 2 * tmp_max + u_max + inv_max + hslots;
}

// Large-matrix tree plans: rows ordered by group (as for kernels 11 and 12), each level's
// pivots in as few equal sub-steps as the shared-memory budget allows, and the halving (last
// axis or first) that needs fewer multiply-adds.  Returns the device bytes of depths
// 1 .. L-1, the sub-step scratch and the Hessenberg leaves, or 0 when the problem does not
// suit it (one group, a last group above GBSBIN_BT_MAX_LAST rows, scratch above 8 GB).
size_t btree_layout(gbsbin_plan* P) {
  const int L = P->L, n = P->n;
  if (L < 2) return 0;
  BTreeArgs& t = P->btree;
  t = BTreeArgs{};
  P->tree_perm.clear();
  int nb[GBSBIN_MAX_L], m[GBSBIN_MAX_L];
  for (int l = 0; l < L; ++l) {
    nb[l] = 0;
    for (int q = 0; q < n; ++q)
      if (P->label[q] == l) {
        P->tree_perm.push_back(q);
        ++nb[l];
      }
  }
  int rem = n;
  for (int l = 0; l < L; ++l) {
    m[l] = rem;
    rem -= nb[l];
  }
  t.L = L;
  t.mL = m[L - 1];
  if (t.mL > GBSBIN_BT_MAX_LAST || t.mL < 1) return 0;
  int best = -1;
  double best_macs = 0.0;
  const bool shard = P->grid.e_lo != 0 || P->grid.e_hi != P->grid.n_full;
  for (int h = 0; h < (shard ? 1 : 2); ++h) {       // a shard keeps the last axis halved
    if (!btree_configure(P, h, nb, m)) continue;
    const double w = btree_macs(P);
    if (best < 0 || w < best_macs) {
      best = h;
      best_macs = w;
    }
  }
  if (best < 0) return 0;
  const size_t total = btree_configure(P, best, nb, m);
  if (total * sizeof(float4) > (8ull << 30)) return 0;
  return total * sizeof(float4);
}

// Device pointers of a large-matrix tree plan (the layout of btree_layout) and the sub-step
// list's inputs and outputs.
void btree_pointers(gbsbin_plan* P, const Stage& sl) {
  BTreeArgs& t = P->btree;
  const int L = P->L, n = P->n;
  float4* A0 = (float4*)(P->d_state + sl.off_tree);
  t.mat[0] = A0;
  t.path[0] = A0 + (size_t)(n + 1) * (n + 1);
  float4* q = (float4*)P->d_tree;
  long long nodes = 1;
  int m = n;
  for (int l = 0; l + 1 < L; ++l) {
    nodes *= t.cnt[l];
    int nbl = 0;
    for (int x : P->label) nbl += x == l;
    m -= nbl;
    t.mat[l + 1] = q;
    q += (size_t)nodes * (m + 1) * (m + 1);
    t.path[l + 1] = q;
    q += 2 * (size_t)nodes;
  }
  const size_t tmp_max = P->bt_scratch[0], u_max = P->bt_scratch[1], inv_max = P->bt_scratch[2];
  float4* tmp[2] = {q, q + tmp_max};
  q += 2 * tmp_max;
  t.U = q;
  q += u_max;
  t.inv = q;
  q += inv_max;
  t.H = q;
  q += (size_t)nodes * t.mL * t.mL;
  t.hv = q;
  // sub-step inputs and outputs: a level's later sub-steps read the previous trailing blocks;
  // the last one writes depth l + 1
  int cur = 0;
  for (size_t k = 0; k < P->btree_steps.size(); ++k) {
    BTreeStep& st = P->btree_steps[k];
    const bool last = k + 1 == P->btree_steps.size() || P->btree_steps[k + 1].first;
    st.in = st.first ? nullptr : tmp[cur];
    if (!st.first) cur ^= 1;
    st.out = last ? t.mat[st.l + 1] : tmp[cur];
  }
}

void tree_pointers(gbsbin_plan* P, const Stage& sl) {
  TreeArgs& t = P->tree;
  const int n = P->n;
  float4* A0 = (float4*)(P->d_state + sl.off_tree);
  t.A[0] = A0;
  t.c[0] = A0 + (size_t)n * n;
  t.u[0] = t.c[0] + n;
  t.path[0] = t.u[0] + n;
  float4* q = (float4*)P->d_tree;
  long long nodes = 1;
  for (int l = 0; l + 1 < P->L; ++l) {
    nodes *= P->grid.radix[l];
    const size_t mc = (size_t)t.m[l + 1];
    t.A[l + 1] = q;
    q += (size_t)nodes * mc * mc;
    t.c[l + 1] = q;
    q += (size_t)nodes * mc;
    t.u[l + 1] = q;
    q += (size_t)nodes * mc;
    t.path[l + 1] = q;
    q += (size_t)nodes * 3;
  }
}

// The reverse pass along the large-matrix tree (gbsbin_backward_tree.cu): E = the rows of
// groups 0 .. L-2, F = the last group's; per parent the inverse of M_EE and its products, per
// leaf the inverse of the mF x mF Schur complement.  Taken when its multiply-adds are under
// half those of one n x n inverse per evaluated point; parents in waves whose buffers stay
// within 512 MB.
int backward_tree_setup(gbsbin_plan* P) {
  const int n = P->n, L = P->L;
  if (L < 2) return GBSBIN_OK;
  int mF = 0;
  for (int x : P->label) mF += x == L - 1;
  const int mE = n - mF;
  const GridDesc& g = P->grid;
  const long long parents = g.npts / g.radix[L - 1], half = g.half;
  const double E = mE, F = mF;
  const double per_parent = E * E * E + 2.0 * E * E * F + E * F * F + (F * F * E + E * E * F + E * F * F);
  const double tree = (double)parents * per_parent + (double)g.n_eval * F * F * F;
  if (!(tree < 0.5 * (double)g.n_eval * (double)n * n * n)) return GBSBIN_OK;
  BwdTree& t = P->bt;
  t.L = L;
  t.mE = mE;
  t.mF = mF;
  t.D = n + 1;
  t.A0 = P->btree.mat[0];
  t.half = half;
  t.pstride = (long long)n * n + 2LL * n;
  t.lstride = 2LL * mF * mF + 2LL * mF + 1;
  int off = 0;
  for (int l = 0; l < L; ++l) {
    t.goff[l] = off;
    for (int x : P->label) off += x == l;
  }
  t.goff[L] = off;
  const long long budget = 512LL << 20;
  const long long wave = std::max(1LL, std::min(parents, budget / (t.pstride * 16)));
  // leaves: two CTAs per SM where two mF x mF matrices fit in an SM's n x n slot
  t.leaf_ctas = 2LL * mF * mF <= (long long)n * n ? 2 * P->num_sms : P->num_sms;
  t.per = (int)((wave * half + t.leaf_ctas - 1) / t.leaf_ctas);
  t.maxspan = (int)((t.per - 1) / half + 2);
  t.nparts = (int)std::min<long long>(parents, P->num_sms);
  const size_t pbuf = (size_t)wave * t.pstride * 16;
  const size_t part = (size_t)t.leaf_ctas * t.maxspan * t.lstride * 16;
  const size_t pinv = ((size_t)n * sizeof(int) + 15) / 16 * 16;
  int st = dalloc(&P->d_bt, pbuf + part + pinv);
  if (st) return st;
  t.pbuf = P->d_bt;
  t.part = P->d_bt + pbuf;
  std::vector<int> inv(n);
  for (int a = 0; a < n; ++a) inv[P->tree_perm[a]] = a;
  int* d_pinv = reinterpret_cast<int*>(P->d_bt + pbuf + part);
  if (cudaMemcpy(d_pinv, inv.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  t.pinv = d_pinv;
  P->bt_parents = parents;
  P->bt_wave = wave;
  P->bwd_tree = true;
  return GBSBIN_OK;
}

int choose_kernel(int n, int L, int precision, int override_id, int has_gamma) {
  if (override_id) return override_id;
  if (L == 1) return precision == GBSBIN_FP32_REFINE ? GBSBIN_KERNEL_HESS_DF32 : GBSBIN_KERNEL_HESS_FP64;   // one group
  if (precision == GBSBIN_FP32_REFINE && n <= 32) return GBSBIN_KERNEL_WARP_FP32R;
  if (precision == GBSBIN_FP32_REFINE && n > GBSBIN_SMEM_MAX_N && n <= GBSBIN_BLK_MAX_N) return GBSBIN_KERNEL_BLK_FP32R;
  if (precision == GBSBIN_FP64)
    return points_per_cta(GBSBIN_KERNEL_SMEM_FP64, n, L) > 0 ? GBSBIN_KERNEL_SMEM_FP64 : GBSBIN_KERNEL_GMEM_FP64;
  return points_per_cta(GBSBIN_KERNEL_SMEM_FP32R, n, L) > 0 ? GBSBIN_KERNEL_SMEM_FP32R : GBSBIN_KERNEL_GMEM_FP32R;
}

}  // namespace

namespace gbsbin {

int host_state(const gbsbin_problem* p, int n, std::vector<cd>& XA, std::vector<cd>& gamma,
               std::vector<cd>& Xgamma) {
  int has_gamma = 0;
  return build_state(p, n, XA, gamma, Xgamma, &has_gamma);
}

cd host_logq1(const std::vector<cd>& XA, const std::vector<cd>& gamma, const std::vector<cd>& Xgamma, int n,
              double* minpiv) {
  std::vector<cd> K((size_t)n * n);
  std::vector<cd> x(Xgamma);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - XA[(size_t)i * n + j];
  cd ld = 0.0;
  double mn = 1e300;
  for (int k = 0; k < n; ++k) {
    const cd piv = K[(size_t)k * n + k];
    ld += std::log(piv);
    mn = std::min(mn, piv.real());
    for (int i = k + 1; i < n; ++i) {
      const cd l = K[(size_t)i * n + k] / piv;
      if (l == cd(0.0)) continue;
      for (int j = k + 1; j < n; ++j) K[(size_t)i * n + j] -= l * K[(size_t)k * n + j];
      x[i] -= l * x[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {                 // x = U^-1 (L^-1 X gamma)
    cd acc = x[i];
    for (int j = i + 1; j < n; ++j) acc -= K[(size_t)i * n + j] * x[j];
    x[i] = acc / K[(size_t)i * n + i];
  }
  cd gx = 0.0;
  for (int i = 0; i < n; ++i) gx += gamma[i] * x[i];
  if (minpiv) *minpiv = mn;
  return 0.5 * gx - 0.5 * ld;
}

}  // namespace gbsbin

extern "C" {

void gbsbin_default_options(gbsbin_options* o) {
  if (!o) return;
  o->precision = GBSBIN_FP64;
  o->oversample = 1;
  o->want_diagnostics = 1;
  o->tile_override = 0;
  o->want_timing = 0;
  o->want_backward = 0;
  o->shard_begin = 0;
  o->shard_end = 0;
}

const char* gbsbin_strerror(int status) {
  switch (status) {
    case GBSBIN_OK: return "ok";
    case GBSBIN_ERR_ARG: return "invalid argument";
    case GBSBIN_ERR_PARTITION: return "detector grouping is not a set partition of the ports";
    case GBSBIN_ERR_CUTOFF: return "invalid cutoff or grid too large";
    case GBSBIN_ERR_NONPHYSICAL: return "covariance is not Hermitian or Sigma - I/2 is not positive definite";
    case GBSBIN_ERR_CUDA: return "CUDA runtime error";
    case GBSBIN_ERR_NOMEM: return "out of memory";
    case GBSBIN_ERR_NUMERIC: return "non-positive or non-finite pivot at some grid point";
    case GBSBIN_ERR_UNSUPPORTED: return "size not supported by this build";
    case GBSBIN_ERR_TIMEOUT: return "bounded device wait timed out";
    case GBSBIN_ERR_PRECISION: return "result lost its significant digits to cancellation (value still written)";
  }
  return "unknown status";
}

static int plan_create_impl(const gbsbin_problem* p, const gbsbin_options* o, gbsbin_plan** out, int p_override,
                            bool alloc_gws, bool allow_tree);

int gbsbin_plan_create(const gbsbin_problem* p, const gbsbin_options* o, gbsbin_plan** out) {
  return plan_create_impl(p, o, out, 0, true, true);
}

// p_override > 0 forces the points per CTA (autotuning); alloc_gws = false leaves the
// workspace to a batch that shares one across its problems; allow_tree lets the automatic
// choice take a tree of block eliminations (standalone plans, and batch problems large enough
// to run apart from the batch's per-point launches).
static int plan_create_impl(const gbsbin_problem* p, const gbsbin_options* o, gbsbin_plan** out, int p_override,
                            bool alloc_gws, bool allow_tree) {
  if (!out) return GBSBIN_ERR_ARG;
  *out = nullptr;
  gbsbin_options opt;
  gbsbin_default_options(&opt);
  if (o) opt = *o;
  int st = validate_shape(p, &opt);
  if (st) return st;
  gbsbin_plan* P = new (std::nothrow) gbsbin_plan();
  if (!P) return GBSBIN_ERR_NOMEM;
  P->M = p->M;
  P->K = p->K;
  P->L = p->L;
  P->n = 2 * p->M * p->K;
  P->opt = opt;
  P->cutoff.assign(p->cutoff, p->cutoff + p->L);
  P->bin_of_mode.assign(p->bin_of_mode, p->bin_of_mode + p->M);
  const int n = P->n, MK = p->M * p->K;
  P->label.resize(n);
  for (int q = 0; q < MK; ++q) P->label[q] = P->label[MK + q] = p->bin_of_mode[q / p->K];
  // grid
  GridDesc& g = P->grid;
  g.L = p->L;
  g.npts = 1;
  P->table_size = 1;
  for (int l = 0; l < p->L; ++l) {
    g.radix[l] = opt.oversample * (p->cutoff[l] + 1);
    g.nout[l] = p->cutoff[l] + 1;
    g.npts *= g.radix[l];
    P->table_size *= g.nout[l];
  }
  g.half = g.radix[p->L - 1] / 2 + 1;
  g.n_full = g.npts / g.radix[p->L - 1] * g.half;
  g.e_lo = 0;
  g.e_hi = g.n_full;
  g.n_eval = g.n_full;
  if (opt.shard_end != 0 || opt.shard_begin != 0) {   // a shard: point 0, then [begin, end)
    if (opt.shard_begin < 0 || opt.shard_end <= opt.shard_begin || opt.shard_end > g.n_full) {
      delete P;
      return GBSBIN_ERR_ARG;
    }
    g.e_lo = opt.shard_begin;
    g.e_hi = opt.shard_end;
    g.n_eval = (g.e_hi - g.e_lo) + (g.e_lo > 0 ? 1 : 0);
  }
  st = build_state(p, n, P->XA, P->gamma, P->Xgamma, &P->has_gamma, &P->zbar);
  if (st) {
    delete P;
    return st;
  }
  record_inputs(P, p);
  P->kernel = choose_kernel(n, p->L, opt.precision, opt.tile_override, P->has_gamma);
  if (is_hess(P->kernel) && p->L != 1) {
    delete P;
    return GBSBIN_ERR_UNSUPPORTED;
  }
  // the tree: asked for, or by default for standalone FP32 + refinement plans it suits
  // (batches run their own per-point launches)
  const bool sharded = opt.shard_end != 0 || opt.shard_begin != 0;
  size_t tree_bytes = 0;
  if (is_tree(P->kernel) || (allow_tree && !opt.tile_override && p->L >= 2)) {
    tree_bytes = !sharded ? tree_layout(P) : 0;
    if (tree_bytes && !is_tree(P->kernel))
      P->kernel = opt.precision == GBSBIN_FP64 ? GBSBIN_KERNEL_TREE_FP64 : GBSBIN_KERNEL_TREE_DF32;
    else if (!tree_bytes && is_tree(P->kernel)) {
      delete P;
      return GBSBIN_ERR_UNSUPPORTED;
    }
  }
  // the large-matrix tree: asked for, or by default for standalone plans the small tree does
  // not take (n > 64, or a last group above 16 rows) where it needs under half the work of one
  // LU per evaluated point
  if (is_btree(P->kernel) || (!is_tree(P->kernel) && allow_tree && !opt.tile_override && p->L >= 2)) {
    tree_bytes = btree_layout(P);
    bool take = tree_bytes > 0;
    if (take && !is_btree(P->kernel))
      take = btree_macs(P) < 0.5 * (double)g.n_eval * (double)n * (double)n * (double)n / 3.0;
    if (!take) {
      tree_bytes = 0;
      if (is_btree(P->kernel)) {
        delete P;
        return GBSBIN_ERR_UNSUPPORTED;
      }
    } else if (!is_btree(P->kernel)) {
      P->kernel = opt.precision == GBSBIN_FP64 ? GBSBIN_KERNEL_BTREE_FP64 : GBSBIN_KERNEL_BTREE_DF32;
    }
  }
  P->P = is_hess(P->kernel) || is_tree(P->kernel) || is_btree(P->kernel) ? 1
         : P->kernel == GBSBIN_KERNEL_WARP_FP32R ? (n <= 32 ? 1 : 0)
         : is_blk(P->kernel) ? (n <= GBSBIN_BLK_MAX_N ? 1 : 0)
                                                 : points_per_cta(P->kernel, n, p->L);
  if (p_override > 0 && P->P > 0 && (P->kernel == GBSBIN_KERNEL_SMEM_FP64 || P->kernel == GBSBIN_KERNEL_SMEM_FP32R)) {
    if (points_smem_bytes(P->kernel, n, p_override, p->L) > 225 * 1024) {
      delete P;
      return GBSBIN_ERR_UNSUPPORTED;
    }
    P->P = p_override;
  }
  if (P->P < 1) {  // a variant forced on a matrix it cannot hold
    delete P;
    return GBSBIN_ERR_UNSUPPORTED;
  }
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  const size_t nn = (size_t)n * n;
  Stage sl = stage_layout(n, tree_region_slots(n, P->kernel));
  (void)nn;
  if ((st = dalloc(&P->d_state, sl.total)) || (st = dalloc(&P->d_label, n)) || (st = dalloc(&P->d_logq, g.n_eval)) ||
      (st = dalloc(&P->d_minpiv, g.n_eval)) || (st = dalloc(&P->d_bufA, g.n_full)) ||
      (st = dalloc(&P->d_bufB, g.n_full)) || (st = dalloc(&P->d_diag, GBSBIN_DIAG_DOUBLES)) ||
      (st = dalloc(&P->d_bar, 4)) ||
      (st = dalloc(&P->d_table, (size_t)P->table_size))) {
    free_device(P);
    delete P;
    return st;
  }
  P->d_NXA = (double2*)(P->d_state + sl.off_XA);          // all offsets are multiples of 16
  P->d_gamma = (double2*)(P->d_state + sl.off_g);
  P->d_Xgamma = (double2*)(P->d_state + sl.off_Xg);
  P->d_NXA_hi = (float2*)(P->d_state + sl.off_XAhi);
  P->d_NXA_lo = (float2*)(P->d_state + sl.off_XAlo);
  P->d_Xg_hi = (float2*)(P->d_state + sl.off_Xghi);
  P->d_Xg_lo = (float2*)(P->d_state + sl.off_Xglo);
  P->d_g_hi = (float2*)(P->d_state + sl.off_ghi);
  P->d_g_lo = (float2*)(P->d_state + sl.off_glo);
  P->d_NXA_fix = (longlong2*)(P->d_state + sl.off_XAfix);
  if (cudaMemset(P->d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(P->d_diag, 0, GBSBIN_DIAG_DOUBLES * sizeof(double)) != cudaSuccess) {
    free_device(P);
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  long long twn = 0;
  for (int l = 0; l < p->L; ++l) twn += g.radix[l];
  if ((st = dalloc(&P->d_tw, (size_t)twn))) {
    free_device(P);
    delete P;
    return st;
  }
  if ((P->kernel == GBSBIN_KERNEL_WARP_FP32R || is_hess(P->kernel) ||
       is_tree(P->kernel) || is_btree(P->kernel)) &&
      (st = dalloc(&P->d_ldfin, (size_t)6 * g.n_eval))) {
    free_device(P);
    delete P;
    return st;
  }
  if (is_tree(P->kernel)) {
    if ((st = dalloc(&P->d_tree, tree_bytes))) {
      free_device(P);
      delete P;
      return st;
    }
    tree_pointers(P, sl);
  }
  if (is_btree(P->kernel)) {
    if ((st = dalloc(&P->d_tree, tree_bytes))) {
      free_device(P);
      delete P;
      return st;
    }
    btree_pointers(P, sl);
  }
  if (is_hess(P->kernel) && (st = dalloc(&P->d_H, nn + 2 * (size_t)n))) {
    free_device(P);
    delete P;
    return st;
  }
  if (alloc_gws && (P->kernel == GBSBIN_KERNEL_GMEM_FP64 || P->kernel == GBSBIN_KERNEL_GMEM_FP32R ||
                    is_blk(P->kernel))) {
    P->gws_slot_bytes = is_blk(P->kernel) ? (long long)points_blk_slot_bytes(n)
                                                             : (long long)points_matrix_bytes(P->kernel, n, P->P);
    P->gws_slot_bytes = (P->gws_slot_bytes + 255) / 256 * 256;
    size_t bytes = (size_t)P->gws_slot_bytes * (size_t)P->num_sms *
                   (is_blk(P->kernel) ? GBSBIN_BLK_CTAS_PER_SM : 1);
    cudaError_t e = cudaMalloc(&P->d_gws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_device(P);
      delete P;
      return e == cudaErrorMemoryAllocation ? GBSBIN_ERR_NOMEM : GBSBIN_ERR_CUDA;
    }
  }
  for (int b = 0; b < 2; ++b) {
    if (cudaMallocHost(&P->h_stage[b], sl.total) != cudaSuccess) {
      cudaGetLastError();
      free_device(P);
      delete P;
      return GBSBIN_ERR_NOMEM;
    }
    if (cudaEventCreateWithFlags(&P->ev_stage[b], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_device(P);
      delete P;
      return GBSBIN_ERR_CUDA;
    }
  }
  P->h_stage_bytes = sl.total;
  if (opt.want_backward) {
    const size_t adj = (size_t)std::max<long long>(P->table_size, g.n_full);
    const size_t parts = (size_t)P->num_sms;
    P->bws_slot_bytes = ((long long)nn * 16 + 255) / 256 * 256;
    if ((st = dalloc(&P->d_adjA, adj)) ||
        (st = dalloc(&P->d_adjB, adj)) ||
        (st = dalloc(&P->d_bws, parts * (size_t)P->bws_slot_bytes / sizeof(double2))) ||
        (st = dalloc(&P->d_partS, parts * nn)) || (st = dalloc(&P->d_partg, parts * n)) ||
        (st = dalloc(&P->d_outS, nn)) || (st = dalloc(&P->d_outg, (size_t)n))) {
      free_device(P);
      delete P;
      return st;
    }
  }
  if (opt.want_backward && is_btree(P->kernel) && !sharded && (st = backward_tree_setup(P))) {
    free_device(P);
    delete P;
    return st;
  }
  if (opt.want_timing &&
      (cudaEventCreate(&P->ev0) != cudaSuccess || cudaEventCreate(&P->ev1) != cudaSuccess ||
       (opt.want_backward && (cudaEventCreate(&P->ev_b0) != cudaSuccess || cudaEventCreate(&P->ev_b1) != cudaSuccess)))) {
    cudaGetLastError();
    free_device(P);
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  // twiddles exp(-2 pi i m / R) and labels: synchronous one-off uploads
  std::vector<double2> tw((size_t)twn);
  long long off = 0;
  const double TWO_PI = 6.283185307179586476925286766559;
  for (int l = 0; l < p->L; ++l) {
    int R = g.radix[l];
    for (int m = 0; m < R; ++m) {
      double a = -TWO_PI * (double)m / (double)R;
      tw[off + m] = make_double2(std::cos(a), std::sin(a));
    }
    off += R;
  }
  if (cudaMemcpy(P->d_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P->d_label, P->label.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    free_device(P);
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  if (is_tree(P->kernel) || is_btree(P->kernel)) {   // the roots w = conj(twiddle) as FP32 pairs
    std::vector<float4> twdf((size_t)twn);
    for (size_t j = 0; j < twdf.size(); ++j) twdf[j] = split4(cd(tw[j].x, -tw[j].y));
    if (cudaMalloc(&P->d_twdf, twdf.size() * sizeof(float4)) != cudaSuccess ||
        cudaMemcpy(P->d_twdf, twdf.data(), twdf.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      free_device(P);
      delete P;
      return GBSBIN_ERR_CUDA;
    }
  }
  st = upload_state(P, 0);
  if (!st && cudaStreamSynchronize(0) != cudaSuccess) st = GBSBIN_ERR_CUDA;
  if (st) {
    cudaGetLastError();
    free_device(P);
    delete P;
    return st;
  }
  *out = P;
  return GBSBIN_OK;
}

int gbsbin_plan_set_state(gbsbin_plan* P, const gbsbin_problem* p, void* stream) {
  if (!P || !p) return GBSBIN_ERR_ARG;
  if (p->M != P->M || p->K != P->K || p->L != P->L) return GBSBIN_ERR_ARG;
  int st = validate_shape(p, &P->opt);
  if (st) return st;
  for (int l = 0; l < P->L; ++l)
    if (p->cutoff[l] != P->cutoff[l]) return GBSBIN_ERR_ARG;
  for (int j = 0; j < P->M; ++j)
    if (p->bin_of_mode[j] != P->bin_of_mode[j]) return GBSBIN_ERR_ARG;
  std::vector<cd> XA, gamma, Xgamma, zbar;
  int has_gamma = 0;
  st = build_state(p, P->n, XA, gamma, Xgamma, &has_gamma, &zbar);
  if (st) return st;
  record_inputs(P, p);
  P->logq_valid = false;
  P->zbar.swap(zbar);
  P->XA.swap(XA);
  P->gamma.swap(gamma);
  P->Xgamma.swap(Xgamma);
  P->has_gamma = has_gamma;
  return upload_state(P, (cudaStream_t)stream);
}

int gbsbin_plan_destroy(gbsbin_plan* P) {
  if (!P) return GBSBIN_ERR_ARG;
  cudaDeviceSynchronize();
  free_device(P);
  delete P;
  return GBSBIN_OK;
}

long long gbsbin_plan_table_size(const gbsbin_plan* P) { return P ? P->table_size : -1; }

static PointArgs make_point_args(gbsbin_plan* P) {
  PointArgs a{};
  a.n = P->n;
  a.has_gamma = P->has_gamma;
  a.P = P->P;
  a.logP = 0;
  while ((1 << a.logP) < P->P) ++a.logP;
  a.NXA = P->d_NXA;
  a.Xgamma = P->d_Xgamma;
  a.gamma = P->d_gamma;
  a.NXA_hi = P->d_NXA_hi;
  a.NXA_lo = P->d_NXA_lo;
  a.NXA_fix = P->d_NXA_fix;
  a.Xg_hi = P->d_Xg_hi;
  a.Xg_lo = P->d_Xg_lo;
  a.g_hi = P->d_g_hi;
  a.g_lo = P->d_g_lo;
  a.label = P->d_label;
  a.tw = P->d_tw;
  a.grid = P->grid;
  a.logq = P->d_logq;
  a.minpiv = P->d_minpiv;
  a.gws = P->d_gws;
  a.gws_slot_bytes = P->gws_slot_bytes;
  a.ldfin = P->d_ldfin;
  a.H = P->d_H;
  return a;
}

static DftArgs make_dft_args(gbsbin_plan* P, double* P_out) {
  DftArgs d{};
  d.grid = P->grid;
  d.logq = P->d_logq;
  d.ldfin = P->d_ldfin;
  d.logq_fin = P->d_logq;
  d.tw = P->d_tw;
  d.bufA = P->d_bufA;
  d.bufB = P->d_bufB;
  d.P = P_out;
  d.diag = P->opt.want_diagnostics ? P->d_diag : nullptr;
  d.minpiv = P->d_minpiv;
  d.table_size = P->table_size;
  d.df = P->kernel == GBSBIN_KERNEL_TREE_DF32 ? 1 : 0;
  return d;
}

int gbsbin_execute(gbsbin_plan* P, double* P_out, void* stream) {
  if (!P || !P_out) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PointArgs a = make_point_args(P);
  P->logq_valid = true;
  if (P->ev0 && cudaEventRecord(P->ev0, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  if (is_tree(P->kernel)) {
    TreeArgs t = P->tree;
    t.has_gamma = P->has_gamma;
    t.tw = P->d_tw;
    t.twdf = P->d_twdf;
    t.grid = P->grid;
    t.ldfin = P->d_ldfin;
    t.minpiv = P->d_minpiv;
    t.gout = P->tree_g ? P->d_bufA : nullptr;
    // pairs plans whose transform runs in pairs take G as pairs (no FP64 round trip)
    t.gout_df = (P->tree_g && P->kernel == GBSBIN_KERNEL_TREE_DF32 && dft_two_phase(P->grid)) ? 1 : 0;
    int nl = 0;
    if (launch_points_tree(t, P->kernel == GBSBIN_KERNEL_TREE_FP64, P->num_sms, s, &nl) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
    P->last_launches = nl + 1;                    // the tree's launches and the fused DFT
    if (P->ev1 && cudaEventRecord(P->ev1, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
    DftArgs d = make_dft_args(P, P_out);
    if (P->dft_plain) {                           // G again from the leaves' records (ldfin)
      P->last_launches = nl + 2 + P->grid.L + (P->opt.want_diagnostics ? 1 : 0);
      return launch_dft(d, s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
    }
    d.g_ready = P->tree_g ? 1 : 0;
    d.g_df = t.gout_df;
    return launch_dft_fused(d, P->d_bar, P->num_sms, s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
  }
  if (is_btree(P->kernel)) {
    BTreeArgs t = P->btree;
    t.has_gamma = P->has_gamma;
    t.tw = P->d_tw;
    t.twdf = P->d_twdf;
    t.grid = P->grid;
    t.ldfin = P->d_ldfin;
    t.minpiv = P->d_minpiv;
    t.q1re = P->logq1.real();
    t.q1im = P->logq1.imag();
    t.q1minpiv = P->logq1_minpiv;
    int nl = 0;
    if (launch_points_btree(t, P->btree_steps.data(), (int)P->btree_steps.size(),
                            P->kernel == GBSBIN_KERNEL_BTREE_FP64, P->num_sms, s, &nl) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
    P->last_launches = nl + 1;                    // the tree's launches and the fused DFT
    if (P->ev1 && cudaEventRecord(P->ev1, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
    if (P->dft_plain) {
      P->last_launches = nl + 1 + P->grid.L + (P->opt.want_diagnostics ? 1 : 0);
      return launch_dft(make_dft_args(P, P_out), s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
    }
    return launch_dft_fused(make_dft_args(P, P_out), P->d_bar, P->num_sms, s) == cudaSuccess ? GBSBIN_OK
                                                                                             : GBSBIN_ERR_CUDA;
  }
  cudaError_t e = P->kernel == GBSBIN_KERNEL_WARP_FP32R  ? launch_points_warp(a, P->num_sms, s)
                  : is_hess(P->kernel) ? launch_points_hess(a, PointBatch{}, 0, P->num_sms, s, P->kernel == GBSBIN_KERNEL_HESS_DF32)
                  : is_blk(P->kernel) ? launch_points_blk(a, PointBatch{}, 0, P->num_sms, s, P->kernel == GBSBIN_KERNEL_BLK_TC_FP32R)
                                                         : launch_points(a, P->kernel, P->num_sms, s);
  if (e != cudaSuccess) return GBSBIN_ERR_CUDA;
  P->last_launches = 2;                           // the point kernel and the fused DFT
  if (P->ev1 && cudaEventRecord(P->ev1, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  e = launch_dft_fused(make_dft_args(P, P_out), P->d_bar, P->num_sms, s);
  return e == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
}

int gbsbin_execute_host_async(gbsbin_plan* P, double* P_out_host, void* stream) {
  if (!P || !P_out_host) return GBSBIN_ERR_ARG;
  int st = gbsbin_execute(P, P->d_table, stream);
  if (!st && cudaMemcpyAsync(P_out_host, P->d_table, (size_t)P->table_size * sizeof(double),
                             cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    st = GBSBIN_ERR_CUDA;
  return st;
}

int gbsbin_execute_host(gbsbin_plan* P, double* P_out_host, void* stream) {
  int st = gbsbin_execute_host_async(P, P_out_host, stream);
  if (st == GBSBIN_ERR_ARG) return st;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess && !st) st = GBSBIN_ERR_CUDA;
  return st;
}

int gbsbin_diagnostics(gbsbin_plan* P, gbsbin_diag* out, void* stream) {
  if (!P || !out) return GBSBIN_ERR_ARG;
  std::vector<double> part(GBSBIN_DIAG_DOUBLES, 0.0);
  double h[5] = {0.0, 0.0, 1.0e300, 0.0, 0.0};
  if (P->opt.want_diagnostics) {
    if (cudaMemcpyAsync(part.data(), P->d_diag, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
    const int nblk = std::min(GBSBIN_DIAG_SLOTS, std::max(0, (int)part[4 * GBSBIN_DIAG_SLOTS + 2]));
    for (int b = 0; b < nblk; ++b) {  // fixed order: deterministic
      h[0] += part[4 * b];
      h[1] = std::fmax(h[1], part[4 * b + 1]);
      h[2] = std::fmin(h[2], part[4 * b + 2]);
      h[3] += part[4 * b + 3];
    }
    h[4] = part[4 * GBSBIN_DIAG_SLOTS];
  }
  out->sum_P = h[0];
  out->max_imag = h[1];
  out->min_pivot_re = h[2];
  out->n_bad_points = (long long)h[3];
  out->log_q1_re = (is_tree(P->kernel) && P->tree_g) ? P->tree_logq0 : h[4];
  out->n_points = P->grid.npts;
  out->n_evaluated = P->grid.n_eval;
  out->table_size = P->table_size;
  out->n = P->n;
  out->kernel = P->kernel;
  out->point_kernel_ms = 0.0;
  out->state_upload_bytes = P->upload_bytes;
  out->launches = P->last_launches;
  if (P->ev1 && P->last_launches > 0) {          // the timing events exist once an execute has run
    float ms = 0.f;
    if (cudaEventSynchronize(P->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, P->ev0, P->ev1) != cudaSuccess) {
      cudaGetLastError();
      return GBSBIN_ERR_CUDA;
    }
    out->point_kernel_ms = ms;
  }
  out->backward_kernel_ms = 0.0;
  out->backward_path = !P->opt.want_backward ? 0 : P->bwd_tree ? 2 : 1;
  if (P->ev_b1 && P->backward_ran) {
    float ms = 0.f;
    if (cudaEventSynchronize(P->ev_b1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, P->ev_b0, P->ev_b1) != cudaSuccess) {
      cudaGetLastError();
      return GBSBIN_ERR_CUDA;
    }
    out->backward_kernel_ms = ms;
  }
  if (!P->opt.want_diagnostics) return GBSBIN_OK;
  if (part[4 * GBSBIN_DIAG_SLOTS + 1] != 0.0) return GBSBIN_ERR_CUDA;   // a grid barrier gave up waiting
  return out->n_bad_points > 0 ? GBSBIN_ERR_NUMERIC : GBSBIN_OK;
}

int gbsbin_read_points(gbsbin_plan* P, double* logq_host, double* minpiv_host, void* stream) {
  if (!P || !logq_host) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ne = (size_t)P->grid.n_eval;
  // plans whose DFT took G directly left log q unfinished
  if (is_tree(P->kernel) && P->tree_g &&
      launch_finish_logq(P->d_ldfin, P->d_logq, (long long)ne, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  if (cudaMemcpyAsync(logq_host, P->d_logq, ne * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  if (minpiv_host &&
      cudaMemcpyAsync(minpiv_host, P->d_minpiv, ne * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
}


// Enqueue the reverse pass to the bilinear adjoints d_outS (n x n) and d_outg (n).
static int backward_enqueue(gbsbin_plan* P, const double* dLdP, cudaStream_t s) {
  int st = GBSBIN_OK;
  if (!P->logq_valid && (st = gbsbin_execute(P, P->d_table, s))) return st;   // log q of the current state
  if (is_tree(P->kernel) && P->tree_g &&        // the tree's DFT took G directly: finish log q
      launch_finish_logq(P->d_ldfin, P->d_logq, P->grid.n_eval, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  BackwardArgs b{};
  b.n = P->n;
  b.df = P->opt.precision == GBSBIN_FP32_REFINE ? 1 : 0;
  b.nb = backward_block(P->n);
  b.grid = P->grid;
  b.n_eval = P->grid.n_eval;
  b.NXA = P->d_NXA;
  b.Xgamma = P->d_Xgamma;
  b.label = P->d_label;
  b.gamma = P->d_gamma;
  b.logq = P->d_logq;
  b.tw = P->d_tw;
  b.bufA = P->d_adjA;
  b.bufB = P->d_adjB;
  b.ws = P->d_bws;
  b.ws_slot_bytes = P->bws_slot_bytes;
  b.partS = P->d_partS;
  b.partg = P->d_partg;
  b.nparts = P->num_sms;
  b.outS = P->d_outS;
  b.outg = P->d_outg;
  b.ev0 = P->ev_b0;
  b.ev1 = P->ev_b1;
  cudaError_t e;
  if (!P->bwd_tree) {
    e = launch_backward(b, dLdP, s);
  } else {                                          // along the tree, parents in waves
    e = launch_backward_weights(b, dLdP, s, &b.beta);
    if (e == cudaSuccess && b.ev0) e = cudaEventRecord(b.ev0, s);
    for (long long p0 = 0; e == cudaSuccess && p0 < P->bt_parents; p0 += P->bt_wave) {
      BwdTree t = P->bt;
      t.p0 = p0;
      t.p1 = std::min(P->bt_parents, p0 + P->bt_wave);
      t.zero_partials = p0 == 0;
      e = launch_backward_tree_wave(b, t, s);
    }
    if (e == cudaSuccess && b.ev1) e = cudaEventRecord(b.ev1, s);
    if (e == cudaSuccess) e = launch_backward_reduce(b, P->bt.nparts, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  P->backward_ran = true;
  return GBSBIN_OK;
}

int gbsbin_backward_device(gbsbin_plan* P, const double* dLdP, gbsbin_complex* dL_dXA, gbsbin_complex* dL_dgamma,
                           void* stream) {
  if (!P || !dLdP || !dL_dXA || !dL_dgamma) return GBSBIN_ERR_ARG;
  if (!P->opt.want_backward) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = backward_enqueue(P, dLdP, s);
  if (st) return st;
  const size_t n = (size_t)P->n;
  if (cudaMemcpyAsync(dL_dXA, P->d_outS, n * n * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dL_dgamma, P->d_outg, n * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  return GBSBIN_OK;
}

int gbsbin_backward(gbsbin_plan* P, const double* dLdP, gbsbin_grads* g, void* stream) {
  if (!P || !dLdP || !g) return GBSBIN_ERR_ARG;
  if (!P->opt.want_backward) return GBSBIN_ERR_ARG;
  if ((g->d_r || g->d_T || g->d_alpha || g->d_V) && !P->physical) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = P->n, MK = n / 2, M = P->M, K = P->K;
  int st = backward_enqueue(P, dLdP, s);
  if (st) return st;
  std::vector<double2> hS((size_t)n * n), hg(n);
  if (cudaMemcpyAsync(hS.data(), P->d_outS, hS.size() * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hg.data(), P->d_outg, hg.size() * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  for (size_t q = 0; q < hS.size(); ++q)
    if (!std::isfinite(hS[q].x) || !std::isfinite(hS[q].y)) return GBSBIN_ERR_NUMERIC;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(hg[i].x) || !std::isfinite(hg[i].y)) return GBSBIN_ERR_NUMERIC;

  // dL = Re( sum_ij S_ij dXA_ij + sum_i s_i dgamma_i ) with XA = I - Sigma^{-1},
  // gamma = X Sigma^{-1} zbar:  dL = Re tr(B dSigma) + Re v^T dzbar, where
  // B = Sinv S^T Sinv - (Sinv zbar)(Sinv^T X s)^T and v = Sinv^T X s.
  std::vector<cd> S((size_t)n * n), sv(n), Sinv((size_t)n * n);
  for (size_t q = 0; q < S.size(); ++q) S[q] = cd(hS[q].x, hS[q].y);
  for (int i = 0; i < n; ++i) sv[i] = cd(hg[i].x, hg[i].y);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Sinv[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - P->XA[(size_t)i * n + j];
  std::vector<cd> T1, B;
  matmul(Sinv, transpose(S, n), T1, n);
  matmul(T1, Sinv, B, n);
  std::vector<cd> u(n, 0.0), w(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) u[i] += Sinv[(size_t)i * n + j] * P->zbar[j];
  for (int i = 0; i < n; ++i)       // w = Sinv^T X s
    for (int j = 0; j < n; ++j) w[i] += Sinv[(size_t)j * n + i] * sv[j < MK ? j + MK : j - MK];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B[(size_t)i * n + j] -= u[i] * w[j];
  if (g->d_sigma1)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cd c = std::conj(B[(size_t)j * n + i]);
        g->d_sigma1[(size_t)i * n + j] = gbsbin_complex{c.real(), c.imag()};
      }
  if (g->d_zbar)
    for (int i = 0; i < n; ++i) g->d_zbar[i] = gbsbin_complex{w[i].real(), -w[i].imag()};
  if (!(g->d_r || g->d_T || g->d_alpha || g->d_V)) return GBSBIN_OK;

  // physical parameters: Sigma^(1) = W Sigma_in W^dag, W = Tf (+) conj(Tf),
  // zbar = (Tf alpha, conj(Tf alpha)), Tf[(j,l),(i,k)] = T_ji V_i[l,k]
  std::vector<cd> Tf((size_t)MK * MK);
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i)
      for (int l = 0; l < K; ++l)
        for (int k = 0; k < K; ++k)
          Tf[(size_t)(j * K + l) * MK + (i * K + k)] = P->T[(size_t)j * M + i] * P->V[((size_t)i * K + l) * K + k];
  std::vector<cd> W((size_t)n * n, 0.0), Wh((size_t)n * n, 0.0), Sin((size_t)n * n, 0.0);
  for (int a = 0; a < MK; ++a)
    for (int c = 0; c < MK; ++c) {
      W[(size_t)a * n + c] = Tf[(size_t)a * MK + c];
      W[(size_t)(a + MK) * n + (c + MK)] = std::conj(Tf[(size_t)a * MK + c]);
    }
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) Wh[(size_t)a * n + c] = std::conj(W[(size_t)c * n + a]);
  for (int q = 0; q < MK; ++q) {
    double sh = std::sinh(P->r[q]), ch = std::cosh(P->r[q]);
    Sin[(size_t)q * n + q] = Sin[(size_t)(q + MK) * n + (q + MK)] = sh * sh;
    Sin[(size_t)q * n + (q + MK)] = Sin[(size_t)(q + MK) * n + q] = sh * ch;
  }
  std::vector<cd> WhB, C, SinWhB, BW, A;
  matmul(Wh, B, WhB, n);
  if (g->d_r) {
    matmul(WhB, W, C, n);
    for (int q = 0; q < MK; ++q) {
      const int p = q + MK;
      double s2 = std::sinh(2.0 * P->r[q]), c2 = std::cosh(2.0 * P->r[q]);
      cd v = s2 * (C[(size_t)q * n + q] + C[(size_t)p * n + p]) + c2 * (C[(size_t)p * n + q] + C[(size_t)q * n + p]);
      g->d_r[q] = v.real();
    }
  }
  if (!(g->d_T || g->d_alpha || g->d_V)) return GBSBIN_OK;
  matmul(Sin, WhB, SinWhB, n);
  matmul(B, W, BW, n);
  matmul(BW, Sin, A, n);
  // G_W = conj(c1) + A with c1 = (Sigma_in W^dag B)^T; G_Tf = G_W11 + conj(G_W22) + z-bar terms
  std::vector<cd> GTf((size_t)MK * MK);
  for (int a = 0; a < MK; ++a)
    for (int c = 0; c < MK; ++c) {
      cd g11 = std::conj(SinWhB[(size_t)c * n + a]) + A[(size_t)a * n + c];
      cd g22 = std::conj(SinWhB[(size_t)(c + MK) * n + (a + MK)]) + A[(size_t)(a + MK) * n + (c + MK)];
      cd v1a = w[a], v2a = w[a + MK], al = P->alpha[c];
      GTf[(size_t)a * MK + c] = g11 + std::conj(g22) + std::conj(v1a * al) + v2a * std::conj(al);
    }
  if (g->d_alpha)
    for (int c = 0; c < MK; ++c) {
      cd uu = 0.0;
      for (int a = 0; a < MK; ++a) uu += Tf[(size_t)a * MK + c] * (w[a] + std::conj(w[a + MK]));
      g->d_alpha[c] = gbsbin_complex{uu.real(), -uu.imag()};
    }
  if (g->d_T)
    for (int j = 0; j < M; ++j)
      for (int i = 0; i < M; ++i) {
        cd acc = 0.0;
        for (int l = 0; l < K; ++l)
          for (int k = 0; k < K; ++k)
            acc += GTf[(size_t)(j * K + l) * MK + (i * K + k)] * std::conj(P->V[((size_t)i * K + l) * K + k]);
        g->d_T[(size_t)j * M + i] = gbsbin_complex{acc.real(), acc.imag()};
      }
  if (g->d_V)
    for (int i = 0; i < M; ++i)
      for (int l = 0; l < K; ++l)
        for (int k = 0; k < K; ++k) {
          cd acc = 0.0;
          for (int j = 0; j < M; ++j)
            acc += GTf[(size_t)(j * K + l) * MK + (i * K + k)] * std::conj(P->T[(size_t)j * M + i]);
          g->d_V[((size_t)i * K + l) * K + k] = gbsbin_complex{acc.real(), acc.imag()};
        }
  return GBSBIN_OK;
}

// ---------------------------------------------------------------- binned moments
// Inverse of a general complex n x n matrix (row-major) by Gauss-Jordan with partial
// pivoting, FP64; returns false if a pivot vanishes.
static bool invert(std::vector<cd>& A, int n) {
  std::vector<cd> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + k]) > std::abs(A[(size_t)piv * n + k])) piv = i;
    if (std::abs(A[(size_t)piv * n + k]) == 0.0) return false;
    if (piv != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)k * n + j], A[(size_t)piv * n + j]);
        std::swap(I[(size_t)k * n + j], I[(size_t)piv * n + j]);
      }
    const cd inv = 1.0 / A[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) {
      A[(size_t)k * n + j] *= inv;
      I[(size_t)k * n + j] *= inv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const cd f = A[(size_t)i * n + k];
      if (f == cd(0.0)) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        I[(size_t)i * n + j] -= f * I[(size_t)k * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

}  // extern "C"

// The algebra both moment calls share (Sec. VI, coarse-grained moments and cumulants):
// R = (I - XA)^{-1}, W = XA R, u = R X gamma, v = R^T gamma and the group label of each
// row of the state.
static int moment_algebra(const gbsbin_problem* p, int& n, std::vector<int>& lab, std::vector<cd>& W,
                          std::vector<cd>& u, std::vector<cd>& v) {
  gbsbin_options o;
  gbsbin_default_options(&o);
  int st = validate_shape(p, &o);
  if (st) return st;
  const int MK = p->M * p->K;
  n = 2 * MK;
  std::vector<cd> C, gamma, Xgamma;
  int has_gamma = 0;
  if ((st = build_state(p, n, C, gamma, Xgamma, &has_gamma))) return st;
  lab.assign(n, 0);
  for (int q = 0; q < MK; ++q) lab[q] = lab[MK + q] = p->bin_of_mode[q / p->K];
  std::vector<cd> R((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - C[(size_t)i * n + j];
  if (!invert(R, n)) return GBSBIN_ERR_NONPHYSICAL;
  W.assign((size_t)n * n, 0.0);
  u.assign(n, 0.0);
  v.assign(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const cd c = C[(size_t)i * n + k];
      if (c == cd(0.0)) continue;
      const cd* rrow = &R[(size_t)k * n];
      cd* wrow = &W[(size_t)i * n];
      for (int j = 0; j < n; ++j) wrow[j] += c * rrow[j];
    }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      u[i] += R[(size_t)i * n + k] * Xgamma[k];
      v[i] += R[(size_t)k * n + i] * gamma[k];
    }
  return GBSBIN_OK;
}

extern "C" {

int gbsbin_moments(const gbsbin_problem* p, double* mean, double* cov) {
  if (!p || !mean || !cov) return GBSBIN_ERR_ARG;
  int n = 0;
  std::vector<int> lab;
  std::vector<cd> W, u, v;
  int st = moment_algebra(p, n, lab, W, u, v);
  if (st) return st;
  const int L = p->L;
  // mean_l = 1/2 sum_{i in l} (v_i u_i + W_ii)
  std::vector<cd> mu(L, 0.0), s(L * L, 0.0);
  for (int i = 0; i < n; ++i) mu[lab[i]] += 0.5 * (v[i] * u[i] + W[(size_t)i * n + i]);
  // cov_lm = 1/2 [sum_{i in m, j in l} v_i W_ij u_j + sum_{i in l, j in m} v_i W_ij u_j
  //               + d_lm sum_{i in l} v_i u_i + sum_{i in m, j in l} W_ij W_ji + d_lm sum_{i in l} W_ii]
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const cd t = v[i] * W[(size_t)i * n + j] * u[j];
      const cd ww = W[(size_t)i * n + j] * W[(size_t)j * n + i];
      const int li = lab[i], lj = lab[j];
      s[lj * L + li] += 0.5 * t;                 // i in m = li, j in l = lj: entry (l, m)
      s[li * L + lj] += 0.5 * t;                 // i in l = li, j in m = lj
      s[lj * L + li] += 0.5 * ww;
    }
  for (int i = 0; i < n; ++i) s[lab[i] * L + lab[i]] += 0.5 * (v[i] * u[i] + W[(size_t)i * n + i]);
  for (int l = 0; l < L; ++l) mean[l] = mu[l].real();
  for (int q = 0; q < L * L; ++q) cov[q] = s[q].real();
  return GBSBIN_OK;
}

int gbsbin_cumulants3(const gbsbin_problem* p, double* k3) {
  if (!p || !k3) return GBSBIN_ERR_ARG;
  int n = 0;
  std::vector<int> lab;
  std::vector<cd> W, u, v;
  int st = moment_algebra(p, n, lab, W, u, v);
  if (st) return st;
  const int L = p->L;
  // log G(e^t) in e_l = e^{t_l} - 1: sum_l c1_l e_l + sum_lm a_lm e_l e_m + sum_lmn b_lmn e_l e_m e_n
  std::vector<cd> c1(L, 0.0), a((size_t)L * L, 0.0), b((size_t)L * L * L, 0.0);
  for (int i = 0; i < n; ++i) c1[lab[i]] += 0.5 * (W[(size_t)i * n + i] + v[i] * u[i]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      a[(size_t)lab[i] * L + lab[j]] +=
          0.25 * W[(size_t)i * n + j] * W[(size_t)j * n + i] + 0.5 * v[i] * W[(size_t)i * n + j] * u[j];
  // b_lmn = 1/6 sum_{i in l, j in m, k in n} W_ij W_jk W_ki + 1/2 sum v_i W_ij W_jk u_k; the second
  // sum is sum_{j in m} x^(l)_j y^(n)_j with x^(l)_j = sum_{i in l} v_i W_ij, y^(n)_j = sum_{k in n} W_jk u_k
  std::vector<cd> Wt((size_t)n * n), acc(L);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Wt[(size_t)j * n + i] = W[(size_t)i * n + j];
  for (int i = 0; i < n; ++i) {
    const cd* wcol_i = &Wt[(size_t)i * n];          // W_ki over k
    for (int j = 0; j < n; ++j) {
      const cd* wrow_j = &W[(size_t)j * n];         // W_jk over k
      std::fill(acc.begin(), acc.end(), cd(0.0));
      for (int k = 0; k < n; ++k) acc[lab[k]] += wrow_j[k] * wcol_i[k];
      const cd wij = W[(size_t)i * n + j] / 6.0;
      cd* brow = &b[((size_t)lab[i] * L + lab[j]) * L];
      for (int l = 0; l < L; ++l) brow[l] += wij * acc[l];
    }
  }
  std::vector<cd> x((size_t)L * n, 0.0), y((size_t)L * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      x[(size_t)lab[i] * n + j] += v[i] * W[(size_t)i * n + j];
      y[(size_t)lab[j] * n + i] += W[(size_t)i * n + j] * u[j];
    }
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < n; ++j)
      for (int m = 0; m < L; ++m) b[((size_t)l * L + lab[j]) * L + m] += 0.5 * x[(size_t)l * n + j] * y[(size_t)m * n + j];
  // kappa_lmn = sum over the 6 orders of (l, m, n) of b + the chain-rule terms of e(t):
  // d_lm Q_ln + d_ln Q_lm + d_mn Q_ml + d_lm d_mn c1_l, Q = a + a^T
  auto B = [&](int i, int j, int k) { return b[((size_t)i * L + j) * L + k]; };
  auto Q = [&](int i, int j) { return a[(size_t)i * L + j] + a[(size_t)j * L + i]; };
  for (int l = 0; l < L; ++l)
    for (int m = 0; m < L; ++m)
      for (int q = 0; q < L; ++q) {
        cd kap = B(l, m, q) + B(l, q, m) + B(m, l, q) + B(m, q, l) + B(q, l, m) + B(q, m, l);
        if (l == m) kap += Q(l, q);
        if (l == q) kap += Q(l, m);
        if (m == q) kap += Q(m, l);
        if (l == m && m == q) kap += c1[l];
        k3[((size_t)l * L + m) * L + q] = kap.real();
      }
  return GBSBIN_OK;
}

// Fourth cumulants: the order-1..4 coefficients C_r of log G in e (C_r = tr((EW)^r) / (2r)
// + 1/2 v^T E (W E)^(r-1) u, summed per group of each index) from block products of W, then
// the chain rule from e_l = e^{t_l} - 1 (every derivative of e^t is 1 at 0, and e_l depends
// on t_l alone): kappa_{l1..l4} = sum over the set partitions of the four slots whose blocks
// each carry one group of F_r(the blocks' groups), F_r the fully symmetrised C_r.
int gbsbin_cumulants4(const gbsbin_problem* p, double* k4) {
  if (!p || !k4) return GBSBIN_ERR_ARG;
  int n = 0;
  std::vector<int> lab;
  std::vector<cd> W, u, v;
  int st = moment_algebra(p, n, lab, W, u, v);
  if (st) return st;
  const int L = p->L;
  std::vector<std::vector<int>> rows(L);             // the rows of each group
  for (int i = 0; i < n; ++i) rows[lab[i]].push_back(i);
  // blocks W_ab (rows of a, columns of b), dense row-major
  auto blk = [&](int a, int b) {
    std::vector<cd> B(rows[a].size() * rows[b].size());
    for (size_t i = 0; i < rows[a].size(); ++i)
      for (size_t j = 0; j < rows[b].size(); ++j) B[i * rows[b].size() + j] = W[(size_t)rows[a][i] * n + rows[b][j]];
    return B;
  };
  std::vector<std::vector<cd>> Wb((size_t)L * L);
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b) Wb[(size_t)a * L + b] = blk(a, b);
  auto Wab = [&](int a, int b) -> const std::vector<cd>& { return Wb[(size_t)a * L + b]; };
  auto sz = [&](int a) { return rows[a].size(); };
  // X_abc = W_ab W_bc (|a| x |c|)
  std::vector<std::vector<cd>> X((size_t)L * L * L);
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b)
      for (int c = 0; c < L; ++c) {
        std::vector<cd>& x = X[((size_t)a * L + b) * L + c];
        x.assign(sz(a) * sz(c), 0.0);
        const std::vector<cd>& A = Wab(a, b);
        const std::vector<cd>& B = Wab(b, c);
        for (size_t i = 0; i < sz(a); ++i)
          for (size_t k = 0; k < sz(b); ++k) {
            const cd aik = A[i * sz(b) + k];
            for (size_t j = 0; j < sz(c); ++j) x[i * sz(c) + j] += aik * B[k * sz(c) + j];
          }
      }
  auto Xabc = [&](int a, int b, int c) -> const std::vector<cd>& { return X[((size_t)a * L + b) * L + c]; };
  auto vg = [&](int a, size_t i) { return v[rows[a][i]]; };
  auto ug = [&](int a, size_t i) { return u[rows[a][i]]; };
  const size_t L2 = (size_t)L * L, L3 = L2 * L;
  std::vector<cd> C1(L, 0.0), C2(L2, 0.0), C3(L3, 0.0), C4(L3 * L, 0.0);
  for (int a = 0; a < L; ++a)
    for (size_t i = 0; i < sz(a); ++i) C1[a] += 0.5 * (Wab(a, a)[i * sz(a) + i] + vg(a, i) * ug(a, i));
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b) {
      cd tr = 0.0, vec = 0.0;
      const std::vector<cd>& A = Wab(a, b);
      const std::vector<cd>& B = Wab(b, a);
      for (size_t i = 0; i < sz(a); ++i)
        for (size_t j = 0; j < sz(b); ++j) {
          tr += A[i * sz(b) + j] * B[j * sz(a) + i];
          vec += vg(a, i) * A[i * sz(b) + j] * ug(b, j);
        }
      C2[(size_t)a * L + b] = tr / 4.0 + 0.5 * vec;
    }
  // q_cd = W_cd u_d (over the rows of c), p_abc = v_a^T X_abc (over the rows of c)
  std::vector<std::vector<cd>> q(L2), pv(L3);
  for (int c = 0; c < L; ++c)
    for (int d = 0; d < L; ++d) {
      std::vector<cd>& y = q[(size_t)c * L + d];
      y.assign(sz(c), 0.0);
      for (size_t i = 0; i < sz(c); ++i)
        for (size_t j = 0; j < sz(d); ++j) y[i] += Wab(c, d)[i * sz(d) + j] * ug(d, j);
    }
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b)
      for (int c = 0; c < L; ++c) {
        std::vector<cd>& y = pv[((size_t)a * L + b) * L + c];
        y.assign(sz(c), 0.0);
        const std::vector<cd>& x = Xabc(a, b, c);
        for (size_t i = 0; i < sz(a); ++i)
          for (size_t j = 0; j < sz(c); ++j) y[j] += vg(a, i) * x[i * sz(c) + j];
      }
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b)
      for (int c = 0; c < L; ++c) {
        cd tr = 0.0, vec = 0.0;
        const std::vector<cd>& x = Xabc(a, b, c);
        const std::vector<cd>& w = Wab(c, a);
        for (size_t i = 0; i < sz(a); ++i)
          for (size_t k = 0; k < sz(c); ++k) tr += x[i * sz(c) + k] * w[k * sz(a) + i];
        const std::vector<cd>& y = pv[((size_t)a * L + b) * L + c];
        for (size_t k = 0; k < sz(c); ++k) vec += y[k] * ug(c, k);
        C3[((size_t)a * L + b) * L + c] = tr / 6.0 + 0.5 * vec;
      }
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b)
      for (int c = 0; c < L; ++c)
        for (int d = 0; d < L; ++d) {
          // tr(X_abc X_cda) and p_abc . q_cd
          cd tr = 0.0, vec = 0.0;
          const std::vector<cd>& x1 = Xabc(a, b, c);
          const std::vector<cd>& x2 = Xabc(c, d, a);
          for (size_t i = 0; i < sz(a); ++i)
            for (size_t k = 0; k < sz(c); ++k) tr += x1[i * sz(c) + k] * x2[k * sz(a) + i];
          const std::vector<cd>& y = pv[((size_t)a * L + b) * L + c];
          const std::vector<cd>& z = q[(size_t)c * L + d];
          for (size_t k = 0; k < sz(c); ++k) vec += y[k] * z[k];
          C4[(((size_t)a * L + b) * L + c) * L + d] = tr / 8.0 + 0.5 * vec;
        }
  // F_r: the r-th mixed partial at e = 0, the sum of C_r over the orders of its indices
  auto F1 = [&](int a) { return C1[a]; };
  auto F2 = [&](int a, int b) { return C2[(size_t)a * L + b] + C2[(size_t)b * L + a]; };
  auto F3 = [&](int a, int b, int c) {
    const int m[3] = {a, b, c};
    static const int P3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    cd t = 0.0;
    for (const auto& o : P3) t += C3[((size_t)m[o[0]] * L + m[o[1]]) * L + m[o[2]]];
    return t;
  };
  auto F4 = [&](int a, int b, int c, int d) {
    int o[4] = {0, 1, 2, 3};
    const int m[4] = {a, b, c, d};
    cd t = 0.0;
    do {
      t += C4[(((size_t)m[o[0]] * L + m[o[1]]) * L + m[o[2]]) * L + m[o[3]]];
    } while (std::next_permutation(o, o + 4));
    return t;
  };
  for (int l0 = 0; l0 < L; ++l0)
    for (int l1 = 0; l1 < L; ++l1)
      for (int l2 = 0; l2 < L; ++l2)
        for (int l3 = 0; l3 < L; ++l3) {
          const int g[4] = {l0, l1, l2, l3};
          cd kap = F4(l0, l1, l2, l3);                 // four singletons
          // one pair, two singletons (6 pairs)
          for (int x = 0; x < 4; ++x)
            for (int y = x + 1; y < 4; ++y) {
              if (g[x] != g[y]) continue;
              int r[2], k = 0;
              for (int z = 0; z < 4; ++z)
                if (z != x && z != y) r[k++] = g[z];
              kap += F3(g[x], r[0], r[1]);
            }
          // two pairs (3 ways)
          const int PP[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
          for (const auto& pp : PP)
            if (g[pp[0]] == g[pp[1]] && g[pp[2]] == g[pp[3]]) kap += F2(g[pp[0]], g[pp[2]]);
          // a triple and a singleton (4 ways)
          for (int z = 0; z < 4; ++z) {
            int t[3], k = 0;
            for (int w = 0; w < 4; ++w)
              if (w != z) t[k++] = g[w];
            if (t[0] == t[1] && t[1] == t[2]) kap += F2(t[0], g[z]);
          }
          // all four in one block
          if (l0 == l1 && l1 == l2 && l2 == l3) kap += F1(l0);
          k4[(((size_t)l0 * L + l1) * L + l2) * L + l3] = kap.real();
        }
  return GBSBIN_OK;
}

// The cumulants of orders 1-4 on the GPU: the host state algebra (validation included), the
// rows sorted by group, then gbsbin_moments.cu's launches.  With XA = I - Sigma^{-1} (Sigma =
// I + Sigma^(1)), R = (I - XA)^{-1} = Sigma and W = XA R = Sigma^(1): the device starts from
// Sigma^(1), made exactly Hermitian ((S + S^H) / 2; the state was validated Hermitian).
int gbsbin_cumulants_device(const gbsbin_problem* p, int precision, double* mean, double* cov, double* k3, double* k4,
                            double* kernel_ms, void* stream) {
  if (!p || (precision != GBSBIN_FP64 && precision != GBSBIN_FP32_REFINE)) return GBSBIN_ERR_ARG;
  const int order = k4 ? 4 : k3 ? 3 : cov ? 2 : mean ? 1 : 0;
  if (order == 0) return GBSBIN_ERR_ARG;
  gbsbin_options o;
  gbsbin_default_options(&o);
  int st = validate_shape(p, &o);
  if (st) return st;
  if (p->L > GBSBIN_MOM_MAX_L) return GBSBIN_ERR_UNSUPPORTED;
  const int MK = p->M * p->K, n = 2 * MK, L = p->L;
  std::vector<cd> XA, gamma, Xgamma, S1;
  int has_gamma = 0;
  if ((st = build_state(p, n, XA, gamma, Xgamma, &has_gamma, nullptr, &S1))) return st;
  std::vector<int> perm, goff(L + 1, 0);
  for (int l = 0; l < L; ++l) {
    goff[l] = (int)perm.size();
    for (int i = 0; i < n; ++i)
      if (p->bin_of_mode[(i % MK) / p->K] == l) perm.push_back(i);
  }
  goff[L] = n;
  std::vector<cd> Wp((size_t)n * n), gp(n), Xgp(n);
  for (int a = 0; a < n; ++a) {
    for (int b = 0; b < n; ++b)
      Wp[(size_t)a * n + b] = 0.5 * (S1[(size_t)perm[a] * n + perm[b]] + std::conj(S1[(size_t)perm[b] * n + perm[a]]));
    gp[a] = gamma[perm[a]];
    Xgp[a] = Xgamma[perm[a]];
  }
  double* out[4] = {mean, cov, k3, k4};
  float ms = 0.f;
  st = cumulants_device(n, L, goff.data(), reinterpret_cast<const double*>(Wp.data()),
                        reinterpret_cast<const double*>(gp.data()), reinterpret_cast<const double*>(Xgp.data()), order,
                        precision == GBSBIN_FP32_REFINE, out, (cudaStream_t)stream, kernel_ms ? &ms : nullptr);
  if (!st && kernel_ms) *kernel_ms = ms;
  return st;
}

// Total photon-number distribution by the power series of App. A (a second evaluator beside
// the roots-of-unity transform): log q(eta) = sum_k a_k eta^k with a_k = tr((XA)^k) / (2k)
// + 1/2 gamma^T (XA)^(k-1) X gamma; q's Taylor coefficients e_m follow from e = exp(sum a_k
// eta^k) by m e_m = sum_{k=1}^m k a_k e_{m-k}; Pr(N) = Pr(0) e_N with Pr(0) = 1 / q(1) from an
// unpivoted LU of I - XA.  Powers of XA by repeated multiplication: O(Nmax n^3), host FP64.
int gbsbin_total_photon_series(const gbsbin_problem* p, int Nmax, double* P_out) {
  if (!p || !P_out || Nmax < 0) return GBSBIN_ERR_ARG;
  if (Nmax > (1 << 20)) return GBSBIN_ERR_UNSUPPORTED;
  gbsbin_options o;
  gbsbin_default_options(&o);
  int st = validate_shape(p, &o);
  if (st) return st;
  const int n = 2 * p->M * p->K;
  std::vector<cd> XA, gamma, Xgamma;
  int has_gamma = 0;
  st = build_state(p, n, XA, gamma, Xgamma, &has_gamma);
  if (st) return st;
  const cd logq1 = host_logq1(XA, gamma, Xgamma, n, nullptr);
  // a_k, k = 1..Nmax: traces of M = (XA)^k and w = (XA)^(k-1) X gamma
  std::vector<cd> a((size_t)Nmax + 1, 0.0), M(XA), T((size_t)n * n), w(Xgamma), w2(n);
  for (int k = 1; k <= Nmax; ++k) {
    cd tr = 0.0, g = 0.0;
    for (int i = 0; i < n; ++i) tr += M[(size_t)i * n + i];
    for (int i = 0; i < n; ++i) g += gamma[i] * w[i];
    a[k] = tr / (2.0 * k) + 0.5 * g;
    if (k == Nmax) break;
    std::fill(T.begin(), T.end(), cd(0.0));          // M <- M XA
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < n; ++q) {
        const cd m = M[(size_t)i * n + q];
        if (m == cd(0.0)) continue;
        const cd* xr = &XA[(size_t)q * n];
        cd* tr_ = &T[(size_t)i * n];
        for (int j = 0; j < n; ++j) tr_[j] += m * xr[j];
      }
    M.swap(T);
    for (int i = 0; i < n; ++i) {                    // w <- XA w
      cd acc = 0.0;
      for (int j = 0; j < n; ++j) acc += XA[(size_t)i * n + j] * w[j];
      w2[i] = acc;
    }
    w.swap(w2);
  }
  std::vector<cd> e((size_t)Nmax + 1, 0.0);
  e[0] = 1.0;
  for (int m = 1; m <= Nmax; ++m) {
    cd acc = 0.0;
    for (int k = 1; k <= m; ++k) acc += (double)k * a[k] * e[m - k];
    e[m] = acc / (double)m;
  }
  const cd pr0 = std::exp(-logq1);
  for (int m = 0; m <= Nmax; ++m) P_out[m] = (pr0 * e[m]).real();
  return GBSBIN_OK;
}

// Joint cumulant of the counts of a set S of distinct groups (the coarse-grained loop
// Montrealer): with distinct groups only the all-singleton partition enters the chain rule,
// so kappa_S = sum over the orders of S of C_|S| = 1/2 sum over the directed Hamiltonian
// cycles through S of tr(W_ab W_bc ... W_za) + 1/2 sum over the Hamiltonian paths of
// v_a^T W_ab ... W_yz u_z.  Both by dynamic programming over the subsets of S: cycles start
// at the smallest group of S (one rotation each), paths at any group.
int gbsbin_cumulant_groups(const gbsbin_problem* p, unsigned mask, double* kappa) {
  if (!p || !kappa || mask == 0u) return GBSBIN_ERR_ARG;
  int n = 0;
  std::vector<int> lab;
  std::vector<cd> W, u, v;
  int st = moment_algebra(p, n, lab, W, u, v);
  if (st) return st;
  const int L = p->L;
  if (L > 16 || (mask >> L) != 0u) return GBSBIN_ERR_ARG;
  std::vector<int> grp;                               // the groups of S, ascending
  for (int l = 0; l < L; ++l)
    if (mask >> l & 1u) grp.push_back(l);
  const int r = (int)grp.size();
  std::vector<std::vector<int>> rows(L);
  for (int i = 0; i < n; ++i) rows[lab[i]].push_back(i);
  auto sz = [&](int g) { return rows[grp[g]].size(); };
  // 2^r x r blocks of |group 0| x |e| entries: at most ten groups and about 1 GB
  size_t big = 0;
  for (int g = 0; g < r; ++g) big = std::max(big, sz(g));
  if (r > 10 || ((size_t)1 << r) * (size_t)r * sz(0) * big * sizeof(cd) > ((size_t)1 << 30))
    return GBSBIN_ERR_UNSUPPORTED;
  auto wblk = [&](int a, int b) {                     // W restricted to S's groups a, b
    std::vector<cd> B(sz(a) * sz(b));
    for (size_t i = 0; i < sz(a); ++i)
      for (size_t j = 0; j < sz(b); ++j) B[i * sz(b) + j] = W[(size_t)rows[grp[a]][i] * n + rows[grp[b]][j]];
    return B;
  };
  std::vector<std::vector<cd>> Wb((size_t)r * r);
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) Wb[(size_t)a * r + b] = wblk(a, b);
  const unsigned full = (1u << r) - 1u;
  // cycles: Pc[m][e] = sum over paths from group 0 through the set m ending at e of the block
  // products (|0| x |e|); paths: Qp[m][e] = the same for row vectors starting at v_start
  std::vector<std::vector<cd>> Pc((size_t)(full + 1) * r), Qp((size_t)(full + 1) * r);
  Pc[(size_t)1u * r + 0].assign(sz(0) * sz(0), 0.0);
  for (size_t i = 0; i < sz(0); ++i) Pc[(size_t)1u * r + 0][i * sz(0) + i] = 1.0;
  for (int a = 0; a < r; ++a) {
    std::vector<cd>& q = Qp[(size_t)(1u << a) * r + a];
    q.resize(sz(a));
    for (size_t i = 0; i < sz(a); ++i) q[i] = v[rows[grp[a]][i]];
  }
  for (unsigned m = 1; m <= full; ++m)
    for (int e = 0; e < r; ++e) {
      if (!(m >> e & 1u) || m == (1u << e)) continue;
      const unsigned prev = m & ~(1u << e);
      std::vector<cd>& pc = Pc[(size_t)m * r + e];
      std::vector<cd>& qp = Qp[(size_t)m * r + e];
      for (int b = 0; b < r; ++b) {
        if (!(prev >> b & 1u)) continue;
        const std::vector<cd>& B = Wb[(size_t)b * r + e];
        const std::vector<cd>& P0 = Pc[(size_t)prev * r + b];
        if ((m & 1u) && !P0.empty() && e != 0) {     // cycles keep group 0 as their start
          if (pc.empty()) pc.assign(sz(0) * sz(e), 0.0);
          for (size_t i = 0; i < sz(0); ++i)
            for (size_t k = 0; k < sz(b); ++k) {
              const cd x = P0[i * sz(b) + k];
              if (x == cd(0.0)) continue;
              for (size_t j = 0; j < sz(e); ++j) pc[i * sz(e) + j] += x * B[k * sz(e) + j];
            }
        }
        const std::vector<cd>& Q0 = Qp[(size_t)prev * r + b];
        if (!Q0.empty()) {
          if (qp.empty()) qp.assign(sz(e), 0.0);
          for (size_t k = 0; k < sz(b); ++k)
            for (size_t j = 0; j < sz(e); ++j) qp[j] += Q0[k] * B[k * sz(e) + j];
        }
      }
    }
  cd cyc = 0.0, path = 0.0;
  for (int e = 0; e < r; ++e) {
    const std::vector<cd>& pc = Pc[(size_t)full * r + e];
    if (!pc.empty()) {                                 // close the cycle: tr(P W_e0)
      const std::vector<cd>& B = Wb[(size_t)e * r + 0];
      for (size_t i = 0; i < sz(0); ++i)
        for (size_t k = 0; k < sz(e); ++k) cyc += pc[i * sz(e) + k] * B[k * sz(0) + i];
    }
    const std::vector<cd>& qp = Qp[(size_t)full * r + e];
    for (size_t k = 0; k < qp.size(); ++k) path += qp[k] * u[rows[grp[e]][k]];
  }
  *kappa = (0.5 * cyc + 0.5 * path).real();
  return GBSBIN_OK;
}

// Fine-grained Pr(n) of an undisplaced state whose internal modes are fully
// distinguishable (App. D): XA (rows and columns of internal mode l: (j K + l) and
// (MK + j K + l), j < M) is block diagonal over the internal modes with blocks B_l of rank
// <= 2.  The finite differences at integer points m <= n give
//   Pr(n) = Pr(0) / prod n_k! * sum_{m <= n} prod C(n_k, m_k) (-1)^(N - |m|) f_N(m),
// f_N(m) = [eta^N] exp(sum_j p_j(m) eta^j / (2j)), p_j(m) = tr((D(m) XA)^j) = sum_l
// (lambda1^j + lambda2^j), the two eigenvalues of sqrt(D) B_l sqrt(D) from its trace T and
// Frobenius norm F (lambda = T/2 +- sqrt(2 F^2 - T^2)/2), D(m) = diag(m) (+) diag(m).
// The App. D sum's result: Pr(n) = Pr(0) / n! x sum, an estimate of its absolute rounding
// error from the sum of the terms' magnitudes (each term carries ~N + 16 roundings of its own
// size: the power sums, the series recurrence, the binomial weight), and the status: the
// value has fewer than three significant digits left when that estimate exceeds 1e-3 of it.
static int dist_finish(double pr0, double fact, double sum, double abs_sum, int N, double* prob, double* abs_err) {
  const double scale = pr0 / fact;
  const double err = (double)(N + 16) * 2.220446049250313e-16 * abs_sum * scale;
  *prob = scale * sum;
  if (abs_err) *abs_err = err;
  return err > 1e-3 * std::fabs(*prob) ? GBSBIN_ERR_PRECISION : GBSBIN_OK;
}

static int dist_eval(const gbsbin_problem* p, const int* pattern, double* prob, double* abs_err, bool device,
                     void* stream) {
  if (!p || !pattern || !prob) return GBSBIN_ERR_ARG;
  gbsbin_options o;
  gbsbin_default_options(&o);
  int st = validate_shape(p, &o);
  if (st) return st;
  const int M = p->M, K = p->K, MK = M * K, n = 2 * MK;
  int N = 0;
  long long npts = 1;                                // evaluation points, at most 2^40
  for (int k = 0; k < M; ++k) {
    if (pattern[k] < 0) return GBSBIN_ERR_ARG;
    N += pattern[k];
    npts *= (long long)pattern[k] + 1;
    if (npts > (1ll << 40)) return GBSBIN_ERR_UNSUPPORTED;
  }
  std::vector<cd> XA, gamma, Xgamma;
  int has_gamma = 0;
  st = build_state(p, n, XA, gamma, Xgamma, &has_gamma);
  if (st) return st;
  if (has_gamma) return GBSBIN_ERR_UNSUPPORTED;       // App. D: undisplaced states
  auto idx = [&](int l, int a) { return a < M ? a * K + l : MK + (a - M) * K + l; };   // a < 2M
  double scale = 0.0;
  for (const cd& x : XA) scale = std::max(scale, std::abs(x));
  // block-diagonal over internal modes?
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int li = (i % MK) % K, lj = (j % MK) % K;
      if (li != lj && std::abs(XA[(size_t)i * n + j]) > 1e-12 * std::max(scale, 1.0)) return GBSBIN_ERR_UNSUPPORTED;
    }
  // blocks B_l (2M x 2M); rank <= 2 checked through tr(B^3) and tr(B^4) against the two
  // eigenvalues from the trace and the Frobenius norm
  const int m2 = 2 * M;
  std::vector<std::vector<cd>> B(K, std::vector<cd>((size_t)m2 * m2));
  for (int l = 0; l < K; ++l)
    for (int a = 0; a < m2; ++a)
      for (int b = 0; b < m2; ++b) B[l][(size_t)a * m2 + b] = XA[(size_t)idx(l, a) * n + idx(l, b)];
  auto eig2 = [&](const std::vector<cd>& Bl, const std::vector<double>& w, double& l1, double& l2) {
    double T = 0.0, F2 = 0.0;                        // of sqrt(D) B sqrt(D), D = diag(w)
    for (int a = 0; a < m2; ++a) {
      T += w[a] * Bl[(size_t)a * m2 + a].real();
      for (int b = 0; b < m2; ++b) F2 += w[a] * w[b] * std::norm(Bl[(size_t)a * m2 + b]);
    }
    const double disc = std::sqrt(std::max(0.0, 2.0 * F2 - T * T));
    l1 = 0.5 * (T + disc);
    l2 = 0.5 * (T - disc);
  };
  for (int l = 0; l < K; ++l) {
    std::vector<double> ones(m2, 1.0);
    double l1, l2;
    eig2(B[l], ones, l1, l2);
    std::vector<cd> B2((size_t)m2 * m2, 0.0);
    for (int a = 0; a < m2; ++a)
      for (int c = 0; c < m2; ++c)
        for (int b = 0; b < m2; ++b) B2[(size_t)a * m2 + b] += B[l][(size_t)a * m2 + c] * B[l][(size_t)c * m2 + b];
    cd t3 = 0.0, t4 = 0.0;
    for (int a = 0; a < m2; ++a)
      for (int c = 0; c < m2; ++c) {
        t3 += B2[(size_t)a * m2 + c] * B[l][(size_t)c * m2 + a];
        t4 += B2[(size_t)a * m2 + c] * B2[(size_t)c * m2 + a];
      }
    const double ref = std::max(1.0, l1 * l1 + l2 * l2);
    if (std::abs(t3 - (l1 * l1 * l1 + l2 * l2 * l2)) > 1e-9 * ref ||
        std::abs(t4 - (l1 * l1 * l1 * l1 + l2 * l2 * l2 * l2)) > 1e-9 * ref)
      return GBSBIN_ERR_UNSUPPORTED;                 // a block of rank above 2
  }
  // Pr(0) = sqrt(det(I - XA)), the blocks' determinants det(I - B_l) = (1 - l1)(1 - l2)
  double pr0 = 1.0;
  for (int l = 0; l < K; ++l) {
    std::vector<double> ones(m2, 1.0);
    double l1, l2;
    eig2(B[l], ones, l1, l2);
    pr0 *= std::sqrt((1.0 - l1) * (1.0 - l2));
  }
  // the sum over m <= n in reflected mixed-radix Gray order (one digit changes by +-1 per
  // point): per block the trace T = sum_k m_k d_k and F^2 = sum_kj m_k m_j S_kj update in
  // O(M), F^2(m + s e_k) = F^2(m) + 2 s sum_j m_j S_kj + S_kk (App. D), with
  // d_k = Re(B_kk + B_k+M,k+M), S_kj = |B_kj|^2 + |B_k+M,j+M|^2 + |B_k+M,j|^2 + |B_k,j+M|^2;
  // both are recomputed from m every 1024 points (rounding cannot drift)
  std::vector<double> d((size_t)K * M), S((size_t)K * M * M);
  for (int l = 0; l < K; ++l)
    for (int k = 0; k < M; ++k) {
      d[(size_t)l * M + k] = B[l][(size_t)k * m2 + k].real() + B[l][(size_t)(k + M) * m2 + k + M].real();
      for (int jj = 0; jj < M; ++jj)
        S[((size_t)l * M + k) * M + jj] = std::norm(B[l][(size_t)k * m2 + jj]) +
                                          std::norm(B[l][(size_t)(k + M) * m2 + jj + M]) +
                                          std::norm(B[l][(size_t)(k + M) * m2 + jj]) +
                                          std::norm(B[l][(size_t)k * m2 + jj + M]);
    }
  double fact = 1.0;
  for (int k = 0; k < M; ++k)
    for (int q = 2; q <= pattern[k]; ++q) fact *= (double)q;
  if (device) {                                      // one thread per point on the GPU
    double sum = 0.0, abs_sum = 0.0;
    st = distinguishable_sum_device(M, K, N, pattern, d.data(), S.data(), &sum, &abs_sum, (cudaStream_t)stream);
    if (st) return st;
    return dist_finish(pr0, fact, sum, abs_sum, N, prob, abs_err);
  }
  std::vector<int> m(M, 0), dir(M, 1);
  std::vector<double> Tl(K, 0.0), F2l(K, 0.0), ps((size_t)N + 1), e((size_t)N + 1);
  auto recompute = [&]() {
    for (int l = 0; l < K; ++l) {
      double T = 0.0, F2 = 0.0;
      for (int k = 0; k < M; ++k) {
        T += m[k] * d[(size_t)l * M + k];
        for (int jj = 0; jj < M; ++jj) F2 += (double)m[k] * m[jj] * S[((size_t)l * M + k) * M + jj];
      }
      Tl[l] = T;
      F2l[l] = F2;
    }
  };
  double binom = 1.0;                                // prod C(n_k, m_k), m = 0
  int msum = 0;
  double total = 0.0, comp = 0.0, abs_sum = 0.0;     // Neumaier-compensated signed sum
  long long count = 0;
  while (true) {
    if ((count & 1023) == 0) recompute();
    std::fill(ps.begin(), ps.end(), 0.0);
    for (int l = 0; l < K; ++l) {
      const double disc = std::sqrt(std::max(0.0, 2.0 * F2l[l] - Tl[l] * Tl[l]));
      const double l1 = 0.5 * (Tl[l] + disc), l2 = 0.5 * (Tl[l] - disc);
      double x1 = 1.0, x2 = 1.0;
      for (int jj = 1; jj <= N; ++jj) {
        x1 *= l1;
        x2 *= l2;
        ps[jj] += x1 + x2;
      }
    }
    e[0] = 1.0;                                      // e = exp(sum_j ps_j eta^j / (2j))
    for (int q = 1; q <= N; ++q) {
      double acc = 0.0;
      for (int jj = 1; jj <= q; ++jj) acc += 0.5 * ps[jj] * e[q - jj];   // j a_j = ps_j / 2
      e[q] = acc / (double)q;
    }
    const double term = (((N - msum) & 1) ? -1.0 : 1.0) * binom * e[N];
    const double t = total + term;
    comp += std::fabs(total) >= std::fabs(term) ? (total - t) + term : (term - t) + total;
    total = t;
    abs_sum += std::fabs(term);
    ++count;
    int k = 0;                                       // next point: the lowest digit that can move
    while (k < M && (m[k] + dir[k] < 0 || m[k] + dir[k] > pattern[k])) {
      dir[k] = -dir[k];
      ++k;
    }
    if (k == M) break;
    const int sgn = dir[k];
    for (int l = 0; l < K; ++l) {
      double cross = 0.0;
      for (int jj = 0; jj < M; ++jj) cross += m[jj] * S[((size_t)l * M + k) * M + jj];
      F2l[l] += 2.0 * sgn * cross + S[((size_t)l * M + k) * M + k];
      Tl[l] += sgn * d[(size_t)l * M + k];
    }
    // C(n, m + 1) = C(n, m) (n - m) / (m + 1); C(n, m - 1) = C(n, m) m / (n - m + 1)
    binom *= sgn > 0 ? (double)(pattern[k] - m[k]) / (double)(m[k] + 1)
                     : (double)m[k] / (double)(pattern[k] - m[k] + 1);
    m[k] += sgn;
    msum += sgn;
  }
  return dist_finish(pr0, fact, total + comp, abs_sum, N, prob, abs_err);
}

int gbsbin_prob_distinguishable(const gbsbin_problem* p, const int* pattern, double* prob, double* abs_err) {
  return dist_eval(p, pattern, prob, abs_err, false, nullptr);
}

int gbsbin_prob_distinguishable_device(const gbsbin_problem* p, const int* pattern, double* prob, double* abs_err,
                                       void* stream) {
  return dist_eval(p, pattern, prob, abs_err, true, stream);
}

int gbsbin_alu_peak(int precision, int blocks, double* tflops, void* stream) {
  if (!tflops || blocks <= 0) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return GBSBIN_ERR_NOMEM;
  const int fp64 = precision == GBSBIN_FP64 ? 1 : precision == GBSBIN_ALU_INT64 ? 2 : 0;
  const int iters = fp64 == 1 ? 256 : fp64 == 2 ? 2048 : 8192;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int st = GBSBIN_OK;
  if (launch_alu_peak(fp64, blocks, sink, iters, s) != cudaSuccess) st = GBSBIN_ERR_CUDA;  // warm-up
  cudaEventRecord(e0, s);
  if (!st && launch_alu_peak(fp64, blocks, sink, iters, s) != cudaSuccess) st = GBSBIN_ERR_CUDA;
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) st = GBSBIN_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
  *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}

}  // extern "C"

// =============================================================== autotuning
// Measured choice of the point-kernel variant and points per CTA for a matrix size.
// Candidates (per precision): the warp kernel (FP32R, n <= 32), the shared-memory CTA
// kernel with P = 1, 2, 4, 8 where the footprint fits, and the workspace kernel.  Each is
// timed with CUDA events on a synthetic state of that size (the unpivoted LU does the same
// arithmetic for any values) over a one-group grid of ~1024 evaluated points; results are
// cached per (size bucket of 16, precision) for the life of the process.
#include <map>
#include <mutex>

namespace {

struct TuneKey {
  int nb, precision;
  bool operator<(const TuneKey& o) const { return nb != o.nb ? nb < o.nb : precision < o.precision; }
};
struct TuneVal {
  int kernel, P;
  double us_per_point;
};
std::map<TuneKey, TuneVal> g_tune;
std::mutex g_tune_mu;

int tune_size(int n, int precision, TuneVal* best) {
  const int M = n / 2;
  std::vector<double> r(M, 0.7);
  std::vector<gbsbin_complex> T((size_t)M * M);
  const double TWO_PI = 6.283185307179586476925286766559;
  for (int j = 0; j < M; ++j)  // 0.8 x unitary DFT matrix: dense, ||T|| < 1
    for (int i = 0; i < M; ++i) {
      double a = TWO_PI * (double)i * (double)j / (double)M;
      T[(size_t)j * M + i] = gbsbin_complex{0.8 * std::cos(a) / std::sqrt((double)M), 0.8 * std::sin(a) / std::sqrt((double)M)};
    }
  std::vector<int> bins(M, 0);
  int cutoff = 2047;  // one axis, half = 1025 evaluated points
  gbsbin_problem pr{};
  pr.M = M;
  pr.K = 1;
  pr.r = r.data();
  pr.T = T.data();
  pr.bin_of_mode = bins.data();
  pr.L = 1;
  pr.cutoff = &cutoff;
  struct Cand {
    int kernel, P;
  };
  std::vector<Cand> cands;
  if (precision == GBSBIN_FP32_REFINE && n <= 32) cands.push_back({GBSBIN_KERNEL_WARP_FP32R, 1});
  const int smem_k = precision == GBSBIN_FP64 ? GBSBIN_KERNEL_SMEM_FP64 : GBSBIN_KERNEL_SMEM_FP32R;
  const int gmem_k = precision == GBSBIN_FP64 ? GBSBIN_KERNEL_GMEM_FP64 : GBSBIN_KERNEL_GMEM_FP32R;
  for (int Pc = 1; Pc <= 8; Pc *= 2)
    if (points_smem_bytes(smem_k, n, Pc, 1) <= 225 * 1024) cands.push_back({smem_k, Pc});
  if (precision == GBSBIN_FP32_REFINE && n > 32 && n <= GBSBIN_BLK_MAX_N) {
    cands.push_back({GBSBIN_KERNEL_BLK_FP32R, 1});
    cands.push_back({GBSBIN_KERNEL_BLK_TC_FP32R, 1});
  }
  cands.push_back({gmem_k, 1});
  best->us_per_point = 1e300;
  best->kernel = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GBSBIN_ERR_CUDA;
  double* table = nullptr;
  if (cudaMalloc(&table, sizeof(double) * (cutoff + 1)) != cudaSuccess) return GBSBIN_ERR_NOMEM;
  int status = GBSBIN_OK;
  for (const Cand& c : cands) {
    gbsbin_options o;
    gbsbin_default_options(&o);
    o.precision = precision;
    o.tile_override = c.kernel;
    o.want_diagnostics = 0;
    gbsbin_plan* P = nullptr;
    if (plan_create_impl(&pr, &o, &P, c.P, true, false) != GBSBIN_OK) continue;
    PointArgs a = make_point_args(P);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, 0);
      cudaError_t err = P->kernel == GBSBIN_KERNEL_WARP_FP32R  ? launch_points_warp(a, P->num_sms, 0)
                        : is_blk(P->kernel) ? launch_points_blk(a, PointBatch{}, 0, P->num_sms, 0, P->kernel == GBSBIN_KERNEL_BLK_TC_FP32R)
                                                               : launch_points(a, P->kernel, P->num_sms, 0);
      cudaEventRecord(e1, 0);
      if (err != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        status = GBSBIN_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best_ms) best_ms = ms;  // first launch is a warm-up
    }
    const double us = 1e3 * best_ms / (double)P->grid.n_eval;
    if (status == GBSBIN_OK && us < best->us_per_point) *best = TuneVal{c.kernel, P->P, us};
    gbsbin_plan_destroy(P);
    if (status) break;
  }
  cudaFree(table);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best->kernel ? status : (status ? status : GBSBIN_ERR_UNSUPPORTED);
}

int autotune_lookup(int n, int precision, TuneVal* out) {
  const int nb = (n + 15) / 16 * 16;
  const int ntune = std::min(std::max(nb, 16), GBSBIN_MAX_N);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(TuneKey{nb, precision});
    if (it != g_tune.end()) {
      *out = it->second;
      return GBSBIN_OK;
    }
  }
  TuneVal v{};
  int st = tune_size(ntune, precision, &v);
  if (st) return st;
  // a choice tuned at the bucket's top size must still be legal for n itself
  if (v.kernel == GBSBIN_KERNEL_WARP_FP32R && n > 32) v = TuneVal{GBSBIN_KERNEL_SMEM_FP32R, 1, v.us_per_point};
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[TuneKey{nb, precision}] = v;
  *out = v;
  return GBSBIN_OK;
}

}  // namespace

// ================================================================== batches
struct gbsbin_batch {
  std::vector<gbsbin_plan*> plans;
  std::vector<char> own;              // problem i runs its own plan's launches (a tree), not the queue
  struct Class {
    int kernel = 0, threads = 0, np = 0;
    size_t smem = 0;
    std::vector<PointJob> jobs;
    PointJob* d_jobs = nullptr;
  };
  std::vector<Class> classes;
  PointArgs* d_probs = nullptr;
  unsigned long long* d_queue = nullptr;
  void* d_gws = nullptr;
  long long gws_slot = 0;
  int num_sms = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // the tree problems, largest first, dealt round-robin to side streams that fork from and
  // join back to the caller's stream with events (also inside a captured graph)
  std::vector<int> tree_order;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
};

namespace {

void batch_free(gbsbin_batch* B) {
  if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& c : B->classes)
    if (c.d_jobs) cudaFree(c.d_jobs);
  if (B->d_probs) cudaFree(B->d_probs);
  if (B->d_queue) cudaFree(B->d_queue);
  if (B->d_gws) cudaFree(B->d_gws);
  for (cudaStream_t st : B->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : B->ev_join)
    if (ev) cudaEventDestroy(ev);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  for (gbsbin_plan* P : B->plans)
    if (P) gbsbin_plan_destroy(P);
  delete B;
}

// Side streams of a batch's tree problems: 8, or the environment variable
// GBSBIN_BATCH_STREAMS (1 .. 64).
int batch_side_streams() {
  static const int n = [] {
    int v = 8;
    if (const char* e = std::getenv("GBSBIN_BATCH_STREAMS")) v = std::atoi(e);
    return std::max(1, std::min(v, 64));
  }();
  return n;
}

int batch_launch(gbsbin_batch* B, double* const* P_out, cudaStream_t s) {
  for (size_t i = 0; i < B->plans.size(); ++i)
    if (!P_out[i]) return GBSBIN_ERR_ARG;
  // the trees on the side streams from the start, beside the per-point classes' persistent
  // launches and the per-point problems' transforms on s; then s waits for every side stream
  const int ns = (int)B->side.size();
  if (ns > 0 && cudaEventRecord(B->ev_fork, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(B->side[k], B->ev_fork, 0) != cudaSuccess) return GBSBIN_ERR_CUDA;
  for (size_t q = 0; q < B->tree_order.size(); ++q) {
    const int i = B->tree_order[q];
    const int st = gbsbin_execute(B->plans[i], P_out[i], ns > 0 ? B->side[q % ns] : s);
    if (st) return st;
  }
  for (size_t c = 0; c < B->classes.size(); ++c) {
    auto& C = B->classes[c];
    if (C.jobs.empty()) continue;
    if (cudaMemsetAsync(B->d_queue + c, 0, sizeof(unsigned long long), s) != cudaSuccess) return GBSBIN_ERR_CUDA;
    PointBatch pb{B->d_probs, C.d_jobs, (long long)C.jobs.size(), B->d_queue + c};
    cudaError_t e = C.kernel == GBSBIN_KERNEL_WARP_FP32R  ? launch_points_warp_batch(pb, C.np, B->num_sms, s)
                    : is_hess(C.kernel) ? launch_points_hess(PointArgs{}, pb, C.np, B->num_sms, s, C.kernel == GBSBIN_KERNEL_HESS_DF32)
                    : is_blk(C.kernel) ? launch_points_blk(PointArgs{}, pb, C.smem, B->num_sms, s, C.kernel == GBSBIN_KERNEL_BLK_TC_FP32R)
                                                          : launch_points_batch(pb, C.kernel, C.threads, C.smem, B->num_sms, s);
    if (e != cudaSuccess) return GBSBIN_ERR_CUDA;
  }
  for (size_t i = 0; i < B->plans.size(); ++i) {
    if (B->own[i]) continue;
    if (launch_dft_fused(make_dft_args(B->plans[i], P_out[i]), B->plans[i]->d_bar, B->num_sms, s) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
  }
  for (int k = 0; k < ns; ++k)
    if (cudaEventRecord(B->ev_join[k], B->side[k]) != cudaSuccess ||
        cudaStreamWaitEvent(s, B->ev_join[k], 0) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
  return GBSBIN_OK;
}

}  // namespace

extern "C" {

int gbsbin_autotune(int n, int precision, int* kernel, int* points_per_cta_out, double* us_per_point) {
  if (n < 2 || n > GBSBIN_MAX_N || (n & 1)) return GBSBIN_ERR_ARG;
  if (precision != GBSBIN_FP64 && precision != GBSBIN_FP32_REFINE) return GBSBIN_ERR_ARG;
  TuneVal v{};
  int st = autotune_lookup(n, precision, &v);
  if (st) return st;
  if (kernel) *kernel = v.kernel;
  if (points_per_cta_out) *points_per_cta_out = v.P;
  if (us_per_point) *us_per_point = v.us_per_point;
  return GBSBIN_OK;
}

int gbsbin_batch_create(const gbsbin_problem* probs, int nprob, const gbsbin_options* o, int autotune,
                        gbsbin_batch** out) {
  if (!out || !probs || nprob <= 0) return GBSBIN_ERR_ARG;
  *out = nullptr;
  gbsbin_options opt;
  gbsbin_default_options(&opt);
  if (o) opt = *o;
  if (opt.want_backward || opt.want_timing) return GBSBIN_ERR_ARG;  // per-plan features only
  if (opt.shard_begin || opt.shard_end) return GBSBIN_ERR_UNSUPPORTED;
  gbsbin_batch* B = new (std::nothrow) gbsbin_batch();
  if (!B) return GBSBIN_ERR_NOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete B;
    return GBSBIN_ERR_CUDA;
  }
  B->plans.assign(nprob, nullptr);
  B->own.assign(nprob, 0);
  std::vector<PointArgs> args(nprob);
  std::map<std::tuple<int, int, int>, int> class_of;
  for (int i = 0; i < nprob; ++i) {
    gbsbin_options oi = opt;
    int p_override = 0;
    const int n = 2 * probs[i].M * probs[i].K;
    // problems whose per-point LUs would take ~50 us or more of the batch run a tree of block
    // eliminations of their own where one suits them (the automatic choice of a standalone
    // plan), outside the per-point job queue
    if (!opt.tile_override && probs[i].L >= 2 && n <= GBSBIN_MAX_N) {
      double evald = 1.0;
      for (int l = 0; l < probs[i].L; ++l) {
        const double R = (double)opt.oversample * (probs[i].cutoff[l] + 1);
        evald *= l + 1 < probs[i].L ? R : std::floor(R / 2) + 1;
      }
      if (evald * n * (double)n * n / 3.0 >= 2e7) {
        gbsbin_plan* T = nullptr;
        const int st = plan_create_impl(&probs[i], &opt, &T, 0, false, true);
        if (st == GBSBIN_OK && (is_tree(T->kernel) || is_btree(T->kernel))) {
          B->plans[i] = T;
          B->own[i] = 1;
          T->dft_plain = true;
          args[i] = make_point_args(T);
          continue;
        }
        if (T) gbsbin_plan_destroy(T);
      }
    }
    // one-group problems keep the Hessenberg path whatever the size's tuning
    const bool one_group = probs[i].L == 1;
    if (autotune && !opt.tile_override && n <= GBSBIN_MAX_N && !one_group) {
      TuneVal v{};
      int st = autotune_lookup(n, opt.precision, &v);
      if (st) {
        batch_free(B);
        return st;
      }
      oi.tile_override = v.kernel;
      p_override = v.P;
    }
    int st = plan_create_impl(&probs[i], &oi, &B->plans[i], p_override, false, false);
    if (st == GBSBIN_ERR_UNSUPPORTED && p_override)
      st = plan_create_impl(&probs[i], &opt, &B->plans[i], 0, false, false);
    if (st) {
      batch_free(B);
      return st;
    }
    gbsbin_plan* P = B->plans[i];
    args[i] = make_point_args(P);
    const int threads = (P->kernel == GBSBIN_KERNEL_WARP_FP32R || is_hess(P->kernel)) ? 128
                        : is_blk(P->kernel) ? 256
                                                               : points_threads(P->kernel, P->n);
    // warp kernel: padded size class; blocked kernel: problems whose shared memory allows
    // two CTAs per SM run apart from the larger ones (a class launches with its largest need);
    // Hessenberg kernels: the row slots per lane of the instantiation
    const int np = P->kernel == GBSBIN_KERNEL_WARP_FP32R ? (P->n <= 8 ? 8 : P->n <= 16 ? 16 : 32)
                   : is_blk(P->kernel) ? points_blk_ctas_per_sm(P->n)
                   : is_hess(P->kernel) ? hess_slots(P->n)
                                                          : 0;
    auto key = std::make_tuple(P->kernel, threads, np);
    if (!class_of.count(key)) {
      class_of[key] = (int)B->classes.size();
      B->classes.emplace_back();
      B->classes.back().kernel = P->kernel;
      B->classes.back().threads = threads;
      B->classes.back().np = np;
    }
    auto& C = B->classes[class_of[key]];
    const int group = (P->kernel == GBSBIN_KERNEL_WARP_FP32R || is_hess(P->kernel)) ? 4 : P->P;
    for (long long e0 = 0; e0 < P->grid.n_eval; e0 += group) C.jobs.push_back(PointJob{i, 0, e0});
    if (P->kernel == GBSBIN_KERNEL_SMEM_FP64 || P->kernel == GBSBIN_KERNEL_SMEM_FP32R ||
        P->kernel == GBSBIN_KERNEL_GMEM_FP64 || P->kernel == GBSBIN_KERNEL_GMEM_FP32R)
      C.smem = std::max(C.smem, points_smem_bytes(P->kernel, P->n, P->P, P->L));
    if (is_blk(P->kernel)) C.smem = std::max(C.smem, points_blk_smem_bytes(P->n));
    if (P->kernel == GBSBIN_KERNEL_GMEM_FP64 || P->kernel == GBSBIN_KERNEL_GMEM_FP32R ||
        is_blk(P->kernel))
      B->gws_slot = std::max(B->gws_slot, ((long long)(is_blk(P->kernel)
                                                               ? points_blk_slot_bytes(P->n)
                                                               : points_matrix_bytes(P->kernel, P->n, 1)) + 255) /
                                              256 * 256);
  }
  if (B->gws_slot > 0) {
    if (cudaMalloc(&B->d_gws, (size_t)B->gws_slot * B->num_sms * GBSBIN_BLK_CTAS_PER_SM) != cudaSuccess) {
      cudaGetLastError();
      batch_free(B);
      return GBSBIN_ERR_NOMEM;
    }
    for (auto& a : args) {
      a.gws = B->d_gws;
      a.gws_slot_bytes = B->gws_slot;
    }
  }
  // largest jobs first: cost ~ n^3 x points per job, so the queue ends on small jobs
  for (auto& C : B->classes) {
    std::stable_sort(C.jobs.begin(), C.jobs.end(), [&](const PointJob& x, const PointJob& y) {
      double cx = std::pow((double)B->plans[x.prob]->n, 3) * B->plans[x.prob]->P;
      double cy = std::pow((double)B->plans[y.prob]->n, 3) * B->plans[y.prob]->P;
      return cx > cy;
    });
    if (cudaMalloc(&C.d_jobs, C.jobs.size() * sizeof(PointJob)) != cudaSuccess ||
        cudaMemcpy(C.d_jobs, C.jobs.data(), C.jobs.size() * sizeof(PointJob), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      batch_free(B);
      return GBSBIN_ERR_NOMEM;
    }
  }
  if (cudaMalloc(&B->d_probs, sizeof(PointArgs) * nprob) != cudaSuccess ||
      cudaMemcpy(B->d_probs, args.data(), sizeof(PointArgs) * nprob, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&B->d_queue, sizeof(unsigned long long) * std::max<size_t>(1, B->classes.size())) != cudaSuccess) {
    cudaGetLastError();
    batch_free(B);
    return GBSBIN_ERR_NOMEM;
  }
  // tree problems, largest per-point work first, over up to batch_side_streams() side streams
  std::vector<std::pair<double, int>> trees;
  for (int i = 0; i < nprob; ++i)
    if (B->own[i]) {
      const gbsbin_plan* P = B->plans[i];
      trees.emplace_back(-(double)P->grid.n_eval * P->n * P->n * P->n, i);
    }
  std::sort(trees.begin(), trees.end());
  for (auto& t : trees) B->tree_order.push_back(t.second);
  const int ns = (int)std::min<size_t>((size_t)batch_side_streams(), trees.size());
  B->side.assign(ns, nullptr);
  B->ev_join.assign(ns, nullptr);
  bool ok = ns == 0 || cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < ns; ++k)
    ok = cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    batch_free(B);
    return GBSBIN_ERR_CUDA;
  }
  *out = B;
  return GBSBIN_OK;
}

int gbsbin_batch_destroy(gbsbin_batch* B) {
  if (!B) return GBSBIN_ERR_ARG;
  cudaDeviceSynchronize();
  batch_free(B);
  return GBSBIN_OK;
}

long long gbsbin_batch_table_size(const gbsbin_batch* B, int i) {
  if (!B || i < 0 || i >= (int)B->plans.size()) return -1;
  return B->plans[i]->table_size;
}

int gbsbin_batch_execute(gbsbin_batch* B, double* const* P_out, void* stream) {
  if (!B || !P_out) return GBSBIN_ERR_ARG;
  return batch_launch(B, P_out, (cudaStream_t)stream);
}

int gbsbin_batch_capture_graph(gbsbin_batch* B, double* const* P_out, void* stream) {
  if (!B || !P_out) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) return GBSBIN_ERR_ARG;  // the legacy default stream cannot be captured
  if (B->graph_exec) {
    cudaGraphExecDestroy(B->graph_exec);
    B->graph_exec = nullptr;
  }
  if (B->graph) {
    cudaGraphDestroy(B->graph);
    B->graph = nullptr;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GBSBIN_ERR_CUDA;
  int st = batch_launch(B, P_out, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || !g) return GBSBIN_ERR_CUDA;
  B->graph = g;
  if (cudaGraphInstantiate(&B->graph_exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  return GBSBIN_OK;
}

int gbsbin_batch_replay(gbsbin_batch* B, void* stream) {
  if (!B || !B->graph_exec) return GBSBIN_ERR_ARG;
  return cudaGraphLaunch(B->graph_exec, (cudaStream_t)stream) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
}

int gbsbin_batch_diagnostics(gbsbin_batch* B, int i, gbsbin_diag* out, void* stream) {
  if (!B || i < 0 || i >= (int)B->plans.size()) return GBSBIN_ERR_ARG;
  return gbsbin_diagnostics(B->plans[i], out, stream);
}

int gbsbin_batch_read_points(gbsbin_batch* B, int i, double* logq_host, double* minpiv_host, void* stream) {
  if (!B || i < 0 || i >= (int)B->plans.size()) return GBSBIN_ERR_ARG;
  return gbsbin_read_points(B->plans[i], logq_host, minpiv_host, stream);
}

}  // extern "C"
