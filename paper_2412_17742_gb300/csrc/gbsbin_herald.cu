// Heralded (conditional) states of a Gaussian state (arXiv:2412.17742, Sec. VII, Eqs.
// heralded_state_internal and lhaf_heralded_offd_internal_1), from the generating function.
//
// The modes are heralding (group l), traced or kept.  With lhaf(A_p, gamma_p) the p-th
// derivative of exp(xi^T A xi / 2 + gamma^T xi) at 0, the sum over the heralding and traced
// photon patterns with weights w^n / n! is the complex-Gaussian expectation of that
// exponential with xi = sqrt(w) (alpha, conj alpha) on those modes, and the kept modes' Fock
// indices (u on the first half, v on the second) are Taylor coefficients of the rest:
//
//   sum_{n, t} lhaf(A_{(n,t,u)+(n,t,v)}, ...) w^n / (n! t!) = u! v! [x^u y^v] F(w; x, y),
//   F = exp(xi_F^T M xi_F / 2 + l^T xi_F + e) / sqrt(det(I - X D(w) A_DD)),
//   N = (I - X D(w) A_DD)^-1 X D(w),  M = A_FF + A_DF^T N A_DF,  l = gamma_F + A_DF^T N gamma_D,
//   e = gamma_D^T N gamma_D / 2,
//
// D the heralding and traced indices (both halves; w = 1 on traced modes), F the kept ones.
// Hence <v|rho(b)|u> = Pr(0) sqrt(u! v!) [w^b][x^u y^v] F.  Per point of the roots-of-unity grid
// over the heralding groups a CTA eliminates I - X D(w) A_DD without pivoting (a principal
// block of I - D(w) XA with ||XA|| < 1: every pivot has Re > 0 and Sum Log is the branch of
// the square root continuous from w = 0), solves for the kept modes' columns and gamma_D,
// forms M, l, e, and the Taylor coefficients of exp(xi^T M xi / 2 + l^T xi) by
// (p_i + 1) c_{p + e_i} = l_i c_p + sum_j M_ij c_{p - e_j} (shells of equal total degree in
// parallel, from a table of each coefficient's neighbours).  The heralding probability's
// generating function (every non-heralding mode traced, w = 1 on the kept ones) continues the
// same elimination into the kept block: its Schur complement is I - X_F M, so it is
// exp(e + l^T (I - X_F M)^{-1} X_F l / 2) / sqrt(det(I - X D A_DD) det(I - X_F M)), the
// branch Sum Log of the pivots of the whole unpivoted elimination.  An inverse DFT over the
// grid, one axis per launch, then extracts [w^b] for every coefficient.  FP64 throughout.
#include <cuda_runtime.h>

#include "gbsbin_device.cuh"
#include "gbsbin_herald.h"

namespace gbsbin {
namespace {

constexpr int HT = 256;

__device__ __forceinline__ double2 cadd2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cneg2(double2 a) { return make_double2(-a.x, -a.y); }

// Unpivoted elimination of the nr x nr block of G (row stride ld) with ncol right-hand-side
// columns after it, then back substitution (column by column: each solved entry updates the
// rows above it in parallel): the columns become the block's inverse times themselves.
// Returns sum Log(pivots) (each Re > 0) and the smallest pivot real part in thread 0's
// registers; all threads call it.
// Sum Log of a sequence of pivots (each Re > 0) without a log or an atan2 per pivot (FP64
// transcendentals are slow on this GPU): the running product, renormalised by powers of two,
// and the FP32 sum of the pivots' arguments, which fixes the winding of the product's argument
// (each argument lies in (-pi/2, pi/2); the FP32 sum errs by far less than pi).
struct LogDet {
  double2 prod = make_double2(1.0, 0.0);
  int e2 = 0, count = 0;
  float args = 0.f;
  double mn = 1e300;
  __device__ void add(double2 p) {
    prod = cmul(prod, p);
    args += atan2f((float)p.y, (float)p.x);
    mn = fmin(mn, p.x);
    if (!(p.x == p.x) || !(p.y == p.y)) mn = -1e300;
    if ((++count & 7) == 0) renorm();
  }
  __device__ void renorm() {
    const double m = fmax(fabs(prod.x), fabs(prod.y));
    if (!(m > 0.0) || !(m < 1e300)) return;
    const int ex = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1022;
    const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
    prod = make_double2(prod.x * sc, prod.y * sc);
    e2 += ex;
  }
  __device__ double2 value() {
    renorm();
    const double TWO_PI = 6.283185307179586476925286766559, LN2 = 0.693147180559945309417232121458;
    const double a0 = atan2(prod.y, prod.x);
    const double wind = rint(((double)args - a0) / TWO_PI);
    return make_double2(0.5 * log(fma(prod.x, prod.x, prod.y * prod.y)) + e2 * LN2, a0 + TWO_PI * wind);
  }
};

__device__ void solve_block(double2* G, int nr, int ncol, int ld, double2* ldet, double* minre) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int cols = nr + ncol;
  LogDet acc;
  for (int k = 0; k < nr; ++k) {
    const double2 piv = G[k * ld + k];
    const double2 r = crecip(piv);
    if (tid == 0) acc.add(piv);
    const int w = cols - k - 1;
    for (int idx = tid; idx < (nr - k - 1) * w; idx += T) {
      const int i = k + 1 + idx / w, j = k + 1 + idx % w;
      const double2 li = cmul(G[i * ld + k], r);
      G[i * ld + j] = cfnma(G[i * ld + j], li, G[k * ld + j]);
    }
    __syncthreads();
  }
  for (int k = nr - 1; k >= 0; --k) {                // x_k = rhs_k / u_kk; rhs_i -= u_ik x_k, i < k
    if (tid < ncol) G[k * ld + nr + tid] = cmul(G[k * ld + nr + tid], crecip(G[k * ld + k]));
    __syncthreads();
    for (int idx = tid; idx < k * ncol; idx += T) {
      const int i = idx / ncol, c = idx - (idx / ncol) * ncol;
      G[i * ld + nr + c] = cfnma(G[i * ld + nr + c], G[i * ld + k], G[k * ld + nr + c]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    *ldet = acc.value();
    *minre = acc.mn;
  }
}

__global__ void __launch_bounds__(HT) k_herald_points(HeraldArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const long long k = blockIdx.x;
  const int nd = a.nd, nf = a.nf, tid = threadIdx.x, T = blockDim.x;
  const int cols = nd + nf + 1;
  double2* G = reinterpret_cast<double2*>(sm_raw);   // nd x cols
  double2* Mq = G + (size_t)nd * cols;                // nf x nf
  double2* lq = Mq + nf * nf;                         // nf
  double2* sc = lq + nf;                              // e, log det
  double2* wg = sc + 2;                               // the heralding groups' roots at this point
  double2* wd = wg + GBSBIN_MAX_L;                    // the root of each D row's mode
  if (tid < a.L) {                                    // digit of group tid, w = exp(2 pi i d / R)
    long long rest = k;
    for (int q = a.L - 1; q > tid; --q) rest /= a.radix[q];
    const int d = (int)(rest % a.radix[tid]);
    int off = 0;
    for (int q = 0; q < tid; ++q) off += a.radix[q];
    const double2 t = a.tw[off + d];
    wg[tid] = make_double2(t.x, -t.y);
  }
  __syncthreads();
  for (int i = tid; i < nd; i += T) wd[i] = a.dgroup[i] >= 0 ? wg[a.dgroup[i]] : make_double2(1.0, 0.0);
  __syncthreads();
  // I - X D(w) A_DD with the right-hand sides X D(w) [A_DF | gamma_D]; row i of X D A is
  // w_{partner(i)} A_{partner(i), .}
  for (int idx = tid; idx < nd * cols; idx += T) {
    const int i = idx / cols, j = idx - (idx / cols) * cols;
    const int pi = a.dpart[i];                        // X partner of row i within D
    const double2 w = wd[pi];
    double2 v;
    if (j < nd) v = cneg2(cmul(w, a.ADD[(size_t)pi * nd + j]));
    else if (j < nd + nf) v = cmul(w, a.ADF[(size_t)pi * nf + (j - nd)]);
    else v = cmul(w, a.gD[pi]);
    if (j == i) v.x += 1.0;
    G[idx] = v;
  }
  __syncthreads();
  double2 ld;
  double mn;
  solve_block(G, nd, nf + 1, cols, &ld, &mn);
  // M = A_FF + A_DF^T Y_F, l = gamma_F + A_DF^T y, e = gamma_D^T y / 2
  for (int idx = tid; idx < nf * (nf + 1); idx += T) {
    const int i = idx / (nf + 1), c = idx - (idx / (nf + 1)) * (nf + 1);
    double2 s = c < nf ? a.AFF[i * nf + c] : a.gF[i];
    for (int d = 0; d < nd; ++d) s = cadd2(s, cmul(a.ADF[(size_t)d * nf + i], G[d * cols + nd + c]));
    if (c < nf) Mq[i * nf + c] = s;
    else lq[i] = s;
  }
  if (tid == 0) {
    double2 e = make_double2(0.0, 0.0);
    for (int d = 0; d < nd; ++d) e = cadd2(e, cmul(a.gD[d], G[d * cols + nd + nf]));
    sc[0] = make_double2(0.5 * e.x, 0.5 * e.y);
    sc[1] = ld;
  }
  __syncthreads();
  // the heralding probability's value: the kept block's Schur complement I - X_F M (X_F swaps
  // the kept modes' halves) with the right-hand side X_F l, eliminated by one thread
  if (tid == 0) {
    const int h = nf / 2;
    double2 Tm[GBSBIN_HERALD_MAX_F][GBSBIN_HERALD_MAX_F + 1];
    for (int i = 0; i < nf; ++i) {
      const int pi = i < h ? i + h : i - h;
      for (int j = 0; j < nf; ++j) Tm[i][j] = cneg2(Mq[pi * nf + j]);
      Tm[i][i].x += 1.0;
      Tm[i][nf] = lq[pi];
    }
    LogDet accf;
    for (int c = 0; c < nf; ++c) {
      const double2 piv = Tm[c][c];
      accf.add(piv);
      const double2 r = crecip(piv);
      for (int i = c + 1; i < nf; ++i) {
        const double2 li = cmul(Tm[i][c], r);
        for (int j = c + 1; j <= nf; ++j) Tm[i][j] = cfnma(Tm[i][j], li, Tm[c][j]);
      }
    }
    double2 y[GBSBIN_HERALD_MAX_F];
    for (int i = nf - 1; i >= 0; --i) {
      double2 s = Tm[i][nf];
      for (int j = i + 1; j < nf; ++j) s = cfnma(s, Tm[i][j], y[j]);
      y[i] = cmul(s, crecip(Tm[i][i]));
    }
    double2 ly = make_double2(0.0, 0.0);
    for (int i = 0; i < nf; ++i) ly = cadd2(ly, cmul(lq[i], y[i]));
    const double2 lf = accf.value();
    const double mnf = accf.mn;
    const double re = sc[0].x + 0.5 * ly.x - 0.5 * (ld.x + lf.x), im = sc[0].y + 0.5 * ly.y - 0.5 * (ld.y + lf.y);
    const double m = exp(re);
    double s, c;
    sincos(im, &s, &c);
    a.gcoef[(size_t)k * (a.ncoef + 1) + a.ncoef] = make_double2(m * c, m * s);
    a.minpiv[k] = fmin(mn, mnf);
  }
  // Taylor coefficients by shells of total degree, in this point's slot of ncoef + 1 entries
  // (index p = sum_i p_i (c + 1)^(nf - 1 - i)), from the plan's table of neighbours
  double2* C = a.gcoef + (size_t)k * (a.ncoef + 1);
  const double2 e = sc[0], l0 = sc[1];
  const double m0 = exp(e.x - 0.5 * l0.x);
  double s0, c0;
  sincos(e.y - 0.5 * l0.y, &s0, &c0);
  if (tid == 0) C[0] = make_double2(m0 * c0, m0 * s0);   // exp(e) / sqrt(det) times c_0 = 1
  __syncthreads();
  for (int shell = 1; shell <= nf * a.cut; ++shell) {
    for (int t = a.shell[shell] + tid; t < a.shell[shell + 1]; t += T) {
      const int i0 = a.ti0[t];
      double2 val = cmul(lq[i0], C[a.tqm[t]]);
      const int* nb = a.tnb + (size_t)t * nf;
      for (int j = 0; j < nf; ++j)
        if (nb[j] >= 0) val = cadd2(val, cmul(Mq[i0 * nf + j], C[nb[j]]));
      const double inv = 1.0 / (double)a.tp[t];
      C[a.tq[t]] = make_double2(val.x * inv, val.y * inv);
    }
    __syncthreads();
  }
}

// One axis of the inverse DFT over the heralding grid: out[pre][b][post][ch] = sum over
// k < R_l of in[pre][k][post][ch] exp(-2 pi i k b / R_l), b < nout_l (pre runs over the
// axes already transformed, extent nout; post over the later ones, extent radix; ch over the
// ncoef Taylor coefficients and the heralding probability's value).  One thread per output
// element, consecutive threads on consecutive channels (coalesced reads of the input).  The
// last axis scales by Pr(0) / N (and prod sqrt(p_i!) per coefficient) and writes rho and
// Pr(b).
__global__ void k_herald_dft_axis(HeraldArgs a, int l, const double2* __restrict__ in, double2* __restrict__ out,
                                  double2* __restrict__ rho, double* __restrict__ prob) {
  const long long nch = a.ncoef + 1;
  long long pre = 1, post = 1;
  for (int q = 0; q < l; ++q) pre *= a.nout[q];
  for (int q = l + 1; q < a.L; ++q) post *= a.radix[q];
  const int R = a.radix[l], nb = a.nout[l];
  int off = 0;
  for (int q = 0; q < l; ++q) off += a.radix[q];
  const bool last = l == a.L - 1;
  const long long total = pre * nb * post * nch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long rest = t;
    const long long ch = rest % nch;
    rest /= nch;
    const long long pi = rest % post;
    rest /= post;
    const int b = (int)(rest % nb);
    const long long pr = rest / nb;
    const double2* src = in + ((pr * R) * post + pi) * nch + ch;
    const long long step = post * nch;
    double2 acc = make_double2(0.0, 0.0);
    int idx = 0;                                     // k b mod R, advanced by b per k
    for (int k = 0; k < R; ++k) {
      acc = cadd2(acc, cmul(src[(long long)k * step], a.tw[off + idx]));
      idx += b;
      if (idx >= R) idx -= R;
    }
    if (!last) {
      out[((pr * nb + b) * post + pi) * nch + ch] = acc;
      continue;
    }
    const long long cell = pr * nb + b;              // post = 1 on the last axis
    const double s = a.pr0 / (double)a.npts;
    if (ch < a.ncoef) {
      const double f = s * a.chscale[ch];
      rho[cell * a.ncoef + ch] = make_double2(acc.x * f, acc.y * f);
    } else {
      prob[cell] = acc.x * s;
      a.prob_own[cell] = acc.x * s;
    }
  }
}

}  // namespace

size_t herald_smem_bytes(int nd, int nf, int n2) {
  (void)n2;
  return sizeof(double2) * ((size_t)nd * (nd + nf + 1) + (size_t)nf * nf + nf + 2 + GBSBIN_MAX_L + nd);
}

cudaError_t launch_herald(const HeraldArgs& a, double2* out, double* prob, cudaStream_t s) {
  const size_t smem = herald_smem_bytes(a.nd, a.nf, a.n2);
  cudaError_t err = cudaSuccess;
  if (smem > 48 * 1024) {
    err = cudaFuncSetAttribute(k_herald_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  k_herald_points<<<(unsigned)a.npts, HT, smem, s>>>(a);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // axis by axis, ping-pong between the coefficient slots and the scratch buffer (each
  // output is at most as large as its input)
  const long long nch = a.ncoef + 1;
  long long pre = 1;
  const double2* in = a.gcoef;
  for (int l = 0; l < a.L; ++l) {
    long long post = 1;
    for (int q = l + 1; q < a.L; ++q) post *= a.radix[q];
    const long long work = pre * a.nout[l] * post * nch;
    long long blocks = (work + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    double2* o = (in == a.gcoef) ? a.scratch : a.gcoef;
    k_herald_dft_axis<<<(unsigned)blocks, 256, 0, s>>>(a, l, in, o, out, prob);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    in = o;
    pre *= a.nout[l];
  }
  return cudaSuccess;
}

}  // namespace gbsbin
