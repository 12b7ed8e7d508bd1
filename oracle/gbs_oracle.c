/*
 * Plain FP64 CPU oracle for binned photon-number distributions of Gaussian states
 * (arXiv:2412.17742).  TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU
 * baseline leg of the benchmark call it; the CUDA library never does.  It is written
 * for checking by eye against the paper, not for speed: no blocking, no fusion.
 *
 * Per grid point (Sec. III, Eq. q_d; Sec. VI, Eq. Lamb_lhaf_master):
 *   w_l   = exp(2 pi i k_l / R_l)                 roots of unity, from the integer k_l
 *   D(w)  = diag(w_{label(i)})                    one w per detector group, both halves
 *   K     = I - D(w) XA
 *   K     = L U                                   Doolittle, no pivoting
 *   ld    = sum_i Log u_ii                        principal Log of each pivot
 *   x     = K^{-1} D(w) X gamma                   forward + back substitution
 *   log q = 1/2 gamma^T x - 1/2 ld
 * The probability generating function is G(w) = q(w) / q(1)   (Eq. sum_lhafs gives
 * Pr(0) = 1/q(1)), and the folded binned table is its inverse DFT
 *   P~(b) = (1/N_pts) sum_k G(omega^k) omega^{-k.b}.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NUMERIC = 7, OR_ERR_NOMEM = 6 };

static const double TWO_PI = 6.283185307179586476925286766559;

/* Mixed-radix digits of the flattened point index f, last axis fastest. */
static void point_digits(long f, int L, const int *radix, int *k) {
  for (int l = L - 1; l >= 0; --l) {
    k[l] = (int)(f % radix[l]);
    f /= radix[l];
  }
}

/* exp(2 pi i m / R) for an integer m reduced mod R, so no angle accumulates. */
static cplx unit_root(long m, int R) {
  long r = m % R;
  if (r < 0) r += R;
  double a = TWO_PI * (double)r / (double)R;
  return cos(a) + I * sin(a);
}

/*
 * log q at one point.  Kw is n*n scratch, x and b are n scratch.
 * Returns 0, or OR_ERR_NUMERIC if a pivot has Re <= 0 or is not finite (the pivots of
 * I - D(w) XA have positive real part for every physical state, because ||XA|| < 1 and
 * D(w) is unitary).
 */
static int point_logq(int n, const cplx *XA, const cplx *gamma, const cplx *Xgamma,
                      const cplx *d, cplx *Kw, cplx *x, cplx *out_logq, double *out_minre) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      Kw[(long)i * n + j] = (i == j ? 1.0 : 0.0) - d[i] * XA[(long)i * n + j];

  int status = OR_OK;
  double minre = INFINITY;
  for (int k = 0; k < n; ++k) {
    cplx piv = Kw[(long)k * n + k];
    if (!(creal(piv) > 0.0) || !isfinite(creal(piv)) || !isfinite(cimag(piv))) status = OR_ERR_NUMERIC;
    if (creal(piv) < minre) minre = creal(piv);
    for (int i = k + 1; i < n; ++i) {
      cplx lik = Kw[(long)i * n + k] / piv;
      Kw[(long)i * n + k] = lik;
      for (int j = k + 1; j < n; ++j) Kw[(long)i * n + j] -= lik * Kw[(long)k * n + j];
    }
  }

  cplx ld = 0.0;
  for (int k = 0; k < n; ++k) ld += clog(Kw[(long)k * n + k]);

  /* right-hand side D(w) X gamma, then L y = b (unit lower), U x = y */
  for (int i = 0; i < n; ++i) {
    cplx s = d[i] * Xgamma[i];
    for (int j = 0; j < i; ++j) s -= Kw[(long)i * n + j] * x[j];
    x[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx s = x[i];
    for (int j = i + 1; j < n; ++j) s -= Kw[(long)i * n + j] * x[j];
    x[i] = s / Kw[(long)i * n + i];
  }
  cplx expo = 0.0;
  for (int i = 0; i < n; ++i) expo += gamma[i] * x[i];

  *out_logq = 0.5 * expo - 0.5 * ld;
  *out_minre = minre;
  return status;
}

/*
 * log q at every point of the grid prod(radix).
 *   XA      n*n complex (interleaved re,im), row-major
 *   gamma   n complex
 *   label   n ints: detector group of row i (both halves of the mode vector)
 *   radix   L ints R_l >= 1
 *   logq    out: N_pts complex
 *   minre   out: N_pts doubles, smallest Re u_ii at each point
 *   status  out: N_pts ints
 */
int oracle_logq_grid(int n, const double *XA_, const double *gamma_, const int *label, int L,
                     const int *radix, double *logq_, double *minre, int *status,
                     int nthreads) {
  if (n <= 0 || L <= 0 || !XA_ || !gamma_ || !label || !radix || !logq_) return OR_ERR_ARG;
  const cplx *XA = (const cplx *)XA_;
  const cplx *gamma = (const cplx *)gamma_;
  cplx *logq = (cplx *)logq_;
  long npts = 1;
  for (int l = 0; l < L; ++l) {
    if (radix[l] <= 0) return OR_ERR_ARG;
    npts *= radix[l];
  }
  /* X gamma swaps the two halves */
  cplx *Xgamma = (cplx *)malloc(sizeof(cplx) * n);
  if (!Xgamma) return OR_ERR_NOMEM;
  int h = n / 2;
  for (int i = 0; i < n; ++i) Xgamma[i] = gamma[i < h ? i + h : i - h];

  int nerr = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : nerr)
  {
    cplx *Kw = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
    cplx *x = (cplx *)malloc(sizeof(cplx) * n);
    cplx *d = (cplx *)malloc(sizeof(cplx) * n);
    int *k = (int *)malloc(sizeof(int) * L);
#pragma omp for schedule(dynamic, 4)
    for (long f = 0; f < npts; ++f) {
      point_digits(f, L, radix, k);
      for (int i = 0; i < n; ++i) d[i] = unit_root(k[label[i]], radix[label[i]]);
      double mr;
      int st = point_logq(n, XA, gamma, Xgamma, d, Kw, x, &logq[f], &mr);
      if (minre) minre[f] = mr;
      if (status) status[f] = st;
      if (st) nerr += 1;
    }
    free(Kw);
    free(x);
    free(d);
    free(k);
  }
  free(Xgamma);
  return nerr ? OR_ERR_NUMERIC : OR_OK;
}

/*
 * log q at selected points only: idx[c] are flattened indices into the grid prod(radix)
 * (last axis fastest); outputs as in oracle_logq_grid, one entry per selected point.
 */
int oracle_logq_points(int n, const double *XA_, const double *gamma_, const int *label, int L,
                       const int *radix, const long long *idx, long count, double *logq_,
                       double *minre, int *status, int nthreads) {
  if (n <= 0 || L <= 0 || !XA_ || !gamma_ || !label || !radix || !idx || !logq_) return OR_ERR_ARG;
  const cplx *XA = (const cplx *)XA_;
  const cplx *gamma = (const cplx *)gamma_;
  cplx *logq = (cplx *)logq_;
  cplx *Xgamma = (cplx *)malloc(sizeof(cplx) * n);
  if (!Xgamma) return OR_ERR_NOMEM;
  int h = n / 2;
  for (int i = 0; i < n; ++i) Xgamma[i] = gamma[i < h ? i + h : i - h];
  int nerr = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : nerr)
  {
    cplx *Kw = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
    cplx *x = (cplx *)malloc(sizeof(cplx) * n);
    cplx *d = (cplx *)malloc(sizeof(cplx) * n);
    int *k = (int *)malloc(sizeof(int) * L);
#pragma omp for schedule(dynamic, 1)
    for (long c = 0; c < count; ++c) {
      point_digits((long)idx[c], L, radix, k);
      for (int i = 0; i < n; ++i) d[i] = unit_root(k[label[i]], radix[label[i]]);
      double mr;
      int st = point_logq(n, XA, gamma, Xgamma, d, Kw, x, &logq[c], &mr);
      if (minre) minre[c] = mr;
      if (status) status[c] = st;
      if (st) nerr += 1;
    }
    free(Kw);
    free(x);
    free(d);
    free(k);
  }
  free(Xgamma);
  return nerr ? OR_ERR_NUMERIC : OR_OK;
}

/* Neumaier-compensated accumulation of one real sum. */
typedef struct {
  double s, c;
} nsum;
static void nsum_add(nsum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

/*
 * Direct multidimensional DFT with the sign of the inverse transform used here:
 *   out(b) = (1/N_pts) sum_k in(k) prod_l exp(-2 pi i k_l b_l / R_l)
 * done one axis at a time, each line summed with Neumaier compensation.  in and out
 * are N_pts complex (interleaved), row-major over the axes, last axis fastest.
 */
int oracle_dft(int L, const int *radix, const double *in_, double *out_) {
  if (L <= 0 || !radix || !in_ || !out_) return OR_ERR_ARG;
  long npts = 1;
  for (int l = 0; l < L; ++l) {
    if (radix[l] <= 0) return OR_ERR_ARG;
    npts *= radix[l];
  }
  cplx *a = (cplx *)malloc(sizeof(cplx) * npts);
  cplx *b = (cplx *)malloc(sizeof(cplx) * npts);
  if (!a || !b) {
    free(a);
    free(b);
    return OR_ERR_NOMEM;
  }
  memcpy(a, in_, sizeof(cplx) * npts);
  long inner = npts;
  for (int l = 0; l < L; ++l) {
    int R = radix[l];
    inner /= R;                 /* stride of axis l */
    long outer = npts / (inner * R);
#pragma omp parallel for collapse(2)
    for (long o = 0; o < outer; ++o)
      for (long s = 0; s < inner; ++s) {
        long base = o * R * inner + s;
        for (int bl = 0; bl < R; ++bl) {
          nsum re = {0, 0}, im = {0, 0};
          for (int kl = 0; kl < R; ++kl) {
            cplx t = a[base + (long)kl * inner] * unit_root(-(long)kl * bl, R);
            nsum_add(&re, creal(t));
            nsum_add(&im, cimag(t));
          }
          b[base + (long)bl * inner] = ((re.s + re.c) + I * (im.s + im.c)) / (double)R;
        }
      }
    cplx *t = a;
    a = b;
    b = t;
  }
  memcpy(out_, a, sizeof(cplx) * npts);
  free(a);
  free(b);
  return OR_OK;
}

/*
 * Fully distinguishable sources (App. D, its limit of one source per internal mode): source
 * s is a single-mode squeezed vacuum whose photons leave on output port k with probability
 * p[k*S + s] = |T_ks|^2 and are lost otherwise, independently of the other sources.  Its
 * output generating function is g_s(1 - P_s + sum_k p_ks z_k), P_s = sum_k p_ks, with
 * g_s(y) = sum_j a[s*(M+1) + j] (y - (1 - P_s))^j given as Taylor coefficients, and the
 * joint one is the product over sources.  The probability of one photon on every one of the
 * M ports is the coefficient of z_1 ... z_M: each source covers a subset T of the ports, with
 * coefficient a_{s,|T|} |T|! prod_{k in T} p_ks, so a dynamic programme over the subsets of
 * covered ports (sources added one at a time, every subset of the uncovered ports tried)
 * sums only positive terms.  O(S 3^M); M <= 24.
 */
int oracle_distinguishable_ones(int M, int S, const double *p, const double *a, double *out) {
  if (M < 1 || M > 24 || S < 1) return OR_ERR_ARG;
  const long full = 1L << M;
  double *dp = (double *)calloc(full, sizeof(double));
  double *nx = (double *)malloc(full * sizeof(double));
  double *f = (double *)malloc(full * sizeof(double));
  if (!dp || !nx || !f) {
    free(dp);
    free(nx);
    free(f);
    return OR_ERR_NOMEM;
  }
  dp[0] = 1.0;
  double fact[25];
  fact[0] = 1.0;
  for (int j = 1; j <= 24; ++j) fact[j] = fact[j - 1] * j;
  for (int s = 0; s < S; ++s) {
    /* f(T) = a_{s,|T|} |T|! prod_{k in T} p_ks */
    for (long T = 0; T < full; ++T) {
      double prod = 1.0;
      int size = 0;
      for (int k = 0; k < M; ++k)
        if (T >> k & 1) {
          prod *= p[(long)k * S + s];
          ++size;
        }
      f[T] = a[(long)s * (M + 1) + size] * fact[size] * prod;
    }
    /* nx(U) = sum over T subset of U of dp(U \ T) f(T) */
#pragma omp parallel for schedule(dynamic, 64)
    for (long U = 0; U < full; ++U) {
      double acc = 0.0;
      for (long T = U;; T = (T - 1) & U) {
        acc += dp[U ^ T] * f[T];
        if (T == 0) break;
      }
      nx[U] = acc;
    }
    double *t = dp;
    dp = nx;
    nx = t;
  }
  *out = dp[full - 1];
  free(dp);
  free(nx);
  free(f);
  return OR_OK;
}
