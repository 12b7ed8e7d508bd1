// Fine-grained Pr(n) of fully distinguishable internal modes (arXiv:2412.17742, App. D) on
// the GPU: the sum over the evaluation points m <= n of the finite differences,
//
//   sum_{m <= n} prod_k C(n_k, m_k) (-1)^(N - |m|) f_N(m),
//   f_N(m) = [eta^N] exp(sum_j p_j(m) eta^j / (2j)),  p_j(m) = sum_l (lambda1^j + lambda2^j),
//
// one thread per point (grid-stride): the digits of m, per rank-2 block l its trace
// T = sum_k m_k d_lk and squared Frobenius norm F^2 = sum_kj m_k m_j S_lkj, the two eigenvalues
// T/2 +- sqrt(2 F^2 - T^2)/2, the power sums and the series coefficient.  FP64 throughout (the
// alternating sum cancels): each thread sums its terms with Neumaier compensation, each CTA
// reduces its threads' (sum, error) pairs by TwoSum in a fixed order into its own partial, and
// the host adds the partials in order, compensated; the terms' magnitudes are summed alongside
// for the caller's error estimate.  The points run in launches of a bounded number of points
// (a bounded amount of FP64 work each).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr int kThreads = 128;

struct DistArgs {
  int M, K, N, nmax;
  long long p0, p1;        // this launch's points [p0, p1) of prod (n_k + 1)
  const int* radix;        // M: n_k + 1
  const double* d;         // K x M
  const double* S;         // K x M x M
  const double* binom;     // M x (nmax + 1): C(n_k, m), m <= n_k
  double* partial;         // 3 x gridDim.x: sum, its rounding error, sum of magnitudes
};

__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__global__ void __launch_bounds__(kThreads) k_distinguishable(DistArgs a) {
  double ps[kDistMaxN + 1], e[kDistMaxN + 1];
  int m[kDistMaxM];
  double acc = 0.0, comp = 0.0, mag = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = a.p0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.p1; t += stride) {
    long long rest = t;
    int msum = 0;
    double bin = 1.0;
    for (int k = 0; k < a.M; ++k) {
      const int R = a.radix[k];
      const int mk = (int)(rest % R);
      rest /= R;
      m[k] = mk;
      msum += mk;
      bin *= a.binom[k * (a.nmax + 1) + mk];
    }
    for (int j = 0; j <= a.N; ++j) ps[j] = 0.0;
    for (int l = 0; l < a.K; ++l) {
      const double* dl = a.d + (size_t)l * a.M;
      const double* Sl = a.S + (size_t)l * a.M * a.M;
      double T = 0.0, F2 = 0.0;
      for (int k = 0; k < a.M; ++k) {
        if (m[k] == 0) continue;
        T += m[k] * dl[k];
        double row = 0.0;
        for (int j = 0; j < a.M; ++j) row += m[j] * Sl[k * a.M + j];
        F2 += m[k] * row;
      }
      const double disc = sqrt(fmax(0.0, 2.0 * F2 - T * T));
      const double l1 = 0.5 * (T + disc), l2 = 0.5 * (T - disc);
      double x1 = 1.0, x2 = 1.0;
      for (int j = 1; j <= a.N; ++j) {
        x1 *= l1;
        x2 *= l2;
        ps[j] += x1 + x2;
      }
    }
    e[0] = 1.0;                                      // e = exp(sum_j ps_j eta^j / (2j))
    for (int q = 1; q <= a.N; ++q) {
      double s = 0.0;
      for (int j = 1; j <= q; ++j) s += 0.5 * ps[j] * e[q - j];
      e[q] = s / q;
    }
    const double term = (((a.N - msum) & 1) ? -1.0 : 1.0) * bin * e[a.N];
    double sn, er;
    two_sum_d(acc, term, sn, er);
    acc = sn;
    comp += er;
    mag += fabs(term);
  }
  __shared__ double sh[kThreads], se[kThreads], sm[kThreads];
  sh[threadIdx.x] = acc;
  se[threadIdx.x] = comp;
  sm[threadIdx.x] = mag;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      double sn, er;
      two_sum_d(sh[threadIdx.x], sh[threadIdx.x + o], sn, er);
      sh[threadIdx.x] = sn;
      se[threadIdx.x] += se[threadIdx.x + o] + er;
      sm[threadIdx.x] += sm[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.partial[blockIdx.x] = sh[0];
    a.partial[gridDim.x + blockIdx.x] = se[0];
    a.partial[2 * gridDim.x + blockIdx.x] = sm[0];
  }
}

}  // namespace

int distinguishable_sum_device(int M, int K, int N, const int* pattern, const double* d, const double* S,
                               double* total, double* abs_total, cudaStream_t s) {
  if (M > kDistMaxM || N > kDistMaxN) return GBSBIN_ERR_UNSUPPORTED;
  int nmax = 0;
  long long npts = 1;
  std::vector<int> radix(M);
  for (int k = 0; k < M; ++k) {
    radix[k] = pattern[k] + 1;
    nmax = pattern[k] > nmax ? pattern[k] : nmax;
    npts *= radix[k];
    if (npts > (1ll << 40)) return GBSBIN_ERR_UNSUPPORTED;
  }
  // FP64 operations per point: digits and binomials, per block the trace and the norm's double
  // sum and the power sums, the series recurrence
  const double per_point = 4.0 * M + (double)K * (2.0 * M * M + 2.0 * M + 4.0 * N + 20.0) + (double)N * N + 4.0 * N;
  if (per_point * (double)npts > kDistMaxFlops) return GBSBIN_ERR_UNSUPPORTED;
  const long long chunk = std::max<long long>(kThreads, (long long)(kDistChunkFlops / per_point));
  std::vector<double> binom((size_t)M * (nmax + 1), 0.0);
  for (int k = 0; k < M; ++k) {
    double c = 1.0;
    for (int q = 0; q <= pattern[k]; ++q) {
      binom[(size_t)k * (nmax + 1) + q] = c;
      c = c * (double)(pattern[k] - q) / (double)(q + 1);
    }
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  const long long max_blocks = 8ll * sms;
  int* d_radix = nullptr;
  double *d_d = nullptr, *d_S = nullptr, *d_binom = nullptr, *d_part = nullptr;
  auto release = [&]() {
    if (d_radix) cudaFree(d_radix);
    if (d_d) cudaFree(d_d);
    if (d_S) cudaFree(d_S);
    if (d_binom) cudaFree(d_binom);
    if (d_part) cudaFree(d_part);
  };
  if (cudaMalloc(&d_radix, sizeof(int) * M) != cudaSuccess || cudaMalloc(&d_d, sizeof(double) * K * M) != cudaSuccess ||
      cudaMalloc(&d_S, sizeof(double) * (size_t)K * M * M) != cudaSuccess ||
      cudaMalloc(&d_binom, sizeof(double) * binom.size()) != cudaSuccess ||
      cudaMalloc(&d_part, sizeof(double) * 3 * max_blocks) != cudaSuccess) {
    cudaGetLastError();
    release();
    return GBSBIN_ERR_NOMEM;
  }
  std::vector<double> part((size_t)(3 * max_blocks));
  cudaError_t err = cudaMemcpyAsync(d_radix, radix.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_d, d, sizeof(double) * K * M, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_S, S, sizeof(double) * (size_t)K * M * M, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(d_binom, binom.data(), sizeof(double) * binom.size(), cudaMemcpyHostToDevice, s);
  double sum = 0.0, comp = 0.0, mag = 0.0;           // the partials, Neumaier-compensated, in order
  auto add = [&](double v) {
    const double t = sum + v;
    comp += std::fabs(sum) >= std::fabs(v) ? (sum - t) + v : (v - t) + sum;
    sum = t;
  };
  for (long long p0 = 0; err == cudaSuccess && p0 < npts; p0 += chunk) {
    const long long p1 = std::min(npts, p0 + chunk);
    long long blocks = (p1 - p0 + kThreads - 1) / kThreads;
    if (blocks > max_blocks) blocks = max_blocks;
    DistArgs a{M, K, N, nmax, p0, p1, d_radix, d_d, d_S, d_binom, d_part};
    k_distinguishable<<<(unsigned)blocks, kThreads, 0, s>>>(a);
    err = cudaGetLastError();
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * 3 * blocks, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess)
      for (long long b = 0; b < blocks; ++b) {       // fixed order
        add(part[b]);
        comp += part[blocks + b];
        mag += part[2 * blocks + b];
      }
  }
  release();
  if (err != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  *total = sum + comp;
  *abs_total = mag;
  return GBSBIN_OK;
}

}  // namespace gbsbin
