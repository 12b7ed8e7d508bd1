// Table stage without device allocation.
//
// gbsbin_table_from_logq_noalloc turns per-point log q values into the binned table, like
// the DFT stage of gbsbin_execute, but it never allocates: its scratch (the twiddle tables
// and the two intermediate transform buffers) lives in one fixed array in this file,
// reserved on every GPU that loads the library for the life of the process.  It is for
// callers that must not allocate device memory: code running under a device-memory
// budget owned by another framework's pool allocator (where a stray cudaMalloc can fail
// or fragment the pool), and latency-critical loops where cudaMalloc/cudaFree would
// synchronise the device and stall work queued on other streams.
#include <mutex>

#include "gbsbin_internal.h"

namespace gbsbin {
namespace {

constexpr long long kMaxEval = GBSBIN_NOALLOC_MAX_EVAL;
constexpr long long kMaxTwiddles = GBSBIN_NOALLOC_MAX_TWIDDLES;
constexpr int kMaxDevices = 64;

// [twiddles | transform buffer A | transform buffer B], complex FP64.  Shared by every call
// on a device; it keeps the last call's contents.  Nothing in it needs to start at zero:
// every element is written before it is read within a call.
static __device__ __align__(256) double2 g_table_scratch[kMaxTwiddles + 2 * kMaxEval];

// Device address of g_table_scratch, looked up once per device.  In host code the array's
// name is only a host-side stand-in, so it is never passed to a kernel directly.
double2* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

int scratch_for_current_device(double2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return GBSBIN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_table_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GBSBIN_ERR_CUDA;
    }
    g_scratch_addr[dev] = (double2*)p;
  }
  *out = g_scratch_addr[dev];
  return GBSBIN_OK;
}

// tw[off_l + m] = exp(-2 pi i m / radix_l) for every axis, from the exact integer m
__global__ void k_fill_twiddles(double2* __restrict__ tw, GridDesc g, long long total) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long off = 0;
    int l = 0;
    while (l < g.L - 1 && t >= off + g.radix[l]) off += g.radix[l++];
    const int R = g.radix[l];
    const long long m = t - off;
    double s, c;
    sincospi(-2.0 * (double)m / (double)R, &s, &c);
    tw[t] = make_double2(c, s);
  }
}

}  // namespace
}  // namespace gbsbin

using namespace gbsbin;

extern "C" int gbsbin_table_from_logq_noalloc(int L, const int* cutoff, int oversample, const double* logq,
                                              double* P_out, void* stream) {
  if (L < 1 || L > GBSBIN_MAX_L || !cutoff || !logq || !P_out || oversample < 1) return GBSBIN_ERR_ARG;
  GridDesc g{};
  g.L = L;
  g.npts = 1;
  long long table = 1, twiddles = 0;
  for (int l = 0; l < L; ++l) {
    if (cutoff[l] < 0) return GBSBIN_ERR_CUTOFF;
    long long R = (long long)oversample * (cutoff[l] + 1LL);
    if (R > (1LL << 26)) return GBSBIN_ERR_CUTOFF;
    g.radix[l] = (int)R;
    g.nout[l] = cutoff[l] + 1;
    g.npts *= R;
    if (g.npts > GBSBIN_MAX_POINTS) return GBSBIN_ERR_CUTOFF;
    table *= g.nout[l];
    twiddles += R;
  }
  g.half = g.radix[L - 1] / 2 + 1;
  g.n_eval = g.npts / g.radix[L - 1] * g.half;
  g.n_full = g.n_eval;   // the whole half grid: no shard
  g.e_lo = 0;
  g.e_hi = g.n_eval;
  if (g.n_eval > kMaxEval || twiddles > kMaxTwiddles) return GBSBIN_ERR_UNSUPPORTED;

  double2* base = nullptr;
  int st = scratch_for_current_device(&base);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  long long blocks = (twiddles + 255) / 256;
  k_fill_twiddles<<<(unsigned)(blocks > 1024 ? 1024 : blocks), 256, 0, s>>>(base, g, twiddles);
  if (cudaGetLastError() != cudaSuccess) return GBSBIN_ERR_CUDA;
  DftArgs d{};
  d.grid = g;
  d.logq = (const double2*)logq;
  d.tw = base;
  d.bufA = base + kMaxTwiddles;
  d.bufB = base + kMaxTwiddles + kMaxEval;
  d.P = P_out;
  d.diag = nullptr;
  d.minpiv = nullptr;
  d.table_size = table;
  return launch_dft(d, s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
}
