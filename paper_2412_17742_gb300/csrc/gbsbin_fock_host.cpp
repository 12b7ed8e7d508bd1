// Host side of the Fock-input path (arXiv:2412.17742, App. C): validation, the FP64
// coefficient matrices I - T^dag T and T_l^dag T_l restricted to the occupied inputs, the
// node and output-group roots, device workspaces and the two launches (nodes x points,
// then the inverse DFT of the output groups).
#include <algorithm>
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "gbsbin_internal.h"

using cd = std::complex<double>;
using namespace gbsbin;

struct gbsbin_fock_plan {
  int M = 0, L = 0;
  gbsbin_options opt{};
  std::vector<int> photons, bin_of_mode, cutoff;
  std::vector<int> pos_input;            // input port of each position (position 0: held)
  bool df = false;
  int zt = 1;                            // output-group points per thread
  int kernel = 0;
  int num_sms = 0;
  long long table_size = 0;
  FockArgs args{};
  size_t coef_count = 0;                 // (L + 1) nin^2
  bool executed = false;                 // an execute has been enqueued
  // device
  unsigned char* d_state = nullptr;      // coef (double2) then coef_df (float4)
  double2* d_xtw = nullptr;
  float4* d_xtw_df = nullptr;
  double2* d_zr = nullptr;
  float4* d_zr_df = nullptr;
  double2* d_tw = nullptr;               // inverse-DFT twiddles exp(-2 pi i m / R)
  double2* d_parts = nullptr;
  double2* d_bufA = nullptr;
  double2* d_bufB = nullptr;
  double* d_diag = nullptr;
  unsigned* d_bar = nullptr;
  double* d_table = nullptr;
  unsigned char* h_stage = nullptr;      // pinned copy of the state block
  size_t state_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

float4 split_df(cd v) {
  const float hr = (float)v.real(), hi = (float)v.imag();
  return make_float4(hr, hi, (float)(v.real() - (double)hr), (float)(v.imag() - (double)hi));
}

template <typename T>
int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? GBSBIN_ERR_NOMEM : GBSBIN_ERR_CUDA;
  }
  return GBSBIN_OK;
}

void free_all(gbsbin_fock_plan* P) {
  void* ptrs[] = {P->d_state, P->d_xtw, P->d_xtw_df, P->d_zr, P->d_zr_df, P->d_tw, P->d_parts,
                  P->d_bufA, P->d_bufB, P->d_diag, P->d_bar, P->d_table};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (P->h_stage) cudaFreeHost(P->h_stage);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
}

// ||T||_2 <= 1: (1 + 1e-10) I - T^dag T must admit a Cholesky factor.
bool contraction(const std::vector<cd>& T, int M) {
  std::vector<cd> A((size_t)M * M);
  for (int j = 0; j < M; ++j)
    for (int k = 0; k < M; ++k) {
      cd s = 0.0;
      for (int i = 0; i < M; ++i) s += std::conj(T[(size_t)i * M + j]) * T[(size_t)i * M + k];
      A[(size_t)j * M + k] = (j == k ? 1.0 + 1e-10 : 0.0) - s;
    }
  for (int j = 0; j < M; ++j) {
    double d = A[(size_t)j * M + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(A[(size_t)j * M + k]);
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * M + j] = d;
    for (int i = j + 1; i < M; ++i) {
      cd s = A[(size_t)i * M + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * M + k] * std::conj(A[(size_t)j * M + k]);
      A[(size_t)i * M + j] = s / d;
    }
  }
  return true;
}

// Coefficient matrices into the pinned staging block: m = 0: I - T^dag T, m = 1 + l:
// T_l^dag T_l, over the occupied inputs in position order, stored [m][k][j]; then the same
// as FP32 pairs.
int stage_transfer(gbsbin_fock_plan* P, const gbsbin_complex* Tin) {
  const int M = P->M, L = P->L, nin = P->args.nin;
  std::vector<cd> T((size_t)M * M);
  for (size_t q = 0; q < T.size(); ++q) {
    T[q] = cd(Tin[q].re, Tin[q].im);
    if (!std::isfinite(Tin[q].re) || !std::isfinite(Tin[q].im)) return GBSBIN_ERR_ARG;
  }
  if (!contraction(T, M)) return GBSBIN_ERR_NONPHYSICAL;
  double2* coef = reinterpret_cast<double2*>(P->h_stage);
  float4* coef_df = reinterpret_cast<float4*>(P->h_stage + P->coef_count * sizeof(double2));
  for (int m = 0; m <= L; ++m)
    for (int k = 0; k < nin; ++k)
      for (int j = 0; j < nin; ++j) {
        const int jj = P->pos_input[j], kk = P->pos_input[k];
        cd s = 0.0;
        for (int i = 0; i < M; ++i)
          if (m == 0 || P->bin_of_mode[i] == m - 1) s += std::conj(T[(size_t)i * M + jj]) * T[(size_t)i * M + kk];
        if (m == 0) s = (j == k ? 1.0 : 0.0) - s;
        const size_t q = ((size_t)m * nin + k) * nin + j;
        coef[q] = make_double2(s.real(), s.imag());
        coef_df[q] = split_df(s);
      }
  return GBSBIN_OK;
}

}  // namespace

extern "C" {

int gbsbin_fock_plan_create(const gbsbin_fock_problem* p, const gbsbin_options* o, gbsbin_fock_plan** out) {
  if (!out) return GBSBIN_ERR_ARG;
  *out = nullptr;
  if (!p || p->M <= 0 || !p->T || !p->photons || !p->bin_of_mode || !p->cutoff) return GBSBIN_ERR_ARG;
  gbsbin_options opt;
  gbsbin_default_options(&opt);
  if (o) opt = *o;
  if (opt.oversample < 1 || (opt.precision != GBSBIN_FP64 && opt.precision != GBSBIN_FP32_REFINE))
    return GBSBIN_ERR_ARG;
  if (opt.tile_override != 0 && opt.tile_override != GBSBIN_KERNEL_FOCK_FP64 &&
      opt.tile_override != GBSBIN_KERNEL_FOCK_DF32)
    return GBSBIN_ERR_ARG;
  if (opt.want_backward) return GBSBIN_ERR_UNSUPPORTED;
  const int M = p->M, L = p->L;
  if (L < 1 || L > M) return GBSBIN_ERR_ARG;
  if (L > GBSBIN_FOCK_MAX_GROUPS) return GBSBIN_ERR_UNSUPPORTED;
  std::vector<int> seen(L, 0);
  for (int i = 0; i < M; ++i) {
    if (p->bin_of_mode[i] < 0 || p->bin_of_mode[i] >= L) return GBSBIN_ERR_PARTITION;
    seen[p->bin_of_mode[i]] = 1;
  }
  for (int l = 0; l < L; ++l)
    if (!seen[l]) return GBSBIN_ERR_PARTITION;
  long long npts = 1;
  for (int l = 0; l < L; ++l) {
    if (p->cutoff[l] < 0) return GBSBIN_ERR_CUTOFF;
    npts *= (long long)opt.oversample * (p->cutoff[l] + 1);
    if (npts > GBSBIN_MAX_POINTS) return GBSBIN_ERR_CUTOFF;
  }
  // occupied inputs; position 0 holds the one with the fewest photons (lowest port on ties)
  std::vector<int> occ;
  for (int j = 0; j < M; ++j) {
    if (p->photons[j] < 0) return GBSBIN_ERR_ARG;
    if (p->photons[j] > GBSBIN_FOCK_MAX_PER_INPUT) return GBSBIN_ERR_UNSUPPORTED;
    if (p->photons[j] > 0) occ.push_back(j);
  }
  if ((int)occ.size() > GBSBIN_FOCK_MAX_INPUTS) return GBSBIN_ERR_UNSUPPORTED;
  {
    std::vector<cd> T((size_t)M * M);
    for (size_t q = 0; q < T.size(); ++q) {
      if (!std::isfinite(p->T[q].re) || !std::isfinite(p->T[q].im)) return GBSBIN_ERR_ARG;
      T[q] = cd(p->T[q].re, p->T[q].im);
    }
    if (!contraction(T, M)) return GBSBIN_ERR_NONPHYSICAL;
  }
  gbsbin_fock_plan* P = new (std::nothrow) gbsbin_fock_plan();
  if (!P) return GBSBIN_ERR_NOMEM;
  P->M = M;
  P->L = L;
  P->opt = opt;
  P->photons.assign(p->photons, p->photons + M);
  P->bin_of_mode.assign(p->bin_of_mode, p->bin_of_mode + M);
  P->cutoff.assign(p->cutoff, p->cutoff + L);
  if (!occ.empty()) {
    int h = 0;
    for (int t = 1; t < (int)occ.size(); ++t)
      if (p->photons[occ[t]] < p->photons[occ[h]]) h = t;
    P->pos_input.push_back(occ[h]);
    for (int t = 0; t < (int)occ.size(); ++t)
      if (t != h) P->pos_input.push_back(occ[t]);
  }
  FockArgs& a = P->args;
  a.nin = (int)P->pos_input.size();
  a.L = L;
  a.nd = a.nin > 0 ? a.nin - 1 : 0;
  for (int j = 0; j < a.nin; ++j) a.pw[j] = p->photons[P->pos_input[j]];
  a.dstride[0] = 1;
  int xoff = 0;
  for (int d = 0; d < a.nd; ++d) {
    a.drad[d] = a.pw[d + 1] + 1;
    a.doff[d] = xoff;
    xoff += a.drad[d];
    if ((double)a.dstride[d] * a.drad[d] > (double)GBSBIN_FOCK_MAX_NODES) {
      delete P;
      return GBSBIN_ERR_UNSUPPORTED;
    }
    a.dstride[d + 1] = a.dstride[d] * a.drad[d];
  }
  a.S = a.dstride[a.nd];
  // a shard walks the nodes [shard_begin, shard_end) only; its table is the partial sum of
  // their terms (normalised by the whole node count), so the shards' tables add up
  a.x_lo = 0;
  a.x_hi = a.S;
  if (opt.shard_end != 0 || opt.shard_begin != 0) {
    if (opt.shard_begin < 0 || opt.shard_end <= opt.shard_begin || opt.shard_end > a.S) {
      delete P;
      return GBSBIN_ERR_ARG;
    }
    a.x_lo = opt.shard_begin;
    a.x_hi = opt.shard_end;
  }
  const long long nodes = a.x_hi - a.x_lo;
  // output-group grid, as for Gaussian states
  GridDesc& g = a.grid;
  g.L = L;
  g.npts = 1;
  P->table_size = 1;
  a.roff[0] = 0;
  for (int l = 0; l < L; ++l) {
    g.radix[l] = opt.oversample * (p->cutoff[l] + 1);
    g.nout[l] = p->cutoff[l] + 1;
    g.npts *= g.radix[l];
    P->table_size *= g.nout[l];
    a.roff[l + 1] = a.roff[l] + g.radix[l];
  }
  a.rsum = a.roff[L];
  g.half = g.radix[L - 1] / 2 + 1;
  g.n_full = g.npts / g.radix[L - 1] * g.half;
  g.e_lo = 0;
  g.e_hi = g.n_full;
  g.n_eval = g.n_full;
  P->kernel = opt.tile_override ? opt.tile_override
                                : (opt.precision == GBSBIN_FP32_REFINE ? GBSBIN_KERNEL_FOCK_DF32 : GBSBIN_KERNEL_FOCK_FP64);
  P->df = P->kernel == GBSBIN_KERNEL_FOCK_DF32;
  // restarts bound the drift of the incrementally updated state (FP32 pairs drift faster)
  const long long chunk_max = P->df ? 256 : 1024;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  const size_t smem = fock_smem_bytes(a.nin, L, a.rsum);
  P->zt = fock_points_per_thread(P->df, g.n_full);
  const int per_sm = smem <= 200 * 1024 ? fock_ctas_per_sm(P->df, P->zt, smem) : 0;
  if (per_sm < 1) {
    delete P;
    return GBSBIN_ERR_UNSUPPORTED;
  }
  const long long per_cta = (long long)GBSBIN_FOCK_THREADS * P->zt;
  const long long tiles = (g.n_full + per_cta - 1) / per_cta;
  // node ranges: two whole waves of resident CTAs where the nodes allow (a partial last wave
  // idles SMs), each range at least 32 nodes; ranges longer than chunk_max are walked as
  // several restarts dealt cyclically
  const long long slots = (long long)per_sm * P->num_sms;
  long long xr = 2 * slots / tiles;
  const long long cap = (512LL << 20) / (16 * g.n_full);            // parts <= 512 MB
  if (xr > cap) xr = cap;
  if (xr > 65535) xr = 65535;
  if (xr > (nodes + 31) / 32) xr = (nodes + 31) / 32;
  if (xr < 1) xr = 1;
  a.chunk = (nodes + xr - 1) / xr;
  if (a.chunk > chunk_max) a.chunk = chunk_max;
  a.nchunks = (nodes + a.chunk - 1) / a.chunk;
  if (xr > a.nchunks) xr = a.nchunks;
  a.xr = (int)xr;
  P->coef_count = (size_t)(L + 1) * a.nin * a.nin;
  P->state_bytes = P->coef_count * (sizeof(double2) + sizeof(float4));
  int st = GBSBIN_OK;
  if ((st = dalloc(&P->d_state, P->state_bytes)) || (st = dalloc(&P->d_xtw, (size_t)xoff)) ||
      (st = dalloc(&P->d_xtw_df, (size_t)xoff)) || (st = dalloc(&P->d_zr, (size_t)a.rsum)) ||
      (st = dalloc(&P->d_zr_df, (size_t)a.rsum)) || (st = dalloc(&P->d_tw, (size_t)a.rsum)) ||
      (st = dalloc(&P->d_parts, (size_t)xr * g.n_full)) || (st = dalloc(&P->d_bufA, (size_t)g.n_full)) ||
      (st = dalloc(&P->d_bufB, (size_t)g.n_full)) || (st = dalloc(&P->d_diag, GBSBIN_DIAG_DOUBLES)) ||
      (st = dalloc(&P->d_bar, 4)) || (st = dalloc(&P->d_table, (size_t)P->table_size))) {
    free_all(P);
    delete P;
    return st;
  }
  if (cudaMallocHost(&P->h_stage, P->state_bytes ? P->state_bytes : 1) != cudaSuccess) {
    cudaGetLastError();
    P->h_stage = nullptr;
    free_all(P);
    delete P;
    return GBSBIN_ERR_NOMEM;
  }
  if (opt.want_timing &&
      (cudaEventCreate(&P->ev0) != cudaSuccess || cudaEventCreate(&P->ev1) != cudaSuccess)) {
    cudaGetLastError();
    free_all(P);
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  a.coef = reinterpret_cast<const double2*>(P->d_state);
  a.coef_df = reinterpret_cast<const float4*>(P->d_state + P->coef_count * sizeof(double2));
  a.xtw = P->d_xtw;
  a.xtw_df = P->d_xtw_df;
  a.zr = P->d_zr;
  a.zr_df = P->d_zr_df;
  a.parts = P->d_parts;
  // roots from exact integer indices
  const double TWO_PI = 6.283185307179586476925286766559;
  std::vector<double2> xtw((size_t)std::max(xoff, 1)), zr((size_t)a.rsum), tw((size_t)a.rsum);
  std::vector<float4> xtw_df((size_t)std::max(xoff, 1)), zr_df((size_t)a.rsum);
  for (int d = 0; d < a.nd; ++d)
    for (int q = 0; q < a.drad[d]; ++q) {
      const cd v = std::polar(1.0, TWO_PI * (double)q / (double)a.drad[d]);
      xtw[a.doff[d] + q] = make_double2(v.real(), v.imag());
      xtw_df[a.doff[d] + q] = split_df(v);
    }
  for (int l = 0; l < L; ++l)
    for (int q = 0; q < g.radix[l]; ++q) {
      const cd v = std::polar(1.0, TWO_PI * (double)q / (double)g.radix[l]);
      zr[a.roff[l] + q] = make_double2(v.real(), v.imag());
      zr_df[a.roff[l] + q] = split_df(v);
      tw[a.roff[l] + q] = make_double2(v.real(), -v.imag());
    }
  st = stage_transfer(P, p->T);
  if (!st) {
    if (cudaMemcpy(P->d_xtw, xtw.data(), (size_t)xoff * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_xtw_df, xtw_df.data(), (size_t)xoff * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_zr, zr.data(), zr.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_zr_df, zr_df.data(), zr_df.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->d_state, P->h_stage, P->state_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(P->d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(P->d_diag, 0, GBSBIN_DIAG_DOUBLES * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      st = GBSBIN_ERR_CUDA;
    }
  }
  if (st) {
    free_all(P);
    delete P;
    return st;
  }
  *out = P;
  return GBSBIN_OK;
}

int gbsbin_fock_plan_set_transfer(gbsbin_fock_plan* P, const gbsbin_complex* T, void* stream) {
  if (!P || !T) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the staging block may still feed an earlier upload on this stream
  if (cudaStreamSynchronize(s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  int st = stage_transfer(P, T);
  if (st) return st;
  if (P->state_bytes &&
      cudaMemcpyAsync(P->d_state, P->h_stage, P->state_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GBSBIN_ERR_CUDA;
  return GBSBIN_OK;
}

long long gbsbin_fock_plan_table_size(const gbsbin_fock_plan* P) { return P ? P->table_size : -1; }

long long gbsbin_fock_plan_nodes(const gbsbin_fock_plan* P) { return P ? P->args.S : -1; }

int gbsbin_fock_execute(gbsbin_fock_plan* P, double* P_out, void* stream) {
  if (!P || !P_out) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (P->ev0 && cudaEventRecord(P->ev0, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  if (launch_fock(P->args, P->df, P->zt, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  P->executed = true;
  if (P->ev1 && cudaEventRecord(P->ev1, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  DftArgs d{};
  d.grid = P->args.grid;
  d.parts = P->d_parts;
  d.nparts = P->args.xr;
  d.pscale = 1.0 / (double)P->args.S;
  d.tw = P->d_tw;
  d.bufA = P->d_bufA;
  d.bufB = P->d_bufB;
  d.P = P_out;
  d.diag = P->opt.want_diagnostics ? P->d_diag : nullptr;
  d.table_size = P->table_size;
  return launch_dft_fused(d, P->d_bar, P->num_sms, s) == cudaSuccess ? GBSBIN_OK : GBSBIN_ERR_CUDA;
}

int gbsbin_fock_execute_host(gbsbin_fock_plan* P, double* P_out_host, void* stream) {
  if (!P || !P_out_host) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = gbsbin_fock_execute(P, P->d_table, stream);
  if (!st && cudaMemcpyAsync(P_out_host, P->d_table, (size_t)P->table_size * sizeof(double),
                             cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = GBSBIN_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = GBSBIN_ERR_CUDA;
  return st;
}

int gbsbin_fock_diagnostics(gbsbin_fock_plan* P, gbsbin_diag* out, void* stream) {
  if (!P || !out) return GBSBIN_ERR_ARG;
  std::vector<double> part(GBSBIN_DIAG_DOUBLES, 0.0);
  double sum = 0.0, im = 0.0;
  if (P->opt.want_diagnostics) {
    if (cudaMemcpyAsync(part.data(), P->d_diag, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
      return GBSBIN_ERR_CUDA;
    const int nblk = std::min(GBSBIN_DIAG_SLOTS, std::max(0, (int)part[4 * GBSBIN_DIAG_SLOTS + 2]));
    for (int b = 0; b < nblk; ++b) {   // fixed order: deterministic
      sum += part[4 * b];
      im = std::fmax(im, part[4 * b + 1]);
    }
  }
  out->sum_P = sum;
  out->max_imag = im;
  out->min_pivot_re = 1.0;
  out->n_bad_points = 0;
  out->log_q1_re = 0.0;
  out->n_points = P->args.grid.npts;
  out->n_evaluated = P->args.grid.n_full;
  out->table_size = P->table_size;
  out->n = P->args.nin;
  out->kernel = P->kernel;
  out->point_kernel_ms = 0.0;
  out->backward_kernel_ms = 0.0;
  out->backward_path = 0;
  out->state_upload_bytes = (long long)P->state_bytes;
  out->launches = P->executed ? 2 : 0;            // the Fock kernel and the fused DFT
  if (P->ev1 && P->executed) {
    float ms = 0.f;
    if (cudaEventSynchronize(P->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, P->ev0, P->ev1) != cudaSuccess) {
      cudaGetLastError();
      return GBSBIN_ERR_CUDA;
    }
    out->point_kernel_ms = ms;
  }
  if (P->opt.want_diagnostics && part[4 * GBSBIN_DIAG_SLOTS + 1] != 0.0) return GBSBIN_ERR_CUDA;
  if (P->opt.want_diagnostics && !(std::isfinite(sum))) return GBSBIN_ERR_NUMERIC;
  return GBSBIN_OK;
}

int gbsbin_fock_plan_destroy(gbsbin_fock_plan* P) {
  if (!P) return GBSBIN_OK;
  cudaDeviceSynchronize();
  free_all(P);
  delete P;
  return GBSBIN_OK;
}

}  // extern "C"
