// Host side of heralded states (arXiv:2412.17742, Sec. VII): validation, the adjacency blocks
// A = X XA split by mode role, the heralding grid's twiddles, Pr(0), device buffers and the
// two launches (points, then the inverse DFT over the heralding grid).
#include <algorithm>
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "gbsbin_herald.h"
#include "gbsbin_host_state.h"

using cd = std::complex<double>;
using namespace gbsbin;

struct gbsbin_herald_plan {
  gbsbin_options opt{};
  HeraldArgs args{};
  int n2 = 0;
  long long table_size = 0;              // complex elements of rho
  bool executed = false;
  double logq1_re = 0.0;
  size_t upload_bytes = 0;
  // device
  unsigned char* d_const = nullptr;      // role, dpart, dmode, tw, blocks, chscale
  double2* d_gcoef = nullptr;
  double2* d_scratch = nullptr;
  double* d_minpiv = nullptr;
  double* d_prob = nullptr;              // the plan's copy of Pr(b)
  double2* d_rho_tmp = nullptr;          // execute_host's device result
  double* d_prob_tmp = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

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

void free_all(gbsbin_herald_plan* P) {
  void* ptrs[] = {P->d_const, P->d_gcoef, P->d_scratch, P->d_minpiv, P->d_prob, P->d_rho_tmp, P->d_prob_tmp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
}

// Byte image of the constant inputs, each piece 16-byte aligned.
struct Blob {
  std::vector<unsigned char> bytes;
  size_t put(const void* src, size_t n) {
    const size_t off = (bytes.size() + 15) & ~(size_t)15;
    bytes.resize(off + n);
    if (n) std::copy((const unsigned char*)src, (const unsigned char*)src + n, bytes.begin() + off);
    return off;
  }
};

std::vector<double2> to_d2(const std::vector<cd>& v) {
  std::vector<double2> o(v.size());
  for (size_t q = 0; q < v.size(); ++q) o[q] = make_double2(v[q].real(), v[q].imag());
  return o;
}

}  // namespace

extern "C" {

int gbsbin_herald_plan_create(const gbsbin_herald_problem* p, const gbsbin_options* o, gbsbin_herald_plan** out) {
  if (!out) return GBSBIN_ERR_ARG;
  *out = nullptr;
  if (!p || !p->role || !p->cutoff) return GBSBIN_ERR_ARG;
  const gbsbin_problem* s = &p->state;
  if (s->M <= 0 || s->K <= 0 || (!s->sigma1 && (!s->r || !s->T))) return GBSBIN_ERR_ARG;
  gbsbin_options opt;
  gbsbin_default_options(&opt);
  if (o) opt = *o;
  if (opt.precision != GBSBIN_FP64 || opt.oversample < 1 || opt.want_backward || opt.shard_end != 0 ||
      opt.shard_begin != 0 || (opt.tile_override != 0 && opt.tile_override != GBSBIN_KERNEL_HERALD_FP64))
    return GBSBIN_ERR_ARG;
  const int L = p->L, nm = s->M * s->K, n2 = 2 * nm;
  if (L < 1 || L > GBSBIN_MAX_L || p->fock_cutoff < 0) return GBSBIN_ERR_ARG;
  if (n2 > GBSBIN_HERALD_MAX_MODES2) return GBSBIN_ERR_UNSUPPORTED;
  std::vector<int> cnt(L, 0), Dm, kept;
  for (int m = 0; m < nm; ++m) {
    const int r = p->role[m];
    if (r < GBSBIN_HERALD_KEPT || r >= L) return GBSBIN_ERR_ARG;
    if (r >= 0) cnt[r]++;
    if (r == GBSBIN_HERALD_KEPT) kept.push_back(m);
    else Dm.push_back(m);
  }
  for (int l = 0; l < L; ++l)
    if (cnt[l] == 0) return GBSBIN_ERR_PARTITION;
  const int nk = (int)kept.size();
  if (nk < 1 || nk > GBSBIN_HERALD_MAX_KEPT) return GBSBIN_ERR_UNSUPPORTED;
  const int nf = 2 * nk, nd = 2 * (int)Dm.size(), cut = p->fock_cutoff;
  long long ncoef = 1;
  for (int i = 0; i < nf; ++i) {
    ncoef *= cut + 1;
    if (ncoef > GBSBIN_HERALD_MAX_COEF) return GBSBIN_ERR_UNSUPPORTED;
  }
  HeraldArgs a{};
  a.L = L;
  a.nd = nd;
  a.nf = nf;
  a.n2 = n2;
  a.cut = cut;
  a.ncoef = ncoef;
  a.npts = 1;
  a.table = 1;
  int rsum = 0;
  for (int l = 0; l < L; ++l) {
    if (p->cutoff[l] < 0) return GBSBIN_ERR_CUTOFF;
    const long long R = (long long)opt.oversample * (p->cutoff[l] + 1LL);
    if (R > (1LL << 26)) return GBSBIN_ERR_CUTOFF;
    a.radix[l] = (int)R;
    a.nout[l] = p->cutoff[l] + 1;
    a.npts *= R;
    a.table *= a.nout[l];
    rsum += (int)R;
    if (a.npts > GBSBIN_MAX_POINTS || rsum > (1 << 26)) return GBSBIN_ERR_CUTOFF;
  }
  // the per-point coefficient tensors and the DFT's scratch (16 bytes an entry) stay within 8 GiB
  if ((double)a.npts * (double)(ncoef + 1) > (double)(1LL << 28)) return GBSBIN_ERR_UNSUPPORTED;
  std::vector<cd> XA, gamma, Xgamma;
  int st = host_state(s, n2, XA, gamma, Xgamma);
  if (st) return st;
  // A = X XA: row i of A is row partner(i) of XA
  std::vector<cd> A((size_t)n2 * n2);
  for (int i = 0; i < n2; ++i) {
    const int pi = i < nm ? i + nm : i - nm;
    for (int j = 0; j < n2; ++j) A[(size_t)i * n2 + j] = XA[(size_t)pi * n2 + j];
  }
  std::vector<int> D, F;
  for (int m : Dm) D.push_back(m);
  for (int m : Dm) D.push_back(m + nm);
  for (int m : kept) F.push_back(m);
  for (int m : kept) F.push_back(m + nm);
  std::vector<cd> ADD((size_t)nd * nd), ADF((size_t)nd * nf), AFF((size_t)nf * nf), gD(nd), gF(nf);
  for (int i = 0; i < nd; ++i) {
    for (int j = 0; j < nd; ++j) ADD[(size_t)i * nd + j] = A[(size_t)D[i] * n2 + D[j]];
    for (int j = 0; j < nf; ++j) ADF[(size_t)i * nf + j] = A[(size_t)D[i] * n2 + F[j]];
    gD[i] = gamma[D[i]];
  }
  for (int i = 0; i < nf; ++i) {
    for (int j = 0; j < nf; ++j) AFF[(size_t)i * nf + j] = A[(size_t)F[i] * n2 + F[j]];
    gF[i] = gamma[F[i]];
  }
  std::vector<int> dpart(nd), dgroup(nd);
  const int hd = nd / 2;
  for (int i = 0; i < nd; ++i) {
    dpart[i] = i < hd ? i + hd : i - hd;
    dgroup[i] = p->role[Dm[i % hd]] >= 0 ? p->role[Dm[i % hd]] : -1;
  }
  // the Taylor coefficients in order of total degree, each with its predecessor p - e_i0 (i0
  // its first non-zero digit) and that predecessor's neighbours p - e_i0 - e_j
  const int cp1 = cut + 1, nsh = nf * cut;
  std::vector<std::vector<int>> by_shell((size_t)nsh + 1);
  for (long long q = 1; q < ncoef; ++q) {
    long long r = q;
    int tot = 0;
    for (int i = 0; i < nf; ++i) {
      tot += (int)(r % cp1);
      r /= cp1;
    }
    by_shell[tot].push_back((int)q);
  }
  std::vector<int> shell((size_t)nsh + 2, 0), tq, tqm, ti0, tp, tnb;
  std::vector<long long> stride(nf);
  stride[nf - 1] = 1;
  for (int i = nf - 2; i >= 0; --i) stride[i] = stride[i + 1] * cp1;
  for (int sh = 1; sh <= nsh; ++sh) {
    shell[sh] = (int)tq.size();
    for (int q : by_shell[sh]) {
      int dig[GBSBIN_HERALD_MAX_F];
      for (int i = 0; i < nf; ++i) dig[i] = (int)((q / stride[i]) % cp1);
      int i0 = 0;
      while (dig[i0] == 0) ++i0;
      const long long qm = q - stride[i0];
      tq.push_back(q);
      tqm.push_back((int)qm);
      ti0.push_back(i0);
      tp.push_back(dig[i0]);
      for (int j = 0; j < nf; ++j) {
        const int dj = dig[j] - (j == i0 ? 1 : 0);
        tnb.push_back(dj > 0 ? (int)(qm - stride[j]) : -1);
      }
    }
  }
  shell[nsh + 1] = (int)tq.size();
  const double TWO_PI = 6.283185307179586476925286766559;
  std::vector<double2> tw((size_t)rsum);
  for (int l = 0, off = 0; l < L; off += a.radix[l], ++l)
    for (int d = 0; d < a.radix[l]; ++d) {
      const cd v = std::polar(1.0, -TWO_PI * (double)d / (double)a.radix[l]);
      tw[off + d] = make_double2(v.real(), v.imag());
    }
  std::vector<double> fs(cut + 1), chs((size_t)ncoef);
  fs[0] = 1.0;
  for (int i = 1; i <= cut; ++i) fs[i] = fs[i - 1] * std::sqrt((double)i);   // sqrt(i!)
  for (long long q = 0; q < ncoef; ++q) {
    long long r = q;
    double v = 1.0;
    for (int i = 0; i < nf; ++i) {
      v *= fs[r % (cut + 1)];
      r /= cut + 1;
    }
    chs[q] = v;
  }
  double mp = 0.0;
  const cd lq1 = host_logq1(XA, gamma, Xgamma, n2, &mp);
  if (!(mp > 0.0) || !std::isfinite(lq1.real())) return GBSBIN_ERR_NONPHYSICAL;
  a.pr0 = std::exp(-lq1.real());

  Blob b;
  const size_t o_dgroup = b.put(dgroup.data(), dgroup.size() * sizeof(int));
  const size_t o_dpart = b.put(dpart.data(), dpart.size() * sizeof(int));
  const size_t o_tw = b.put(tw.data(), tw.size() * sizeof(double2));
  const std::vector<double2> vADD = to_d2(ADD), vADF = to_d2(ADF), vAFF = to_d2(AFF), vgD = to_d2(gD),
                             vgF = to_d2(gF);
  const size_t o_ADD = b.put(vADD.data(), vADD.size() * sizeof(double2));
  const size_t o_ADF = b.put(vADF.data(), vADF.size() * sizeof(double2));
  const size_t o_AFF = b.put(vAFF.data(), vAFF.size() * sizeof(double2));
  const size_t o_gD = b.put(vgD.data(), vgD.size() * sizeof(double2));
  const size_t o_gF = b.put(vgF.data(), vgF.size() * sizeof(double2));
  const size_t o_chs = b.put(chs.data(), chs.size() * sizeof(double));
  const size_t o_shell = b.put(shell.data(), shell.size() * sizeof(int));
  const size_t o_tq = b.put(tq.data(), tq.size() * sizeof(int));
  const size_t o_tqm = b.put(tqm.data(), tqm.size() * sizeof(int));
  const size_t o_ti0 = b.put(ti0.data(), ti0.size() * sizeof(int));
  const size_t o_tp = b.put(tp.data(), tp.size() * sizeof(int));
  const size_t o_tnb = b.put(tnb.data(), tnb.size() * sizeof(int));

  gbsbin_herald_plan* P = new (std::nothrow) gbsbin_herald_plan();
  if (!P) return GBSBIN_ERR_NOMEM;
  P->opt = opt;
  P->n2 = n2;
  P->table_size = a.table * ncoef;
  P->logq1_re = lq1.real();
  P->upload_bytes = b.bytes.size();
  if ((st = dalloc(&P->d_const, b.bytes.size())) || (st = dalloc(&P->d_gcoef, (size_t)(a.npts * (ncoef + 1)))) ||
      (st = dalloc(&P->d_scratch, (size_t)(a.npts * (ncoef + 1)))) || (st = dalloc(&P->d_minpiv, (size_t)a.npts)) ||
      (st = dalloc(&P->d_prob, (size_t)a.table))) {
    free_all(P);
    delete P;
    return st;
  }
  if (cudaMemcpy(P->d_const, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(P->d_prob, 0, (size_t)a.table * sizeof(double)) != cudaSuccess ||
      (opt.want_timing && (cudaEventCreate(&P->ev0) != cudaSuccess || cudaEventCreate(&P->ev1) != cudaSuccess))) {
    cudaGetLastError();
    free_all(P);
    delete P;
    return GBSBIN_ERR_CUDA;
  }
  unsigned char* c = P->d_const;
  a.dgroup = reinterpret_cast<const int*>(c + o_dgroup);
  a.dpart = reinterpret_cast<const int*>(c + o_dpart);
  a.tw = reinterpret_cast<const double2*>(c + o_tw);
  a.ADD = reinterpret_cast<const double2*>(c + o_ADD);
  a.ADF = reinterpret_cast<const double2*>(c + o_ADF);
  a.AFF = reinterpret_cast<const double2*>(c + o_AFF);
  a.gD = reinterpret_cast<const double2*>(c + o_gD);
  a.gF = reinterpret_cast<const double2*>(c + o_gF);
  a.chscale = reinterpret_cast<const double*>(c + o_chs);
  a.shell = reinterpret_cast<const int*>(c + o_shell);
  a.tq = reinterpret_cast<const int*>(c + o_tq);
  a.tqm = reinterpret_cast<const int*>(c + o_tqm);
  a.ti0 = reinterpret_cast<const int*>(c + o_ti0);
  a.tp = reinterpret_cast<const int*>(c + o_tp);
  a.tnb = reinterpret_cast<const int*>(c + o_tnb);
  a.gcoef = P->d_gcoef;
  a.scratch = P->d_scratch;
  a.minpiv = P->d_minpiv;
  a.prob_own = P->d_prob;
  P->args = a;
  *out = P;
  return GBSBIN_OK;
}

long long gbsbin_herald_table_size(const gbsbin_herald_plan* P) { return P ? P->table_size : -1; }

long long gbsbin_herald_prob_size(const gbsbin_herald_plan* P) { return P ? P->args.table : -1; }

int gbsbin_herald_execute(gbsbin_herald_plan* P, gbsbin_complex* rho_out, double* prob_out, void* stream) {
  if (!P || !rho_out || !prob_out) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (P->ev0 && cudaEventRecord(P->ev0, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  if (launch_herald(P->args, reinterpret_cast<double2*>(rho_out), prob_out, s) != cudaSuccess) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  P->executed = true;
  if (P->ev1 && cudaEventRecord(P->ev1, s) != cudaSuccess) return GBSBIN_ERR_CUDA;
  return GBSBIN_OK;
}

int gbsbin_herald_execute_host(gbsbin_herald_plan* P, gbsbin_complex* rho_host, double* prob_host, void* stream) {
  if (!P || !rho_host || !prob_host) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = GBSBIN_OK;
  if (!P->d_rho_tmp && ((st = dalloc(&P->d_rho_tmp, (size_t)P->table_size)) ||
                        (st = dalloc(&P->d_prob_tmp, (size_t)P->args.table))))
    return st;
  st = gbsbin_herald_execute(P, reinterpret_cast<gbsbin_complex*>(P->d_rho_tmp), P->d_prob_tmp, stream);
  if (!st && (cudaMemcpyAsync(rho_host, P->d_rho_tmp, (size_t)P->table_size * sizeof(double2),
                              cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaMemcpyAsync(prob_host, P->d_prob_tmp, (size_t)P->args.table * sizeof(double),
                              cudaMemcpyDeviceToHost, s) != cudaSuccess))
    st = GBSBIN_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && !st) st = GBSBIN_ERR_CUDA;
  return st;
}

int gbsbin_herald_diagnostics(gbsbin_herald_plan* P, gbsbin_diag* out, void* stream) {
  if (!P || !out) return GBSBIN_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const HeraldArgs& a = P->args;
  std::vector<double> mp((size_t)a.npts, 1.0), pr((size_t)a.table, 0.0);
  if (P->executed &&
      (cudaMemcpyAsync(mp.data(), P->d_minpiv, mp.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaMemcpyAsync(pr.data(), P->d_prob, pr.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess)) {
    cudaGetLastError();
    return GBSBIN_ERR_CUDA;
  }
  double sum = 0.0, mn = 1e300;
  long long bad = 0;
  for (double v : pr) sum += v;
  for (double v : mp) {
    if (!(v > 0.0)) ++bad;
    mn = std::fmin(mn, v);
  }
  *out = gbsbin_diag{};
  out->sum_P = sum;
  out->max_imag = 0.0;
  out->min_pivot_re = P->executed ? mn : 1.0;
  out->n_bad_points = bad;
  out->n_points = a.npts;
  out->n_evaluated = a.npts;
  out->table_size = P->table_size;
  out->n = P->n2;
  out->kernel = GBSBIN_KERNEL_HERALD_FP64;
  out->log_q1_re = P->logq1_re;
  out->point_kernel_ms = 0.0;
  out->state_upload_bytes = (long long)P->upload_bytes;
  out->launches = P->executed ? 1 + a.L : 0;
  if (P->ev1 && P->executed) {
    float ms = 0.f;
    if (cudaEventSynchronize(P->ev1) != cudaSuccess || cudaEventElapsedTime(&ms, P->ev0, P->ev1) != cudaSuccess) {
      cudaGetLastError();
      return GBSBIN_ERR_CUDA;
    }
    out->point_kernel_ms = ms;
  }
  if (bad > 0 || !std::isfinite(sum)) return GBSBIN_ERR_NUMERIC;
  return GBSBIN_OK;
}

int gbsbin_herald_plan_destroy(gbsbin_herald_plan* P) {
  if (!P) return GBSBIN_OK;
  cudaDeviceSynchronize();
  free_all(P);
  delete P;
  return GBSBIN_OK;
}

}  // extern "C"
