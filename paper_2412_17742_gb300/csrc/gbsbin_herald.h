// Heralded states (gbsbin_herald.cu, gbsbin_herald_host.cpp).  Not part of the public ABI.
#pragma once

#include "gbsbin_internal.h"

namespace gbsbin {

// D: the heralding and traced modes' indices (first halves, then second halves, nd in all),
// F: the kept modes' (nf).  A = X XA blocks row-major.  The Taylor coefficients are visited
// in order of total degree from a table built with the plan: entry t of shell s (s = 1 ..
// nf cut, entries shell[s] .. shell[s + 1] - 1) is coefficient q = tq[t], computed from
// p - e_i0 (index tqm[t], i0 = ti0[t] the first non-zero digit, p_i0 = tp[t]) and its
// neighbours p - e_i0 - e_j (tnb[t nf + j], -1 where that digit is zero).
#define GBSBIN_HERALD_MAX_F (2 * GBSBIN_HERALD_MAX_KEPT)
struct HeraldArgs {
  int L, nd, nf, n2, cut;
  int radix[GBSBIN_MAX_L];           // oversample (cutoff + 1) per heralding group
  int nout[GBSBIN_MAX_L];            // cutoff + 1
  long long npts;                    // prod radix
  long long ncoef;                   // (cut + 1)^nf
  long long table;                   // prod nout
  double pr0;                        // Pr(0) of the whole state
  const int* dgroup;                 // [nd] heralding group of D index i, or -1 (traced)
  const int* dpart;                  // [nd] the X partner of D index i (within D)
  const double2* tw;                 // exp(-2 pi i d / radix[l]), d < radix[l], group after group
  const double2* ADD;                // nd x nd
  const double2* ADF;                // nd x nf
  const double2* AFF;                // nf x nf
  const double2* gD;                 // nd
  const double2* gF;                 // nf
  const double* chscale;             // [ncoef] prod_i sqrt(p_i!)
  const int* shell;                  // [nf cut + 2] first table entry of each shell
  const int* tq;                     // [ncoef - 1] coefficient of each entry
  const int* tqm;
  const int* ti0;
  const int* tp;
  const int* tnb;                    // [(ncoef - 1) nf]
  double2* gcoef;                    // npts x (ncoef + 1): Taylor coefficients at each point, then
                                     // the heralding probability's generating function
  double2* scratch;                  // npts x (ncoef + 1): the inverse DFT's other buffer
  double* minpiv;                    // npts: smallest pivot real part of both eliminations
  double* prob_own;                  // table: the plan's copy of Pr(b) (diagnostics)
};
size_t herald_smem_bytes(int nd, int nf, int n2);
cudaError_t launch_herald(const HeraldArgs& a, double2* out, double* prob, cudaStream_t s);

}  // namespace gbsbin
