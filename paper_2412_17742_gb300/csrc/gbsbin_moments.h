// Exact binned cumulants of orders 1-4 on the GPU (gbsbin_moments.cu).  Not part of the public
// ABI.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gbsbin.h"

#define GBSBIN_MOM_MAX_L 16

namespace gbsbin {

// n x n W = Sigma^(1) (Hermitian) and the vectors gamma, X gamma (interleaved complex FP64,
// host memory) with the rows sorted by group: group l holds rows goff[l] .. goff[l + 1] - 1 (goff[0] = 0, goff[L] = n).
// For r = 1 .. order, kappa[r - 1] (host memory, L^r doubles, row-major; may be null) receives
// the r-th cumulant tensor of the counts.  Device buffers are allocated and freed per call;
// synchronous on s.  *ms (may be null) receives the device time of the launches (CUDA events).
// pairs: the products and block sums in pairs of FP32 (~46 bits) instead of FP64.
int cumulants_device(int n, int L, const int* goff, const double* W, const double* gamma, const double* Xgamma,
                     int order, bool pairs, double* const* kappa, cudaStream_t s, float* ms);

}  // namespace gbsbin
