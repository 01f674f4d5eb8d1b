// FP64-accurate residual on the BF16 tensor cores (residual_ozaki.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace spdinv {

// Bytes of workspace ozaki_residual needs for order n and S slices.
size_t ozaki_workspace_bytes(int64_t n, int S);

// R = I - A X (n x n, ld n), A symmetric given by its lower triangle (lda),
// X full (ld n); S slices per operand, slice pairs with s + t <= L.  The slice
// products run on tcgen05 (tc = true) or on mma.sync.  err: device int that
// records a device-side timeout.  Queues its kernels on s and adds their
// number to *launches.
cudaError_t ozaki_residual(int64_t n, const double* A, int64_t lda, const double* X, double* R, void* ws, int S,
                           int L, bool tc, int* err, cudaStream_t s, int* launches);

// The slice products with tcgen05 (residual_tc.cu): output = base + sign *
// sum of the pairs' products, where base is the given matrix, or the identity
// (identity = true) or zero when base is nullptr.  SA / SB: slice planes held
// by the two operands.  lower: only the 128 x 128 output tiles on and below
// the diagonal (products known to be symmetric).  The planes are atom-major
// (residual_ozaki.cu, plane_index).
cudaError_t ozaki_products_tc(int64_t n, int64_t npad, const void* Asl, int SA, const void* Xsl, int SB,
                              const int* ps, const int* pt, int npairs, const int* e, const int* f, double* R,
                              const double* base, bool identity, double sign, bool lower, int* err, cudaStream_t s);

// Workspace bytes of ozaki_refine_step for order n.
size_t ozaki_refine_workspace_bytes(int64_t n);

// One correction step of order p (2 <= p <= 8) of the hyperpower family
// X <- X (I + R + ... + R^{p-1}), R = I - A X, whose new residual is R^p:
//   R = I - A X from 7 slices per operand, pairs with levels <= levelsR;
//   X R, X R^2, ... as (X R^{m-1}) R, each symmetric, lower tiles only, with
//   fewer slices as the terms shrink; each term is added into X.
// X is symmetric, read from and updated in its lower triangle (ld n); R
// (n x n) and Y (n x n, the current term) are scratch.  A (lower, lda) is
// sliced only when slice_A (its slices are kept in ws between steps).
cudaError_t ozaki_refine_step(int64_t n, const double* A, int64_t lda, double* X, double* R, double* Y, void* ws,
                              int levelsR, int order, bool slice_A, int* err, cudaStream_t s, int* launches);

}  // namespace spdinv
