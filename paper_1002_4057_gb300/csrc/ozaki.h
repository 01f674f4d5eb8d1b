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

// The slice products with tcgen05 (residual_tc.cu).
cudaError_t ozaki_products_tc(int64_t n, int64_t npad, const void* Asl, const void* Xsl, int S, const int* ps,
                              const int* pt, int npairs, const int* e, const int* f, double* R, const double* base,
                              double sign, int* err, cudaStream_t s);

// Xn = X + X R on the tensor cores (X symmetric, stored full; R full; all ld
// n): the same exact-slice products with S slices and pairs s + t <= L.
cudaError_t ozaki_correction(int64_t n, const double* X, const double* R, double* Xn, void* ws, int S, int L,
                             int* err, cudaStream_t s, int* launches);

}  // namespace spdinv
