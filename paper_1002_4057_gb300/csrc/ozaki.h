// FP64-accurate residual on the BF16 tensor cores (residual_ozaki.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace spdinv {

// Bytes of workspace ozaki_residual needs for order n and S slices.
size_t ozaki_workspace_bytes(int64_t n, int S);

// R = I - A X (n x n, ld n), A symmetric given by its lower triangle (lda),
// X full (ld n); S slices per operand, slice pairs with s + t <= L.
// Queues its kernels on s and adds their number to *launches.
cudaError_t ozaki_residual(int64_t n, const double* A, int64_t lda, const double* X, double* R, void* ws, int S,
                           int L, cudaStream_t s, int* launches);

}  // namespace spdinv
