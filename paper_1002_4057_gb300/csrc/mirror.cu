// Fills the strictly upper triangle of column-major matrices from their lower
// triangle (A_ij = A_ji for i < j), so that the lower-triangle result of the
// inversion becomes the full symmetric A^{-1}.  One block per 32 x 32 tile of
// the upper part, transposed through shared memory so both the reads and the
// writes are coalesced.
#include <cuda_runtime.h>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

template <typename T>
__global__ void mirror_lower_kernel(int64_t n, T* A, int64_t lda, int64_t stride) {
    __shared__ T s[32][33];
    const int64_t tj = blockIdx.x, ti = blockIdx.y;  // target tile (ti, tj) with ti < tj
    if (ti > tj) return;
    T* M = A + (int64_t)blockIdx.z * stride;
    // read the source tile (tj, ti) of the lower triangle
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t gr = tj * 32 + threadIdx.x, gc = ti * 32 + r;  // source (row, col)
        if (gr < n && gc < n) s[r][threadIdx.x] = M[gr + gc * lda];
    }
    cta_sync();
    for (int c = threadIdx.y; c < 32; c += blockDim.y) {
        const int64_t gr = ti * 32 + threadIdx.x, gc = tj * 32 + c;  // target (row, col), row < col
        if (gr < n && gc < n && gr < gc) M[gr + gc * lda] = s[threadIdx.x][c];
    }
}

template <typename T>
spdinv_status run_mirror(int batch, int64_t n, T* dA, int64_t lda, int64_t stride, cudaStream_t s) {
    if (batch < 0 || n < 0 || batch > 65535) return SPDINV_ERR_N;
    if (lda < (n > 1 ? n : 1)) return SPDINV_ERR_LDA;
    if (batch == 0 || n == 0) return SPDINV_OK;
    if (!dA) return SPDINV_ERR_NULL;
    const int64_t t = (n + 31) / 32;
    if (t > 65535) return SPDINV_ERR_N;
    mirror_lower_kernel<T><<<dim3((unsigned)t, (unsigned)t, (unsigned)batch), dim3(32, 8), 0, s>>>(n, dA, lda, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return SPDINV_OK;
}

}  // namespace
}  // namespace spdinv

using namespace spdinv;

extern "C" {
SPDINV_API spdinv_status spdinv_mirror_lower(int batch, int64_t n, double* dA, int64_t lda, int64_t stride,
                                             cudaStream_t stream) {
    return log_status("spdinv_mirror_lower", "n", n, run_mirror<double>(batch, n, dA, lda, stride, stream));
}
SPDINV_API spdinv_status spdinv_smirror_lower(int batch, int64_t n, float* dA, int64_t lda, int64_t stride,
                                              cudaStream_t stream) {
    return log_status("spdinv_smirror_lower", "n", n, run_mirror<float>(batch, n, dA, lda, stride, stream));
}
}
