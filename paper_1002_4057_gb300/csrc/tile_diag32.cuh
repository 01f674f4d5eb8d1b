// FP32 factorisation (POTRF) and inversion (TRTRI) of one 32 x 32 diagonal
// tile, column-major in shared memory with leading dimension LD, inside a CTA
// of 128 threads: the diagonal tasks of the mixed-precision tile DAG at tile
// 32.  A block-wide column sweep takes a CTA barrier and a shared-memory
// round trip per column; on the critical path of the tile DAG that latency,
// not the arithmetic, is what counts.  Here one warp keeps the block in
// registers (lane r holds row r) and the column values travel by shuffles:
// no CTA barrier inside the sweep.  sqrtf and the divisions are IEEE
// (correctly rounded); no math function is reproduced.
#pragma once
#include <utility>

#include "ptx.cuh"

namespace spdinv {
namespace diag32 {

// Column C of the register sweeps: a template, so that every index into the
// row held in registers is a compile-time constant.
template <int C>
__device__ __forceinline__ void potrf_col(float (&a)[32], int r, int& fail) {
    const float d = __shfl_sync(0xffffffffu, a[C], C);
    if (fail == 0 && !(d > 0.f)) fail = C + 1;  // uniform: every lane sees the same pivot
    if (fail) return;
    const float l = sqrtf(d);
    const float inv = 1.f / l;
    if (r == C) a[C] = l;
    else if (r > C) a[C] = a[C] * inv;
#pragma unroll
    for (int k = C + 1; k < 32; ++k) {
        const float lk = __shfl_sync(0xffffffffu, a[C], k);  // L(k, C)
        if (r >= k) a[k] -= a[C] * lk;
    }
}
template <int... C>
__device__ __forceinline__ void potrf_cols(float (&a)[32], int r, int& fail, std::integer_sequence<int, C...>) {
    (potrf_col<C>(a, r, fail), ...);
}

template <int J>
__device__ __forceinline__ void trtri_col(float (&x)[32], int r) {
    const float xjj = 1.f / __shfl_sync(0xffffffffu, x[J], J);
    float s = 0.f;
#pragma unroll
    for (int k = J + 1; k < 32; ++k) {
        const float lkj = __shfl_sync(0xffffffffu, x[J], k);  // L(k, J): lane k's column J is not yet replaced
        if (k <= r) s += x[k] * lkj;                           // X(r, k) L(k, J)
    }
    if (r == J) x[J] = xjj;
    else if (r > J) x[J] = -s * xjj;
}
template <int... J>
__device__ __forceinline__ void trtri_cols(float (&x)[32], int r, std::integer_sequence<int, J...>) {
    (trtri_col<31 - J>(x, r), ...);  // last column first
}

// Cholesky of the lower triangle of the 32 x 32 block at T, in place; one
// full warp.  Returns 0 or c+1 for the first column c whose pivot is not > 0.
template <int LD>
__device__ __forceinline__ int warp_potrf32(float* T) {
    const int r = threadIdx.x & 31;
    float a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = (k <= r) ? T[k * LD + r] : 0.f;
    int fail = 0;
    potrf_cols(a, r, fail, std::make_integer_sequence<int, 32>{});
#pragma unroll
    for (int k = 0; k < 32; ++k)
        if (k <= r) T[k * LD + r] = a[k];
    return fail;
}

// Inverse of the lower-triangular 32 x 32 block at T, in place; one full warp.
template <int LD>
__device__ __forceinline__ void warp_trtri32(float* T) {
    const int r = threadIdx.x & 31;
    float x[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = (k <= r) ? T[k * LD + r] : 0.f;
    trtri_cols(x, r, std::make_integer_sequence<int, 32>{});
#pragma unroll
    for (int k = 0; k < 32; ++k)
        if (k <= r) T[k * LD + r] = x[k];
}

}  // namespace diag32

// POTRF of a 32 x 32 FP32 tile (128 threads; called by all): 0 or c+1 for
// the first column c whose pivot is not > 0 (uniform).
template <int LD>
__device__ int diag_potrf32_f32(float* T, int* s_fail) {
    if (threadIdx.x == 0) *s_fail = 0;
    cta_sync();
    if ((threadIdx.x >> 5) == 0) {
        const int f = diag32::warp_potrf32<LD>(T);
        if (threadIdx.x == 0) *s_fail = f;
    }
    cta_sync();
    return *s_fail;
}

// TRTRI of a lower-triangular 32 x 32 FP32 tile (128 threads; called by all).
template <int LD>
__device__ void diag_trtri32_f32(float* T) {
    cta_sync();
    if ((threadIdx.x >> 5) == 0) diag32::warp_trtri32<LD>(T);
    cta_sync();
}

}  // namespace spdinv
