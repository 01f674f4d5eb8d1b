// FP32 tile kernels (device functions) for b x b tiles held column-major in
// shared memory with leading dimension b+1 (the padding keeps the transposed
// accesses free of bank conflicts), run by one CTA of 128 threads arranged
// 16 x 8, each thread owning an (b/16) x (b/8) block of the output.
// Same operations as the FP64 tile kernels (Algorithm 1, Sec. 2), in FP32
// CUDA-core arithmetic (fused multiply-add).
#pragma once
#include "tile_fp64.cuh"

namespace spdinv {

template <int B>
struct Cfg32 {
    static constexpr int LD = B + 1;
    static constexpr int RM = B / 16;  // rows per thread
    static constexpr int CN = B / 8;   // columns per thread
};

template <int B>
struct Acc32 {
    float v[Cfg32<B>::RM][Cfg32<B>::CN];
};

template <int B>
__device__ __forceinline__ void acc_zero(Acc32<B>& a) {
#pragma unroll
    for (int r = 0; r < Cfg32<B>::RM; ++r)
#pragma unroll
        for (int c = 0; c < Cfg32<B>::CN; ++c) a.v[r][c] = 0.f;
}

template <int B>
__device__ __forceinline__ void acc_store(const Acc32<B>& a, float* T) {
    constexpr int RM = Cfg32<B>::RM, CN = Cfg32<B>::CN, LD = Cfg32<B>::LD;
    const int r0 = (threadIdx.x % 16) * RM, c0 = (threadIdx.x / 16) * CN;
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) T[(c0 + c) * LD + r0 + r] = a.v[r][c];
}

template <int B>
__device__ __forceinline__ void acc_load(Acc32<B>& a, const float* T) {
    constexpr int RM = Cfg32<B>::RM, CN = Cfg32<B>::CN, LD = Cfg32<B>::LD;
    const int r0 = (threadIdx.x % 16) * RM, c0 = (threadIdx.x / 16) * CN;
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) a.v[r][c] = T[(c0 + c) * LD + r0 + r];
}

// acc (+|-)= op(P) op(Q), FP32 FMA.  A triangular right operand lets each
// warp skip the k-range that multiplies its zero part; the bounds are
// uniform across the warp (a warp owns all rows and 2*CN columns), so no warp
// diverges.  (A triangular left operand gives no warp-wide skip here.)
template <int B, bool TA, bool TB, bool NEG, int SP, int SQ>
__device__ __forceinline__ void tile_mma(Acc32<B>& acc, const float* P, const float* Q) {
    constexpr int RM = Cfg32<B>::RM, CN = Cfg32<B>::CN, LD = Cfg32<B>::LD;
    const int r0 = (threadIdx.x % 16) * RM, c0 = (threadIdx.x / 16) * CN;
    const int cw = (threadIdx.x / 32) * 2 * CN;  // the warp's first column
    int kb = 0, ke = B;
    if (SQ == LOWER) {
        if (TB) ke = cw + 2 * CN; else kb = cw;
    }
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        float a[RM], b[CN];
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const float v = TA ? P[(r0 + r) * LD + k] : P[k * LD + r0 + r];
            a[r] = NEG ? -v : v;
        }
#pragma unroll
        for (int c = 0; c < CN; ++c) b[c] = TB ? Q[k * LD + c0 + c] : Q[(c0 + c) * LD + k];
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
            for (int c = 0; c < CN; ++c) acc.v[r][c] = fmaf(a[r], b[c], acc.v[r][c]);
    }
}

template <int B>
__device__ __forceinline__ void tile_zero_upper(float* T) {
    constexpr int LD = Cfg32<B>::LD;
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        if (r < c) T[c * LD + r] = 0.f;
    }
}

// Unblocked Cholesky of one FP32 tile (same sweep as the FP64 version).
template <int B>
__device__ int tile_potrf(float* T, int* s_fail) {
    constexpr int LD = Cfg32<B>::LD, RS = kThreads / B > 0 ? kThreads / B : 1;
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    const bool active = threadIdx.x < RS * B;
    if (threadIdx.x == 0) *s_fail = 0;
    cta_sync();
    for (int c = 0; c < B; ++c) {
        if (threadIdx.x == 0) {
            const float d = T[c * LD + c];
            if (d > 0.f) T[c * LD + c] = sqrtf(d);
            else *s_fail = c + 1;
        }
        cta_sync();
        if (*s_fail) return *s_fail;
        const float l = T[c * LD + c];
        if (active && cs == 0 && r > c) T[c * LD + r] = T[c * LD + r] / l;
        cta_sync();
        if (active && r > c) {
            const float lr = T[c * LD + r];
            for (int k = c + 1 + cs; k <= r; k += RS) T[k * LD + r] -= lr * T[c * LD + k];
        }
        cta_sync();
    }
    return 0;
}

// Inverse of one lower-triangular FP32 tile (trti2 column sweep).
// tmp: kThreads floats.
template <int B>
__device__ void tile_trtri(float* T, float* tmp) {
    constexpr int LD = Cfg32<B>::LD, RS = kThreads / B > 0 ? kThreads / B : 1;
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    const bool active = threadIdx.x < RS * B;
    cta_sync();
    for (int j = B - 1; j >= 0; --j) {
        const float xjj = 1.f / T[j * LD + j];
        float s = 0.f;
        if (active && r > j)
            for (int k = j + 1 + cs; k <= r; k += RS) s += T[k * LD + r] * T[j * LD + k];
        if (active && RS > 1) tmp[cs * B + r] = s;
        cta_sync();
        if (active && cs == 0 && r > j) {
            float tot = s;
            for (int u = 1; u < RS; ++u) tot += tmp[u * B + r];
            T[j * LD + r] = -tot * xjj;
        }
        cta_sync();
        if (threadIdx.x == 0) T[j * LD + j] = xjj;
        cta_sync();
    }
}

}  // namespace spdinv
