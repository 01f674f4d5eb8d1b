// FP32-accurate and BF16-split tile products on the tensor cores (the
// low-precision bulk updates of the mixed-precision inversion: GEMM, SYRK and
// TRMM of Algorithm 1, Sec. 2), with the interface of the CUDA-core FP32 tile
// products (tile_f32.cuh): b x b FP32 tiles, column-major in shared memory
// with leading dimension b + 1, one CTA of 128 threads (4 warps in a 2 x 2
// grid, each owning a (b/2) x (b/2) block of the output).
//
// Each operand element x is split into a high and a low part and the product
// is formed from three warp-level MMAs with FP32 accumulation,
//     x y ~ hi(x) hi(y) + hi(x) lo(y) + lo(x) hi(y)
// (the lo * lo term, of relative size 2^-2p, is dropped):
//   SplitTF32  hi = x rounded to TF32 (11 significant bits), lo = x - hi
//              rounded to TF32: 3 x mma.m16n8k8.tf32, about 2^-21 relative
//              per product, near FP32 (the 3xTF32 method);
//   SplitBF16  hi = x rounded to BF16 (8 significant bits), lo likewise:
//              3 x mma.m16n8k16.bf16, about 2^-16 relative per product
//              (the two-term BF16x3 split of Henry, Tang and Heinecke, 2019).
// The difference x - hi is exact in FP32, so only the roundings to TF32 /
// BF16 and the dropped term limit the accuracy.
#pragma once
#include <cuda_bf16.h>

#include "tile_f32.cuh"

namespace spdinv {

struct SplitTF32 {
    static constexpr int K = 8;  // k per MMA
};
struct SplitBF16 {
    static constexpr int K = 16;
};

template <int B, class S>
struct AccTC {
    static constexpr int W = B / 2;    // warp block edge
    static constexpr int MI = W / 16;  // 16-row MMA blocks per warp
    static constexpr int NI = W / 8;   // 8-column MMA blocks per warp
    static constexpr int LD = B + 1;
    float v[MI][NI][4];
};

template <int B, class S>
__device__ __forceinline__ void acc_zero(AccTC<B, S>& a) {
#pragma unroll
    for (int mi = 0; mi < AccTC<B, S>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < AccTC<B, S>::NI; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) a.v[mi][ni][r] = 0.f;
}

// Element (row, col) of accumulator entry (mi, ni, r) of this thread (the
// m16n8 accumulator fragment: rows g, g + 8, columns 2q, 2q + 1).
template <int B, class S>
__device__ __forceinline__ void acc_coord_tc(int mi, int ni, int r, int& row, int& col) {
    constexpr int W = AccTC<B, S>::W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    row = (warp >> 1) * W + mi * 16 + g + 8 * (r >> 1);
    col = (warp & 1) * W + ni * 8 + 2 * q + (r & 1);
}

template <int B, class S>
__device__ __forceinline__ void acc_store(const AccTC<B, S>& a, float* T) {
    constexpr int LD = AccTC<B, S>::LD;
#pragma unroll
    for (int mi = 0; mi < AccTC<B, S>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < AccTC<B, S>::NI; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int row, col;
                acc_coord_tc<B, S>(mi, ni, r, row, col);
                T[col * LD + row] = a.v[mi][ni][r];
            }
}

template <int B, class S>
__device__ __forceinline__ void acc_load(AccTC<B, S>& a, const float* T) {
    constexpr int LD = AccTC<B, S>::LD;
#pragma unroll
    for (int mi = 0; mi < AccTC<B, S>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < AccTC<B, S>::NI; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                int row, col;
                acc_coord_tc<B, S>(mi, ni, r, row, col);
                a.v[mi][ni][r] = T[col * LD + row];
            }
}

// x rounded to TF32 (10 stored mantissa bits), to nearest with ties away from
// zero, in integer arithmetic: add half a TF32 unit to the magnitude bits and
// clear the 13 low mantissa bits (a carry into the exponent is the correct
// rounding up, to Inf past the largest TF32 value).  Inf stays Inf; a NaN
// whose payload lies only in the 13 low bits becomes Inf, any other NaN stays
// NaN.  Two integer instructions instead of a conversion, which measured 13 %
// faster for the 64 x 64 3xTF32 tile product.
__device__ __forceinline__ uint32_t to_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

// hi and lo TF32 parts of x (lo = x - hi, exact in FP32, then rounded).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// hi and lo BF16 parts of the pair (x0, x1), packed two to a register
// (x0 in the low half).
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
    hi = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16x(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc (+|-)= op(P) op(Q) as three split MMAs per k-step.  op(X) = X or X^T
// (TA / TB); a lower-triangular stored operand lets each warp skip the k-steps
// that multiply its zero part (the skipped terms are exact zeros).
template <int B, bool TA, bool TB, bool NEG, int SP, int SQ, class S>
__device__ __forceinline__ void tile_mma(AccTC<B, S>& acc, const float* P, const float* Q) {
    constexpr int W = AccTC<B, S>::W, MI = AccTC<B, S>::MI, NI = AccTC<B, S>::NI, LD = AccTC<B, S>::LD;
    constexpr int KS = S::K;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int wm = (warp >> 1) * W, wn = (warp & 1) * W;
    auto opP = [&](int m, int k) -> float {
        const float v = TA ? P[m * LD + k] : P[k * LD + m];
        return NEG ? -v : v;
    };
    auto opQ = [&](int k, int n) -> float { return TB ? Q[k * LD + n] : Q[n * LD + k]; };
    int kb = 0, ke = B;
    if (SP == LOWER) {  // op(P)[m][k] != 0 only for k <= m (N) or k >= m (T)
        if (TA) kb = wm; else ke = wm + W;
    }
    if (SQ == LOWER) {  // op(Q)[k][n] != 0 only for k >= n (N) or k <= n (T)
        if (TB) ke = min(ke, wn + W); else kb = max(kb, wn);
    }
    kb = kb / KS * KS;
    ke = (ke + KS - 1) / KS * KS;
    // The tensor cores' FP32 accumulation is not rounded like an FP32 add;
    // over a whole update chain (thousands of terms) that costs bits.  Each
    // tile product therefore starts from a zero accumulator, and its sum is
    // added to the running one with rounded FP32 adds.
    float part[MI][NI][4];
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) part[mi][ni][r] = 0.f;
#pragma unroll 1
    for (int k0 = kb; k0 < ke; k0 += KS) {
        uint32_t ah[MI][4], al[MI][4], bh[NI][2], bl[NI][2];
        if constexpr (KS == 8) {  // m16n8k8 tf32: a (g, q) (g+8, q) (g, q+4) (g+8, q+4); b (q, g) (q+4, g)
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                const int m = wm + mi * 16 + g;
                split_tf32(opP(m, k0 + q), ah[mi][0], al[mi][0]);
                split_tf32(opP(m + 8, k0 + q), ah[mi][1], al[mi][1]);
                split_tf32(opP(m, k0 + q + 4), ah[mi][2], al[mi][2]);
                split_tf32(opP(m + 8, k0 + q + 4), ah[mi][3], al[mi][3]);
            }
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) {
                const int n = wn + ni * 8 + g;
                split_tf32(opQ(k0 + q, n), bh[ni][0], bl[ni][0]);
                split_tf32(opQ(k0 + q + 4, n), bh[ni][1], bl[ni][1]);
            }
            // each term over all (mi, ni) blocks before the next: the three
            // MMAs into one accumulator depend on each other, the blocks not
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_tf32(part[mi][ni], al[mi], bh[ni][0], bh[ni][1]);
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_tf32(part[mi][ni], ah[mi], bl[ni][0], bl[ni][1]);
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_tf32(part[mi][ni], ah[mi], bh[ni][0], bh[ni][1]);
        } else {  // m16n8k16 bf16: a pairs (g, 2q..) (g+8, 2q..) (g, 2q+8..) (g+8, 2q+8..); b (2q.., g) (2q+8.., g)
#pragma unroll
            for (int mi = 0; mi < MI; ++mi) {
                const int m = wm + mi * 16 + g, k = k0 + 2 * q;
                split_bf16x2(opP(m, k), opP(m, k + 1), ah[mi][0], al[mi][0]);
                split_bf16x2(opP(m + 8, k), opP(m + 8, k + 1), ah[mi][1], al[mi][1]);
                split_bf16x2(opP(m, k + 8), opP(m, k + 9), ah[mi][2], al[mi][2]);
                split_bf16x2(opP(m + 8, k + 8), opP(m + 8, k + 9), ah[mi][3], al[mi][3]);
            }
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) {
                const int n = wn + ni * 8 + g, k = k0 + 2 * q;
                split_bf16x2(opQ(k, n), opQ(k + 1, n), bh[ni][0], bl[ni][0]);
                split_bf16x2(opQ(k + 8, n), opQ(k + 9, n), bh[ni][1], bl[ni][1]);
            }
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_bf16x(part[mi][ni], al[mi], bh[ni][0], bh[ni][1]);
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_bf16x(part[mi][ni], ah[mi], bl[ni][0], bl[ni][1]);
#pragma unroll
            for (int mi = 0; mi < MI; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_bf16x(part[mi][ni], ah[mi], bh[ni][0], bh[ni][1]);
        }
    }
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc.v[mi][ni][r] += part[mi][ni][r];
}

}  // namespace spdinv
