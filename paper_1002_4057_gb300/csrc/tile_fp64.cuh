// FP64 tile kernels (device functions) for b x b tiles held column-major in
// shared memory, run by one CTA of 128 threads arranged 8 x 16, each thread
// owning a (b/8) x (b/16) block of the output.  The products are FP64 fused
// multiply-adds on register blocks: on GB300 the FP64 FMA pipe measures
// 1.255 TFLOP/s against 1.10 for the FP64 tensor-core MMA (mma.sync m8n8k4),
// and at about two FP64 FMAs per clock per SM the pipe, not instruction
// issue or shared memory, bounds the product.  The diagonal-tile
// factorisation (POTRF) and inversion (TRTRI) are column sweeps in shared
// memory.
//
// The tile operations are the BLAS/LAPACK kernels of Algorithm 1 (Sec. 2):
//   GEMM / SYRK / TRMM  -> tile_mma with the operands' transposes and
//                          triangular shapes as template parameters
//   POTRF               -> tile_potrf (unblocked Cholesky of one tile)
//   TRTRI               -> tile_trtri (inverse of one lower-triangular tile)
//   LAUUM               -> tile_mma of X_ii^T X_ii (lower part kept)
#pragma once
#include "ptx.cuh"

namespace spdinv {

constexpr int kThreads = 128;

template <int B>
struct TileCfg {
    static_assert(B % 16 == 0, "tiles of 16, 32 or 64");
    static constexpr int RM = B / 8;   // rows per thread (8 thread rows)
    static constexpr int CN = B / 16;  // columns per thread (16 thread columns)
};

template <int B>
struct Acc {
    double v[TileCfg<B>::RM][TileCfg<B>::CN];
};

template <int B>
__device__ __forceinline__ void acc_zero(Acc<B>& a) {
#pragma unroll
    for (int i = 0; i < TileCfg<B>::RM; ++i)
#pragma unroll
        for (int j = 0; j < TileCfg<B>::CN; ++j) a.v[i][j] = 0.0;
}

// Element (row, col) of the accumulator entry (i, j) of this thread.
template <int B>
__device__ __forceinline__ void acc_coord(int i, int j, int& row, int& col) {
    row = (threadIdx.x % 8) * TileCfg<B>::RM + i;
    col = (threadIdx.x / 8) * TileCfg<B>::CN + j;
}

template <int B>
__device__ __forceinline__ void acc_store(const Acc<B>& a, double* T) {
#pragma unroll
    for (int i = 0; i < TileCfg<B>::RM; ++i)
#pragma unroll
        for (int j = 0; j < TileCfg<B>::CN; ++j) {
            int r, c;
            acc_coord<B>(i, j, r, c);
            T[c * B + r] = a.v[i][j];
        }
}

template <int B>
__device__ __forceinline__ void acc_load(Acc<B>& a, const double* T) {
#pragma unroll
    for (int i = 0; i < TileCfg<B>::RM; ++i)
#pragma unroll
        for (int j = 0; j < TileCfg<B>::CN; ++j) {
            int r, c;
            acc_coord<B>(i, j, r, c);
            a.v[i][j] = T[c * B + r];
        }
}

// acc += T (a b x b column-major tile in shared memory), element by element.
template <int B>
__device__ __forceinline__ void acc_add(Acc<B>& a, const double* T) {
#pragma unroll
    for (int i = 0; i < TileCfg<B>::RM; ++i)
#pragma unroll
        for (int j = 0; j < TileCfg<B>::CN; ++j) {
            int r, c;
            acc_coord<B>(i, j, r, c);
            a.v[i][j] += T[c * B + r];
        }
}

// Shape of a stored operand.
enum TriShape { FULL = 0, LOWER = 1 };

// acc (+|-)= op(P) * op(Q) for b x b column-major tiles P, Q in shared memory,
// op(X) = X (TA/TB false) or X^T (true), one FP64 FMA per product term in
// increasing k.  When a stored operand is lower triangular (its upper part
// exactly zero), each thread skips the k-range that multiplies zeros of its
// own rows or columns.
template <int B, bool TA, bool TB, bool NEG, int SP, int SQ>
__device__ __forceinline__ void tile_mma(Acc<B>& acc, const double* P, const double* Q) {
    constexpr int RM = TileCfg<B>::RM, CN = TileCfg<B>::CN;
    const int r0 = (threadIdx.x % 8) * RM, c0 = (threadIdx.x / 8) * CN;
    int kb = 0, ke = B;
    // op(P)[m][k] != 0 only for k <= m (P lower, N) or k >= m (P lower, T)
    if (SP == LOWER) {
        if (TA) kb = r0; else ke = r0 + RM;
    }
    // op(Q)[k][n] != 0 only for k >= n (Q lower, N) or k <= n (Q lower, T)
    if (SQ == LOWER) {
        if (TB) ke = min(ke, c0 + CN); else kb = max(kb, c0);
    }
#pragma unroll 4
    for (int k = kb; k < ke; ++k) {
        double a[RM], b[CN];
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const double v = TA ? P[(r0 + i) * B + k] : P[k * B + r0 + i];
            a[i] = NEG ? -v : v;
        }
#pragma unroll
        for (int j = 0; j < CN; ++j) b[j] = TB ? Q[k * B + c0 + j] : Q[(c0 + j) * B + k];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < CN; ++j) acc.v[i][j] = fma(a[i], b[j], acc.v[i][j]);
    }
}

// Zero the strictly upper part of a b x b tile (NT threads).
template <int B, int NT = kThreads>
__device__ __forceinline__ void tile_zero_upper(double* T) {
    for (int idx = threadIdx.x; idx < B * B; idx += NT) {
        const int r = idx % B, c = idx / B;
        if (r < c) T[idx] = 0.0;
    }
}

// Unblocked Cholesky of the lower triangle of a b x b tile, in place
// (right-looking column sweep; each column is scaled by the reciprocal of its
// pivot, one FP64 division per column instead of one per element).  Returns
// 0, or c+1 for the first local column c whose pivot is not > 0 (or is NaN);
// the tile is then partly updated.
// Must be called by all threads; the return value is uniform.
template <int B, int NT = kThreads>
__device__ int tile_potrf(double* T, int* s_fail) {
    constexpr int RS = NT / B;  // threads per row (2 for b=64, 4 for b=32 with 128 threads)
    static_assert(RS >= 1 && NT % B == 0, "whole rows per thread group");
    __shared__ double s_inv;  // 1 / L_cc of the current column
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    if (threadIdx.x == 0) *s_fail = 0;
    cta_sync();
    for (int c = 0; c < B; ++c) {
        if (threadIdx.x == 0) {
            const double d = T[c * B + c];
            if (d > 0.0) {
                const double l = sqrt(d);
                T[c * B + c] = l;
                s_inv = 1.0 / l;  // one division per column; the column is scaled by products
            } else {
                *s_fail = c + 1;
            }
        }
        cta_sync();
        if (*s_fail) return *s_fail;
        const double inv = s_inv;
        if (cs == 0 && r > c) T[c * B + r] = T[c * B + r] * inv;
        cta_sync();
        if (r > c) {
            const double lr = T[c * B + r];
            for (int k = c + 1 + cs; k <= r; k += RS) T[k * B + r] -= lr * T[c * B + k];
        }
        cta_sync();
    }
    return 0;
}

// Inverse of a lower-triangular, non-singular b x b tile, in place
// (column sweep from the last column, as in LAPACK's unblocked trti2):
//   X_jj = 1/L_jj,  X_ij = -(sum_{k=j+1..i} X_ik L_kj) X_jj   (i > j).
// tmp: NT doubles of shared scratch.  The strictly upper part is not touched.
// The b reciprocals are formed once, in parallel, into tmp[0 .. b-1] (the
// partial sums use tmp[b ..]): an FP64 division is a sequence of FP64-pipe
// instructions, and this chip's FP64 pipe issues two FMAs per clock per SM.
template <int B, int NT = kThreads>
__device__ void tile_trtri(double* T, double* tmp) {
    constexpr int RS = NT / B;
    static_assert(RS >= 1 && NT % B == 0, "whole rows per thread group");
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    cta_sync();
    if (threadIdx.x < B) tmp[threadIdx.x] = 1.0 / T[threadIdx.x * B + threadIdx.x];
    cta_sync();
    for (int j = B - 1; j >= 0; --j) {
        const double xjj = tmp[j];
        // rows i > j: partial sums over k split among the RS threads of a row
        double s = 0.0;
        if (r > j)
            for (int k = j + 1 + cs; k <= r; k += RS) s += T[k * B + r] * T[j * B + k];
        // combine the RS partial sums: thread group cs > 0 leaves its sum in
        // tmp[cs * b + r] (tmp[0 .. b-1] holds the reciprocals)
        if (RS > 1 && cs > 0) tmp[cs * B + r] = s;
        cta_sync();
        if (cs == 0 && r > j) {
            double tot = s;
            for (int u = 1; u < RS; ++u) tot += tmp[u * B + r];
            T[j * B + r] = -tot * xjj;
        }
        cta_sync();
        if (threadIdx.x == 0) T[j * B + j] = xjj;
        // the next column reads T[j*B+j] only through X_ik (k > j'), written
        // above by this thread; the barrier at the top of the next iteration
        // orders it.
        cta_sync();
    }
}

}  // namespace spdinv
