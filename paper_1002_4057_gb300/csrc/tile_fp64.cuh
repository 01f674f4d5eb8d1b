// FP64 tile kernels (device functions) for b x b tiles held column-major in
// shared memory, run by one CTA of 128 threads (4 warps in a 2 x 2 grid, each
// warp owning a (b/2) x (b/2) block of the output).  The products use the
// FP64 tensor-core MMA (m8n8k4); the diagonal-tile factorisation (POTRF) and
// inversion (TRTRI) are column sweeps in shared memory.
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
    static constexpr int W = B / 2;   // warp block edge
    static constexpr int MI = W / 8;  // 8x8 MMA blocks per warp, rows
    static constexpr int NI = W / 8;  // ... columns
};

template <int B>
struct Acc {
    double v[TileCfg<B>::MI][TileCfg<B>::NI][2];
};

template <int B>
__device__ __forceinline__ void acc_zero(Acc<B>& a) {
#pragma unroll
    for (int mi = 0; mi < TileCfg<B>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < TileCfg<B>::NI; ++ni) a.v[mi][ni][0] = a.v[mi][ni][1] = 0.0;
}

// Element (row, col) of the accumulator entry (mi, ni, h) of this thread.
template <int B>
__device__ __forceinline__ void acc_coord(int mi, int ni, int h, int& row, int& col) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    row = (warp >> 1) * TileCfg<B>::W + mi * 8 + (lane >> 2);
    col = (warp & 1) * TileCfg<B>::W + ni * 8 + 2 * (lane & 3) + h;
}

template <int B>
__device__ __forceinline__ void acc_store(const Acc<B>& a, double* T) {
#pragma unroll
    for (int mi = 0; mi < TileCfg<B>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < TileCfg<B>::NI; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int r, c;
                acc_coord<B>(mi, ni, h, r, c);
                T[c * B + r] = a.v[mi][ni][h];
            }
}

template <int B>
__device__ __forceinline__ void acc_load(Acc<B>& a, const double* T) {
#pragma unroll
    for (int mi = 0; mi < TileCfg<B>::MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < TileCfg<B>::NI; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int r, c;
                acc_coord<B>(mi, ni, h, r, c);
                a.v[mi][ni][h] = T[c * B + r];
            }
}

// Shape of a stored operand.
enum TriShape { FULL = 0, LOWER = 1 };

// acc (+|-)= op(P) * op(Q) for b x b column-major tiles P, Q in shared memory,
// op(X) = X (TA/TB false) or X^T (true).  When a stored operand is lower
// triangular, each warp skips the k-range that multiplies its zero part.
template <int B, bool TA, bool TB, bool NEG, int SP, int SQ>
__device__ __forceinline__ void tile_mma(Acc<B>& acc, const double* P, const double* Q) {
    constexpr int W = TileCfg<B>::W, MI = TileCfg<B>::MI, NI = TileCfg<B>::NI;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int wm = (warp >> 1) * W, wn = (warp & 1) * W;
    int kb = 0, ke = B;
    // op(P)[m][k] != 0 only for k <= m (P lower, N) or k >= m (P lower, T)
    if (SP == LOWER) {
        if (TA) kb = wm; else ke = wm + W;
    }
    // op(Q)[k][n] != 0 only for k >= n (Q lower, N) or k <= n (Q lower, T)
    if (SQ == LOWER) {
        if (TB) ke = min(ke, wn + W); else kb = max(kb, wn);
    }
#pragma unroll 2
    for (int k0 = kb; k0 < ke; k0 += 4) {
        const int k = k0 + q;
        double a[MI], b[NI];
#pragma unroll
        for (int mi = 0; mi < MI; ++mi) {
            const int m = wm + mi * 8 + g;
            const double v = TA ? P[m * B + k] : P[k * B + m];
            a[mi] = NEG ? -v : v;
        }
#pragma unroll
        for (int ni = 0; ni < NI; ++ni) {
            const int n = wn + ni * 8 + g;
            b[ni] = TB ? Q[k * B + n] : Q[n * B + k];
        }
#pragma unroll
        for (int mi = 0; mi < MI; ++mi)
#pragma unroll
            for (int ni = 0; ni < NI; ++ni) dmma_m8n8k4(acc.v[mi][ni][0], acc.v[mi][ni][1], a[mi], b[ni]);
    }
}

// Zero the strictly upper part of a b x b tile.
template <int B>
__device__ __forceinline__ void tile_zero_upper(double* T) {
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        if (r < c) T[idx] = 0.0;
    }
}

// Unblocked Cholesky of the lower triangle of a b x b tile, in place
// (right-looking column sweep).  Returns 0, or c+1 for the first local column
// c whose pivot is not > 0 (or is NaN); the tile is then partly updated.
// Must be called by all threads; the return value is uniform.
template <int B>
__device__ int tile_potrf(double* T, int* s_fail) {
    constexpr int RS = kThreads / B;  // threads per row (2 for b=64, 4 for b=32)
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    if (threadIdx.x == 0) *s_fail = 0;
    cta_sync();
    for (int c = 0; c < B; ++c) {
        if (threadIdx.x == 0) {
            const double d = T[c * B + c];
            if (d > 0.0) T[c * B + c] = sqrt(d);
            else *s_fail = c + 1;
        }
        cta_sync();
        if (*s_fail) return *s_fail;
        const double l = T[c * B + c];
        if (cs == 0 && r > c) T[c * B + r] = T[c * B + r] / l;
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
// tmp: b doubles of shared scratch.  The strictly upper part is not touched.
template <int B>
__device__ void tile_trtri(double* T, double* tmp) {
    constexpr int RS = kThreads / B;
    const int r = threadIdx.x % B, cs = threadIdx.x / B;
    cta_sync();
    for (int j = B - 1; j >= 0; --j) {
        const double xjj = 1.0 / T[j * B + j];
        // rows i > j: partial sums over k split among the RS threads of a row
        double s = 0.0;
        if (r > j)
            for (int k = j + 1 + cs; k <= r; k += RS) s += T[k * B + r] * T[j * B + k];
        // combine the RS partial sums (RS consecutive... rows share lanes across warps)
        if (RS > 1) {
            tmp[cs * B + r] = s;
        }
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
