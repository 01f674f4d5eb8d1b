// Mixed-precision inversion (an added form): the tile DAG of Algorithm 1
// (Sec. 2) with renaming and pipelining (Sec. 3) runs with its bulk updates
// (GEMM, SYRK, TRMM) at FP32 accuracy (FP32 FMA, or three TF32 or BF16
// tensor-core products of split operands) and its diagonal-tile POTRF and
// TRTRI in FP32 (warp-level register sweeps for 32-tiles, block-wide sweeps
// for 64-tiles) or, with spdinv_opts.diag_fp64, in native FP64; then `refine_steps` residual corrections of order p bring the
// result back to FP64 accuracy:
//      R = I - A X         (FP64-accurate; A read from its lower triangle)
//      X <- X + X R + X R^2 + ... + X R^{p-1}
// (the hyperpower family of iterations for the inverse; p = 2 is the
// Newton-Schulz step; the new residual is R^p), and the lower triangle of X
// is written into A.  By default every product runs on the BF16 tensor cores
// as a sum of exact slice products (residual_ozaki.cu, residual_tc.cu): R from
// 7 slices per operand, 28 slice pairs in every step but the last and 34 in
// the last one, whose residual error stays in the result; the terms X R^m are
// formed as (X R^{m-1}) R, symmetric, so only their lower tiles, with 15, 10,
// 6, ... pairs as the terms shrink.  SPDINV_RESIDUAL_FP64 (and the mma.sync
// comparison path) forms R with native FP64 MMA (or mma.sync slices) and X R
// in FP32 on the CUDA cores instead, for p = 2 only.
//
// The persistent FP32 kernel follows the FP64 one task for task.  Its
// renamed stores hold FP32 tiles padded to b x (b+1) -- the layout the
// CUDA-core tile products read without bank conflicts -- so that each tile
// still moves as a single bulk (TMA) copy.  Step 3 writes the full symmetric X
// (FP64) into a workspace matrix instead of A, which stays intact for the
// residual.
#include <climits>

#include "api_internal.h"
#include "kernels.h"
#include "ozaki.h"
#include "persist.cuh"
#include "tile_f32.cuh"
#include "tile_tc32.cuh"
#include "tile_diag32.cuh"
#include "tile_fp64.cuh"

namespace spdinv {

struct KParamsMixed {
    int64_t n, lda;
    int t, b, ntasks;
    const double* A;
    float* Bw;
    float* Cw;
    float* Dw;
    double* X;  // full symmetric X, n x n, leading dimension n
    const uint32_t* tasks;
    int* flags;
    int* ctrl;
    long long timeout_ns;
    int drop_task;
};

namespace {

template <int B>
__host__ __device__ constexpr int padded_tile() {
    return B * (B + 1);
}

template <int B>
__device__ __forceinline__ const float* tB(const KParamsMixed& p, int i, int j) {
    return p.Bw + ((int64_t)i * (i - 1) / 2 + j) * (int64_t)padded_tile<B>();
}
template <int B>
__device__ __forceinline__ const float* tC(const KParamsMixed& p, int i, int j) {
    return p.Cw + ((int64_t)i * (i - 1) / 2 + j) * (int64_t)padded_tile<B>();
}
template <int B>
__device__ __forceinline__ const float* tD(const KParamsMixed& p, int j) {
    return p.Dw + (int64_t)j * padded_tile<B>();
}

// Tile of A (FP64) into an FP32 shared tile (LD = B+1), padded.
template <int B>
__device__ void load_A32(const KParamsMixed& p, int ti, int tj, float* T, bool lower_only) {
    constexpr int LD = B + 1;
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + c;
        float v;
        if (gr < p.n && gc < p.n) v = (lower_only && r < c) ? 0.f : (float)p.A[gr + gc * p.lda];
        else v = (ti == tj && r == c) ? 1.f : 0.f;
        T[c * LD + r] = v;
    }
}

template <int B>
__device__ void store_ws32(float* g, const float* T) {
    const float4* s = reinterpret_cast<const float4*>(T);
    float4* d = reinterpret_cast<float4*>(g);
    for (int idx = threadIdx.x; idx < padded_tile<B>() / 4; idx += kThreads) d[idx] = s[idx];
}

// Tile (ti, tj) of X (and, mirrored, (tj, ti)); diagonal tiles are written
// from their lower part on both sides, so X is exactly symmetric.
template <int B>
__device__ void store_X(const KParamsMixed& p, int ti, int tj, const float* T) {
    constexpr int LD = B + 1;
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + c;
        if (gr >= p.n || gc >= p.n) continue;
        if (ti == tj) {
            const float v = r >= c ? T[c * LD + r] : T[r * LD + c];
            p.X[gr + gc * p.n] = (double)v;
        } else {
            p.X[gr + gc * p.n] = (double)T[c * LD + r];
        }
    }
    if (ti != tj) {
        for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
            const int r = idx % B, c = idx / B;  // target (tj*B + r, ti*B + c)
            const int64_t gr = (int64_t)tj * B + r, gc = (int64_t)ti * B + c;
            if (gr < p.n && gc < p.n) p.X[gr + gc * p.n] = (double)T[r * LD + c];
        }
    }
}

// ACC: the bulk tile products' accumulator, which selects their arithmetic --
// Acc32<B> FP32 FMA on the CUDA cores, AccTC<B, SplitTF32> three TF32 MMAs
// (3xTF32), AccTC<B, SplitBF16> three BF16 MMAs (BF16x3).
//
// Shared memory: two sets of two tile buffers for the double-buffered update
// chains (run_chain); the Step-1 diagonal task's scratch (the FP32 TRTRI's, or
// the FP64 copy of the tile and its TRTRI scratch) reuses the second set once
// that task's chain is done, and extends past it where the FP64 copy needs.
template <int B>
__host__ __device__ constexpr int mixed_tile_bytes() {
    return round_up128(padded_tile<B>() * (int)sizeof(float));
}
template <int B>
__host__ __device__ constexpr int mixed_diag64_bytes() {
    return (B * B + kThreads) * (int)sizeof(double);
}
template <int B, bool DIAG64>
__host__ __device__ constexpr int mixed_smem_bytes() {
    return 2 * mixed_tile_bytes<B>() + (DIAG64 && mixed_diag64_bytes<B>() > 2 * mixed_tile_bytes<B>()
                                            ? mixed_diag64_bytes<B>()
                                            : 2 * mixed_tile_bytes<B>());
}

template <int B, class ACC, bool DIAG64>
__global__ void __launch_bounds__(kThreads) potri_mixed_persistent(const KParamsMixed prm) {
    unsigned char* const smem_raw = dynamic_smem();
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_task, s_fail, s_state[3];
    constexpr int LD = B + 1;
    constexpr uint32_t kBytes = (uint32_t)(padded_tile<B>() * sizeof(float));
    const KParamsMixed& p = prm;
    constexpr int kT = mixed_tile_bytes<B>();
    float* const T0 = reinterpret_cast<float*>(smem_raw);  // set 0: T0, T1; set 1: T2, T3
    float* const T1 = reinterpret_cast<float*>(smem_raw + kT);
    float* const T2 = reinterpret_cast<float*>(smem_raw + 2 * kT);
    float* const T3 = reinterpret_cast<float*>(smem_raw + 3 * kT);
    float* const tmpf = reinterpret_cast<float*>(smem_raw + 2 * kT);  // TRTRI scratch, kThreads floats (set 1)
    double* const Td = reinterpret_cast<double*>(smem_raw + 2 * kT);  // FP64 diagonal tile, stride B (set 1 on)
    double* const tmpd = Td + B * B;                                   // its TRTRI scratch, kThreads doubles
    PCtx c;
    c.T0 = T0;
    c.T1 = T1;
    c.bar = nullptr;
    c.s_flag = nullptr;
    c.phase = 0;
    c.ctrl = p.ctrl;
    c.timeout_ns = p.timeout_ns;
    c.drop_task = p.drop_task;
    c.wait_ns = nullptr;
    Chain2 ch;
    ch.base = smem_raw;
    ch.stride = (uint32_t)kT;
    ch.bar = bars;
    ch.phase = 0;
    ch.s_state = s_state;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_proxy_async_shared();
    }
    cta_sync();
    if (!layout_ok(T0, T2, p.Bw, p.Cw, p.Dw, p.ctrl)) return;
    if (!layout_ok(T1, T3, p.Bw, p.Cw, p.Dw, p.ctrl)) return;
    const int t = p.t;
    int* const fL = p.flags;
    int* const fX = p.flags + (int64_t)t * t;
    int* const fD = p.flags + 2 * (int64_t)t * t;
    auto el = [](const int* f0, const int* f1, const float* g0, const float* g1) {
        return ChainElem{f0, f1, g0, g1};
    };

    for (;;) {
        const int ticket = next_ticket(p.ctrl, p.ntasks, &s_task);
        if (ticket < 0) return;
        const uint32_t e = p.tasks[ticket];
        const int kind = (int)task_kind(e), i = (int)task_i(e), j = (int)task_j(e);
        ACC acc;

        if (kind == K_S1_DIAG) {
            load_A32<B>(p, j, j, T0, true);
            cta_sync();
            acc_load<B>(acc, T0);
            if (j > 0 &&
                !run_chain(ch, c, j, kBytes, [&](int k) { return el(&fL[j * t + k], nullptr, tB<B>(p, j, k), nullptr); },
                           [&](int, const void* Ta, const void*) {  // SYRK chain (FP32)
                               const float* A = static_cast<const float*>(Ta);
                               tile_mma<B, false, true, true, FULL, FULL>(acc, A, A);
                           }))
                return;
            cta_sync();
            acc_store<B>(acc, T0);
            if constexpr (DIAG64) {  // FP64 block-wide sweeps (tile_fp64.cuh) on an FP64 copy of the tile
                cta_sync();
                for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
                    const int r = idx % B, cc = idx / B;
                    Td[idx] = r >= cc ? (double)T0[cc * LD + r] : 0.0;
                }
                const int fail = tile_potrf<B>(Td, &s_fail);
                if (fail) {
                    if (threadIdx.x == 0) record_info(p.ctrl, j * B + fail);
                    return;
                }
                tile_zero_upper<B>(Td);
                tile_trtri<B>(Td, tmpd);
                for (int idx = threadIdx.x; idx < padded_tile<B>(); idx += kThreads) {  // X_jj back to FP32
                    const int r = idx % LD, cc = idx / LD;
                    T0[idx] = (r < B && r >= cc) ? (float)Td[cc * B + r] : 0.f;
                }
                cta_sync();
            } else if constexpr (B == 32) {  // warp-level FP32 sweeps in registers (tile_diag32.cuh)
                const int fail = diag_potrf32_f32<LD>(T0, &s_fail);
                if (fail) {
                    if (threadIdx.x == 0) record_info(p.ctrl, j * B + fail);
                    return;
                }
                for (int idx = threadIdx.x; idx < padded_tile<B>(); idx += kThreads) {  // upper part, pad row
                    const int r = idx % LD, cc = idx / LD;
                    if (r < cc || r == B) T0[idx] = 0.f;
                }
                diag_trtri32_f32<LD>(T0);
            } else {  // FP32 block-wide column sweeps (tile_f32.cuh)
                const int fail = tile_potrf<B>(T0, &s_fail);
                if (fail) {
                    if (threadIdx.x == 0) record_info(p.ctrl, j * B + fail);
                    return;
                }
                for (int idx = threadIdx.x; idx < padded_tile<B>(); idx += kThreads) {  // upper part, pad row
                    const int r = idx % LD, cc = idx / LD;
                    if (r < cc || r == B) T0[idx] = 0.f;
                }
                tile_trtri<B>(T0, tmpf);
                cta_sync();
            }
            store_ws32<B>(const_cast<float*>(tD<B>(p, j)), T0);
            publish(c, &fD[j], ticket);
        } else if (kind == K_S1_OFF) {
            load_A32<B>(p, i, j, T0, false);
            cta_sync();
            acc_load<B>(acc, T0);
            // GEMM chain k < j, then the TRSM as a product with X_jj^T
            if (!run_chain(
                    ch, c, j + 1, kBytes,
                    [&](int k) {
                        return k < j ? el(&fL[i * t + k], &fL[j * t + k], tB<B>(p, i, k), tB<B>(p, j, k))
                                     : el(&fD[j], nullptr, nullptr, tD<B>(p, j));
                    },
                    [&](int k, const void* Ta, const void* Tb) {
                        float* P = static_cast<float*>(const_cast<void*>(Ta));
                        const float* Q = static_cast<const float*>(Tb);
                        if (k < j) {
                            tile_mma<B, false, true, true, FULL, FULL>(acc, P, Q);
                        } else {
                            acc_store<B>(acc, P);  // P's slot received no copy for this element
                            cta_sync();
                            acc_zero<B>(acc);
                            tile_mma<B, false, true, false, FULL, LOWER>(acc, P, Q);
                        }
                    }))
                return;
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            store_ws32<B>(const_cast<float*>(tB<B>(p, i, j)), T0);
            publish(c, &fL[i * t + j], ticket);
        } else if (kind == K_S2_OFF) {
            acc_zero<B>(acc);
            const int m = i - j + 1;  // TRMM by X_ii, GEMMs k = i-1 .. j+1, TRMM by -X_jj
            if (!run_chain(
                    ch, c, m, kBytes,
                    [&](int q) {
                        if (q == 0) return el(&fD[i], &fL[i * t + j], tD<B>(p, i), tB<B>(p, i, j));
                        if (q == m - 1) return el(&fD[j], nullptr, nullptr, tD<B>(p, j));
                        const int k = i - q;
                        return el(&fX[i * t + k], &fL[k * t + j], tC<B>(p, i, k), tB<B>(p, k, j));
                    },
                    [&](int q, const void* Ta, const void* Tb) {
                        float* P = static_cast<float*>(const_cast<void*>(Ta));
                        const float* Q = static_cast<const float*>(Tb);
                        if (q == 0) {
                            tile_mma<B, false, false, false, LOWER, FULL>(acc, P, Q);
                        } else if (q < m - 1) {
                            tile_mma<B, false, false, false, FULL, FULL>(acc, P, Q);
                        }
                        if (q == m - 1) {
                            acc_store<B>(acc, P);  // P's slot received no copy for this element
                            cta_sync();
                            acc_zero<B>(acc);
                            tile_mma<B, false, false, true, FULL, LOWER>(acc, P, Q);
                        }
                    }))
                return;
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            store_ws32<B>(const_cast<float*>(tC<B>(p, i, j)), T0);
            publish(c, &fX[i * t + j], ticket);
        } else if (kind == K_S3_OFF) {
            acc_zero<B>(acc);
            if (!run_chain(
                    ch, c, t - i, kBytes,
                    [&](int q) {
                        if (q == 0) return el(&fD[i], &fX[i * t + j], tD<B>(p, i), tC<B>(p, i, j));
                        const int k = i + q;
                        return el(&fX[k * t + i], &fX[k * t + j], tC<B>(p, k, i), tC<B>(p, k, j));
                    },
                    [&](int q, const void* Ta, const void* Tb) {
                        const float* P = static_cast<const float*>(Ta);
                        const float* Q = static_cast<const float*>(Tb);
                        if (q == 0) tile_mma<B, true, false, false, LOWER, FULL>(acc, P, Q);
                        else tile_mma<B, true, false, false, FULL, FULL>(acc, P, Q);
                    }))
                return;
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            store_X<B>(p, i, j, T0);
        } else if (kind == K_S3_DIAG) {
            acc_zero<B>(acc);
            if (!run_chain(
                    ch, c, t - i, kBytes,
                    [&](int q) {
                        if (q == 0) return el(&fD[i], nullptr, tD<B>(p, i), nullptr);
                        return el(&fX[(i + q) * t + i], nullptr, tC<B>(p, i + q, i), nullptr);
                    },
                    [&](int q, const void* Ta, const void*) {
                        const float* P = static_cast<const float*>(Ta);
                        if (q == 0) tile_mma<B, true, false, false, LOWER, LOWER>(acc, P, P);
                        else tile_mma<B, true, false, false, FULL, FULL>(acc, P, P);
                    }))
                return;
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            store_X<B>(p, i, i, T0);
        }
    }
}

}  // namespace

constexpr int RB = 64;  // output tile of the refinement products

__device__ __forceinline__ bool aborted(const int* ctrl) { return ctrl[2] != 0 || ctrl[3] != 0; }

// R = I - A X with A symmetric, read from its lower triangle; FP64 MMA.
__global__ void __launch_bounds__(kThreads) residual_kernel(int64_t n, const double* A, int64_t lda,
                                                            const double* X, double* R, const int* ctrl) {
    unsigned char* const smem_raw = dynamic_smem();
    if (aborted(ctrl)) return;
    double* S0 = reinterpret_cast<double*>(smem_raw);
    double* S1 = S0 + RB * RB;
    const int t = (int)((n + RB - 1) / RB);
    const int ti = blockIdx.x % t, tj = blockIdx.x / t;
    Acc<RB> acc;
    acc_zero<RB>(acc);
    for (int kt = 0; kt < t; ++kt) {
        cta_sync();
        for (int idx = threadIdx.x; idx < RB * RB; idx += kThreads) {
            const int r = idx % RB, c = idx / RB;
            // A tile (ti, kt): below/on the diagonal read directly, above it
            // read the mirrored lower tile (kt, ti), coalesced, and transpose.
            if (ti >= kt) {
                const int64_t gr = (int64_t)ti * RB + r, gc = (int64_t)kt * RB + c;
                double v = 0.0;
                if (gr < n && gc < n) v = gr >= gc ? A[gr + gc * lda] : A[gc + gr * lda];
                S0[c * RB + r] = v;
            } else {
                const int64_t gr = (int64_t)kt * RB + r, gc = (int64_t)ti * RB + c;  // lower element
                S0[r * RB + c] = (gr < n && gc < n) ? A[gr + gc * lda] : 0.0;
            }
            const int64_t xr = (int64_t)kt * RB + r, xc = (int64_t)tj * RB + c;
            S1[c * RB + r] = (xr < n && xc < n) ? X[xr + xc * n] : 0.0;
        }
        cta_sync();
        tile_mma<RB, false, false, false, FULL, FULL>(acc, S0, S1);
    }
#pragma unroll
    for (int a = 0; a < TileCfg<RB>::RM; ++a)
#pragma unroll
        for (int b = 0; b < TileCfg<RB>::CN; ++b) {
            int r, cc;
            acc_coord<RB>(a, b, r, cc);
            const int64_t gr = (int64_t)ti * RB + r, gc = (int64_t)tj * RB + cc;
            if (gr < n && gc < n) R[gr + gc * n] = (gr == gc ? 1.0 : 0.0) - acc.v[a][b];
        }
}

// Xn = X + X R, the product in FP32 (R is small), the sum in FP64.
__global__ void __launch_bounds__(kThreads) correct_kernel(int64_t n, const double* X, const double* R, double* Xn,
                                                           const int* ctrl) {
    unsigned char* const smem_raw = dynamic_smem();
    if (aborted(ctrl)) return;
    constexpr int LD = RB + 1;
    float* S0 = reinterpret_cast<float*>(smem_raw);
    float* S1 = S0 + RB * LD;
    const int t = (int)((n + RB - 1) / RB);
    const int ti = blockIdx.x % t, tj = blockIdx.x / t;
    Acc32<RB> acc;
    acc_zero<RB>(acc);
    for (int kt = 0; kt < t; ++kt) {
        cta_sync();
        for (int idx = threadIdx.x; idx < RB * RB; idx += kThreads) {
            const int r = idx % RB, c = idx / RB;
            const int64_t ar = (int64_t)ti * RB + r, ac = (int64_t)kt * RB + c;
            S0[c * LD + r] = (ar < n && ac < n) ? (float)X[ar + ac * n] : 0.f;
            const int64_t br = (int64_t)kt * RB + r, bc = (int64_t)tj * RB + c;
            S1[c * LD + r] = (br < n && bc < n) ? (float)R[br + bc * n] : 0.f;
        }
        cta_sync();
        tile_mma<RB, false, false, false, FULL, FULL>(acc, S0, S1);
    }
    cta_sync();
    acc_store<RB>(acc, S0);
    cta_sync();
    for (int idx = threadIdx.x; idx < RB * RB; idx += kThreads) {
        const int r = idx % RB, c = idx / RB;
        const int64_t gr = (int64_t)ti * RB + r, gc = (int64_t)tj * RB + c;
        if (gr < n && gc < n) Xn[gr + gc * n] = X[gr + gc * n] + (double)S0[c * LD + r];
    }
}

namespace {

// Lower triangle of X (ld n) into A (ld lda).
__global__ void store_lower_kernel(int64_t n, const double* X, double* A, int64_t lda, const int* ctrl) {
    if (aborted(ctrl)) return;
    const int64_t j = blockIdx.x;
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) A[i + j * lda] = X[i + j * n];
}

__global__ void finalize_info_mixed(const int* ctrl, int* d_info) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_info = ctrl[2] != 0 ? ctrl[2] : ctrl[3];
}

template <int B, class ACC, bool DIAG64>
cudaError_t launch_mixed_dag_t(const KParamsMixed& p, int ctas_per_sm, int num_sms, cudaStream_t s) {
    auto kern = potri_mixed_persistent<B, ACC, DIAG64>;
    const int sm = mixed_smem_bytes<B, DIAG64>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int per = ctas_per_sm > 0 ? ctas_per_sm : occ;
    per = per < occ ? per : occ;
    int grid = num_sms * per;
    if (grid > p.ntasks) grid = p.ntasks;
    kern<<<grid, kThreads, sm, s>>>(p);
    return cudaGetLastError();
}

template <int B, class ACC>
cudaError_t launch_mixed_dag(const KParamsMixed& p, bool diag64, int ctas_per_sm, int num_sms, cudaStream_t s) {
    return diag64 ? launch_mixed_dag_t<B, ACC, true>(p, ctas_per_sm, num_sms, s)
                  : launch_mixed_dag_t<B, ACC, false>(p, ctas_per_sm, num_sms, s);
}

}  // namespace

// 7 slices of 8 bits cover the 53-bit significands.  Products of slice
// levels s + t <= 6 (28 pairs) leave an error small enough for every step
// but the last, whose residual error stays in the result: it keeps the
// levels up to 7 (34 pairs), which matches the native FP64 residual.
constexpr int kSlices = 7, kLevels = 6, kLevelsLast = 7;

spdinv_status mixed_layout(int64_t n, const spdinv_opts* o, MixedLayout* out) {
    if (n < 0) return SPDINV_ERR_N;
    if (!o || (o->precision != SPDINV_PREC_MIXED_FP32 && o->precision != SPDINV_PREC_MIXED_BF16X3 &&
               o->precision != SPDINV_PREC_MIXED_TF32X3))
        return SPDINV_ERR_UNSUPPORTED;
    if (o->variant != 0) return SPDINV_ERR_UNSUPPORTED;  // the execution variants are FP64 only
    if (o->diag_fp64 != 0 && o->diag_fp64 != 1) return SPDINV_ERR_UNSUPPORTED;
    // default tile: 32 up to n = 8192, 64 above.  The diagonal tasks lie on the
    // critical path, and a 32-tile's sweeps cost 8x less (measured with FP64
    // sweeps: 9.2 against 13.0 ms at n = 4096); at n = 16384 the 64-tile DAG
    // has the shorter run (110 against 155 ms, FP64 sweeps).
    const int b = o->tile > 0 ? o->tile : (n <= 8192 ? 32 : 64);
    if (b != 32 && b != 64) return SPDINV_ERR_UNSUPPORTED;
    if (o->refine_steps < 0 || o->refine_steps > 16) return SPDINV_ERR_UNSUPPORTED;
    const int order = o->refine_order == 0 ? 2 : o->refine_order;
    if (order < 2 || order > 8) return SPDINV_ERR_UNSUPPORTED;
    if (order > 2 && o->residual != SPDINV_RESIDUAL_EMULATED) return SPDINV_ERR_UNSUPPORTED;
    if (o->residual != SPDINV_RESIDUAL_EMULATED && o->residual != SPDINV_RESIDUAL_EMULATED_MMA_SYNC &&
        o->residual != SPDINV_RESIDUAL_FP64)
        return SPDINV_ERR_UNSUPPORTED;
    const int64_t t64 = (n + b - 1) / b;
    if (t64 > 16383) return SPDINV_ERR_N;
    MixedLayout L;
    L.b = b;
    L.t = (int)t64;
    L.order = order;
    if (n > 0) {
        auto align = [](size_t v) { return (v + 255) / 256 * 256; };
        const size_t tileb = (size_t)b * (b + 1) * sizeof(float);
        const size_t ntri = (size_t)L.t * (L.t - 1) / 2;
        L.ctrl = align(sizeof(int) * (4 + 2 * (size_t)L.t * L.t + L.t));
        L.BC = align(ntri * tileb);
        L.D = align((size_t)L.t * tileb);
        L.nn = align((size_t)n * n * sizeof(double));
        const int steps = o->refine_steps;
        const bool emulated =
            o->residual == SPDINV_RESIDUAL_EMULATED || o->residual == SPDINV_RESIDUAL_EMULATED_MMA_SYNC;
        const bool chain = o->residual == SPDINV_RESIDUAL_EMULATED;
        L.oz = (steps > 0 && emulated)
                   ? align(chain ? ozaki_refine_workspace_bytes(n) : ozaki_workspace_bytes(n, kSlices))
                   : 0;
        L.total = L.ctrl + 2 * L.BC + L.D + L.nn * (steps > 0 ? 3 : 1) + L.oz;
    }
    *out = L;
    return SPDINV_OK;
}

spdinv_status residual_workspace(int64_t n, int residual, size_t* bytes) {
    if (n < 0) return SPDINV_ERR_N;
    const bool emulated = residual == SPDINV_RESIDUAL_EMULATED || residual == SPDINV_RESIDUAL_EMULATED_MMA_SYNC;
    if (!emulated && residual != SPDINV_RESIDUAL_FP64) return SPDINV_ERR_UNSUPPORTED;
    // status words (zero: no abort) + the slices
    *bytes = n == 0 ? 0 : 256 + (emulated ? ozaki_workspace_bytes(n, kSlices) : 0);
    return SPDINV_OK;
}

spdinv_status run_mixed(int64_t n, double* dA, int64_t lda, const spdinv_opts* o, int* d_info,
                        cudaStream_t stream) {
    if (n < 0) return SPDINV_ERR_N;
    if (lda < (n > 1 ? n : 1)) return SPDINV_ERR_LDA;
    if (n > 0 && dA == nullptr) return SPDINV_ERR_NULL;
    MixedLayout W;
    const spdinv_status ls = mixed_layout(n, o, &W);
    if (ls != SPDINV_OK) return ls;
    if (n == 0) {
        if (d_info) {
            cudaError_t e = cudaMemsetAsync(d_info, 0, sizeof(int), stream);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        return SPDINV_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    DeviceState& ds = device_state(dev);
    std::lock_guard<std::mutex> lk(ds.mu);
    const int t = W.t, b = W.b, order = W.order;
    const size_t ctrl_bytes = W.ctrl, bytesBC = W.BC, bytesD = W.D, nn = W.nn, oz = W.oz;
    const int steps = o->refine_steps;
    const bool emulated = o->residual == SPDINV_RESIDUAL_EMULATED || o->residual == SPDINV_RESIDUAL_EMULATED_MMA_SYNC;
    const bool chain = o->residual == SPDINV_RESIDUAL_EMULATED;  // order-p step on tcgen05
    void* wsp = nullptr;
    const spdinv_status ws = ds.acquire(W.total, &wsp);
    if (ws != SPDINV_OK) return ws;
    char* base = static_cast<char*>(wsp);
    KParamsMixed p{};
    p.n = n;
    p.lda = lda;
    p.t = t;
    p.b = b;
    p.A = dA;
    p.ctrl = reinterpret_cast<int*>(base);
    p.flags = p.ctrl + 4;
    p.Bw = reinterpret_cast<float*>(base + ctrl_bytes);
    p.Cw = reinterpret_cast<float*>(base + ctrl_bytes + bytesBC);
    p.Dw = reinterpret_cast<float*>(base + ctrl_bytes + 2 * bytesBC);
    double* X0 = reinterpret_cast<double*>(base + ctrl_bytes + 2 * bytesBC + bytesD);
    double* R = steps > 0 ? reinterpret_cast<double*>(reinterpret_cast<char*>(X0) + nn) : nullptr;
    double* X1 = steps > 0 ? reinterpret_cast<double*>(reinterpret_cast<char*>(X0) + 2 * nn) : nullptr;
    void* ozws = oz ? static_cast<void*>(reinterpret_cast<char*>(X0) + 3 * nn) : nullptr;
    p.X = X0;
    p.timeout_ns = (long long)(wait_timeout_s(o) * 1e9);
    p.drop_task = (o->wait_timeout_s > 0 && o->fault_drop_task >= 0) ? o->fault_drop_task : -1;
    e = ds.exec_plan(t, STEPS_ALL, &p.tasks, &p.ntasks);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemsetAsync(p.ctrl, 0, ctrl_bytes, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    void* tok = nullptr;
    timing_begin(SPDINV_TIMED_MIXED_DAG, stream, &tok);
    switch (o->precision) {
        case SPDINV_PREC_MIXED_TF32X3:
            e = b == 64 ? launch_mixed_dag<64, AccTC<64, SplitTF32>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream)
                        : launch_mixed_dag<32, AccTC<32, SplitTF32>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream);
            break;
        case SPDINV_PREC_MIXED_BF16X3:
            e = b == 64 ? launch_mixed_dag<64, AccTC<64, SplitBF16>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream)
                        : launch_mixed_dag<32, AccTC<32, SplitBF16>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream);
            break;
        default:
            e = b == 64 ? launch_mixed_dag<64, Acc32<64>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream)
                        : launch_mixed_dag<32, Acc32<32>>(p, o->diag_fp64 != 0, o->ctas_per_sm, ds.num_sms, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    timing_end(SPDINV_TIMED_MIXED_DAG, stream, tok, (double)n * (double)n * (double)n);
    int launches = 1;
    const int rt = (int)((n + RB - 1) / RB);
    const int rsm = 2 * RB * RB * (int)sizeof(double);
    const int csm = 2 * RB * (RB + 1) * (int)sizeof(float);
    e = cudaFuncSetAttribute(residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rsm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(correct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, csm);
    if (e != cudaSuccess) return cuda_fail(e);
    double* Xc = X0;
    for (int s = 0; s < steps && chain; ++s) {
        // X (lower triangle) is updated in place; X1 holds the current term.
        e = ozaki_refine_step(n, dA, lda, X0, R, X1, ozws, s == steps - 1 ? kLevelsLast : kLevels, order, s == 0,
                              p.ctrl + 2, stream, &launches);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    for (int s = 0; s < steps && !chain; ++s) {
        double* Xn = (Xc == X0) ? X1 : X0;
        if (emulated) {
            e = ozaki_residual(n, dA, lda, Xc, R, ozws, kSlices, s == steps - 1 ? kLevelsLast : kLevels,
                               o->residual == SPDINV_RESIDUAL_EMULATED, p.ctrl + 2, stream, &launches);
            if (e != cudaSuccess) return cuda_fail(e);
        } else {
            residual_kernel<<<(unsigned)((int64_t)rt * rt), kThreads, rsm, stream>>>(n, dA, lda, Xc, R, p.ctrl);
            launches += 1;
        }
        correct_kernel<<<(unsigned)((int64_t)rt * rt), kThreads, csm, stream>>>(n, Xc, R, Xn, p.ctrl);
        Xc = Xn;
        launches += 1;
    }
    store_lower_kernel<<<(unsigned)n, 256, 0, stream>>>(n, Xc, dA, lda, p.ctrl);
    launches += 1;
    if (d_info) {
        finalize_info_mixed<<<1, 32, 0, stream>>>(p.ctrl, d_info);
        launches += 1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(launches);
    return SPDINV_OK;
}

}  // namespace spdinv

using namespace spdinv;

static spdinv_status inverse_residual_impl(int64_t n, const double* dA, int64_t lda, const double* dX,
                                                            double* dR, int residual, cudaStream_t stream) {
    if (n < 0) return SPDINV_ERR_N;
    if (lda < (n > 1 ? n : 1)) return SPDINV_ERR_LDA;
    if (n == 0) return SPDINV_OK;
    if (!dA || !dX || !dR) return SPDINV_ERR_NULL;
    size_t need = 0;
    const spdinv_status ls = residual_workspace(n, residual, &need);
    if (ls != SPDINV_OK) return ls;
    const bool emulated = residual == SPDINV_RESIDUAL_EMULATED || residual == SPDINV_RESIDUAL_EMULATED_MMA_SYNC;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    DeviceState& ds = device_state(dev);
    std::lock_guard<std::mutex> lk(ds.mu);
    void* wsp = nullptr;
    const spdinv_status ws = ds.acquire(need, &wsp);
    if (ws != SPDINV_OK) return ws;
    int* ctrl = static_cast<int*>(wsp);
    e = cudaMemsetAsync(ctrl, 0, 256, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int launches = 0;
    if (emulated) {
        e = ozaki_residual(n, dA, lda, dX, dR, static_cast<char*>(wsp) + 256, 7, 7,
                           residual == SPDINV_RESIDUAL_EMULATED, ctrl + 2, stream, &launches);
    } else {
        const int rt = (int)((n + RB - 1) / RB);
        const int rsm = 2 * RB * RB * (int)sizeof(double);
        e = cudaFuncSetAttribute(residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rsm);
        if (e == cudaSuccess) {
            residual_kernel<<<(unsigned)((int64_t)rt * rt), kThreads, rsm, stream>>>(n, dA, lda, dX, dR, ctrl);
            launches = 1;
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(launches);
    return SPDINV_OK;
}

extern "C" SPDINV_API spdinv_status spdinv_inverse_residual(int64_t n, const double* dA, int64_t lda, const double* dX,
                                                            double* dR, int residual, cudaStream_t stream) {
    return log_status("spdinv_inverse_residual", "n", n, inverse_residual_impl(n, dA, lda, dX, dR, residual, stream));
}
