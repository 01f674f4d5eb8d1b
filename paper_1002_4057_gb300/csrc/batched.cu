// Many independent SPD matrices of uneven sizes, inverted in ONE persistent
// launch.  Each CTA takes the next matrix from a device queue ordered by
// decreasing n (largest first, so the long jobs start early and the short
// ones fill the tail) and runs the three steps of Algorithm 1 (Sec. 2) on it
// with b x b tiles, one tile operation after another.  Executed in the
// algorithm's own sequential order the in-place updates have no hazards
// (Step 2 walks i downwards, Step 3 walks i upwards, exactly as Algorithm 1
// prints them), so a matrix needs no workspace, flags or waits: only barriers
// between tile operations.  The inverted diagonal tile X_jj is kept in place
// of L_jj from Step 1 on; nothing after Step 1 reads L_jj.
//
// The tile size of each matrix comes from the autotuner's table for its size
// class, capped per batch by plan tuning (one kernel holds the largest tile
// any matrix uses, and that sets every CTA's occupancy).  Inside each chain of
// products the next tiles are read into registers while the current product
// runs.  FP64 uses the FP64 FMA register-block tile products (tile_fp64.cuh),
// FP32 the CUDA-core FMA ones (tile_f32.cuh).
// spdinv_batch_shard splits a batch across GPUs (host only).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "tile_f32.cuh"
#include "tile_fp64.cuh"

namespace spdinv {
namespace {

template <typename T, int B>
struct Tile;
template <int B>
struct Tile<double, B> {
    using Acc = spdinv::Acc<B>;
    static constexpr int LD = B;
};
template <int B>
struct Tile<float, B> {
    using Acc = Acc32<B>;
    static constexpr int LD = B + 1;
};

template <typename T>
struct BatchParams {
    int batch;
    const int* order;  // matrix indices, largest n first
    const int* n;
    const int* lda;
    const int* tile;   // tile order chosen for each matrix
    T* const* A;
    int* info;         // [batch] or nullptr
    int* counter;      // queue ticket
};

// Tile (ti, tj) of a column-major matrix into shared memory (leading
// dimension LD); padding past n: identity on the diagonal, zeros elsewhere.
template <typename T, int B>
__device__ __forceinline__ void gload(const T* A, int n, int64_t lda, int ti, int tj, T* S, bool lower_only) {
    constexpr int LD = Tile<T, B>::LD;
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int gr = ti * B + r, gc = tj * B + c;
        T v;
        if (gr < n && gc < n) v = (lower_only && r < c) ? T(0) : A[gr + (int64_t)gc * lda];
        else v = (ti == tj && r == c) ? T(1) : T(0);
        S[c * LD + r] = v;
    }
}

template <typename T, int B>
__device__ __forceinline__ void gstore(T* A, int n, int64_t lda, int ti, int tj, const T* S, bool lower_only) {
    constexpr int LD = Tile<T, B>::LD;
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int gr = ti * B + r, gc = tj * B + c;
        if (gr < n && gc < n && !(lower_only && r < c)) A[gr + (int64_t)gc * lda] = S[c * LD + r];
    }
}

// The next tile of a chain of products.  For tiles of at most 8 elements per
// thread (b <= 32) the thread's elements are read into registers while the
// current product runs and placed in shared memory after it; larger tiles
// (b = 64, 32 elements per thread) would take the registers the product
// needs, so they keep only the tile's position and are read when placed.
template <typename T, int B, bool Staged = (B * B / kThreads <= 8)>
struct TileRegs {
    static constexpr int N = B * B / kThreads;
    T v[N];
};
template <typename T, int B>
struct TileRegs<T, B, false> {
    const T* A;
    int n;
    int64_t lda;
    int ti, tj;
};

// Thread t holds row t % B of the tile at columns t / B + q (kThreads / B),
// q = 0 .. N-1 (kThreads is a multiple of B): one pointer and one stride.
template <typename T, int B, bool S>
__device__ __forceinline__ void fetch(const T* A, int n, int64_t lda, int ti, int tj, TileRegs<T, B, S>& r) {
    if constexpr (S) {
        constexpr int CS = kThreads / B;
        const int rr = threadIdx.x % B, c0 = threadIdx.x / B;
        const int gr = ti * B + rr, gc0 = tj * B + c0;
        const T* src = A + gr + (int64_t)gc0 * lda;
        const int64_t step = (int64_t)CS * lda;
#pragma unroll
        for (int q = 0; q < TileRegs<T, B, S>::N; ++q) {
            const bool in = gr < n && gc0 + q * CS < n;
            r.v[q] = in ? src[q * step] : ((ti == tj && rr == c0 + q * CS) ? T(1) : T(0));
        }
    } else {
        r.A = A;
        r.n = n;
        r.lda = lda;
        r.ti = ti;
        r.tj = tj;
    }
}

template <typename T, int B, bool S>
__device__ __forceinline__ void place(const TileRegs<T, B, S>& r, T* Sm) {
    if constexpr (S) {
        constexpr int LD = Tile<T, B>::LD, CS = kThreads / B;
        T* dst = Sm + (threadIdx.x / B) * LD + threadIdx.x % B;
#pragma unroll
        for (int q = 0; q < TileRegs<T, B, S>::N; ++q) dst[q * CS * LD] = r.v[q];
    } else {
        gload<T, B>(r.A, r.n, r.lda, r.ti, r.tj, Sm, false);
    }
}

// Algorithm 1 on one matrix, in place.  Returns LAPACK's info.
template <typename T, int B>
__device__ int run_matrix(T* A, int n, int64_t lda, T* S0, T* S1, T* tmp, int* s_fail) {
    static_assert(B * B % kThreads == 0 && kThreads % B == 0, "whole tiles per thread");
    typename Tile<T, B>::Acc acc;
    TileRegs<T, B> r0, r1;
    const int t = (n + B - 1) / B;
    // ---- Step 1: tile Cholesky (left-looking, k increasing)
    for (int j = 0; j < t; ++j) {
        cta_sync();
        gload<T, B>(A, n, lda, j, j, S0, true);
        cta_sync();
        acc_load<B>(acc, S0);
        if (j > 0) fetch<T, B>(A, n, lda, j, 0, r0);
        for (int k = 0; k < j; ++k) {  // SYRK
            cta_sync();
            place<T, B>(r0, S1);
            cta_sync();
            if (k + 1 < j) fetch<T, B>(A, n, lda, j, k + 1, r0);
            tile_mma<B, false, true, true, FULL, FULL>(acc, S1, S1);
        }
        cta_sync();
        acc_store<B>(acc, S0);
        const int fail = tile_potrf<B>(S0, s_fail);  // POTRF
        if (fail) return j * B + fail;
        tile_zero_upper<B>(S0);
        tile_trtri<B>(S0, tmp);  // X_jj = L_jj^{-1}, kept in place of L_jj
        gstore<T, B>(A, n, lda, j, j, S0, true);
        for (int i = j + 1; i < t; ++i) {
            cta_sync();
            gload<T, B>(A, n, lda, i, j, S0, false);
            cta_sync();
            acc_load<B>(acc, S0);
            if (j > 0) {
                fetch<T, B>(A, n, lda, i, 0, r0);
                fetch<T, B>(A, n, lda, j, 0, r1);
            }
            for (int k = 0; k < j; ++k) {  // GEMM
                cta_sync();
                place<T, B>(r0, S0);
                place<T, B>(r1, S1);
                cta_sync();
                if (k + 1 < j) {
                    fetch<T, B>(A, n, lda, i, k + 1, r0);
                    fetch<T, B>(A, n, lda, j, k + 1, r1);
                }
                tile_mma<B, false, true, true, FULL, FULL>(acc, S0, S1);
            }
            cta_sync();  // TRSM as the product with X_jj^T
            gload<T, B>(A, n, lda, j, j, S1, true);
            acc_store<B>(acc, S0);
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, false, true, false, FULL, LOWER>(acc, S0, S1);
            cta_sync();
            acc_store<B>(acc, S0);
            cta_sync();
            gstore<T, B>(A, n, lda, i, j, S0, false);
        }
    }
    // ---- Step 2: X = L^{-1} (j decreasing, i decreasing, k decreasing)
    for (int j = t - 1; j >= 0; --j) {
        for (int i = t - 1; i > j; --i) {
            cta_sync();
            gload<T, B>(A, n, lda, i, i, S0, true);   // X_ii
            gload<T, B>(A, n, lda, i, j, S1, false);  // L_ij
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, false, false, false, LOWER, FULL>(acc, S0, S1);  // TRMM
            if (i - 1 > j) {
                fetch<T, B>(A, n, lda, i, i - 1, r0);
                fetch<T, B>(A, n, lda, i - 1, j, r1);
            }
            for (int k = i - 1; k > j; --k) {  // GEMM
                cta_sync();
                place<T, B>(r0, S0);  // X_ik
                place<T, B>(r1, S1);  // L_kj
                cta_sync();
                if (k - 1 > j) {
                    fetch<T, B>(A, n, lda, i, k - 1, r0);
                    fetch<T, B>(A, n, lda, k - 1, j, r1);
                }
                tile_mma<B, false, false, false, FULL, FULL>(acc, S0, S1);
            }
            cta_sync();
            gload<T, B>(A, n, lda, j, j, S1, true);  // X_jj
            acc_store<B>(acc, S0);
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, false, false, true, FULL, LOWER>(acc, S0, S1);  // TRMM by -X_jj
            cta_sync();
            acc_store<B>(acc, S0);
            cta_sync();
            gstore<T, B>(A, n, lda, i, j, S0, false);
        }
    }
    // ---- Step 3: A^{-1} = X^T X (i increasing; k increasing)
    for (int i = 0; i < t; ++i) {
        for (int j = 0; j < i; ++j) {
            cta_sync();
            gload<T, B>(A, n, lda, i, i, S0, true);   // X_ii
            gload<T, B>(A, n, lda, i, j, S1, false);  // X_ij
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, true, false, false, LOWER, FULL>(acc, S0, S1);  // TRMM
            if (i + 1 < t) {
                fetch<T, B>(A, n, lda, i + 1, i, r0);
                fetch<T, B>(A, n, lda, i + 1, j, r1);
            }
            for (int k = i + 1; k < t; ++k) {  // GEMM
                cta_sync();
                place<T, B>(r0, S0);
                place<T, B>(r1, S1);
                cta_sync();
                if (k + 1 < t) {
                    fetch<T, B>(A, n, lda, k + 1, i, r0);
                    fetch<T, B>(A, n, lda, k + 1, j, r1);
                }
                tile_mma<B, true, false, false, FULL, FULL>(acc, S0, S1);
            }
            cta_sync();
            acc_store<B>(acc, S0);
            cta_sync();
            gstore<T, B>(A, n, lda, i, j, S0, false);
        }
        cta_sync();
        gload<T, B>(A, n, lda, i, i, S0, true);
        cta_sync();
        acc_zero<B>(acc);
        tile_mma<B, true, false, false, LOWER, LOWER>(acc, S0, S0);  // LAUUM
        if (i + 1 < t) fetch<T, B>(A, n, lda, i + 1, i, r0);
        for (int k = i + 1; k < t; ++k) {  // SYRK
            cta_sync();
            place<T, B>(r0, S0);
            cta_sync();
            if (k + 1 < t) fetch<T, B>(A, n, lda, k + 1, i, r0);
            tile_mma<B, true, false, false, FULL, FULL>(acc, S0, S0);
        }
        cta_sync();
        acc_store<B>(acc, S0);
        cta_sync();
        gstore<T, B>(A, n, lda, i, i, S0, true);
    }
    return 0;
}

// Resident CTAs per SM the register budget is set for: the largest tile's
// accumulator and staged tiles must fit without spilling.
template <typename T, int BMAX>
constexpr int batched_min_blocks() {
    return BMAX >= 64 ? 4 : (BMAX <= 16 ? 12 : (sizeof(T) == 8 ? 5 : 8));
}

template <typename T, int BMAX>
__global__ void __launch_bounds__(kThreads, batched_min_blocks<T, BMAX>()) potri_batched_kernel(const BatchParams<T> p) {
    unsigned char* const smem_raw = dynamic_smem();
    __shared__ int s_m, s_fail;
    constexpr int TS = BMAX * (BMAX + 1);
    T* S0 = reinterpret_cast<T*>(smem_raw);
    T* S1 = S0 + TS;
    T* tmp = S1 + TS;
    for (;;) {
        cta_sync();
        if (threadIdx.x == 0) s_m = atomicAdd(p.counter, 1);
        cta_sync();
        const int m = s_m;
        if (m >= p.batch) return;
        const int idx = p.order[m];
        const int n = p.n[idx];
        const int64_t lda = p.lda[idx];
        T* A = p.A[idx];
        int info = 0;
        const int b = p.tile[idx];
        if (b == 16) info = run_matrix<T, 16>(A, n, lda, S0, S1, tmp, &s_fail);
        if constexpr (BMAX >= 32) {
            if (b == 32) info = run_matrix<T, 32>(A, n, lda, S0, S1, tmp, &s_fail);
        }
        if constexpr (BMAX >= 64) {
            if (b == 64) info = run_matrix<T, 64>(A, n, lda, S0, S1, tmp, &s_fail);
        }
        if (threadIdx.x == 0 && p.info) p.info[idx] = info;
    }
}

template <typename T, int BMAX>
constexpr int batched_smem() {
    return (2 * BMAX * (BMAX + 1) + kThreads) * (int)sizeof(T);
}

template <typename T, int BMAX>
cudaError_t launch_batched_t(const BatchParams<T>& p, int num_sms, cudaStream_t s) {
    auto k = potri_batched_kernel<T, BMAX>;
    constexpr int sm = batched_smem<T, BMAX>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int grid = num_sms * occ;
    if (grid > p.batch) grid = p.batch;
    k<<<grid, kThreads, sm, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batched(const BatchParams<T>& p, int bmax, int num_sms, cudaStream_t s) {
    if (bmax <= 16) return launch_batched_t<T, 16>(p, num_sms, s);
    if (bmax <= 32) return launch_batched_t<T, 32>(p, num_sms, s);
    if constexpr (sizeof(T) == 4) return launch_batched_t<T, 64>(p, num_sms, s);
    return cudaErrorInvalidValue;
}

// A diagonally dominant (hence SPD) test matrix per slot, for the autotuner.
template <typename T>
__global__ void fill_tuning_batch(T* base, int n, int count) {
    const int64_t per = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % per;
        const int r = (int)(q % n), c = (int)(q / n);
        uint32_t h = (uint32_t)(min(r, c) * 73856093u) ^ (uint32_t)(max(r, c) * 19349663u) ^ (uint32_t)(e / per);
        h ^= h >> 13;
        h *= 0x5bd1e995u;
        h ^= h >> 15;
        const T off = (T)((h & 0xFFFF) / 65536.0 - 0.5);
        base[e] = r == c ? (T)n : off;
    }
}

constexpr int kClasses = 8;  // n in (32c, 32(c+1)], c = 0..7; larger n use class 7

struct BatchPlan {
    int* dev = nullptr;  // [n | lda | order | tile | counter] in one allocation
    int batch = 0;
    int bmax = 16;
};

constexpr int kCands = 3;  // candidate tiles 16, 32, 64 (64: FP32 only)
constexpr int kCandTile[kCands] = {16, 32, 64};

struct BatchState {
    std::mutex mu;
    bool tuned[2] = {false, false};
    bool forced[2] = {false, false};        // one tile from SPDINV_BATCHED_TILE
    int tiles[2][kClasses];
    float ms[2][kClasses][kCands];          // per-class timings of each candidate (1e30: not run)
    std::map<std::vector<int>, BatchPlan> plans[2];
};

BatchState& batch_state(int dev) {
    static std::mutex mu;
    static std::map<int, BatchState*> m;
    std::lock_guard<std::mutex> lk(mu);
    auto& s = m[dev];
    if (!s) s = new BatchState();
    return *s;
}

int size_class(int n) {
    const int c = (n - 1) / 32;
    return c < 0 ? 0 : (c >= kClasses ? kClasses - 1 : c);
}

// Autotuner: for every size class, time the batched kernel on a synthetic
// batch of that class's largest size with each candidate tile, keep the
// fastest.  Runs once per device and precision (or takes SPDINV_BATCHED_TILE).
template <typename T>
cudaError_t autotune(BatchState& bs, int num_sms, int* tiles) {
    const int fp = sizeof(T) == 4 ? 1 : 0;
    if (bs.tuned[fp]) {
        std::memcpy(tiles, bs.tiles[fp], sizeof(int) * kClasses);
        return cudaSuccess;
    }
    if (const char* env = std::getenv("SPDINV_BATCHED_TILE")) {
        const int b = std::atoi(env);
        if (b == 16 || b == 32 || (b == 64 && fp == 1)) {
            for (int c = 0; c < kClasses; ++c) bs.tiles[fp][c] = b;
            bs.tuned[fp] = true;
            bs.forced[fp] = true;
            std::memcpy(tiles, bs.tiles[fp], sizeof(int) * kClasses);
            return cudaSuccess;
        }
    }
    const std::vector<int> cands = fp ? std::vector<int>{16, 32, 64} : std::vector<int>{16, 32};
    const int count = 2 * num_sms;
    const int nmax = 32 * kClasses;
    T* data = nullptr;
    T** ptrs = nullptr;
    int* ints = nullptr;
    cudaError_t e = cudaMalloc(&data, sizeof(T) * (size_t)nmax * nmax * count);
    if (e == cudaSuccess) e = cudaMalloc(&ptrs, sizeof(T*) * count);
    if (e == cudaSuccess) e = cudaMalloc(&ints, sizeof(int) * (4 * count + 1));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<T*> hp(count);
    std::vector<int> hints(4 * count);
    for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
        const int n = 32 * (c + 1);
        for (int q = 0; q < count; ++q) {
            hp[q] = data + (size_t)q * n * n;
            hints[q] = n;              // n
            hints[count + q] = n;      // lda
            hints[2 * count + q] = q;  // order
        }
        e = cudaMemcpy(ptrs, hp.data(), sizeof(T*) * count, cudaMemcpyHostToDevice);
        float best = 1e30f;
        int bestb = cands[0];
        for (int k = 0; k < kCands; ++k) bs.ms[fp][c][k] = 1e30f;
        for (int b : cands) {
            if (e != cudaSuccess) break;
            for (int q = 0; q < count; ++q) hints[3 * count + q] = b;
            e = cudaMemcpy(ints, hints.data(), sizeof(int) * 4 * count, cudaMemcpyHostToDevice);
            BatchParams<T> p{count, ints + 2 * count, ints, ints + count, ints + 3 * count, ptrs, nullptr,
                             ints + 4 * count};
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                fill_tuning_batch<T><<<256, 256>>>(data, n, count);
                cudaMemset(ints + 4 * count, 0, sizeof(int));
                cudaEventRecord(e0);
                e = launch_batched<T>(p, b, num_sms, 0);
                cudaEventRecord(e1);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_min = std::min(ms_min, ms);
            }
            bs.ms[fp][c][b == 16 ? 0 : (b == 32 ? 1 : 2)] = ms_min;
            if (ms_min < best) {
                best = ms_min;
                bestb = b;
            }
        }
        bs.tiles[fp][c] = bestb;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(data);
    cudaFree(ptrs);
    cudaFree(ints);
    if (e != cudaSuccess) return e;
    bs.tuned[fp] = true;
    std::memcpy(tiles, bs.tiles[fp], sizeof(int) * kClasses);
    return cudaSuccess;
}

// Fills matrix k of a batch (order n[k], leading dimension n[k]) with a
// diagonally dominant (hence SPD) test matrix, one CTA per matrix.
template <typename T>
__global__ void fill_tuning_mats(T* const* ptrs, const int* n, int batch) {
    for (int k = blockIdx.x; k < batch; k += gridDim.x) {
        const int m = n[k];
        T* A = ptrs[k];
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = e % m, c = e / m;
            uint32_t h = (uint32_t)(min(r, c) * 73856093u) ^ (uint32_t)(max(r, c) * 19349663u) ^ (uint32_t)k;
            h ^= h >> 13;
            h *= 0x5bd1e995u;
            h ^= h >> 15;
            A[e] = r == c ? (T)m : (T)((h & 0xFFFF) / 65536.0 - 0.5);
        }
    }
}

// The per-class table when every tile is at most `cap`: the fastest tile of
// each class among those (one persistent kernel holds the largest tile any
// matrix uses, and its shared memory and registers set the occupancy of all).
int capped_tiles(const BatchState& bs, int fp, int cap, int* out) {
    int bmax = 16;
    for (int c = 0; c < kClasses; ++c) {
        if (bs.forced[fp]) {
            out[c] = bs.tiles[fp][c];
        } else {
            int best = 0;
            for (int k = 1; k < kCands; ++k)
                if (kCandTile[k] <= cap && bs.ms[fp][c][k] < bs.ms[fp][c][best]) best = k;
            out[c] = kCandTile[best];
        }
        bmax = std::max(bmax, out[c]);
    }
    return bmax;
}

// Whole-batch plan tuning: the per-class tables capped at 64, 32 and 16 are
// each timed on a synthetic batch with the caller's sizes; the fastest wins.
// Returns the chosen table in `tiles`.  Skipped (first table kept) when the
// synthetic copy would exceed 2 GiB.
template <typename T>
cudaError_t tune_plan(const BatchState& bs, int fp, int batch, const int* h_n, const std::vector<int>& order,
                      int num_sms, int* tiles) {
    std::vector<std::vector<int>> tables;
    for (int cap : {64, 32, 16}) {
        if (fp == 0 && cap == 64) continue;
        std::vector<int> t(kClasses);
        capped_tiles(bs, fp, cap, t.data());
        if (std::find(tables.begin(), tables.end(), t) == tables.end()) tables.push_back(t);
    }
    std::copy(tables[0].begin(), tables[0].end(), tiles);
    size_t elems = 0;
    for (int k = 0; k < batch; ++k) elems += (size_t)h_n[k] * h_n[k];
    if (tables.size() < 2 || elems * sizeof(T) > (size_t(2) << 30)) return cudaSuccess;
    T* data = nullptr;
    T** ptrs = nullptr;
    int* ints = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&data, sizeof(T) * std::max<size_t>(elems, 1));
    if (e == cudaSuccess) e = cudaMalloc(&ptrs, sizeof(T*) * batch);
    if (e == cudaSuccess) e = cudaMalloc(&ints, sizeof(int) * (4 * (size_t)batch + 1));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<T*> hp(batch);
    std::vector<int> h(4 * (size_t)batch);
    size_t off = 0;
    for (int k = 0; k < batch; ++k) {
        hp[k] = data + off;
        off += (size_t)h_n[k] * h_n[k];
        h[k] = h_n[k];
        h[batch + k] = std::max(h_n[k], 1);
        h[2 * batch + k] = order[k];
    }
    if (e == cudaSuccess) e = cudaMemcpy(ptrs, hp.data(), sizeof(T*) * batch, cudaMemcpyHostToDevice);
    float best = 1e30f;
    for (const auto& t : tables) {
        if (e != cudaSuccess) break;
        int bmax = 16;
        for (int k = 0; k < batch; ++k) {
            h[3 * batch + k] = t[size_class(h_n[k])];
            bmax = std::max(bmax, h[3 * batch + k]);
        }
        e = cudaMemcpy(ints, h.data(), sizeof(int) * 4 * batch, cudaMemcpyHostToDevice);
        BatchParams<T> p{batch, ints + 2 * batch, ints, ints + batch, ints + 3 * batch, ptrs, nullptr, ints + 4 * batch};
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            fill_tuning_mats<T><<<std::min(batch, 4 * num_sms), 256>>>(ptrs, ints, batch);
            cudaMemset(ints + 4 * batch, 0, sizeof(int));
            cudaEventRecord(e0);
            e = launch_batched<T>(p, bmax, num_sms, 0);
            cudaEventRecord(e1);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
        }
        if (e == cudaSuccess && ms_min < best) {
            best = ms_min;
            std::copy(t.begin(), t.end(), tiles);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(data);
    cudaFree(ptrs);
    cudaFree(ints);
    return e;
}

template <typename T>
spdinv_status run_batched(int batch, const int* h_n, T* const* d_Aptrs, const int* h_lda, int* d_info,
                          cudaStream_t stream) {
    if (batch < 0) return SPDINV_ERR_N;
    if (batch == 0) return SPDINV_OK;
    if (!h_n || !h_lda || !d_Aptrs) return SPDINV_ERR_NULL;
    for (int k = 0; k < batch; ++k) {
        if (h_n[k] < 0 || h_n[k] > 4096) return SPDINV_ERR_N;
        if (h_lda[k] < (h_n[k] > 1 ? h_n[k] : 1)) return SPDINV_ERR_LDA;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const int num_sms = device_state(dev).num_sms;
    BatchState& bs = batch_state(dev);
    std::lock_guard<std::mutex> lk(bs.mu);
    const int fp = sizeof(T) == 4 ? 1 : 0;
    std::vector<int> key(h_n, h_n + batch);
    key.insert(key.end(), h_lda, h_lda + batch);
    auto it = bs.plans[fp].find(key);
    if (it == bs.plans[fp].end()) {
        int tiles[kClasses];
        e = autotune<T>(bs, num_sms, tiles);
        if (e != cudaSuccess) return cuda_fail(e);
        std::vector<int> h(4 * batch + 1, 0);
        std::vector<int> order(batch);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
        e = tune_plan<T>(bs, fp, batch, h_n, order, num_sms, tiles);
        if (e != cudaSuccess) return cuda_fail(e);
        int bmax = 16;
        for (int k = 0; k < batch; ++k) {
            h[k] = h_n[k];
            h[batch + k] = h_lda[k];
            h[2 * batch + k] = order[k];
            const int b = tiles[size_class(h_n[k])];
            h[3 * batch + k] = b;
            bmax = std::max(bmax, b);
        }
        BatchPlan bp;
        bp.batch = batch;
        bp.bmax = bmax;
        e = cudaMalloc(&bp.dev, sizeof(int) * h.size());
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaMemcpy(bp.dev, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(bp.dev);
            return cuda_fail(e);
        }
        it = bs.plans[fp].emplace(std::move(key), bp).first;
    }
    const BatchPlan& bp = it->second;
    BatchParams<T> p{batch, bp.dev + 2 * batch, bp.dev, bp.dev + batch, bp.dev + 3 * batch, d_Aptrs, d_info,
                     bp.dev + 4 * batch};
    e = cudaMemsetAsync(p.counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_batched<T>(p, bp.bmax, num_sms, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return SPDINV_OK;
}

}  // namespace
}  // namespace spdinv

using namespace spdinv;

extern "C" {

SPDINV_API spdinv_status spdinv_potri_batched(int batch, const int* h_n, double* const* d_Aptrs, const int* h_lda,
                                              int* d_info, cudaStream_t stream) {
    return log_status("spdinv_potri_batched", "batch", batch, run_batched<double>(batch, h_n, d_Aptrs, h_lda, d_info, stream));
}

SPDINV_API spdinv_status spdinv_spotri_batched(int batch, const int* h_n, float* const* d_Aptrs, const int* h_lda,
                                               int* d_info, cudaStream_t stream) {
    return log_status("spdinv_spotri_batched", "batch", batch, run_batched<float>(batch, h_n, d_Aptrs, h_lda, d_info, stream));
}

SPDINV_API spdinv_status spdinv_batch_shard(int batch, const int* h_n, int world, int* owner, double* load) {
    if (batch < 0) return SPDINV_ERR_N;
    if (world < 1) return SPDINV_ERR_UNSUPPORTED;
    if (batch > 0 && (!h_n || !owner)) return SPDINV_ERR_NULL;
    for (int k = 0; k < batch; ++k)
        if (h_n[k] < 0) return SPDINV_ERR_N;
    // Longest processing time first: matrices by decreasing n (ties: lower
    // index first), each to the rank with the least n^3 so far (ties: lower
    // rank).  Deterministic, so every rank computes the same split.
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
    std::vector<double> sum(world, 0.0);
    for (int k : order) {
        int r = 0;
        for (int q = 1; q < world; ++q)
            if (sum[q] < sum[r]) r = q;
        owner[k] = r;
        sum[r] += (double)h_n[k] * h_n[k] * h_n[k];
    }
    if (load)
        for (int q = 0; q < world; ++q) load[q] = sum[q];
    return SPDINV_OK;
}

SPDINV_API spdinv_status spdinv_batched_tiles(int fp32, int tiles[8]) {
    if (!tiles) return SPDINV_ERR_NULL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const int num_sms = device_state(dev).num_sms;
    BatchState& bs = batch_state(dev);
    std::lock_guard<std::mutex> lk(bs.mu);
    e = fp32 ? autotune<float>(bs, num_sms, tiles) : autotune<double>(bs, num_sms, tiles);
    return e == cudaSuccess ? SPDINV_OK : cuda_fail(e);
}

}  // extern "C"
