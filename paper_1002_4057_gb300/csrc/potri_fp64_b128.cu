// Persistent FP64 kernel with 128 x 128 tiles (tile b = 128 of the tile
// sweep; Sec. 2's tile storage takes b as a parameter).  Same plan, renamed
// stores B, C, D, readiness flags and task protocol as potri_fp64.cu
// (Algorithm 1 with the renaming and pipelining of Sec. 3); what differs is
// how a tile product is fed, because two 128 x 128 FP64 tiles (256 KB) do
// not fit in shared memory:
//   * a CTA has 256 threads (16 x 16, each owning an 8 x 8 block of the
//     128 x 128 accumulator: 64 doubles);
//   * each chain element streams its operands through shared memory in
//     slabs 32 deep -- a 128 x 32 column slab or a 32 x 128 row slab of a
//     stored tile, whichever op(X) needs -- fetched by 2-D TMA loads from
//     tensor maps over the tile-major stores, double-buffered;
//   * the diagonal POTRF and TRTRI work on the whole tile in shared memory
//     (128 KB), as do the TRMMs whose left operand is the task's own
//     intermediate tile.
// The products are FP64 fused multiply-adds on register blocks, like the
// smaller tiles'.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "api_internal.h"
#include "kernels.h"
#include "persist.cuh"
#include "tile_fp64.cuh"

namespace spdinv {
namespace {

constexpr int TB = 128;                  // tile order
constexpr int NT = 256;                  // threads per CTA
constexpr int KS = 32;                   // slab depth
constexpr int RM = 8, CN = 8;            // accumulator block per thread
constexpr int SLAB = TB * KS;            // doubles per slab (32 KB)
constexpr int SLAB_BYTES = SLAB * 8;
// Shared memory: region X (128 KB) holds a whole tile, or the two buffers of
// a chain's slab pairs (P and Q slabs, 2 x 64 KB); region Y (64 KB) holds
// two Q slabs for products whose left operand is resident in X; then NT
// doubles of TRTRI scratch.
constexpr int X_DOUBLES = TB * TB, Y_DOUBLES = 2 * SLAB;
constexpr int SMEM128 = (X_DOUBLES + Y_DOUBLES + NT) * 8;

struct Acc128 {
    double v[RM][CN];
};

// Tensor maps over the three stores, each seen as a 2-D array: x = row of a
// tile (128, contiguous), y = tile * 128 + column.  col: boxes 128 x 32 (a
// column slab), row: boxes 32 x 128 (a row slab).
struct Maps128 {
    CUtensorMap b_col, b_row, c_col, c_row, d_col, d_row;
};

__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int r0_of() { return (threadIdx.x % 16) * RM; }
__device__ __forceinline__ int c0_of() { return (threadIdx.x / 16) * CN; }

__device__ __forceinline__ void acc_zero128(Acc128& a) {
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) a.v[i][j] = 0.0;
}
__device__ __forceinline__ void acc_store128(const Acc128& a, double* T) {
    const int r0 = r0_of(), c0 = c0_of();
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) T[(c0 + j) * TB + r0 + i] = a.v[i][j];
}
__device__ __forceinline__ void acc_load128(Acc128& a, const double* T) {
    const int r0 = r0_of(), c0 = c0_of();
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) a.v[i][j] = T[(c0 + j) * TB + r0 + i];
}

// acc (+|-)= op(P)[:, k0 : k0 + KS] op(Q)[k0 : k0 + KS, :] from slabs in
// shared memory (P resident: the whole column-major tile, op(P) = P).
//   P column slab (TA false): (m, kk) at kk * 128 + m
//   P row slab    (TA true):  (m, kk) at m * 32 + kk
//   Q row slab    (TQ false): (kk, n) at n * 32 + kk
//   Q column slab (TQ true):  (kk, n) at kk * 128 + n
// A lower-triangular stored operand (SP / SQ = LOWER) lets each thread skip
// the k that multiply its zeros.
template <bool TA, bool TQ, bool NEG, int SP, int SQ, bool PRES>
__device__ __forceinline__ void slab_mma(Acc128& acc, const double* P, const double* Q, int k0) {
    const int r0 = r0_of(), c0 = c0_of();
    int kb = k0, ke = k0 + KS;
    if (SP == LOWER) {  // op(P)[m][k] != 0 only for k <= m (N) or k >= m (T)
        if (TA) kb = max(kb, r0); else ke = min(ke, r0 + RM);
    }
    if (SQ == LOWER) {  // op(Q)[k][n] != 0 only for k >= n (N) or k <= n (T)
        if (TQ) ke = min(ke, c0 + CN); else kb = max(kb, c0);
    }
#pragma unroll 2
    for (int k = kb; k < ke; ++k) {
        const int kk = k - k0;
        double a[RM], b[CN];
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const double v = PRES ? P[k * TB + r0 + i] : (TA ? P[(r0 + i) * KS + kk] : P[kk * TB + r0 + i]);
            a[i] = NEG ? -v : v;
        }
#pragma unroll
        for (int j = 0; j < CN; ++j) b[j] = TQ ? Q[kk * TB + c0 + j] : Q[(c0 + j) * KS + kk];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < CN; ++j) acc.v[i][j] = fma(a[i], b[j], acc.v[i][j]);
    }
}

// The CTA's slab pipeline: two buffers, each with an mbarrier that counts
// its copied bytes.
struct Slabs {
    uint64_t* bar;  // [2]
    uint32_t phase[2];
    int* s_flag;
    int* ctrl;
    long long timeout_ns;
};

// Where an operand of a chain element comes from: a tile of a store, sliced
// into row slabs or column slabs.
struct Src {
    const CUtensorMap* map;
    int tile;
};

enum ElemMode {
    STREAM_BOTH = 0,  // P and Q slabs streamed (X holds the two buffers of slab pairs)
    RESIDENT_P = 1,   // P is the whole tile in X, Q slabs streamed through Y
    SAME_SLAB = 2,    // Q is P's slab (SYRK-like products of one tile with itself)
};

// Bounded wait for buffer b's copy (every thread); false = timeout (error raised).
__device__ __forceinline__ bool wait_buf(Slabs& S, int b) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(&S.bar[b], S.phase[b])) {
        if ((long long)(globaltimer_ns() - t0) > 2000000000LL) {
            if (threadIdx.x == 0) raise_error(S.ctrl, SPDINV_ERR_TIMEOUT);
            return false;
        }
    }
    S.phase[b] ^= 1u;
    return true;
}

// One chain element: waits for the input tiles' flags f0, f1 (thread 0,
// bounded), then acc (+|-)= op(P) op(Q) over four slabs, two copies in
// flight.  Called by all threads; false = stop (abort, timeout).
template <bool TA, bool TQ, bool NEG, int SP, int SQ, int MODE>
__device__ bool element(Slabs& S, Acc128& acc, const int* f0, const int* f1, Src P, Src Q, double* X, double* Y) {
    constexpr bool P_ROW = TA;   // op(P) = P^T needs P's rows k
    constexpr bool Q_ROW = !TQ;  // op(Q) = Q needs Q's rows k
    auto buf_p = [&](int b) -> double* { return MODE == RESIDENT_P ? X : X + b * 2 * SLAB; };
    auto buf_q = [&](int b) -> double* {
        return MODE == RESIDENT_P ? Y + b * SLAB : (MODE == SAME_SLAB ? X + b * 2 * SLAB : X + b * 2 * SLAB + SLAB);
    };
    auto issue = [&](int s) {  // thread 0: slab s into buffer s & 1
        const int b = s & 1;
        const uint32_t bytes = (MODE == STREAM_BOTH ? 2u : 1u) * (uint32_t)SLAB_BYTES;
        mbar_arrive_expect_tx(&S.bar[b], bytes);
        if (MODE != RESIDENT_P) {
            if (P_ROW) tma2d(buf_p(b), P.map, s * KS, P.tile * TB, &S.bar[b]);
            else tma2d(buf_p(b), P.map, 0, P.tile * TB + s * KS, &S.bar[b]);
        }
        if (MODE != SAME_SLAB) {
            if (Q_ROW) tma2d(buf_q(b), Q.map, s * KS, Q.tile * TB, &S.bar[b]);
            else tma2d(buf_q(b), Q.map, 0, Q.tile * TB + s * KS, &S.bar[b]);
        }
    };
    fence_proxy_async_shared();  // this thread's reads of the buffers before the copies that reuse them
    cta_sync();
    if (threadIdx.x == 0) {
        const bool ok = wait_flag(f0, S.ctrl, S.timeout_ns) && wait_flag(f1, S.ctrl, S.timeout_ns);
        *S.s_flag = ok ? 0 : 1;
        if (ok) {
            fence_proxy_async_global();
            fence_proxy_async_shared();
            issue(0);
            issue(1);
        }
    }
    cta_sync();
    if (*S.s_flag != 0) return false;
    for (int s = 0; s < TB / KS; ++s) {
        const int b = s & 1;
        if (!wait_buf(S, b)) return false;
        slab_mma<TA, TQ, NEG, SP, SQ, MODE == RESIDENT_P>(acc, buf_p(b), buf_q(b), s * KS);
        if (s + 2 < TB / KS) {
            fence_proxy_async_shared();
            cta_sync();  // everyone is done with buffer b
            if (threadIdx.x == 0) issue(s + 2);
        }
    }
    return true;
}

// Tile (ti, tj) of the column-major A into T (zeros, and the identity on the
// diagonal, past n); lower_only: the diagonal tile's strictly upper part of A
// is not read.
__device__ void load_A128(const KParamsF64& p, int ti, int tj, double* T, bool lower_only) {
    for (int idx = threadIdx.x; idx < TB * TB; idx += NT) {
        const int r = idx % TB, c = idx / TB;
        const int64_t gr = (int64_t)ti * TB + r, gc = (int64_t)tj * TB + c;
        double v;
        if (gr < p.n && gc < p.n) v = (lower_only && r < c) ? 0.0 : p.A[gr + gc * p.lda];
        else v = (ti == tj && r == c) ? 1.0 : 0.0;
        T[idx] = v;
    }
}

__device__ void store_A128(const KParamsF64& p, int ti, int tj, const double* T, bool lower_only) {
    for (int idx = threadIdx.x; idx < TB * TB; idx += NT) {
        const int r = idx % TB, c = idx / TB;
        const int64_t gr = (int64_t)ti * TB + r, gc = (int64_t)tj * TB + c;
        if (gr < p.n && gc < p.n && !(lower_only && r < c)) p.A[gr + gc * p.lda] = T[idx];
    }
}

__device__ void store_ws128(double* g, const double* T) {
    const double2* s = reinterpret_cast<const double2*>(T);
    double2* d = reinterpret_cast<double2*>(g);
    for (int idx = threadIdx.x; idx < TB * TB / 2; idx += NT) d[idx] = s[idx];
}

__global__ void __launch_bounds__(NT, 1)
    potri_fp64_b128(const __grid_constant__ Maps128 mp, const __grid_constant__ KParamsF64 p) {
    unsigned char* const smem_raw = dynamic_smem();
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_task, s_flag, s_fail;
    double* const X = reinterpret_cast<double*>(smem_raw);
    double* const Y = X + X_DOUBLES;
    double* const tmp = Y + Y_DOUBLES;
    Slabs S;
    S.bar = bars;
    S.phase[0] = S.phase[1] = 0;
    S.s_flag = &s_flag;
    S.ctrl = p.ctrl;
    S.timeout_ns = p.timeout_ns;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_proxy_async_shared();
    }
    cta_sync();
    const int t = p.t;
    int* const fL = p.flags;
    int* const fX = p.flags + (int64_t)t * t;
    int* const fD = p.flags + 2 * (int64_t)t * t;
    auto tri = [](int i, int j) { return i * (i - 1) / 2 + j; };  // tile index of (i, j), i > j, in B and C
    auto Bc = [&](int i, int j) { return Src{&mp.b_col, tri(i, j)}; };
    auto Br = [&](int i, int j) { return Src{&mp.b_row, tri(i, j)}; };
    auto Cc = [&](int i, int j) { return Src{&mp.c_col, tri(i, j)}; };
    auto Cr = [&](int i, int j) { return Src{&mp.c_row, tri(i, j)}; };
    auto Dc = [&](int j) { return Src{&mp.d_col, j}; };
    auto Dr = [&](int j) { return Src{&mp.d_row, j}; };
    const Src none{nullptr, 0};
    auto publish_flag = [&](int* flag, int ticket) {
        fence_proxy_async_global();
        __threadfence();
        cta_sync();
        if (threadIdx.x == 0 && ticket != p.drop_task) {
            __threadfence();
            st_release_gpu(flag, 1);
        }
    };

    for (;;) {
        const int ticket = next_ticket(p.ctrl, p.ntasks, &s_task);
        if (ticket < 0) return;
        const uint32_t e = p.tasks[ticket];
        const int kind = (int)task_kind(e), i = (int)task_i(e), j = (int)task_j(e);
        Acc128 acc;
        if (kind == K_S1_DIAG) {
            // A_jj - sum_k L_jk L_jk^T, POTRF, TRTRI -> D_j
            fence_proxy_async_shared();
            cta_sync();
            load_A128(p, j, j, X, true);
            cta_sync();
            acc_load128(acc, X);
            for (int k = 0; k < j; ++k)
                if (!element<false, true, true, FULL, FULL, SAME_SLAB>(S, acc, &fL[j * t + k], nullptr, Bc(j, k), none, X,
                                                                        Y))
                    return;
            cta_sync();
            acc_store128(acc, X);
            const int fail = tile_potrf<TB, NT>(X, &s_fail);
            if (fail) {
                if (threadIdx.x == 0) record_info(p.ctrl, j * TB + fail);
                return;
            }
            tile_zero_upper<TB, NT>(X);
            cta_sync();
            tile_trtri<TB, NT>(X, tmp);
            store_ws128(p.Dw + (int64_t)j * TB * TB, X);
            publish_flag(&fD[j], ticket);
        } else if (kind == K_S1_OFF) {
            // (A_ij - sum_k L_ik L_jk^T) X_jj^T -> B_ij
            fence_proxy_async_shared();
            cta_sync();
            load_A128(p, i, j, X, false);
            cta_sync();
            acc_load128(acc, X);
            for (int k = 0; k < j; ++k)
                if (!element<false, true, true, FULL, FULL, STREAM_BOTH>(S, acc, &fL[i * t + k], &fL[j * t + k], Bc(i, k),
                                                                          Bc(j, k), X, Y))
                    return;
            cta_sync();
            acc_store128(acc, X);  // A'_ij, resident for the TRSM
            acc_zero128(acc);
            if (!element<false, true, false, FULL, LOWER, RESIDENT_P>(S, acc, &fD[j], nullptr, none, Dc(j), X, Y))
                return;
            cta_sync();
            acc_store128(acc, X);
            cta_sync();
            store_ws128(p.Bw + (int64_t)tri(i, j) * TB * TB, X);
            publish_flag(&fL[i * t + j], ticket);
        } else if (kind == K_S2_OFF) {
            // -(X_ii L_ij + sum_{k=i-1..j+1} X_ik L_kj) X_jj -> C_ij
            acc_zero128(acc);
            if (!element<false, false, false, LOWER, FULL, STREAM_BOTH>(S, acc, &fD[i], &fL[i * t + j], Dc(i), Br(i, j),
                                                                          X, Y))
                return;
            for (int k = i - 1; k > j; --k)
                if (!element<false, false, false, FULL, FULL, STREAM_BOTH>(S, acc, &fX[i * t + k], &fL[k * t + j],
                                                                             Cc(i, k), Br(k, j), X, Y))
                    return;
            fence_proxy_async_shared();
            cta_sync();
            acc_store128(acc, X);
            acc_zero128(acc);
            if (!element<false, false, true, FULL, LOWER, RESIDENT_P>(S, acc, &fD[j], nullptr, none, Dr(j), X, Y))
                return;
            cta_sync();
            acc_store128(acc, X);
            cta_sync();
            store_ws128(p.Cw + (int64_t)tri(i, j) * TB * TB, X);
            publish_flag(&fX[i * t + j], ticket);
        } else if (kind == K_S3_OFF) {
            // X_ii^T X_ij + sum_{k>i} X_ki^T X_kj -> A_ij
            acc_zero128(acc);
            if (!element<true, false, false, LOWER, FULL, STREAM_BOTH>(S, acc, &fD[i], &fX[i * t + j], Dr(i), Cr(i, j),
                                                                         X, Y))
                return;
            for (int k = i + 1; k < t; ++k)
                if (!element<true, false, false, FULL, FULL, STREAM_BOTH>(S, acc, &fX[k * t + i], &fX[k * t + j],
                                                                            Cr(k, i), Cr(k, j), X, Y))
                    return;
            fence_proxy_async_shared();
            cta_sync();
            acc_store128(acc, X);
            cta_sync();
            store_A128(p, i, j, X, false);
        } else if (kind == K_S3_DIAG) {
            // X_ii^T X_ii + sum_{k>i} X_ki^T X_ki (lower part) -> A_ii
            acc_zero128(acc);
            if (!element<true, false, false, LOWER, LOWER, SAME_SLAB>(S, acc, &fD[i], nullptr, Dr(i), none, X, Y))
                return;
            for (int k = i + 1; k < t; ++k)
                if (!element<true, false, false, FULL, FULL, SAME_SLAB>(S, acc, &fX[k * t + i], nullptr, Cr(k, i), none,
                                                                          X, Y))
                    return;
            fence_proxy_async_shared();
            cta_sync();
            acc_store128(acc, X);
            cta_sync();
            store_A128(p, i, i, X, true);
        } else {  // no other kind in the plan of the whole inversion
            if (threadIdx.x == 0) raise_error(p.ctrl, SPDINV_ERR_UNSUPPORTED);
            return;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode128() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &ptr, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// A store of `tiles` tile-major 128 x 128 FP64 tiles as a 2-D tensor (x = row
// in the tile, y = tile * 128 + column), with box bx x by.
bool store_map(CUtensorMap* m, const double* base, int64_t tiles, int bx, int by) {
    auto fn = encode128();
    if (!fn || tiles < 1) return false;
    cuuint64_t dims[2] = {(cuuint64_t)TB, (cuuint64_t)(tiles * TB)};
    cuuint64_t strides[1] = {(cuuint64_t)(TB * sizeof(double))};
    cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_potri_fp64_b128(const KParamsF64& p, int num_sms, cudaStream_t s, int* grid_out) {
    if (p.b != TB || p.steps != STEPS_ALL) return cudaErrorInvalidValue;
    const int64_t ntri = (int64_t)p.t * (p.t - 1) / 2;
    // With one tile row there are no off-diagonal tiles: the B and C maps
    // then cover D (valid, never read).
    const double* bw = ntri ? p.Bw : p.Dw;
    const double* cw = ntri ? p.Cw : p.Dw;
    const int64_t nb = ntri ? ntri : p.t;
    Maps128 mp;
    if (!store_map(&mp.b_col, bw, nb, TB, KS) || !store_map(&mp.b_row, bw, nb, KS, TB) ||
        !store_map(&mp.c_col, cw, nb, TB, KS) || !store_map(&mp.c_row, cw, nb, KS, TB) ||
        !store_map(&mp.d_col, p.Dw, p.t, TB, KS) || !store_map(&mp.d_row, p.Dw, p.t, KS, TB))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(potri_fp64_b128, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM128);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, potri_fp64_b128, NT, SMEM128);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int grid = num_sms * occ;
    if (grid > p.ntasks) grid = p.ntasks > 0 ? p.ntasks : 1;
    *grid_out = grid;
    potri_fp64_b128<<<grid, NT, SMEM128, s>>>(mp, p);
    return cudaGetLastError();
}

}  // namespace spdinv
