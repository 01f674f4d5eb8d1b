// The slice products of the emulated FP64 residual (residual_ozaki.cu) on the
// fifth-generation tensor cores: tcgen05.mma (BF16 in, FP32 accumulator in
// tensor memory), operands staged by TMA with 128-byte swizzle.
//
// One CTA computes a 128 x 128 tile of R = I - A X over all slice pairs:
//   warp 0    TMA producer: 64-deep K slices of A's and X's slice planes into
//             a 4-stage shared-memory ring;
//   warp 1    allocates 256 tensor-memory columns (two 128-column FP32
//             accumulators) and issues the MMAs from one thread: 4 stages =
//             one exact 256-deep chunk per accumulator, then a commit;
//   warps 2-9 epilogue: each thread owns half of one accumulator row (its
//             warp's lane quarter, 64 columns), reads a finished chunk with
//             tcgen05.ld, adds the exact FP32 integers into INT32 registers,
//             releases the accumulator, and at the end of a slice pair adds
//             -2^{e_i + f_j - 8(s+t+2)} * sum into R (FP64, global).
// Every wait is bounded; on a timeout the CTA records an error, all roles
// leave their loops, and the tensor memory is freed before exit.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "api_internal.h"
#include "ozaki.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

constexpr int TM = 128, TN = 128, TK = 64;  // output tile; K per stage = one 128-byte swizzle row of bf16
constexpr int NSTAGE = 4;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int CHUNK_STAGES = 256 / TK;  // exact FP32 chunk: 256 products of 8-bit slices
constexpr int FLUSH_CHUNKS = 128;       // INT32 headroom: 128 chunks x 256 x 255^2 < 2^31
constexpr int TMEM_COLS = 256;          // two 128-column FP32 accumulators
constexpr int NTHREADS = 320;          // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int EPI_COLS = TN / 2;        // columns per epilogue thread (two warps per lane quarter)
constexpr uint32_t IDESC = (1u << 4)                        // D: FP32
                           | (1u << 7) | (1u << 10)          // A, B: BF16
                           | ((uint32_t)(TN >> 3) << 17)     // N / 8
                           | ((uint32_t)(TM >> 4) << 24);    // M / 16 (both operands K-major)

struct TcParams {
    int64_t n, npad;
    int npairs;
    int ps[64], pt[64];
    const int* e;
    const int* f;
    double* R;
    int* err;
    long long timeout_ns;
};

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bounded wait that ignores the abort flag (used while draining in-flight work).
__device__ __forceinline__ void drain_bar(uint64_t* bar, uint32_t parity, long long limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if ((long long)(globaltimer_ns() - t0) > limit_ns) return;
}

// Bounded parity wait on an mbarrier; false = gave up (abort or timeout).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* s_abort, const TcParams& p) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*s_abort) return false;
        if ((long long)(globaltimer_ns() - t0) > p.timeout_ns) {
            *s_abort = 1;
            atomicCAS(p.err, 0, SPDINV_ERR_TIMEOUT);
            return false;
        }
    }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const TcParams p) {
    unsigned char* smem = dynamic_smem();  // 1024-byte aligned (swizzled operand tiles)
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int s_f[TN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * TN;
    const int kstages = (int)(p.npad / TK);            // stages per slice pair
    const int chunks_per_pair = kstages / CHUNK_STAGES;
    const int total_stages = p.npairs * kstages;
    const int total_chunks = p.npairs * chunks_per_pair;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 8);  // one arrival per epilogue warp
        }
        mbar_init(&fin, 1);
        s_abort = 0;
        fence_proxy_async_shared();
    }
    for (int j = threadIdx.x; j < TN; j += NTHREADS) s_f[j] = (n0 + j < p.n) ? p.f[n0 + j] : 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer
            int it = 0;
            for (; it < total_stages; ++it) {
                const int s = it % NSTAGE;
                if (!wait_bar(&empty[s], ((it / NSTAGE) & 1) ^ 1, &s_abort, p)) break;
                const int pair = it / kstages, kt = it - pair * kstages;
                unsigned char* st = smem + s * STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(st, &tmA, kt * TK, (int)(p.ps[pair] * p.npad + m0), &full[s]);
                tma_load_2d(st + A_BYTES, &tmB, kt * TK, (int)(p.pt[pair] * p.npad + n0), &full[s]);
            }
            if (s_abort)  // let the copies already issued land before the CTA leaves
                for (int k = it - NSTAGE > 0 ? it - NSTAGE : 0; k < it; ++k)
                    drain_bar(&full[k % NSTAGE], (k / NSTAGE) & 1, 200000000LL);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            int it = 0;
            for (int c = 0; c < total_chunks && !s_abort; ++c) {
                const int b = c & 1;
                if (!wait_bar(&acce[b], ((c >> 1) & 1) ^ 1, &s_abort, p)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * TN);
                bool ok = true;
                for (int q = 0; q < CHUNK_STAGES; ++q, ++it) {
                    const int s = it % NSTAGE;
                    if (!wait_bar(&full[s], (it / NSTAGE) & 1, &s_abort, p)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                    const uint64_t da = sdesc_sw128(sa), db = sdesc_sw128(sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < TK / 16; ++k)  // +32 bytes per K=16 inside the swizzle row
                        umma_bf16(d, da + 2 * k, db + 2 * k, (q | k) != 0);
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accf[b]);
            }
            umma_commit(&fin);  // every MMA issued above has completed when this arrives
            drain_bar(&fin, 0, 2000000000LL);
        }
    } else {  // ---- epilogue: warps 2..9, half an accumulator row per thread
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int64_t i = m0 + row;
        const int ei = (i < p.n) ? p.e[i] : 0;
        int acc[EPI_COLS];
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) acc[j] = 0;
        bool first_flush = true;
        int pair = 0, cin = 0;  // chunk index within the pair
        for (int c = 0; c < total_chunks; ++c) {
            const int b = c & 1;
            if (!wait_bar(&accf[b], (c >> 1) & 1, &s_abort, p)) break;
            tc_fence_after();
#pragma unroll
            for (int cb = 0; cb < EPI_COLS / 32; ++cb) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TN + half * EPI_COLS + cb * 32), r);
#pragma unroll
                for (int u = 0; u < 32; ++u) acc[cb * 32 + u] += __float2int_rn(__uint_as_float(r[u]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
            ++cin;
            const bool pair_end = cin == chunks_per_pair;
            if (pair_end || (cin % FLUSH_CHUNKS) == 0) {
                const int lvl = 8 * (p.ps[pair] + p.pt[pair] + 2);
#pragma unroll
                for (int j = 0; j < EPI_COLS; ++j) {
                    const int64_t jj = n0 + half * EPI_COLS + j;
                    if (i < p.n && jj < p.n) {
                        double* dst = &p.R[i + jj * p.n];
                        const double v = scalbn((double)acc[j], ei + s_f[half * EPI_COLS + j] - lvl);
                        *dst = (first_flush ? (i == jj ? 1.0 : 0.0) : *dst) - v;
                    }
                    acc[j] = 0;
                }
                first_flush = false;
            }
            if (pair_end) {
                ++pair;
                cin = 0;
            }
        }
    }
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 2D map over S slice planes stacked as (S*npad) rows of npad bf16, box 64 x 128.
bool make_map(CUtensorMap* m, const void* base, int64_t npad, int S) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)(S * npad)};
    cuuint64_t strides[1] = {(cuuint64_t)(npad * 2)};
    cuuint32_t box[2] = {(cuuint32_t)TK, 128u};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t ozaki_products_tc(int64_t n, int64_t npad, const void* Asl, const void* Xsl, int S, const int* ps,
                              const int* pt, int npairs, const int* e, const int* f, double* R, int* err,
                              cudaStream_t s) {
    if (npad % TM != 0 || npad % 256 != 0 || npairs > 64) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, Asl, npad, S) || !make_map(&mb, Xsl, npad, S)) return cudaErrorInvalidValue;
    TcParams p{};
    p.n = n;
    p.npad = npad;
    p.npairs = npairs;
    for (int q = 0; q < npairs; ++q) {
        p.ps[q] = ps[q];
        p.pt[q] = pt[q];
    }
    p.e = e;
    p.f = f;
    p.R = R;
    p.err = err;
    p.timeout_ns = 20LL * 1000000000LL;
    const int sm = NSTAGE * STAGE_BYTES;
    cudaError_t rc = cudaFuncSetAttribute(ozaki_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (rc != cudaSuccess) return rc;
    ozaki_tc_kernel<<<dim3((unsigned)(npad / TN), (unsigned)(npad / TM)), NTHREADS, sm, s>>>(ma, mb, p);
    return cudaGetLastError();
}

}  // namespace spdinv
