// FP32 backward of the inversion on the fifth-generation tensor cores (an
// added form; the paper has only the forward method):
//   grad_A = -X sym(G) X,   sym(G) = (G + G^T) / 2,
// as two batched products, each a sum of three TF32 products of split
// operands (3xTF32: lo hi + hi lo + hi hi, the lo lo term dropped) into an
// FP32 accumulator in tensor memory, 128 x 128 output tiles:
//   prep:     Xp = split(X), Gp = split(sym(G)): column-major, leading
//             dimension npad (n rounded up to 128), zero-padded, hi and lo
//             planes.  X and sym(G) are symmetric, so a column is a row and
//             these planes are the K-major operands the MMA reads.
//   phase 0:  Y = X sym(G); the epilogue splits Y and writes it row-major,
//             the K-major A operand of phase 1.
//   phase 1:  grad = -Y X on the tiles on and below the diagonal, each written
//             to (i, j) and, transposed through shared memory, to (j, i); the
//             diagonal tiles are averaged with their transposes, so grad is
//             exactly symmetric.
// Roles in a CTA of 192 threads: warp 0 issues the TMA copies (four 16 KB
// boxes per 32-deep stage: A hi, A lo, B hi, B lo; three stages), warp 1
// allocates 128 tensor-memory columns and issues the MMAs from one thread,
// warps 2-5 read the accumulator (one row per thread) and store.  Every wait
// is bounded; on a timeout the CTA records an error in the workspace word,
// every role leaves its loop, and the tensor memory is freed before exit.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

constexpr int BT = 128;                   // output tile (M = N = 128)
constexpr int KA = 32;                    // K per 128-byte swizzle row of FP32 / TF32
constexpr int NSTAGE = 3;
constexpr int BOX_BYTES = BT * KA * 4;    // 16 KB: 128 rows x 32 entries
constexpr int STAGE_BYTES = 4 * BOX_BYTES;
constexpr int NTHR = 192;                 // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int TMEM_COLS = 128;
constexpr int SLD = BT + 1;               // epilogue staging row stride (floats)
constexpr uint32_t IDESC_TF32 = (1u << 4)                     // D: FP32
                                | (2u << 7) | (2u << 10)       // A, B: TF32
                                | ((uint32_t)(BT >> 3) << 17)  // N / 8
                                | ((uint32_t)(BT >> 4) << 24); // M / 16 (both operands K-major)
static_assert(NSTAGE * STAGE_BYTES >= BT * SLD * 4, "the staging tile reuses the ring");

struct BwdTcParams {
    int64_t n, npad;
    int t;            // tiles per side
    float* Yh;        // phase 0 output planes (row-major Y), phase 1 A operand
    float* Yl;
    float* grad;
    int64_t ldr, sr;
    int* err;
    long long timeout_ns;
};

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

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC_TF32), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this thread's lane, waited for.
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
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// hi = x rounded to TF32 (to nearest, ties away from zero, in integer
// arithmetic), lo = x - hi (exact in FP32; the MMA reads its TF32 part).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
    lo = x - hi;
}

__device__ __forceinline__ void drain(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if ((long long)(globaltimer_ns() - t0) > 200000000LL) return;
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* s_abort, const BwdTcParams& p) {
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

// Xp, Gp (hi, lo): column-major npad x npad per matrix, zero past n; one
// 32 x 32 tile per block, sym(G) through a shared-memory transpose.
__global__ void __launch_bounds__(256) prep_kernel(int64_t n, int64_t npad, const float* X, int64_t ldx, int64_t sx,
                                                   const float* G, int64_t ldg, int64_t sg, float* Xh, float* Xl,
                                                   float* Gh, float* Gl) {
    __shared__ float gt[32][33];
    const int64_t mat = blockIdx.y;
    const int64_t tp = npad / 32;
    const int64_t bi = blockIdx.x % tp, bj = blockIdx.x / tp;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const float* Xm = X + mat * sx;
    const float* Gm = G + mat * sg;
    const int64_t plane = npad * npad * mat;
    for (int c = ty; c < 32; c += 8) {  // G(bj*32 + tx, bi*32 + c) -> gt[tx][c] (the mirrored tile, coalesced)
        const int64_t gr = bj * 32 + tx, gc = bi * 32 + c;
        gt[tx][c] = (gr < n && gc < n) ? Gm[gr + gc * ldg] : 0.f;
    }
    cta_sync();
    for (int c = ty; c < 32; c += 8) {
        const int64_t r = bi * 32 + tx, col = bj * 32 + c;
        const bool in = r < n && col < n;
        const float x = in ? Xm[r + col * ldx] : 0.f;
        const float g = in ? 0.5f * (Gm[r + col * ldg] + gt[c][tx]) : 0.f;
        float h, l;
        split_tf32(x, h, l);
        Xh[plane + col * npad + r] = h;
        Xl[plane + col * npad + r] = l;
        split_tf32(g, h, l);
        Gh[plane + col * npad + r] = h;
        Gl[plane + col * npad + r] = l;
    }
}

// Tile (ti, tj) of launch index pid among the t (t + 1) / 2 tiles with ti >= tj.
__device__ __forceinline__ void lower_tile(int pid, int& ti, int& tj) {
    int r = (int)((sqrt(8.0 * pid + 1.0) - 1.0) / 2.0);
    while ((r + 1) * (r + 2) / 2 <= pid) ++r;
    while (r * (r + 1) / 2 > pid) --r;
    ti = r;
    tj = pid - r * (r + 1) / 2;
}

template <int PHASE>
__global__ void __launch_bounds__(NTHR, 1)
    bwd_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                  const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                  const BwdTcParams p) {
    unsigned char* smem = dynamic_smem();  // 1024-byte aligned
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], accf, fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mat = blockIdx.y;
    int ti, tj;
    if (PHASE == 0) {
        ti = (int)blockIdx.x % p.t;
        tj = (int)blockIdx.x / p.t;
    } else {
        lower_tile((int)blockIdx.x, ti, tj);
    }
    const int rowA = (int)(mat * p.npad + (int64_t)ti * BT), rowB = (int)(mat * p.npad + (int64_t)tj * BT);
    const int ksteps = (int)(p.npad / KA);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accf, 1);
        mbar_init(&fin, 1);
        s_abort = 0;
        fence_proxy_async_shared();
    }
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
            for (; it < ksteps; ++it) {
                const int s = it % NSTAGE;
                if (!wait_bar(&empty[s], ((it / NSTAGE) & 1) ^ 1, &s_abort, p)) break;
                unsigned char* st = smem + s * STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(st, &mAh, it * KA, rowA, &full[s]);
                tma_load_2d(st + BOX_BYTES, &mAl, it * KA, rowA, &full[s]);
                tma_load_2d(st + 2 * BOX_BYTES, &mBh, it * KA, rowB, &full[s]);
                tma_load_2d(st + 3 * BOX_BYTES, &mBl, it * KA, rowB, &full[s]);
            }
            if (s_abort)
                for (int k = it - NSTAGE > 0 ? it - NSTAGE : 0; k < it; ++k) drain(&full[k % NSTAGE], (k / NSTAGE) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            bool ok = true;
            for (int it = 0; it < ksteps; ++it) {
                const int s = it % NSTAGE;
                if (!wait_bar(&full[s], (it / NSTAGE) & 1, &s_abort, p)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint64_t ah = sdesc_sw128(sa), al = sdesc_sw128(sa + BOX_BYTES);
                const uint64_t bh = sdesc_sw128(sa + 2 * BOX_BYTES), bl = sdesc_sw128(sa + 3 * BOX_BYTES);
#pragma unroll
                for (int k = 0; k < KA / 8; ++k) {  // K = 8 per MMA: 32 bytes, +2 in the descriptor
                    umma_tf32(tmem, al + 2 * k, bh + 2 * k, (it | k) != 0);
                    umma_tf32(tmem, ah + 2 * k, bl + 2 * k, 1u);
                    umma_tf32(tmem, ah + 2 * k, bh + 2 * k, 1u);
                }
                umma_commit(&empty[s]);
            }
            if (ok) umma_commit(&accf);
            umma_commit(&fin);  // every MMA issued has finished before the tensor memory is freed
            drain(&fin, 0);
        }
    } else {  // ---- epilogue: warps 2-5, one accumulator row (tensor-memory lane) per thread
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        if (wait_bar(&accf, 0, &s_abort, p)) {
            tc_fence_after();
            if (PHASE == 0) {  // Y row m, split, row-major into the phase 1 operand planes
                const int64_t off = (int64_t)mat * p.npad * p.npad + ((int64_t)ti * BT + row) * p.npad + (int64_t)tj * BT;
                float4* yh = reinterpret_cast<float4*>(p.Yh + off);
                float4* yl = reinterpret_cast<float4*>(p.Yl + off);
#pragma unroll 1
                for (int g = 0; g < BT / 32; ++g) {
                    uint32_t v[32];
                    tmem_ld32(trow + (uint32_t)(g * 32), v);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 h, l;
                        split_tf32(__uint_as_float(v[4 * q + 0]), h.x, l.x);
                        split_tf32(__uint_as_float(v[4 * q + 1]), h.y, l.y);
                        split_tf32(__uint_as_float(v[4 * q + 2]), h.z, l.z);
                        split_tf32(__uint_as_float(v[4 * q + 3]), h.w, l.w);
                        yh[g * 8 + q] = h;
                        yl[g * 8 + q] = l;
                    }
                }
            } else {  // -Y X through a shared staging tile (the ring is idle now)
                float* S = reinterpret_cast<float*>(smem);
#pragma unroll 1
                for (int g = 0; g < BT / 32; ++g) {
                    uint32_t v[32];
                    tmem_ld32(trow + (uint32_t)(g * 32), v);
#pragma unroll
                    for (int u = 0; u < 32; ++u) S[row * SLD + g * 32 + u] = -__uint_as_float(v[u]);
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
                float* R = p.grad + (int64_t)mat * p.sr;
                const int e = threadIdx.x - 64;  // 0 .. 127: a row of the tile
                const int64_t gi = (int64_t)ti * BT + e, gj = (int64_t)tj * BT + e;
#pragma unroll 4
                for (int c = 0; c < BT; ++c) {  // (ti, tj): element (ti*128 + e, tj*128 + c), coalesced in e
                    const int64_t gc = (int64_t)tj * BT + c;
                    if (gi < p.n && gc < p.n)
                        R[gi + gc * p.ldr] = ti == tj ? 0.5f * (S[e * SLD + c] + S[c * SLD + e]) : S[e * SLD + c];
                }
                if (ti != tj) {
#pragma unroll 4
                    for (int c = 0; c < BT; ++c) {  // (tj, ti): element (tj*128 + e, ti*128 + c) = S[c][e]
                        const int64_t gc = (int64_t)ti * BT + c;
                        if (gj < p.n && gc < p.n) R[gj + gc * p.ldr] = S[c * SLD + e];
                    }
                }
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

// 2-D map over `rows` rows of npad FP32 entries (a stack of planes): box of
// 32 entries (one 128-byte swizzle row) x 128 rows.
bool make_map(CUtensorMap* m, const float* base, int64_t npad, int64_t rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(npad * 4)};
    cuuint32_t box[2] = {(cuuint32_t)KA, (cuuint32_t)BT};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcState {
    std::mutex mu;
    void* ws = nullptr;
    size_t bytes = 0;
};

TcState& tc_state(int dev) {
    static std::mutex mu;
    static std::map<int, TcState*> m;
    std::lock_guard<std::mutex> lk(mu);
    auto& s = m[dev];
    if (!s) s = new TcState();
    return *s;
}

}  // namespace

// The FP32 backward on the tensor cores (see the head of this file); the
// argument checks are the caller's (backward.cu).
spdinv_status backward_f32_tc(int batch, int64_t n, const float* dX, int64_t ldx, int64_t sx, const float* dG,
                              int64_t ldg, int64_t sg, float* dGrad, int64_t ldr, int64_t sr, cudaStream_t stream) {
    const int64_t npad = (n + BT - 1) / BT * BT;
    const int64_t t = npad / BT;
    if ((int64_t)batch * npad > 2147483647LL || t * t > 2147483647LL) return SPDINV_ERR_N;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    TcState& st = tc_state(dev);
    std::lock_guard<std::mutex> lk(st.mu);
    const size_t plane = (size_t)npad * npad * batch;  // floats per plane stack
    const size_t need = 6 * plane * sizeof(float) + 256;
    if (need > st.bytes) {
        if (st.ws) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e);
            cudaFree(st.ws);
            st.ws = nullptr;
            st.bytes = 0;
        }
        e = cudaMalloc(&st.ws, need);
        if (e != cudaSuccess) return cuda_fail(e);
        st.bytes = need;
    }
    float* Xh = static_cast<float*>(st.ws);
    float* Xl = Xh + plane;
    float* Gh = Xl + plane;
    float* Gl = Gh + plane;
    float* Yh = Gl + plane;
    float* Yl = Yh + plane;
    int* err = reinterpret_cast<int*>(Yl + plane);
    const int64_t rows = npad * batch;
    CUtensorMap mXh, mXl, mGh, mGl, mYh, mYl;
    if (!make_map(&mXh, Xh, npad, rows) || !make_map(&mXl, Xl, npad, rows) || !make_map(&mGh, Gh, npad, rows) ||
        !make_map(&mGl, Gl, npad, rows) || !make_map(&mYh, Yh, npad, rows) || !make_map(&mYl, Yl, npad, rows))
        return SPDINV_ERR_UNSUPPORTED;
    const int sm = NSTAGE * STAGE_BYTES;
    e = cudaFuncSetAttribute(bwd_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(bwd_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    BwdTcParams p{};
    p.n = n;
    p.npad = npad;
    p.t = (int)t;
    p.Yh = Yh;
    p.Yl = Yl;
    p.grad = dGrad;
    p.ldr = ldr;
    p.sr = sr;
    p.err = err;
    p.timeout_ns = 20LL * 1000000000LL;
    const int64_t tp = npad / 32;
    prep_kernel<<<dim3((unsigned)(tp * tp), (unsigned)batch), dim3(32, 8), 0, stream>>>(n, npad, dX, ldx, sx, dG, ldg,
                                                                                       sg, Xh, Xl, Gh, Gl);
    bwd_tc_kernel<0><<<dim3((unsigned)(t * t), (unsigned)batch), NTHR, sm, stream>>>(mXh, mXl, mGh, mGl, p);
    bwd_tc_kernel<1><<<dim3((unsigned)(t * (t + 1) / 2), (unsigned)batch), NTHR, sm, stream>>>(mYh, mYl, mXh, mXl, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(3);
    return SPDINV_OK;
}

}  // namespace spdinv
