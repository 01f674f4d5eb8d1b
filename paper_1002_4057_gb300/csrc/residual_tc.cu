// The slice products of the emulated FP64 residual (residual_ozaki.cu; the
// error-free splitting of Ozaki, Ogita, Oishi and Rump 2012) on the
// fifth-generation tensor cores: tcgen05.mma (BF16 in, FP32 accumulator in
// tensor memory), operands staged by TMA with 128-byte swizzle.  One CTA
// computes one output tile of R = I - A X (or of a correction term X R^m)
// over all slice pairs.  Two forms:
//
// ozaki_tc_wide (the default): a 128 x 256 tile, 320 threads, 1 CTA per SM.
//   warp 0    TMA producer: per stage one 3-D box of an A-slice plane
//             (128 rows x one 64-deep atom, 16 KB) and one of an X-slice
//             plane (256 rows, 32 KB) into a 4-stage ring;
//   warp 1    allocates the 512 tensor-memory columns and issues the MMAs
//             (M = 128, N = 256) from one thread into one 256-column FP32
//             accumulator, committing at the end of each exact 1024-deep
//             chunk;
//   warps 2-9 epilogue: per chunk each thread loads its half of an
//             accumulator row (128 values) into registers and releases the
//             accumulator at once, then adds the exact FP32 integers into
//             INT32 level sums kept in tensor-memory columns 256-511; per level
//             s + t -- all its pairs share the scale 2^{e_i + f_j - 8(s+t+2)}
//             -- it adds the level once into R (FP64, global), so the FP64
//             work, slow on this chip, happens once per level per tile.
// ozaki_tc_kernel (SPDINV_SLICE_TILE=128): a 128 x 128 tile, two 64-deep atoms
//   per stage and operand, 3 stages, two alternating 128-column accumulators
//   and INT64 level sums; it wins only where too few 128 x 256 tiles exist to
//   fill the GPU.
// Both visit the tiles in a grouped raster (block_of, block_of_wide), replayed
// on the host by spdinv_slice_tile_order.  Every wait is bounded; on a timeout
// the CTA records an error, all roles leave their loops, and the tensor memory
// is freed before exit.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "api_internal.h"
#include "ozaki.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

constexpr int TM = 128, TN = 128;
constexpr int ATOM = 64;                 // K entries of one 128-byte swizzle row of bf16
constexpr int ATOMS = 2;                 // atoms per stage: one 3-D TMA operation per operand
constexpr int TK = ATOM * ATOMS;         // K per stage
constexpr int NSTAGE = 3;                // 192 KB of copies in flight
constexpr int ATOM_BYTES = TM * ATOM * 2;  // one 128-row atom tile, 16 KB
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int CHUNK_STAGES = 1024 / TK;  // exact FP32 chunk: 1024 products of balanced 8-bit digits (<= 2^24)
constexpr int TMEM_COLS = 512;          // two 128-column FP32 accumulators + INT64 level sums (256 columns)
constexpr int LVL_COL = 256;            // first tensor-memory column of the INT64 level sums
constexpr int NTHREADS = 320;          // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int EPI_WARPS = 8;
constexpr int EPI_COLS = TN / 2;        // columns per epilogue thread (two warps per lane quarter)
constexpr uint32_t IDESC = (1u << 4)                        // D: FP32
                           | (1u << 7) | (1u << 10)          // A, B: BF16
                           | ((uint32_t)(TN >> 3) << 17)     // N / 8
                           | ((uint32_t)(TM >> 4) << 24);    // M / 16 (both operands K-major)

struct TcParams {
    int64_t n, npad;
    int npairs;
    int tiles;            // tiles per side
    int lower;            // 1: only the output tiles on and below the diagonal (symmetric products)
    int identity;         // with base == nullptr: 1 = start from the identity, 0 = from zero
    const double* base;   // output = base + sign * A X   (base == nullptr: identity or zero)
    double sign;
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

// One TMA operation: a box of ATOMS atoms x 128 rows x 64 entries of the
// atom-major slice planes (x: entry, y: row, z: plane * (npad / 64) + atom),
// landing as ATOMS consecutive 16 KB swizzled atom tiles.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(z), "r"(smem_u32(bar))
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

// 2^x as a double, exactly, for |x| < 1022.
__device__ __forceinline__ double pow2(int x) { return __longlong_as_double((long long)(x + 1023) << 52); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// After tmem_wait_ld: marks the 32 registers of an earlier tmem load as
// written here, so that no use of them is scheduled above the wait.
__device__ __forceinline__ void reg_fence32(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

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
    reg_fence32(r);
}

// The same load without its wait: several loads in flight, then one wait.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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

// Tile (bm, bn) of a tb_m x tb_n tile grid for launch index `pid`, in a
// grouped raster: GROUP tile rows are swept column by column, so the CTAs
// resident at one time share both operands' slices in L2.  With `lower`
// only the tiles with bm >= bn (tb_m == tb_n): in the group of rows
// [first, first + gm), column c holds the rows r >= c.
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

template <int GROUP>
__host__ __device__ __forceinline__ void block_of(int pid, int tb_m, int tb_n, bool lower, int& bm, int& bn) {
    if (!lower) {
        const int per_group = GROUP * tb_n;
        const int first = (pid / per_group) * GROUP;
        const int gm = imin(tb_m - first, GROUP);
        bm = first + (pid % per_group) % gm;
        bn = (pid % per_group) / gm;
        return;
    }
    int first = 0;
    for (;;) {
        const int gm = imin(tb_m - first, GROUP);
        const int cnt = first * gm + gm * (gm + 1) / 2;
        if (pid < cnt || first + gm >= tb_m) break;
        pid -= cnt;
        first += gm;
    }
    const int gm = imin(tb_m - first, GROUP);
    if (pid < first * gm) {
        bn = pid / gm;
        bm = first + pid % gm;
    } else {
        pid -= first * gm;
        int c = 0;
        while (pid >= gm - c) {
            pid -= gm - c;
            ++c;
        }
        bn = first + c;
        bm = bn + pid;
    }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ TcParams p) {
    unsigned char* smem = dynamic_smem();  // 1024-byte aligned (swizzled operand tiles)
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ int s_f[TN];
    __shared__ int s_za[64], s_zb[64];  // per pair: first atom plane of the A and X slices
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tile_m, tile_n;
    block_of<16>((int)blockIdx.x, p.tiles, p.tiles, p.lower != 0, tile_m, tile_n);
    const int64_t m0 = (int64_t)tile_m * TM, n0 = (int64_t)tile_n * TN;
    const int kstages = (int)(p.npad / TK);            // stages per slice pair
    const int chunks_per_pair = (kstages + CHUNK_STAGES - 1) / CHUNK_STAGES;  // the last one may be shorter
    const int total_stages = p.npairs * kstages;
    const int total_chunks = p.npairs * chunks_per_pair;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], EPI_WARPS);  // one arrival per epilogue warp
        }
        mbar_init(&fin, 1);
        s_abort = 0;
        fence_proxy_async_shared();
    }
    for (int j = threadIdx.x; j < TN; j += NTHREADS) s_f[j] = (n0 + j < p.n) ? p.f[n0 + j] : 0;
    for (int q = threadIdx.x; q < p.npairs; q += NTHREADS) {
        s_za[q] = (int)(p.ps[q] * (p.npad / ATOM));
        s_zb[q] = (int)(p.pt[q] * (p.npad / ATOM));
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
            for (; it < total_stages; ++it) {
                const int s = it % NSTAGE;
                if (!wait_bar(&empty[s], ((it / NSTAGE) & 1) ^ 1, &s_abort, p)) break;
                const int pair = it / kstages, kt = it - pair * kstages;
                unsigned char* st = smem + s * STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tma_load_3d(st, &tmA, (int)m0, s_za[pair] + kt * ATOMS, &full[s]);
                tma_load_3d(st + A_BYTES, &tmB, (int)n0, s_zb[pair] + kt * ATOMS, &full[s]);
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
                const int q0 = (c % chunks_per_pair) * CHUNK_STAGES;
                const int nq = min(CHUNK_STAGES, kstages - q0);
                bool ok = true;
                for (int q = 0; q < nq; ++q, ++it) {
                    const int s = it % NSTAGE;
                    if (!wait_bar(&full[s], (it / NSTAGE) & 1, &s_abort, p)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                    for (int a = 0; a < ATOMS; ++a) {  // each atom: a 128-row swizzled tile of 64 entries
                        const uint64_t da = sdesc_sw128(sa + a * ATOM_BYTES);
                        const uint64_t db = sdesc_sw128(sa + A_BYTES + a * ATOM_BYTES);
#pragma unroll
                        for (int k = 0; k < ATOM / 16; ++k)  // +32 bytes per K=16 inside the swizzle row
                            umma_bf16(d, da + 2 * k, db + 2 * k, (q | a | k) != 0);
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accf[b]);
            }
            umma_commit(&fin);  // every MMA issued above has completed when this arrives
            drain_bar(&fin, 0, 2000000000LL);
        }
    } else {  // ---- epilogue: warps 2..17, a quarter of an accumulator row per thread
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;  // which 32-column part of the row
        const int row = quarter * 32 + lane;
        const int64_t i = m0 + row;
        const int ei = (i < p.n) ? p.e[i] : 0;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t tlvl = trow + (uint32_t)(LVL_COL + half * 2 * EPI_COLS);  // this thread's INT64 sums
        int acc[EPI_COLS];
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) acc[j] = 0;
        bool first_flush = true, level_start = true;
        int pair = 0, cin = 0;  // chunk index within the pair
        for (int c = 0; c < total_chunks; ++c) {
            const int b = c & 1;
            if (!wait_bar(&accf[b], (c >> 1) & 1, &s_abort, p)) break;
            tc_fence_after();
            {  // both 32-column loads in flight, one wait; the sums are exact integers <= 2^24
                uint32_t r0[32], r1[32];
                tmem_ld32_async(trow + (uint32_t)(b * TN + half * EPI_COLS), r0);
                tmem_ld32_async(trow + (uint32_t)(b * TN + half * EPI_COLS + 32), r1);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    acc[u] += __float2int_rn(__uint_as_float(r0[u]));
                    acc[32 + u] += __float2int_rn(__uint_as_float(r1[u]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
            if (++cin < chunks_per_pair) continue;
            // ---- end of a slice pair: INT32 pair sums into the INT64 level sums
            cin = 0;
            const int lv = p.ps[pair] + p.pt[pair];
            ++pair;
            const bool level_end = !(pair < p.npairs && p.ps[pair] + p.pt[pair] == lv);
#pragma unroll
            for (int g = 0; g < EPI_COLS / 8; ++g) {  // 8 INT64 values = 16 columns per step
                uint32_t r[16];
                if (!level_start) tmem_ld16(tlvl + (uint32_t)(g * 16), r);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    long long v = level_start ? 0ll
                                              : (long long)(((unsigned long long)r[2 * u + 1] << 32) | r[2 * u]);
                    v += (long long)acc[g * 8 + u];
                    acc[g * 8 + u] = 0;
                    r[2 * u] = (uint32_t)(unsigned long long)v;
                    r[2 * u + 1] = (uint32_t)((unsigned long long)v >> 32);
                }
                tmem_st16(tlvl + (uint32_t)(g * 16), r);
            }
            level_start = level_end;
            if (!level_end) continue;
            // ---- end of a level: R -= 2^{e_i + f_j - 8(lv+2)} * sum (exact scale, one FMA per entry)
            const double ri = pow2(ei - 8 * (lv + 2));
#pragma unroll 1
            for (int g = 0; g < EPI_COLS / 16; ++g) {
                uint32_t r[32];
                tmem_ld32(tlvl + (uint32_t)(g * 32), r);
                if (i >= p.n) continue;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const long long v = (long long)(((unsigned long long)r[2 * u + 1] << 32) | r[2 * u]);
                    const int j = half * EPI_COLS + g * 16 + u;
                    const int64_t jj = n0 + j;
                    if (jj < p.n) {
                        double* dst = &p.R[i + jj * p.n];
                        const double base =
                            first_flush ? (p.base ? p.base[i + jj * p.n] : (p.identity && i == jj ? 1.0 : 0.0))
                                        : *dst;
                        *dst = fma(p.sign * (double)v, ri * pow2(s_f[j]), base);
                    }
                }
            }
            first_flush = false;
        }
    }
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}


// ---- the wide form: 128 x 256 output tiles ---------------------------------
// Per flop of MMA work it brings three quarters of the operand bytes of the
// 128 x 128 tile: with about 190 KB of copies in flight per SM and the copy
// latency under load, that, not the tensor pipe, sets the rate.  The FP32
// accumulator (256 columns) is single-buffered and the INT32 level sums take
// the other 256 tensor-memory columns; while the epilogue drains a chunk the
// copies keep filling the ring.
constexpr int WN = 256;                        // output columns per tile
constexpr int W_NSTAGE = 4;                    // 4 x 48 KB of copies in flight
constexpr int WA_BYTES = TM * ATOM * 2;        // 16 KB: A, 128 rows x one atom
constexpr int WB_BYTES = WN * ATOM * 2;        // 32 KB: X, 256 rows x one atom
constexpr int W_STAGE = WA_BYTES + WB_BYTES;
constexpr int W_CHUNK = 1024 / ATOM;           // stages per exact 1024-deep chunk
constexpr int W_LVL = 256;                     // tensor-memory column of the INT32 level sums
constexpr int W_COLS = WN / 2;                 // columns per epilogue thread
constexpr uint32_t IDESC_W = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(WN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void umma_bf16_w(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC_W), "r"(accumulate));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Tile (bm, bn) of launch index pid: 128-row block bm, 256-column block bn.
// The full grid sweeps groups of 8 row blocks column by column (at n = 16384
// groups of 8 measured 4 % faster than 16; 4, 12, 32 and 64 were slower).
// lower: only tiles holding an entry on or below the diagonal, bn <= bm / 2,
// in groups of 16 row blocks (8 measured the same), so the CTAs resident at
// one time share the column blocks of X's slices in L2.  In the group of rows [first, first + gm), column bn holds the
// rows max(first, 2 bn) .. first + gm - 1.  (tb_m is even: npad is a multiple
// of 256.)
__host__ __device__ __forceinline__ int lower_group_tiles(int first, int gm) {
    const int h = (first + gm - 1) / 2, f2 = first / 2;  // last column; last full column
    int cnt = (imin(f2, h) + 1) * gm;
    if (h > f2) cnt += (h - f2) * (first + gm) - (h * (h + 1) - f2 * (f2 + 1));
    return cnt;
}
__host__ __device__ __forceinline__ void block_of_wide(int pid, int tb_m, int tb_n, bool lower, int& bm, int& bn) {
    if (!lower) {
        block_of<8>(pid, tb_m, tb_n, false, bm, bn);
        return;
    }
    constexpr int GROUP = 16;
    int first = 0, gm = imin(tb_m, GROUP);
    for (;;) {
        gm = imin(tb_m - first, GROUP);
        const int cnt = lower_group_tiles(first, gm);
        if (pid < cnt || first + gm >= tb_m) break;
        pid -= cnt;
        first += gm;
    }
    for (bn = 0; bn <= (first + gm - 1) / 2; ++bn) {
        const int lo = imax(first, 2 * bn), c = first + gm - lo;
        if (pid < c) {
            bm = lo + pid;
            return;
        }
        pid -= c;
    }
    bm = tb_m;  // past the last tile (the launch has exactly as many CTAs as tiles)
}

__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_tc_wide(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ TcParams p) {
    unsigned char* smem = dynamic_smem();  // 1024-byte aligned (swizzled operand tiles)
    __shared__ __align__(8) uint64_t full[W_NSTAGE], empty[W_NSTAGE], accf, acce, fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb_m = (int)(p.npad / TM), tb_n = (int)(p.npad / WN);
    int tile_m, tile_n;
    block_of_wide((int)blockIdx.x, tb_m, tb_n, p.lower != 0, tile_m, tile_n);
    if (tile_m >= tb_m) return;
    const int64_t m0 = (int64_t)tile_m * TM, n0 = (int64_t)tile_n * WN;
    const int kstages = (int)(p.npad / ATOM);  // stages per slice pair
    const int chunks_per_pair = (kstages + W_CHUNK - 1) / W_CHUNK;
    const int total_stages = p.npairs * kstages;
    const int total_chunks = p.npairs * chunks_per_pair;
    const int zpl = (int)(p.npad / ATOM);  // atom planes per slice plane

    if (threadIdx.x == 0) {
        for (int s = 0; s < W_NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accf, 1);
        mbar_init(&acce, EPI_WARPS);
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
        if (lane == 0) {  // ---- TMA producer: one atom of A (128 rows) and of X (256 rows) per stage
            int it = 0;
            for (; it < total_stages; ++it) {
                const int s = it % W_NSTAGE;
                if (!wait_bar(&empty[s], ((it / W_NSTAGE) & 1) ^ 1, &s_abort, p)) break;
                const int pair = it / kstages, kt = it - pair * kstages;
                unsigned char* st = smem + s * W_STAGE;
                mbar_arrive_expect_tx(&full[s], W_STAGE);
                tma_load_3d(st, &tmA, (int)m0, p.ps[pair] * zpl + kt, &full[s]);
                tma_load_3d(st + WA_BYTES, &tmB, (int)n0, p.pt[pair] * zpl + kt, &full[s]);
            }
            if (s_abort)
                for (int k = it - W_NSTAGE > 0 ? it - W_NSTAGE : 0; k < it; ++k)
                    drain_bar(&full[k % W_NSTAGE], (k / W_NSTAGE) & 1, 200000000LL);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer: one chunk at a time into the single accumulator
            int it = 0;
            for (int c = 0; c < total_chunks && !s_abort; ++c) {
                if (!wait_bar(&acce, (c & 1) ^ 1, &s_abort, p)) break;  // the epilogue drained chunk c - 1
                tc_fence_after();
                const int q0 = (c % chunks_per_pair) * W_CHUNK;
                const int nq = min(W_CHUNK, kstages - q0);
                bool ok = true;
                for (int q = 0; q < nq; ++q, ++it) {
                    const int s = it % W_NSTAGE;
                    if (!wait_bar(&full[s], (it / W_NSTAGE) & 1, &s_abort, p)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * W_STAGE);
                    const uint64_t da = sdesc_sw128(sa), db = sdesc_sw128(sa + WA_BYTES);
#pragma unroll
                    for (int k = 0; k < ATOM / 16; ++k) umma_bf16_w(tmem, da + 2 * k, db + 2 * k, (q | k) != 0);
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accf);
            }
            umma_commit(&fin);
            drain_bar(&fin, 0, 2000000000LL);
        }
    } else {  // ---- epilogue: warps 2..9, half of a row (128 columns) per thread
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int64_t i = m0 + row;
        const int ei = (i < p.n) ? p.e[i] : 0;
        const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t tacc = trow + (uint32_t)(half * W_COLS);          // this thread's FP32 accumulator
        const uint32_t tsum = trow + (uint32_t)(W_LVL + half * W_COLS);  // and INT32 level sums
        bool first_flush = true, fresh = true;  // fresh: the level sums hold nothing yet
        int pair = 0, cin = 0, since_flush = 0;
        for (int c = 0; c < total_chunks; ++c) {
            if (!wait_bar(&accf, c & 1, &s_abort, p)) break;
            tc_fence_after();
            // The whole chunk (128 values per thread) into registers, then the
            // accumulator goes back to the MMA warp at once: the next chunk's
            // products overlap the level-sum update below.
            uint32_t r[W_COLS / 32][32];
#pragma unroll
            for (int g = 0; g < W_COLS / 32; ++g) tmem_ld32_async(tacc + (uint32_t)(g * 32), r[g]);
            tmem_wait_ld();
#pragma unroll
            for (int g = 0; g < W_COLS / 32; ++g) reg_fence32(r[g]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce);
#pragma unroll
            for (int g = 0; g < W_COLS / 32; ++g) {  // sums += int(chunk), exact: chunk entries are integers <= 2^24
                uint32_t l[32];
                if (!fresh) {
                    tmem_ld32(tsum + (uint32_t)(g * 32), l);
#pragma unroll
                    for (int u = 0; u < 32; ++u) l[u] = (uint32_t)(__float2int_rn(__uint_as_float(r[g][u])) + (int)l[u]);
                } else {
#pragma unroll
                    for (int u = 0; u < 32; ++u) l[u] = (uint32_t)__float2int_rn(__uint_as_float(r[g][u]));
                }
                tmem_st32(tsum + (uint32_t)(g * 32), l);
            }
            fresh = false;
            ++since_flush;
            const int lv = p.ps[pair] + p.pt[pair];
            bool flush = since_flush >= 127;  // INT32 headroom: 127 chunks of at most 2^24
            if (++cin == chunks_per_pair) {
                cin = 0;
                ++pair;
                flush = flush || !(pair < p.npairs && p.ps[pair] + p.pt[pair] == lv);  // end of a level
            }
            if (!flush) continue;
            // R = base + sign 2^{e_i + f_j - 8(lv+2)} * sum (exact scale, one FMA per entry)
            const double ri = pow2(ei - 8 * (lv + 2));
#pragma unroll 1
            for (int g = 0; g < W_COLS / 32; ++g) {
                uint32_t l[32];
                tmem_ld32(tsum + (uint32_t)(g * 32), l);
                if (i >= p.n) continue;
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    const int64_t jj = n0 + half * W_COLS + g * 32 + u;
                    if (jj < p.n) {
                        double* dst = &p.R[i + jj * p.n];
                        const double base =
                            first_flush ? (p.base ? p.base[i + jj * p.n] : (p.identity && i == jj ? 1.0 : 0.0))
                                        : *dst;
                        *dst = fma(p.sign * (double)(int)l[u], ri * pow2(p.f[jj]), base);
                    }
                }
            }
            first_flush = false;
            fresh = true;
            since_flush = 0;
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

// 3-D map over S atom-major slice planes (residual_ozaki.cu): x = entry of
// an atom (64, one 128-byte swizzle row), y = row (npad), z = atom plane
// (S * npad / 64, plane s's atoms from s * npad / 64); box 64 x rows x atoms.
bool make_map(CUtensorMap* m, const void* base, int64_t npad, int S, int rows, int atoms) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)ATOM, (cuuint64_t)npad, (cuuint64_t)(S * (npad / ATOM))};
    cuuint64_t strides[2] = {(cuuint64_t)(ATOM * 2), (cuuint64_t)(npad * ATOM * 2)};
    cuuint32_t box[3] = {(cuuint32_t)ATOM, (cuuint32_t)rows, (cuuint32_t)atoms};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Output tile width of the slice GEMM: 256 (the wide form, default) or 128;
// SPDINV_SLICE_TILE=128|256 in the environment chooses.
// Launch size of the slice GEMM for padded order npad: one CTA per output
// tile, 128 x 256 tiles (wide) or 128 x 128; lower: the tiles holding an entry
// on or below the diagonal.
int slice_grid(int64_t npad, bool lower, bool wide) {
    const int tb_m = (int)(npad / TM);
    if (wide) return lower ? (tb_m / 2) * (tb_m / 2 + 1) : tb_m * (int)(npad / WN);
    return lower ? tb_m * (tb_m + 1) / 2 : tb_m * tb_m;
}

static int slice_tile() {
    static const int v = [] {
        const char* env = std::getenv("SPDINV_SLICE_TILE");
        return (env && std::atoi(env) == 128) ? 128 : 256;
    }();
    return v;
}

cudaError_t ozaki_products_tc(int64_t n, int64_t npad, const void* Asl, int SA, const void* Xsl, int SB,
                              const int* ps, const int* pt, int npairs, const int* e, const int* f, double* R,
                              const double* base, bool identity, double sign, bool lower, int* err, cudaStream_t s) {
    if (npad % 256 != 0 || npairs < 1 || npairs > 64) return cudaErrorInvalidValue;  // whole 256-deep chunks
    for (int q = 0; q < npairs; ++q)  // every pair must address planes that the maps cover
        if (ps[q] < 0 || ps[q] >= SA || pt[q] < 0 || pt[q] >= SB) return cudaErrorInvalidValue;
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
    p.base = base;
    p.identity = identity ? 1 : 0;
    p.sign = sign;
    p.lower = lower ? 1 : 0;
    p.tiles = (int)(npad / TM);
    p.err = err;
    p.timeout_ns = 20LL * 1000000000LL;
    CUtensorMap ma, mb;
    cudaError_t rc;
    void* tok = nullptr;
    if (slice_tile() == 256) {  // 128 x 256 output tiles
        if (!make_map(&ma, Asl, npad, SA, TM, 1) || !make_map(&mb, Xsl, npad, SB, WN, 1)) return cudaErrorInvalidValue;
        const int sm = W_NSTAGE * W_STAGE;
        rc = cudaFuncSetAttribute(ozaki_tc_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (rc != cudaSuccess) return rc;
        const int grid = slice_grid(npad, lower, true);
        timing_begin(SPDINV_TIMED_SLICE_GEMM, s, &tok);
        ozaki_tc_wide<<<(unsigned)grid, NTHREADS, sm, s>>>(ma, mb, p);
        rc = cudaGetLastError();
        timing_end(SPDINV_TIMED_SLICE_GEMM, s, tok, 2.0 * TM * WN * (double)npad * (double)npairs * (double)grid);
        return rc;
    }
    if (!make_map(&ma, Asl, npad, SA, TM, ATOMS) || !make_map(&mb, Xsl, npad, SB, TN, ATOMS))
        return cudaErrorInvalidValue;
    const int sm = NSTAGE * STAGE_BYTES;
    rc = cudaFuncSetAttribute(ozaki_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (rc != cudaSuccess) return rc;
    const int grid = slice_grid(npad, lower, false);
    timing_begin(SPDINV_TIMED_SLICE_GEMM, s, &tok);
    ozaki_tc_kernel<<<(unsigned)grid, NTHREADS, sm, s>>>(ma, mb, p);
    rc = cudaGetLastError();
    timing_end(SPDINV_TIMED_SLICE_GEMM, s, tok, 2.0 * TM * TN * (double)npad * (double)npairs * (double)grid);
    return rc;
}

// Host replay of the slice GEMM's launch order: the output tile (bm, bn) that
// launch index pid takes, from the same functions the kernels call.
int slice_tile_order(int64_t n, bool lower, bool wide, int* bm, int* bn) {
    const int64_t npad = (n + 255) / 256 * 256;
    const int tb_m = (int)(npad / TM);
    const int grid = slice_grid(npad, lower, wide);
    if (bm && bn)
        for (int pid = 0; pid < grid; ++pid) {
            if (wide) block_of_wide(pid, tb_m, (int)(npad / WN), lower, bm[pid], bn[pid]);
            else block_of<16>(pid, tb_m, tb_m, lower, bm[pid], bn[pid]);
        }
    return grid;
}

}  // namespace spdinv

extern "C" SPDINV_API spdinv_status spdinv_slice_tile_order(int64_t n, int lower, int wide, int* bm, int* bn,
                                                            int* count) {
    if (n < 1 || n > (int64_t(1) << 20)) return SPDINV_ERR_N;
    if (!count || (bm == nullptr) != (bn == nullptr)) return SPDINV_ERR_NULL;
    *count = spdinv::slice_tile_order(n, lower != 0, wide != 0, bm, bn);
    return SPDINV_OK;
}
