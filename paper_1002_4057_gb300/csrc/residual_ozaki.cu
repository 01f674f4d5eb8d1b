// FP64-accurate residual R = I - A X on the BF16 tensor cores (an added form
// used by the mixed-precision inversion; the paper has none).
//
// Method (error-free splitting of the operands into small integer slices,
// after Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)):
//   * every row i of A (symmetric, read from its lower triangle) is scaled by
//     2^-e_i with 2^e_i > 2 max_k |A_ik|, every column j of X by 2^-f_j;
//   * each scaled entry u in (-1/2, 1/2) is cut into S balanced digits of
//     base 256, u = sum_s a_s 2^{-8(s+1)} + rest with a_s = round(256 u_s),
//     integers in [-128, 128] -- exact in BF16 (8 significant bits);
//   * for a slice pair (s, t) the product sum_k a_s(i,k) x_t(k,j) has terms
//     of at most 2^14 and is exact in FP32 over k-chunks of up to 1024
//     (<= 2^24); chunks are added exactly in INT32, and into R in FP64 with
//     the pair's scale 2^{e_i + f_j - 8(s+t+2)};
//   * pairs with s + t > L are dropped.  Rows are scaled by their largest
//     entry, so smaller entries keep fewer bits.  S = 7 with L = 6 (28 pairs)
//     leaves an error of about 1e-15 relative to |A| |X|, enough for every
//     correction step but the last; L = 7 (34 pairs) brings it to about
//     1e-16, the accuracy of the native FP64 product, which the last step
//     needs because its residual error stays in the result.
// The slice products run on the tcgen05 tensor cores (residual_tc.cu) or, as
// the comparison path, on mma.sync m16n8k16 here (BF16 in, FP32 out, fed from
// shared memory by cp.async and ldmatrix).  This file also holds the slicing
// kernels and the order-p correction step built on them (ozaki_refine_step).
// The mma.sync path adds each flush of its INT32 chunk sums into R in FP64;
// the tcgen05 path first sums each level's pairs exactly in INT64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "api_internal.h"
#include "ozaki.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

constexpr int BM = 128, BN = 64, BK = 32, STAGES = 4, THREADS = 256;
constexpr int LDS = BK + 8;  // shared row stride (bf16): 80 bytes, conflict-free ldmatrix
constexpr int CHUNK_TILES = 256 / BK;  // exact FP32 sums of 8-bit slice products
constexpr int FLUSH_TILES = 128 * CHUNK_TILES;  // INT32 headroom: 128 chunks of 256 x 128^2 = 2^29

// Layout of a slice plane (npad x npad BF16 digits of one slice): "atom
// major" -- for each 64-deep K atom (one 128-byte row of the tensor cores'
// swizzled operand tiles), the atom's 64 entries of every row, row after row.
// Element (row r, k) of a plane sits at (k / 64 * npad + r) * 64 + k % 64, so
// the tensor-core path fetches a 128-row tile two atoms deep (32 KB) with one
// 3-D TMA operation.
__device__ __forceinline__ int64_t plane_index(int64_t npad, int64_t r, int64_t k) {
    return ((k >> 6) * npad + r) * 64 + (k & 63);
}

// Positive doubles order like their bit patterns, so the maxima are kept as
// 64-bit integers updated with atomicMax.
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// Largest |value| of each row of the symmetric A (lower triangle given):
// every lower tile contributes its row maxima and, through the mirror, its
// column maxima (the diagonal tiles' columns hold the rows' upper entries).
__global__ void row_absmax_kernel(int64_t n, const double* A, int64_t lda, unsigned long long* rowmax) {
    __shared__ double cm[32][33];
    const int64_t ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int c = ty; c < 32; c += 8) {
        const int64_t gr = ti * 32 + tx, gc = tj * 32 + c;
        cm[c][tx] = (gr < n && gc < n && gr >= gc) ? fabs(A[gr + gc * lda]) : 0.0;
    }
    cta_sync();
    if (ty == 0) {
        double m = 0.0;
        for (int c = 0; c < 32; ++c) m = fmax(m, cm[c][tx]);
        const int64_t gr = ti * 32 + tx;
        if (gr < n && m > 0.0) atomicMax(&rowmax[gr], dbits(m));
    } else if (ty == 1) {
        double m = 0.0;
        for (int r = 0; r < 32; ++r) m = fmax(m, cm[tx][r]);
        const int64_t gc = tj * 32 + tx;
        if (gc < n && m > 0.0) atomicMax(&rowmax[gc], dbits(m));
    }
}

// Largest |value| of each column of the full matrix X (ld n).
__global__ void col_absmax_kernel(int64_t n, const double* X, unsigned long long* colmax) {
    const int64_t j = blockIdx.x;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(X[i + j * n]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double wmx[32];
    if ((threadIdx.x & 31) == 0) wmx[threadIdx.x >> 5] = m;
    cta_sync();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, wmx[w]);
        colmax[j] = dbits(r);
    }
}

// Exponent e with 2^e > 2 m (m = 0 -> 0).
__global__ void exponents_kernel(int64_t n, const unsigned long long* maxbits, int* expo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = __longlong_as_double((long long)maxbits[i]);
        int e = 0;
        if (m > 0.0) {
            frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
            ++e;
        }
        expo[i] = e;
    }
}

// The S balanced base-256 digits of u = v 2^-e in (-1/2, 1/2), in integer
// arithmetic: W = u 2^(8S), rounded to the nearest integer (half away from
// zero), is formed from v's exponent and 53-bit significand by one shift; its
// digits are then peeled from the least significant end, each the residue of
// W mod 256 taken in [-128, 127], and the top digit is what remains, in
// [-128, 128] because |W| <= 2^(8S-1).  The digits sum to W 2^(-8S), within
// 2^-(8S+1) of u, and each is an exact BF16 integer.  (Digit by digit in FP64
// -- a = rint(256 u), u -= a -- gives a split with the same bounds, but costs
// some 25 FP64 instructions per entry, and the FP64 pipe is this chip's
// slowest.)  A NaN or Inf entry gives NaN digits.
__device__ __forceinline__ void cut(double v, int e, int S, __nv_bfloat16* out, int64_t stride) {
    const long long bits = __double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7ff);
    if (E == 0x7ff) {
        for (int s = 0; s < S; ++s) out[s * stride] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        return;
    }
    const long long M = (bits & 0xFFFFFFFFFFFFFLL) | (E ? (1LL << 52) : 0LL);  // |v| = M 2^(max(E,1) - 1075)
    const int sh = (E ? E : 1) - 1075 + 8 * S - e;                              // |W| = M 2^sh
    long long W;
    if (M == 0 || sh < -60) W = 0;         // below half a unit of the last digit
    else if (sh >= 0) W = M << sh;         // < 2^(8S-1) <= 2^55: no overflow
    else W = (M + (1LL << (-sh - 1))) >> -sh;
    if (bits < 0) W = -W;
    for (int s = S - 1; s > 0; --s) {
        const long long a = ((W + 128) & 255) - 128;  // W mod 256 in [-128, 127]
        out[s * stride] = __float2bfloat16_rn((float)a);
        W = (W - a) >> 8;                              // exact: W - a is a multiple of 256
    }
    out[0] = __float2bfloat16_rn((float)W);
}

// Slices of A, K-major: Asl[s][i][k] = slice s of A(i,k) 2^-e_i (npad x npad,
// zero past n).  Each 32 x 32 lower tile writes its own tile and, with the
// other row's exponent, the mirrored one.
__global__ void slice_A_kernel(int64_t n, int64_t npad, const double* A, int64_t lda, const int* e, int S,
                               __nv_bfloat16* Asl) {
    const int64_t ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int64_t plane = npad * npad;
    __shared__ double tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int c = ty; c < 32; c += 8) {
        const int64_t gr = ti * 32 + tx, gc = tj * 32 + c;
        tile[c][tx] = (gr < n && gc < n && gr >= gc) ? A[gr + gc * lda] : 0.0;  // tile[col][row]
    }
    cta_sync();
    // (i, k) = (ti*32 + r, tj*32 + c): row i, k contiguous along c
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = ti * 32 + r, k = tj * 32 + tx;
        double v = tile[tx][r];
        if (ti == tj && k > i) v = tile[r][tx];  // upper part of a diagonal tile: mirror
        const int ei = i < n ? e[i] : 0;
        cut(v, ei, S, Asl + plane_index(npad, i, k), plane);
    }
    if (ti != tj) {
        // mirrored tile: (i, k) = (tj*32 + r, ti*32 + c), value A(ti*32 + c, tj*32 + r)
        for (int r = ty; r < 32; r += 8) {
            const int64_t i = tj * 32 + r, k = ti * 32 + tx;
            const double v = tile[r][tx];
            const int ei = i < n ? e[i] : 0;
            cut(v, ei, S, Asl + plane_index(npad, i, k), plane);
        }
    }
}

// Slices of X, K-major per column: Xsl[t][j][k] = slice t of X(k,j) 2^-f_j.
__global__ void slice_X_kernel(int64_t n, int64_t npad, const double* X, const int* f, int S, __nv_bfloat16* Xsl) {
    const int64_t plane = npad * npad;
    const int64_t j = blockIdx.x;
    const int fj = j < n ? f[j] : 0;
    for (int64_t k = threadIdx.x; k < npad; k += blockDim.x) {
        const double v = (j < n && k < n) ? X[k + j * n] : 0.0;
        cut(v, fj, S, Xsl + plane_index(npad, j, k), plane);
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p))
                 : "memory");
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct OzParams {
    int64_t n, npad;
    int npairs;
    const __nv_bfloat16* Asl;
    const __nv_bfloat16* Xsl;
    const int* e;  // row exponents of A
    const int* f;  // column exponents of X
    double* R;
    int ps[64], pt[64];  // the slice pairs
};

__global__ void __launch_bounds__(THREADS, 1) ozaki_residual_kernel(const OzParams p) {
    __nv_bfloat16* smem = reinterpret_cast<__nv_bfloat16*>(dynamic_smem());
    __nv_bfloat16* sA = smem;                          // [STAGES][BM][LDS]
    __nv_bfloat16* sB = smem + STAGES * BM * LDS;      // [STAGES][BN][LDS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t plane = p.npad * p.npad;
    const int ktiles = (int)(p.npad / BK);
    const int total = p.npairs * ktiles;

    auto load_stage = [&](int step, int stage) {
        const int pair = step / ktiles, kt = step - pair * ktiles;
        // BK = 32 entries of a row lie inside one 64-deep atom: contiguous
        const __nv_bfloat16* a = p.Asl + p.ps[pair] * plane + plane_index(p.npad, m0, (int64_t)kt * BK);
        const __nv_bfloat16* b = p.Xsl + p.pt[pair] * plane + plane_index(p.npad, n0, (int64_t)kt * BK);
        __nv_bfloat16* da = sA + stage * BM * LDS;
        __nv_bfloat16* db = sB + stage * BN * LDS;
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // A: 128 rows x 4 chunks of 16 bytes
            const int c = tid + u * THREADS, row = c >> 2, col = (c & 3) * 8;
            cp_async16(da + row * LDS + col, a + row * 64 + col);
        }
        {  // B: 64 rows x 4 chunks
            const int row = tid >> 2, col = (tid & 3) * 8;
            cp_async16(db + row * LDS + col, b + row * 64 + col);
        }
    };

    float facc[2][4][4];
    int iacc[2][4][4];
    double racc[2][4][4];
    int er[2][2], fc[4][2];  // exponents of this thread's rows and columns
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = m0 + wm + mi * 16 + g + 8 * h;
            er[mi][h] = i < p.n ? p.e[i] : 0;
        }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t j = n0 + wn + ni * 8 + 2 * q + h;
            fc[ni][h] = j < p.n ? p.f[j] : 0;
        }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = m0 + wm + mi * 16 + g + 8 * (r >> 1);
                const int64_t j = n0 + wn + ni * 8 + 2 * q + (r & 1);
                facc[mi][ni][r] = 0.f;
                iacc[mi][ni][r] = 0;
                racc[mi][ni][r] = (i == j) ? 1.0 : 0.0;
            }

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < total) load_stage(s, s);
        cp_async_commit();
    }
    for (int step = 0; step < total; ++step) {
        cp_async_wait<STAGES - 2>();
        cta_sync();
        const int stage = step % STAGES;
        const __nv_bfloat16* a_s = sA + stage * BM * LDS;
        const __nv_bfloat16* b_s = sB + stage * BN * LDS;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int row = wm + mi * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], a_s + row * LDS + col);
            }
#pragma unroll
            for (int nb = 0; nb < 4; nb += 2) {
                const int row = wn + (nb + (lane >> 4)) * 8 + (lane & 7), col = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bf[nb][0], bf[nb][1], bf[nb + 1][0], bf[nb + 1][1], b_s + row * LDS + col);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(facc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
        // prefetch the step STAGES-1 ahead into the stage freed at this step's start
        const int nxt = step + STAGES - 1;
        if (nxt < total) load_stage(nxt, nxt % STAGES);
        cp_async_commit();

        const int pair = step / ktiles, kt = step - pair * ktiles;
        const bool chunk_end = ((kt + 1) % CHUNK_TILES) == 0 || kt == ktiles - 1;
        if (chunk_end) {  // exact FP32 integers -> INT32
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        iacc[mi][ni][r] += __float2int_rn(facc[mi][ni][r]);
                        facc[mi][ni][r] = 0.f;
                    }
        }
        if (kt == ktiles - 1 || ((kt + 1) % FLUSH_TILES) == 0) {  // R -= 2^{e_i + f_j - 8(s+t+2)} * sum
            const int lvl = 8 * (p.ps[pair] + p.pt[pair] + 2);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ex = er[mi][r >> 1] + fc[ni][r & 1] - lvl;
                        racc[mi][ni][r] -= scalbn((double)iacc[mi][ni][r], ex);
                        iacc[mi][ni][r] = 0;
                    }
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = m0 + wm + mi * 16 + g + 8 * (r >> 1);
                const int64_t j = n0 + wn + ni * 8 + 2 * q + (r & 1);
                if (i < p.n && j < p.n) p.R[i + j * p.n] = racc[mi][ni][r];
            }
}

}  // namespace

size_t ozaki_workspace_bytes(int64_t n, int S) {
    const int64_t npad = (n + 255) / 256 * 256;
    const size_t slices = 2 * (size_t)S * npad * npad * sizeof(__nv_bfloat16);
    return slices + 2 * (size_t)npad * sizeof(int) + 2 * (size_t)npad * sizeof(unsigned long long) + 1024;
}

cudaError_t ozaki_residual(int64_t n, const double* A, int64_t lda, const double* X, double* R, void* ws, int S,
                           int L, bool tc, int* errw, cudaStream_t s, int* launches) {
    const int64_t npad = (n + 255) / 256 * 256;  // whole 256-deep chunks and 128-wide tiles
    char* w = static_cast<char*>(ws);
    __nv_bfloat16* Asl = reinterpret_cast<__nv_bfloat16*>(w);
    __nv_bfloat16* Xsl = Asl + (size_t)S * npad * npad;
    unsigned long long* rmax = reinterpret_cast<unsigned long long*>(Xsl + (size_t)S * npad * npad);
    unsigned long long* cmax = rmax + npad;
    int* e = reinterpret_cast<int*>(cmax + npad);
    int* f = e + npad;
    cudaError_t err = cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * npad, s);
    if (err != cudaSuccess) return err;
    const int64_t t32 = (n + 31) / 32;
    row_absmax_kernel<<<dim3((unsigned)t32, (unsigned)t32), dim3(32, 8), 0, s>>>(n, A, lda, rmax);
    col_absmax_kernel<<<(unsigned)n, 256, 0, s>>>(n, X, cmax);
    exponents_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, rmax, e);
    exponents_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, cmax, f);
    // the slicing grids cover the padded planes, writing zeros past n
    const unsigned tp = (unsigned)(npad / 32);
    slice_A_kernel<<<dim3(tp, tp), dim3(32, 8), 0, s>>>(n, npad, A, lda, e, S, Asl);
    slice_X_kernel<<<(unsigned)npad, 256, 0, s>>>(n, npad, X, f, S, Xsl);
    OzParams p{};
    p.n = n;
    p.npad = npad;
    p.Asl = Asl;
    p.Xsl = Xsl;
    p.e = e;
    p.f = f;
    p.R = R;
    int np = 0;
    for (int lv = 0; lv <= L; ++lv)
        for (int a = 0; a <= lv; ++a) {
            const int b = lv - a;
            if (a < S && b < S && np < 64) {
                p.ps[np] = a;
                p.pt[np] = b;
                ++np;
            }
        }
    p.npairs = np;
    if (tc) {
        err = ozaki_products_tc(n, npad, Asl, S, Xsl, S, p.ps, p.pt, np, e, f, R, nullptr, true, -1.0, false, errw, s);
        if (launches) *launches += 7;
        return err;
    }
    const int sm = STAGES * (BM + BN) * LDS * (int)sizeof(__nv_bfloat16);
    err = cudaFuncSetAttribute(ozaki_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (err != cudaSuccess) return err;
    ozaki_residual_kernel<<<dim3((unsigned)(npad / BN), (unsigned)(npad / BM)), THREADS, sm, s>>>(p);
    if (launches) *launches += 7;
    return cudaGetLastError();
}

}  // namespace spdinv

namespace spdinv {
namespace {

// Slices of a symmetric matrix given by its lower triangle (ld): row maxima,
// exponents and S planes, laid out as rows (equal to the columns).
cudaError_t slice_symmetric(int64_t n, int64_t npad, const double* M, int64_t ld, int S, __nv_bfloat16* planes,
                            unsigned long long* mx, int* ex, cudaStream_t s, int* launches) {
    cudaError_t err = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * npad, s);
    if (err != cudaSuccess) return err;
    const unsigned t32 = (unsigned)((n + 31) / 32), tp = (unsigned)(npad / 32);
    row_absmax_kernel<<<dim3(t32, t32), dim3(32, 8), 0, s>>>(n, M, ld, mx);
    exponents_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, mx, ex);
    slice_A_kernel<<<dim3(tp, tp), dim3(32, 8), 0, s>>>(n, npad, M, ld, ex, S, planes);
    *launches += 3;
    return cudaGetLastError();
}

// Slices of a full matrix (ld n) by columns: column maxima, exponents and S
// planes laid out K-major per column.
cudaError_t slice_columns(int64_t n, int64_t npad, const double* M, int S, __nv_bfloat16* planes,
                          unsigned long long* mx, int* ex, cudaStream_t s, int* launches) {
    col_absmax_kernel<<<(unsigned)n, 256, 0, s>>>(n, M, mx);
    exponents_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, mx, ex);
    slice_X_kernel<<<(unsigned)npad, 256, 0, s>>>(n, npad, M, ex, S, planes);
    *launches += 3;
    return cudaGetLastError();
}

// Lower triangle: X += Y (both ld n).
__global__ void add_lower_kernel(int64_t n, double* X, const double* Y) {
    const int64_t j = blockIdx.x;
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) X[i + j * n] += Y[i + j * n];
}

// Slice pairs (s, t), s < SA, t < SB, by increasing level s + t <= L.
int level_pairs(int SA, int SB, int L, int* ps, int* pt) {
    int np = 0;
    for (int lv = 0; lv <= L; ++lv)
        for (int a = 0; a <= lv; ++a)
            if (a < SA && lv - a < SB && np < 64) {
                ps[np] = a;
                pt[np] = lv - a;
                ++np;
            }
    return np;
}

constexpr int kResSlices = 7;                        // slices of A and X for R
constexpr int kChainLevels[7] = {4, 3, 2, 2, 1, 1, 1};  // level limit of X R^m, m = 1..7
constexpr int kRSlices = 5;                          // slices of R (kChainLevels[0] + 1)
constexpr int kYSlices = 4;                          // slices of X R^m (kChainLevels[1] + 1)

struct RefineWs {
    __nv_bfloat16 *Asl, *Xsl, *Rsl, *Ysl;
    unsigned long long* mx;
    int *eA, *eX, *fR, *eY;
};

RefineWs refine_layout(int64_t n, void* ws) {
    const int64_t npad = (n + 255) / 256 * 256;
    const size_t plane = (size_t)npad * npad;
    RefineWs w;
    w.Asl = static_cast<__nv_bfloat16*>(ws);
    w.Xsl = w.Asl + kResSlices * plane;
    w.Rsl = w.Xsl + kResSlices * plane;
    w.Ysl = w.Rsl + kRSlices * plane;
    w.mx = reinterpret_cast<unsigned long long*>(w.Ysl + kYSlices * plane);
    w.eA = reinterpret_cast<int*>(w.mx + npad);
    w.eX = w.eA + npad;
    w.fR = w.eX + npad;
    w.eY = w.fR + npad;
    return w;
}

}  // namespace

size_t ozaki_refine_workspace_bytes(int64_t n) {
    const int64_t npad = (n + 255) / 256 * 256;
    const size_t plane = (size_t)npad * npad;
    return (2 * kResSlices + kRSlices + kYSlices) * plane * sizeof(__nv_bfloat16) +
           (size_t)npad * (sizeof(unsigned long long) + 4 * sizeof(int)) + 1024;
}

cudaError_t ozaki_refine_step(int64_t n, const double* A, int64_t lda, double* X, double* R, double* Y, void* ws,
                              int levelsR, int order, bool slice_A, int* errw, cudaStream_t s, int* launches) {
    if (order < 2 || order > 8) return cudaErrorInvalidValue;
    const int64_t npad = (n + 255) / 256 * 256;
    const RefineWs w = refine_layout(n, ws);
    cudaError_t err = cudaSuccess;
    if (slice_A) {  // A does not change between steps
        err = slice_symmetric(n, npad, A, lda, kResSlices, w.Asl, w.mx, w.eA, s, launches);
        if (err != cudaSuccess) return err;
    }
    // X is symmetric: its row slices are also its column slices.
    err = slice_symmetric(n, npad, X, n, kResSlices, w.Xsl, w.mx, w.eX, s, launches);
    if (err != cudaSuccess) return err;
    int ps[64], pt[64];
    int np = level_pairs(kResSlices, kResSlices, levelsR, ps, pt);
    err = ozaki_products_tc(n, npad, w.Asl, kResSlices, w.Xsl, kResSlices, ps, pt, np, w.eA, w.eX, R, nullptr, true,
                            -1.0, false, errw, s);  // R = I - A X, every tile
    if (err != cudaSuccess) return err;
    err = slice_columns(n, npad, R, kRSlices, w.Rsl, w.mx, w.fR, s, launches);
    if (err != cudaSuccess) return err;
    *launches += 1;
    // X R^m = (X R^{m-1}) R is symmetric: only its lower tiles are formed.
    const __nv_bfloat16* left = w.Xsl;
    int left_slices = kResSlices;
    const int* eleft = w.eX;
    for (int m = 1; m < order; ++m) {
        const int L = kChainLevels[m - 1];
        np = level_pairs(L + 1, kRSlices, L, ps, pt);
        err = ozaki_products_tc(n, npad, left, left_slices, w.Rsl, kRSlices, ps, pt, np, eleft, w.fR, Y, nullptr,
                                false, 1.0, true, errw, s);
        if (err != cudaSuccess) return err;
        *launches += 1;
        if (m + 1 < order) {
            err = slice_symmetric(n, npad, Y, n, kYSlices, w.Ysl, w.mx, w.eY, s, launches);
            if (err != cudaSuccess) return err;
            left = w.Ysl;
            left_slices = kYSlices;
            eleft = w.eY;
        }
        add_lower_kernel<<<(unsigned)n, 256, 0, s>>>(n, X, Y);
        *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace spdinv
