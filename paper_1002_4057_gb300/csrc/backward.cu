// Backward of the inversion (an added form; the paper has only the forward
// method): for f(A) with X = A^{-1} and incoming gradient G = df/dX,
//   d(A^{-1}) = -X dA X   =>   grad_A = -X sym(G) X,   sym(G) = (G + G^T)/2,
// which is -sym(X G X) for symmetric X.  Two tiled products per matrix:
//   sym:      Gs = sym(G)               (a coalesced tiled transpose, once)
//   phase 0:  Y = X Gs
//   phase 1:  grad = -Y X, lower tiles only, each written to (i, j) and,
//             transposed, to (j, i); the diagonal tiles are averaged with
//             their transpose, so grad is exactly symmetric.
// This file runs FP64: the tile products are FP64 FMAs on register blocks.
// FP32 runs on the tensor cores as 3xTF32 products (backward_tc.cu).
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "tile_fp64.cuh"

namespace spdinv {
namespace {

constexpr int BB = 64;  // output tile

template <typename T>
struct BwdTile;
template <>
struct BwdTile<double> {
    using Acc = spdinv::Acc<BB>;
    static constexpr int LD = BB;
};

template <typename T>
struct BwdParams {
    int64_t n;
    int t;
    const T* X;
    int64_t ldx, sx;
    const T* Gs;  // workspace: sym(G), n x n per matrix, ld n
    T* Y;         // workspace, n x n per matrix, ld n
    T* grad;
    int64_t ldr, sr;
};

// Tile (ti, tj) of a column-major matrix, zero-padded past n.
template <typename T>
__device__ __forceinline__ void load_tile(const T* M, int64_t n, int64_t ld, int ti, int tj, T* S) {
    constexpr int LD = BwdTile<T>::LD;
    for (int idx = threadIdx.x; idx < BB * BB; idx += kThreads) {
        const int r = idx % BB, c = idx / BB;
        const int64_t gr = (int64_t)ti * BB + r, gc = (int64_t)tj * BB + c;
        S[c * LD + r] = (gr < n && gc < n) ? M[gr + gc * ld] : T(0);
    }
}

// Gs = sym(G) = (G + G^T)/2 (ld n, matrix k at k n^2), formed once before
// the products so that they read plain tiles: each CTA reads the 32 x 32
// tiles (bi, bj) and (bj, bi), bi >= bj, with coalesced loads, transposes
// through shared memory, and writes both halves with coalesced stores.
template <typename T>
__global__ void __launch_bounds__(256) sym_kernel(int64_t n, const T* G, int64_t ldg, int64_t sg, T* Gs) {
    __shared__ T a[32][33], b[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int64_t k = blockIdx.y;
    int bi = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) / 2.0);
    while ((bi + 1) * (bi + 2) / 2 <= (int)blockIdx.x) ++bi;
    while (bi * (bi + 1) / 2 > (int)blockIdx.x) --bi;
    const int bj = blockIdx.x - bi * (bi + 1) / 2;
    const T* g = G + k * sg;
    T* o = Gs + k * n * n;
    for (int c = ty; c < 32; c += 8) {  // a[c][r] = G(bi*32 + r, bj*32 + c), b[c][r] = G(bj*32 + r, bi*32 + c)
        const int64_t r0 = (int64_t)bi * 32 + tx, c0 = (int64_t)bj * 32 + c;
        const int64_t r1 = (int64_t)bj * 32 + tx, c1 = (int64_t)bi * 32 + c;
        a[c][tx] = (r0 < n && c0 < n) ? g[r0 + c0 * ldg] : T(0);
        b[c][tx] = (r1 < n && c1 < n) ? g[r1 + c1 * ldg] : T(0);
    }
    cta_sync();
    for (int c = ty; c < 32; c += 8) {
        const int64_t r0 = (int64_t)bi * 32 + tx, c0 = (int64_t)bj * 32 + c;  // Gs(r0, c0) = (a[c][tx] + b[tx][c]) / 2
        if (r0 < n && c0 < n) o[r0 + c0 * n] = T(0.5) * (a[c][tx] + b[tx][c]);
        const int64_t r1 = (int64_t)bj * 32 + tx, c1 = (int64_t)bi * 32 + c;  // Gs(r1, c1) = (b[c][tx] + a[tx][c]) / 2
        if (bi != bj && r1 < n && c1 < n) o[r1 + c1 * n] = T(0.5) * (b[c][tx] + a[tx][c]);
    }
}

template <typename T, int PHASE>
__global__ void __launch_bounds__(kThreads) backward_kernel(const BwdParams<T> p) {
    unsigned char* const smem_raw = dynamic_smem();
    constexpr int LD = BwdTile<T>::LD;
    T* S0 = reinterpret_cast<T*>(smem_raw);
    T* S1 = S0 + BB * LD;
    const int64_t mat = blockIdx.y;
    int ti, tj;
    if (PHASE == 0) {
        ti = blockIdx.x % p.t;
        tj = blockIdx.x / p.t;
    } else {  // lower tiles: blockIdx.x = ti (ti + 1) / 2 + tj
        ti = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) / 2.0);
        while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
        while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
        tj = blockIdx.x - ti * (ti + 1) / 2;
    }
    const T* X = p.X + mat * p.sx;
    const T* G = p.Gs + mat * p.n * p.n;
    T* Y = p.Y + mat * p.n * p.n;
    typename BwdTile<T>::Acc acc;
    acc_zero<BB>(acc);
    for (int kt = 0; kt < p.t; ++kt) {
        cta_sync();
        if (PHASE == 0) {
            load_tile<T>(X, p.n, p.ldx, ti, kt, S0);
            load_tile<T>(G, p.n, p.n, kt, tj, S1);  // sym(G), formed by sym_kernel
        } else {
            load_tile<T>(Y, p.n, p.n, ti, kt, S0);
            load_tile<T>(X, p.n, p.ldx, kt, tj, S1);
        }
        cta_sync();
        tile_mma<BB, false, false, PHASE == 1, FULL, FULL>(acc, S0, S1);
    }
    cta_sync();
    acc_store<BB>(acc, S0);
    cta_sync();
    if (PHASE == 0) {
        for (int idx = threadIdx.x; idx < BB * BB; idx += kThreads) {
            const int r = idx % BB, c = idx / BB;
            const int64_t gr = (int64_t)ti * BB + r, gc = (int64_t)tj * BB + c;
            if (gr < p.n && gc < p.n) Y[gr + gc * p.n] = S0[c * LD + r];
        }
    } else {
        T* R = p.grad + mat * p.sr;
        for (int idx = threadIdx.x; idx < BB * BB; idx += kThreads) {
            const int r = idx % BB, c = idx / BB;
            const int64_t gr = (int64_t)ti * BB + r, gc = (int64_t)tj * BB + c;
            if (gr >= p.n || gc >= p.n) continue;
            if (ti == tj) {
                R[gr + gc * p.ldr] = T(0.5) * (S0[c * LD + r] + S0[r * LD + c]);
            } else {
                R[gr + gc * p.ldr] = S0[c * LD + r];
            }
        }
        if (ti != tj) {  // mirror: grad(j, i) = grad(i, j)^T, coalesced along the target's rows
            for (int idx = threadIdx.x; idx < BB * BB; idx += kThreads) {
                const int r = idx % BB, c = idx / BB;  // target element (tj*B + r, ti*B + c)
                const int64_t gr = (int64_t)tj * BB + r, gc = (int64_t)ti * BB + c;
                if (gr < p.n && gc < p.n) R[gr + gc * p.ldr] = S0[r * LD + c];
            }
        }
    }
}

struct BwdState {
    std::mutex mu;
    void* ws = nullptr;
    size_t bytes = 0;
};

BwdState& bwd_state(int dev) {
    static std::mutex mu;
    static std::map<int, BwdState*> m;
    std::lock_guard<std::mutex> lk(mu);
    auto& s = m[dev];
    if (!s) s = new BwdState();
    return *s;
}

// Argument checks of both precisions: SPDINV_OK with *run = false when there
// is nothing to do.
spdinv_status backward_args(int batch, int64_t n, const void* dX, int64_t ldx, const void* dG, int64_t ldg,
                            const void* dGrad, int64_t ldr, bool* run) {
    *run = false;
    if (batch < 0 || n < 0) return SPDINV_ERR_N;
    const int64_t mn = n > 1 ? n : 1;
    if (ldx < mn || ldg < mn || ldr < mn) return SPDINV_ERR_LDA;
    if (batch == 0 || n == 0) return SPDINV_OK;
    if (!dX || !dG || !dGrad) return SPDINV_ERR_NULL;
    if (batch > 65535) return SPDINV_ERR_N;
    *run = true;
    return SPDINV_OK;
}

template <typename T>
spdinv_status run_backward(int batch, int64_t n, const T* dX, int64_t ldx, int64_t sx, const T* dG, int64_t ldg,
                           int64_t sg, T* dGrad, int64_t ldr, int64_t sr, cudaStream_t stream) {
    bool run = false;
    const spdinv_status a = backward_args(batch, n, dX, ldx, dG, ldg, dGrad, ldr, &run);
    if (!run) return a;
    const int64_t t = (n + BB - 1) / BB;
    if (t * (t + 1) / 2 > 2147483647LL || t * t > 2147483647LL) return SPDINV_ERR_N;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    BwdState& st = bwd_state(dev);
    std::lock_guard<std::mutex> lk(st.mu);
    const size_t need = 2 * sizeof(T) * (size_t)n * n * batch;  // Y and sym(G)
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
    T* Ys = static_cast<T*>(st.ws);
    BwdParams<T> p{n, (int)t, dX, ldx, sx, Ys + (size_t)n * n * batch, Ys, dGrad, ldr, sr};
    T* Gs = Ys + (size_t)n * n * batch;
    const int sm = 2 * BB * BwdTile<T>::LD * (int)sizeof(T);
    auto k0 = backward_kernel<T, 0>;
    auto k1 = backward_kernel<T, 1>;
    e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t t32 = (n + 31) / 32;
    sym_kernel<T><<<dim3((unsigned)(t32 * (t32 + 1) / 2), (unsigned)batch), dim3(32, 8), 0, stream>>>(n, dG, ldg, sg,
                                                                                                    Gs);
    k0<<<dim3((unsigned)(t * t), (unsigned)batch), kThreads, sm, stream>>>(p);
    k1<<<dim3((unsigned)(t * (t + 1) / 2), (unsigned)batch), kThreads, sm, stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(3);
    return SPDINV_OK;
}

}  // namespace
}  // namespace spdinv

using namespace spdinv;

extern "C" {

SPDINV_API spdinv_status spdinv_potri_backward(int batch, int64_t n, const double* dX, int64_t ldx, int64_t sx,
                                               const double* dG, int64_t ldg, int64_t sg, double* dGrad,
                                               int64_t ldr, int64_t sr, cudaStream_t stream) {
    return log_status("spdinv_potri_backward", "n", n, run_backward<double>(batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldr, sr, stream));
}

SPDINV_API spdinv_status spdinv_spotri_backward(int batch, int64_t n, const float* dX, int64_t ldx, int64_t sx,
                                                const float* dG, int64_t ldg, int64_t sg, float* dGrad,
                                                int64_t ldr, int64_t sr, cudaStream_t stream) {
    bool run = false;
    spdinv_status st = backward_args(batch, n, dX, ldx, dG, ldg, dGrad, ldr, &run);
    if (run) st = backward_f32_tc(batch, n, dX, ldx, sx, dG, ldg, sg, dGrad, ldr, sr, stream);
    return log_status("spdinv_spotri_backward", "n", n, st);
}

}  // extern "C"
