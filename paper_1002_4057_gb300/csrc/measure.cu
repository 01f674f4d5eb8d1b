// Measurement utilities (no counterpart in the paper).
//
//  * Peaks of this GPU, as the roofline's denominators: a kernel that keeps
//    one pipe busy on register operands -- the FP64 tensor-core MMA
//    (mma.sync m8n8k4, the instruction of the FP64 tile products), the FP64
//    FMA or the FP32 FMA -- with enough independent accumulators per thread
//    to cover the pipe's latency.  The caller times it with CUDA events on
//    its stream and divides the flop count this call reports by the time.
//  * CUDA-event timing of the library's own launches of selected kernels (the
//    tcgen05 slice GEMM and the persistent DAGs), with each launch's
//    algorithmic work, so that a benchmark can report a kernel's rate inside
//    a whole call.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "ptx.cuh"

namespace spdinv {
namespace {

constexpr int kProbeThreads = 128;
constexpr int kProbeChains = 16;  // independent accumulators per thread

__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(int64_t iters, double* sink) {
    const int lane = threadIdx.x & 31;
    const double a = 1.0 + 1e-3 * lane, b = 1.0 - 1e-3 * (lane & 7);
    double c[kProbeChains][2];
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) c[u][0] = c[u][1] = 0.0;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kProbeChains; ++u) dmma_m8n8k4(c[u][0], c[u][1], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) s += c[u][0] + c[u][1];
    if (lane == 0) sink[blockIdx.x * (kProbeThreads / 32) + (threadIdx.x >> 5)] = s;
}

// FMA chains in T (double: the FP64 pipe; float: the FP32 pipe).
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int64_t iters, double* sink) {
    const T a = (T)(1.0 + 1e-9 * threadIdx.x), b = (T)(1.0 - 1e-9 * (threadIdx.x & 15));
    T c[kProbeChains];
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) c[u] = (T)(1e-3 * u);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kProbeChains; ++u) c[u] = fma(a, c[u], b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) s += (double)c[u];
    if ((threadIdx.x & 31) == 0) sink[blockIdx.x * (kProbeThreads / 32) + (threadIdx.x >> 5)] = s;
}

struct TimingState {
    std::mutex mu;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[SPDINV_TIMED_KERNELS];
    double flops[SPDINV_TIMED_KERNELS] = {};
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};

TimingState& timing() {
    static TimingState s;
    return s;
}

}  // namespace

void timing_begin(int which, cudaStream_t s, void** token) {
    *token = nullptr;
    TimingState& T = timing();
    std::lock_guard<std::mutex> lk(T.mu);
    if (!T.on || which < 0 || which >= SPDINV_TIMED_KERNELS) return;
    cudaEvent_t e = T.take();
    if (e == nullptr || cudaEventRecord(e, s) != cudaSuccess) return;
    *token = e;
}

void timing_end(int which, cudaStream_t s, void* token, double flops) {
    if (token == nullptr) return;
    TimingState& T = timing();
    std::lock_guard<std::mutex> lk(T.mu);
    cudaEvent_t e1 = T.take();
    if (e1 == nullptr || cudaEventRecord(e1, s) != cudaSuccess) {
        T.pool.push_back(static_cast<cudaEvent_t>(token));
        if (e1) T.pool.push_back(e1);
        return;
    }
    T.pending[which].emplace_back(static_cast<cudaEvent_t>(token), e1);
    T.flops[which] += flops;
}

}  // namespace spdinv

using namespace spdinv;

extern "C" {

SPDINV_API spdinv_status spdinv_fp64_peak_probe(int kind, int64_t iters, int blocks_per_sm, double* d_sink,
                                                double* flops, cudaStream_t stream) {
    if (kind != SPDINV_PROBE_DMMA && kind != SPDINV_PROBE_DFMA && kind != SPDINV_PROBE_FFMA)
        return SPDINV_ERR_UNSUPPORTED;
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 16) return SPDINV_ERR_N;
    if (!d_sink || !flops) return SPDINV_ERR_NULL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const int grid = device_state(dev).num_sms * blocks_per_sm;
    const double warps = (double)grid * (kProbeThreads / 32);
    if (kind == SPDINV_PROBE_DMMA) {
        dmma_probe_kernel<<<grid, kProbeThreads, 0, stream>>>(iters, d_sink);
        *flops = warps * (double)iters * kProbeChains * (8.0 * 8.0 * 4.0 * 2.0);
    } else {
        if (kind == SPDINV_PROBE_DFMA) fma_probe_kernel<double><<<grid, kProbeThreads, 0, stream>>>(iters, d_sink);
        else fma_probe_kernel<float><<<grid, kProbeThreads, 0, stream>>>(iters, d_sink);
        *flops = warps * 32.0 * (double)iters * kProbeChains * 2.0;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return SPDINV_OK;
}

SPDINV_API spdinv_status spdinv_set_kernel_timing(int on) {
    TimingState& T = timing();
    std::lock_guard<std::mutex> lk(T.mu);
    T.on = on != 0;
    return SPDINV_OK;
}

SPDINV_API spdinv_status spdinv_kernel_time_ms(int which, double* ms, int* launches, double* flops) {
    if (which < 0 || which >= SPDINV_TIMED_KERNELS) return SPDINV_ERR_UNSUPPORTED;
    if (!ms || !launches || !flops) return SPDINV_ERR_NULL;
    TimingState& T = timing();
    std::lock_guard<std::mutex> lk(T.mu);
    double tot = 0.0;
    int cnt = 0;
    cudaError_t err = cudaSuccess;
    for (auto& pr : T.pending[which]) {
        cudaError_t e = cudaEventSynchronize(pr.second);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, pr.first, pr.second);
        if (e == cudaSuccess) {
            tot += v;
            ++cnt;
        } else if (err == cudaSuccess) {
            err = e;
        }
        T.pool.push_back(pr.first);
        T.pool.push_back(pr.second);
    }
    T.pending[which].clear();
    *flops = T.flops[which];
    T.flops[which] = 0.0;
    *ms = tot;
    *launches = cnt;
    return err == cudaSuccess ? SPDINV_OK : cuda_fail(err);
}

}  // extern "C"
