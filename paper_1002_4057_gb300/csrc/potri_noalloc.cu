// spdinv_potri_noalloc: the FP64 inversion for callers that cannot allocate
// device memory.  Everything the persistent kernel needs besides the caller's
// matrix -- the ticket/status words, the readiness flags, the renamed stores
// B, C, D and the task list -- lives in one fixed array in this file's device
// memory, sized for n <= SPDINV_NOALLOC_MAX_N with 32 x 32 tiles.
//
// The kernel run is the same persistent kernel spdinv_potri queues; only the
// task list differs: instead of the planner's priority order (computed on the
// host and uploaded to an allocation), a small kernel writes Algorithm 1's
// sequential loop order, which is also a topological order of the tile tasks,
// straight into the array.  Each tile's update chain runs in the same order
// either way, so results match spdinv_potri with tile 32.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "kernels.h"
#include "plan.h"

namespace spdinv {
namespace {

constexpr int kTile = 32;
constexpr int kMaxT = (SPDINV_NOALLOC_MAX_N + kTile - 1) / kTile;
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kTileBytes = (size_t)kTile * kTile * sizeof(double);
constexpr size_t kMaxTri = (size_t)kMaxT * (kMaxT - 1) / 2;
constexpr size_t kMaxTasks = (size_t)kMaxT * (kMaxT + 1) / 2 + kMaxTri + (size_t)kMaxT * (kMaxT + 1) / 2;
constexpr size_t kCtrlBytes = align256(sizeof(int) * (4 + 2 * (size_t)kMaxT * kMaxT + kMaxT));
constexpr size_t kTaskBytes = align256(sizeof(uint32_t) * kMaxTasks);
constexpr size_t kScratchBytes = kCtrlBytes + kTaskBytes + 2 * kMaxTri * kTileBytes + (size_t)kMaxT * kTileBytes;
static_assert(kScratchBytes <= 9u * 1024u * 1024u, "scratch must stay modest");

// The scratch.  In host code this name is only a stand-in for the symbol,
// never a device address: host code uses the address cudaGetSymbolAddress
// returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Algorithm 1's loop order for all three steps (Step 2's diagonal inversion
// is part of the Step-1 diagonal task, as in spdinv_potri).
__global__ void write_sequential_plan(uint32_t* tasks, int t) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int m = 0;
    for (int j = 0; j < t; ++j) {
        tasks[m++] = encode_task(K_S1_DIAG, j, j);
        for (int i = j + 1; i < t; ++i) tasks[m++] = encode_task(K_S1_OFF, i, j);
    }
    for (int j = t - 1; j >= 0; --j)
        for (int i = t - 1; i > j; --i) tasks[m++] = encode_task(K_S2_OFF, i, j);
    for (int i = 0; i < t; ++i) {
        for (int j = 0; j < i; ++j) tasks[m++] = encode_task(K_S3_OFF, i, j);
        tasks[m++] = encode_task(K_S3_DIAG, i, i);
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
struct Setup {
    void* addr = nullptr;          // device address of the array in that context
    unsigned long long ctx = 0;    // the context it was looked up in (0 = none)
    int num_sms = 0;
};
Setup g_setup[kMaxDevices];

// Unique id of the calling thread's current CUDA context, or 0 when none is
// current or the driver does not provide the query.  A device reset destroys
// the context, and the module -- with the array -- is loaded again at a new
// address in the next one; keying the cached address on the context makes a
// call after a reset look it up again instead of using a stale address.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static std::once_flag once;
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPoint("cuCtxGetId", &f, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Set-up, once per device (and again in a new context after a device reset),
// with that device current: look up the array's device address.  Without a
// context id the address is looked up on every call.
cudaError_t scratch_for(int dev, void** addr, int* num_sms) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    Setup& su = g_setup[dev];
    const unsigned long long ctx = current_context_id();
    if (su.addr == nullptr || ctx == 0 || ctx != su.ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        su.addr = p;
        su.num_sms = sms;
        su.ctx = current_context_id();  // the lookup has made the device's context current
    }
    *addr = su.addr;
    *num_sms = su.num_sms;
    return cudaSuccess;
}

}  // namespace
}  // namespace spdinv

using namespace spdinv;

static spdinv_status potri_noalloc_impl(int64_t n, double* dA, int64_t lda, int* d_info,
                                                         cudaStream_t stream) {
    if (n < 0 || n > SPDINV_NOALLOC_MAX_N) return SPDINV_ERR_N;
    if (lda < (n > 1 ? n : 1)) return SPDINV_ERR_LDA;
    if (n > 0 && dA == nullptr) return SPDINV_ERR_NULL;
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
    void* base_v = nullptr;
    int num_sms = 0;
    e = scratch_for(dev, &base_v, &num_sms);
    if (e != cudaSuccess) return cuda_fail(e);

    const int t = (int)((n + kTile - 1) / kTile);
    const size_t ntri = (size_t)t * (t - 1) / 2;
    const size_t ctrl_used = sizeof(int) * (4 + 2 * (size_t)t * t + t);
    char* base = static_cast<char*>(base_v);

    KParamsF64 p{};
    p.n = n;
    p.lda = lda;
    p.t = t;
    p.b = kTile;
    p.steps = STEPS_ALL;
    p.ntasks = (int)((size_t)t * (t + 1) / 2 + ntri + (size_t)t * (t + 1) / 2);
    p.A = dA;
    p.ctrl = reinterpret_cast<int*>(base);
    p.flags = p.ctrl + 4;
    uint32_t* tasks = reinterpret_cast<uint32_t*>(base + kCtrlBytes);
    p.tasks = tasks;
    p.Bw = reinterpret_cast<double*>(base + kCtrlBytes + kTaskBytes);
    p.Cw = p.Bw + ntri * (kTileBytes / sizeof(double));
    p.Dw = p.Cw + ntri * (kTileBytes / sizeof(double));
    p.timeout_ns = (long long)(wait_timeout_s(nullptr) * 1e9);  // the same limit as spdinv_potri's
    p.drop_task = -1;

    // The array keeps the previous call's contents: the status words and the
    // readiness flags must start at zero; B, C and D are written before read.
    e = cudaMemsetAsync(p.ctrl, 0, ctrl_used, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    write_sequential_plan<<<1, 32, 0, stream>>>(tasks, t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    int grid = 0;
    e = launch_potri_fp64(p, 0, num_sms, d_info, stream, &grid);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(2 + (d_info ? 1 : 0));
    return SPDINV_OK;
}

extern "C" SPDINV_API spdinv_status spdinv_potri_noalloc(int64_t n, double* dA, int64_t lda, int* d_info,
                                                         cudaStream_t stream) {
    return log_status("spdinv_potri_noalloc", "n", n, potri_noalloc_impl(n, dA, lda, d_info, stream));
}
