// C-ABI of the library (declared in include/spdinv.h): argument checks, the
// per-device plan cache and workspace, and the launch of the persistent
// kernel.  No compute happens here.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/spdinv.h"
#include "api_internal.h"
#include "kernels.h"
#include "plan.h"

namespace spdinv {

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

namespace {
thread_local std::string g_last_cuda_error;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void count_launches(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

spdinv_status cuda_fail(cudaError_t e) {
    g_last_cuda_error = cudaGetErrorString(e);
    return SPDINV_ERR_CUDA;
}

namespace {
const char* status_name(int st) {
    switch (st) {
        case SPDINV_OK: return "SPDINV_OK";
        case SPDINV_ERR_N: return "SPDINV_ERR_N";
        case SPDINV_ERR_LDA: return "SPDINV_ERR_LDA";
        case SPDINV_ERR_NULL: return "SPDINV_ERR_NULL";
        case SPDINV_ERR_CUDA: return "SPDINV_ERR_CUDA";
        case SPDINV_ERR_TIMEOUT: return "SPDINV_ERR_TIMEOUT";
        case SPDINV_ERR_UNSUPPORTED: return "SPDINV_ERR_UNSUPPORTED";
        case SPDINV_ERR_WORKSPACE: return "SPDINV_ERR_WORKSPACE";
    }
    return "unknown status";
}

int log_level() {
    static const int level = [] {
        const char* env = std::getenv("SPDINV_LOG");
        return env ? std::atoi(env) : 0;
    }();
    return level;
}

std::mutex g_log_mu;

std::atomic<unsigned>& debug_flags() {
    static std::atomic<unsigned> flags{[] {
        const char* env = std::getenv("SPDINV_DEBUG");
        return env ? (unsigned)std::strtoul(env, nullptr, 0) : 0u;
    }()};
    return flags;
}
}  // namespace

spdinv_status log_status(const char* fn, const char* size_name, int64_t size, spdinv_status st) {
    const int level = log_level();
    if (level >= 2 || (level >= 1 && st != SPDINV_OK)) {
        std::lock_guard<std::mutex> lk(g_log_mu);
        if (st == SPDINV_ERR_CUDA)
            std::fprintf(stderr, "[spdinv] %s %s=%lld: %s (%s)\n", fn, size_name, (long long)size, status_name(st),
                         g_last_cuda_error.c_str());
        else
            std::fprintf(stderr, "[spdinv] %s %s=%lld: %s\n", fn, size_name, (long long)size, status_name(st));
    }
    return st;
}

DeviceState& device_state(int dev) {
    static std::mutex mu;
    static std::map<int, std::unique_ptr<DeviceState>> states;
    std::lock_guard<std::mutex> lk(mu);
    auto& s = states[dev];
    if (!s) {
        s.reset(new DeviceState());
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return *s;
}

cudaError_t DeviceState::ensure_workspace(size_t bytes) {
    if (bytes <= ws_bytes) return cudaSuccess;
    if (ws) {
        cudaError_t e = cudaDeviceSynchronize();  // earlier work may still use the old buffer
        if (e != cudaSuccess) return e;
        cudaFree(ws);
        ws = nullptr;
        ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ws, bytes);
    if (e == cudaSuccess) ws_bytes = bytes;
    return e;
}

spdinv_status DeviceState::acquire(size_t bytes, void** out) {
    if (user_ws) {
        if (bytes > user_bytes) return SPDINV_ERR_WORKSPACE;
        *out = user_ws;
        return SPDINV_OK;
    }
    cudaError_t e = ensure_workspace(bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    *out = ws;
    return SPDINV_OK;
}

cudaError_t DeviceState::variant_plan(int t, int variant, int seg, const DevicePlan** out) {
    const auto key = std::make_tuple(t, (int)STEPS_ALL, (int)ORDER_BOTTOM_LEVEL, variant, seg);
    auto it = plans.find(key);
    if (it == plans.end()) {
        ExecPlan p;
        if (!build_variant_plan(t, variant, seg, &p)) return cudaErrorInvalidValue;
        const size_t tb = align_up(sizeof(uint32_t) * (p.order.size() + 1), 256);
        const size_t pb = align_up(sizeof(PartTask) * p.parts.size(), 256);
        const size_t sb = sizeof(SplitInfo) * p.split.size();
        DevicePlan dp;
        dp.ntasks = (int)p.order.size();
        cudaError_t e = cudaMalloc(&dp.d_tasks, tb + pb + sb + 256);
        if (e != cudaSuccess) return e;
        char* base = reinterpret_cast<char*>(dp.d_tasks);
        dp.d_parts = reinterpret_cast<const PartTask*>(base + tb);
        dp.d_split = reinterpret_cast<const SplitInfo*>(base + tb + pb);
        e = cudaMemcpy(dp.d_tasks, p.order.data(), sizeof(uint32_t) * p.order.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !p.parts.empty())
            e = cudaMemcpy(base + tb, p.parts.data(), sizeof(PartTask) * p.parts.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !p.split.empty())
            e = cudaMemcpy(base + tb + pb, p.split.data(), sb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dp.d_tasks);
            return e;
        }
        it = plans.emplace(key, dp).first;
    }
    *out = &it->second;
    return cudaSuccess;
}

cudaError_t DeviceState::exec_plan(int t, int steps, const uint32_t** d_tasks, int* ntasks) {
    const int order = current_plan_order();
    const auto key = std::make_tuple(t, steps, order, 0, 0);
    auto it = plans.find(key);
    if (it == plans.end()) {
        ExecPlan p = build_exec_plan(t, steps, false, order);
        DevicePlan dp;
        dp.ntasks = (int)p.order.size();
        cudaError_t e = cudaMalloc(&dp.d_tasks, sizeof(uint32_t) * (p.order.size() + 1));
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(dp.d_tasks, p.order.data(), sizeof(uint32_t) * p.order.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dp.d_tasks);
            return e;
        }
        it = plans.emplace(key, dp).first;
    }
    *d_tasks = it->second.d_tasks;
    *ntasks = it->second.ntasks;
    return cudaSuccess;
}

double wait_timeout_s(const spdinv_opts* o) {
    if (o && o->wait_timeout_s > 0) return o->wait_timeout_s;
    if (const char* env = std::getenv("SPDINV_WAIT_TIMEOUT_S")) {
        const double v = std::atof(env);
        if (v > 0) return v;
    }
    return 60.0;
}

// Tile 32 measured faster than 64 at n = 4096, 8192 and 16384 (1241 against
// 1200 Gflop/s at 16384: more tasks to overlap the dependency waits, and fewer
// wasted flops in the diagonal tiles).  Above n = 16384 the default is 64: it
// runs at the FP64 rate at n = 32768, and it halves t for the first call's
// plan build (the ALAP order takes about 1 s at t = 512, 8 s at t = 1024).
// SPDINV_TILE=32|64 in the environment overrides it.
static int default_tile(int64_t n) {
    static const int forced = [] {
        const char* env = std::getenv("SPDINV_TILE");
        const int v = env ? std::atoi(env) : 0;
        return (v == 32 || v == 64) ? v : 0;
    }();
    if (forced) return forced;
    return n <= 16384 ? 32 : 64;
}

spdinv_status fp64_layout(int64_t n, int steps, const spdinv_opts* o, Fp64Layout* out) {
    if (n < 0) return SPDINV_ERR_N;
    const int b = (o && o->tile > 0) ? o->tile : default_tile(n);
    if (b != 32 && b != 64 && b != 128) return SPDINV_ERR_UNSUPPORTED;
    // tile 128: the whole inversion, default variant, no trace (potri_fp64_b128.cu)
    if (b == 128 && (steps != STEPS_ALL || (o && o->variant != 0))) return SPDINV_ERR_UNSUPPORTED;
    if (o && o->precision != SPDINV_PREC_FP64) return SPDINV_ERR_UNSUPPORTED;
    const int64_t t64 = (n + b - 1) / b;
    if (t64 > 16383) return SPDINV_ERR_N;
    Fp64Layout L;
    L.b = b;
    L.t = (int)t64;
    L.variant = o ? o->variant : 0;
    if (L.variant & ~kVariantMask) return SPDINV_ERR_UNSUPPORTED;
    const bool split = L.variant & VAR_SPLIT3, shared = L.variant & (VAR_SHARE_BC | VAR_INPLACE);
    if (L.variant && steps != STEPS_ALL) return SPDINV_ERR_UNSUPPORTED;
    if (split && shared) return SPDINV_ERR_UNSUPPORTED;
    if (split) {
        L.seg = o->split_segment > 0 ? o->split_segment : 16;
        if (L.seg > 16383) return SPDINV_ERR_UNSUPPORTED;
        for (int i = 0; i < L.t; ++i) {  // the partial tiles of row i: (i + 1) chains of t - 1 - i
            const int m = L.t - 1 - i;
            if (m > L.seg) L.nparts += (int64_t)(i + 1) * ((m + L.seg - 1) / L.seg - 1);
        }
    }
    L.needB = steps != STEPS_LAUUM;
    L.needC = steps != STEPS_POTRF && !shared;  // shared variants keep X in B's slots
    if (n > 0) {
        const size_t tile_bytes = (size_t)b * b * sizeof(double);  // a multiple of 256
        const size_t ntri = (size_t)L.t * (L.t - 1) / 2;
        size_t words = 4 + 2 * (size_t)L.t * L.t + L.t;              // status words, flags
        if (L.variant) words += 2 * (size_t)L.t * L.t + L.t + (size_t)L.nparts;  // read counters, partials' flags
        L.ctrl = align_up(sizeof(int) * words, 256);
        L.B = L.needB ? ntri * tile_bytes : 0;
        L.C = L.needC ? ntri * tile_bytes : 0;
        L.D = (size_t)L.t * tile_bytes;
        L.P = (size_t)L.nparts * tile_bytes;
        L.total = L.ctrl + L.B + L.C + L.D + L.P;
    }
    *out = L;
    return SPDINV_OK;
}

// Shared body of potrf / trtri / lauum / potri (FP64).
spdinv_status run_fp64(int64_t n, double* dA, int64_t lda, int steps, const spdinv_opts* o, int* d_info,
                       cudaStream_t stream, double* d_diag) {
    if (n < 0) return SPDINV_ERR_N;
    if (lda < (n > 1 ? n : 1)) return SPDINV_ERR_LDA;
    if (n > 0 && dA == nullptr) return SPDINV_ERR_NULL;
    if (steps == STEPS_DIAG && n > 0 && d_diag == nullptr) return SPDINV_ERR_NULL;
    Fp64Layout W;
    const spdinv_status ls = fp64_layout(n, steps, o, &W);
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

    const int t = W.t, b = W.b;
    void* wsp = nullptr;
    const spdinv_status ws = ds.acquire(W.total, &wsp);
    if (ws != SPDINV_OK) return ws;
    if (debug_flags().load(std::memory_order_relaxed) & SPDINV_DEBUG_POISON) {
        e = cudaMemsetAsync(static_cast<char*>(wsp) + W.ctrl, 0xFF, W.total - W.ctrl, stream);  // B, C, D
        if (e != cudaSuccess) return cuda_fail(e);
    }

    KParamsF64 p{};
    p.n = n;
    p.lda = lda;
    p.t = t;
    p.b = b;
    p.steps = steps;
    p.A = dA;
    char* base = static_cast<char*>(wsp);
    p.ctrl = reinterpret_cast<int*>(base);
    p.flags = p.ctrl + 4;
    p.Bw = W.needB ? reinterpret_cast<double*>(base + W.ctrl) : nullptr;
    p.Cw = W.needC ? reinterpret_cast<double*>(base + W.ctrl + W.B) : nullptr;
    p.Dw = reinterpret_cast<double*>(base + W.ctrl + W.B + W.C);
    p.timeout_ns = (long long)(wait_timeout_s(o) * 1e9);
    p.drop_task = (o && o->wait_timeout_s > 0 && o->fault_drop_task >= 0) ? o->fault_drop_task : -1;
    p.diag = d_diag;
    p.variant = W.variant;
    if (W.variant) {
        if (W.variant & (VAR_SHARE_BC | VAR_INPLACE)) p.Cw = p.Bw;  // X in L's slots
        const size_t tt = (size_t)t * t;
        p.reads = p.flags + 2 * tt + t;
        p.fP = p.reads + 2 * tt + t;
        p.Pw = reinterpret_cast<double*>(base + W.ctrl + W.B + W.C + W.D);
        const DevicePlan* vp = nullptr;
        e = ds.variant_plan(t, W.variant, W.seg, &vp);
        if (e != cudaSuccess) return cuda_fail(e);
        p.tasks = vp->d_tasks;
        p.ntasks = vp->ntasks;
        p.parts = vp->d_parts;
        p.split = vp->d_split;
    } else {
        e = ds.exec_plan(t, steps, &p.tasks, &p.ntasks);
        if (e != cudaSuccess) return cuda_fail(e);
    }

    if (ds.trace) {
        if (b == 128) return SPDINV_ERR_UNSUPPORTED;
        if (p.ntasks > ds.trace_cap) return SPDINV_ERR_WORKSPACE;
        p.trace = ds.trace;
    }
    e = cudaMemsetAsync(p.ctrl, 0, W.ctrl, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int grid = 0;
    const int per = (o && o->ctas_per_sm > 0) ? o->ctas_per_sm : 0;
    void* tok = nullptr;
    timing_begin(SPDINV_TIMED_FP64_DAG, stream, &tok);
    e = launch_potri_fp64(p, per, ds.num_sms, d_info, stream, &grid);
    if (e != cudaSuccess) return cuda_fail(e);
    const double n3 = (double)n * (double)n * (double)n;  // leading terms: n^3 / 3 per step
    timing_end(SPDINV_TIMED_FP64_DAG, stream, tok,
               steps == STEPS_ALL ? n3 : (steps == STEPS_DIAG ? 2.0 * n3 / 3.0 : n3 / 3.0));
    count_launches(1 + (d_info ? 1 : 0) + ((steps == STEPS_TRTRI || steps == STEPS_LAUUM) ? 1 : 0) +
                   ((W.variant & VAR_INPLACE) ? 1 : 0));
    ds.last_grid = grid;
    return SPDINV_OK;
}

}  // namespace spdinv

using namespace spdinv;

extern "C" {

spdinv_status spdinv_potrf(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream) {
    return log_status("spdinv_potrf", "n", n, run_fp64(n, dA, lda, STEPS_POTRF, nullptr, d_info, stream));
}

spdinv_status spdinv_trtri(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream) {
    return log_status("spdinv_trtri", "n", n, run_fp64(n, dA, lda, STEPS_TRTRI, nullptr, d_info, stream));
}

spdinv_status spdinv_lauum(int64_t n, double* dA, int64_t lda, cudaStream_t stream) {
    return log_status("spdinv_lauum", "n", n, run_fp64(n, dA, lda, STEPS_LAUUM, nullptr, nullptr, stream));
}

spdinv_status spdinv_potri(int64_t n, double* dA, int64_t lda, int* d_info, cudaStream_t stream) {
    return log_status("spdinv_potri", "n", n, run_fp64(n, dA, lda, STEPS_ALL, nullptr, d_info, stream));
}

spdinv_status spdinv_potri_ex(int64_t n, double* dA, int64_t lda, const spdinv_opts* opts, int* d_info,
                              cudaStream_t stream) {
    if (opts && opts->precision != SPDINV_PREC_FP64)
        return log_status("spdinv_potri_ex", "n", n, run_mixed(n, dA, lda, opts, d_info, stream));
    return log_status("spdinv_potri_ex", "n", n, run_fp64(n, dA, lda, STEPS_ALL, opts, d_info, stream));
}

spdinv_status spdinv_potri_diag(int64_t n, const double* dA, int64_t lda, double* d_diag, int* d_info,
                                cudaStream_t stream) {
    // A is only read: Step 3 keeps just the diagonal of each diagonal tile.
    return log_status("spdinv_potri_diag", "n", n,
                      run_fp64(n, const_cast<double*>(dA), lda, STEPS_DIAG, nullptr, d_info, stream, d_diag));
}

spdinv_status spdinv_workspace_size(int64_t n, int routine, const spdinv_opts* opts, size_t* bytes) {
    if (!bytes) return SPDINV_ERR_NULL;
    spdinv_status st = SPDINV_OK;
    if (routine == SPDINV_ROUTINE_INVERSE_RESIDUAL) {
        size_t need = 0;
        st = residual_workspace(n, opts ? opts->residual : SPDINV_RESIDUAL_EMULATED, &need);
        if (st == SPDINV_OK) *bytes = need;
        return st;
    }
    if (routine < SPDINV_ROUTINE_POTRI || routine > SPDINV_ROUTINE_POTRI_DIAG) return SPDINV_ERR_UNSUPPORTED;
    if (routine == SPDINV_ROUTINE_POTRI && opts && opts->precision != SPDINV_PREC_FP64) {
        MixedLayout L;
        st = mixed_layout(n, opts, &L);
        if (st == SPDINV_OK) *bytes = L.total;
        return st;
    }
    // The routine numbers are the plan's step sets; only spdinv_potri_ex takes options.
    Fp64Layout L;
    st = fp64_layout(n, routine, routine == SPDINV_ROUTINE_POTRI ? opts : nullptr, &L);
    if (st == SPDINV_OK) *bytes = L.total;
    return st;
}

static spdinv_status set_workspace(void* d_ws, size_t bytes) {
    if (d_ws && (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return SPDINV_ERR_WORKSPACE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (d_ws) {
        cudaPointerAttributes at{};
        e = cudaPointerGetAttributes(&at, d_ws);
        if (e != cudaSuccess) return cuda_fail(e);
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return SPDINV_ERR_WORKSPACE;
    }
    DeviceState& ds = device_state(dev);
    std::lock_guard<std::mutex> lk(ds.mu);
    ds.user_ws = d_ws;
    ds.user_bytes = d_ws ? bytes : 0;
    return SPDINV_OK;
}

static spdinv_status set_trace(spdinv_trace_record* d_records, int64_t capacity) {
    if (d_records && capacity < 1) return SPDINV_ERR_N;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    DeviceState& ds = device_state(dev);
    std::lock_guard<std::mutex> lk(ds.mu);
    ds.trace = d_records;
    ds.trace_cap = d_records ? capacity : 0;
    return SPDINV_OK;
}

spdinv_status spdinv_set_trace(spdinv_trace_record* d_records, int64_t capacity) {
    return log_status("spdinv_set_trace", "capacity", capacity, set_trace(d_records, capacity));
}

spdinv_status spdinv_set_workspace(void* d_ws, size_t bytes) {
    return log_status("spdinv_set_workspace", "bytes", (int64_t)bytes, set_workspace(d_ws, bytes));
}

spdinv_status spdinv_dag_critical_path(int t, int flags, int64_t out[4]) {
    if (t < 1 || t > 256 || ((flags & (SPDINV_DAG_TREE | SPDINV_DAG_TREE_STEP3)) && t > 128)) return SPDINV_ERR_N;
    if (!out) return SPDINV_ERR_NULL;
    dag_critical_path(t, flags, out);
    return SPDINV_OK;
}

spdinv_status spdinv_dag_task_counts(int t, int64_t out[12]) {
    if (t < 1) return SPDINV_ERR_N;
    if (!out) return SPDINV_ERR_NULL;
    dag_task_counts(t, out);
    return SPDINV_OK;
}

spdinv_status spdinv_plan_check(int t, int steps, int64_t out[3]) {
    if (t < 1 || t > 16383) return SPDINV_ERR_N;
    if (steps < 0 || steps > 4) return SPDINV_ERR_UNSUPPORTED;
    if (!out) return SPDINV_ERR_NULL;
    out[1] = out[2] = 0;
    for (int order : {(int)ORDER_BOTTOM_LEVEL, (int)ORDER_ALAP}) {
        const ExecPlan a = build_exec_plan(t, steps, false, order), b = build_exec_plan(t, steps, true, order);
        int64_t diff = 0;
        for (size_t m = 0; m < a.order.size() && m < b.order.size(); ++m) diff += a.order[m] != b.order[m];
        out[0] = (int64_t)a.order.size();
        out[1] += diff + (int64_t)(a.order.size() > b.order.size() ? a.order.size() - b.order.size()
                                                                    : b.order.size() - a.order.size());
        if (a.crit != b.crit || a.work != b.work) out[2] = 1;
    }
    return SPDINV_OK;
}

spdinv_status spdinv_plan_tasks(int64_t n, int b, int steps, uint32_t* out, int64_t cap, int64_t* ntasks,
                                double* crit) {
    if (n < 1 || b < 1) return SPDINV_ERR_N;
    if (steps < 0 || steps > 4) return SPDINV_ERR_UNSUPPORTED;
    if (!ntasks || (cap > 0 && !out)) return SPDINV_ERR_NULL;
    const int64_t t = (n + b - 1) / b;
    if (t > 16383) return SPDINV_ERR_N;
    ExecPlan p = build_exec_plan((int)t, steps, false, current_plan_order());
    *ntasks = (int64_t)p.order.size();
    if (crit) *crit = p.crit;
    const int64_t m = cap < *ntasks ? cap : *ntasks;
    if (m > 0) std::memcpy(out, p.order.data(), sizeof(uint32_t) * (size_t)m);
    return SPDINV_OK;
}

const char* spdinv_status_name(int status) { return status_name(status); }

int spdinv_set_plan_order(int order) {
    if (order != SPDINV_PLAN_BOTTOM_LEVEL && order != SPDINV_PLAN_ALAP) return SPDINV_ERR_UNSUPPORTED;
    return set_plan_order(order);
}

unsigned spdinv_set_debug_flags(unsigned flags) { return debug_flags().exchange(flags); }

const char* spdinv_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

uint64_t spdinv_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int spdinv_version(void) { return 10200; }

}  // extern "C"
