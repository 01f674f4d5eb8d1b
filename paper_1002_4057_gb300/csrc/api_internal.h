// Host-side state shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "../../include/spdinv.h"
#include "plan.h"

namespace spdinv {

struct DevicePlan {
    uint32_t* d_tasks = nullptr;  // one allocation: tasks, then (split variant) parts and split tables
    const PartTask* d_parts = nullptr;
    const SplitInfo* d_split = nullptr;
    int ntasks = 0;
};

// One per CUDA device: the workspace (renamed stores, flags) and the plans.
struct DeviceState {
    std::mutex mu;
    int num_sms = 0;
    void* ws = nullptr;       // the library's own workspace, grown on demand
    size_t ws_bytes = 0;
    void* user_ws = nullptr;  // a caller's buffer (spdinv_set_workspace), used instead when set
    size_t user_bytes = 0;
    int last_grid = 0;
    spdinv_trace_record* trace = nullptr;  // spdinv_set_trace
    int64_t trace_cap = 0;
    // (t, steps, ticket order, variant, split segment) -> plan
    std::map<std::tuple<int, int, int, int, int>, DevicePlan> plans;
    cudaError_t ensure_workspace(size_t bytes);
    // The workspace of one call: the caller's buffer when one is set
    // (SPDINV_ERR_WORKSPACE when it is too small; nothing is allocated), else
    // the library's own.  Call with mu held.
    spdinv_status acquire(size_t bytes, void** out);
    cudaError_t exec_plan(int t, int steps, const uint32_t** d_tasks, int* ntasks);
    // The plan of an execution variant (STEPS_ALL); cudaErrorInvalidValue for
    // an unsupported combination.
    cudaError_t variant_plan(int t, int variant, int seg, const DevicePlan** out);
};

// Workspace layouts of the single-matrix calls (byte offsets from the
// workspace base; every part starts on a 256-byte boundary).  The same
// functions size the calls and answer spdinv_workspace_size.
struct Fp64Layout {
    int b = 0, t = 0;
    int variant = 0, seg = 0;                         // execution variant (spdinv_opts.variant)
    int64_t nparts = 0;                               // split variant: partial tiles
    bool needB = false, needC = false;                // the call uses the store B (L) / C (X)
    // sizes of the parts, in this order; ctrl holds the status words, the
    // flags and, for the variants, the read counters and the partials' flags
    size_t ctrl = 0, B = 0, C = 0, D = 0, P = 0, total = 0;
};
struct MixedLayout {
    int b = 0, t = 0, order = 2;  // tile, tiles per side, correction order
    size_t ctrl = 0, BC = 0, D = 0, nn = 0, oz = 0, total = 0;  // ctrl, B, C, D, X0 [, R, X1, slices]
};
// Argument checks that need no device (the status of the call, or
// SPDINV_OK) and the layout of a call with those arguments.
spdinv_status fp64_layout(int64_t n, int steps, const spdinv_opts* o, Fp64Layout* out);
spdinv_status mixed_layout(int64_t n, const spdinv_opts* o, MixedLayout* out);
spdinv_status residual_workspace(int64_t n, int residual, size_t* bytes);

DeviceState& device_state(int dev);
void count_launches(int k);
// Kernel timing (spdinv_set_kernel_timing): an event before and after a
// launch of kind `which` (SPDINV_TIMED_*) on stream s when timing is on;
// `flops` is the launch's algorithmic work, summed for the report.
void timing_begin(int which, cudaStream_t s, void** token);
void timing_end(int which, cudaStream_t s, void* token, double flops);
// The default limit of one dependency wait, in seconds: opts->wait_timeout_s
// when positive, else SPDINV_WAIT_TIMEOUT_S from the environment, else 60.
double wait_timeout_s(const spdinv_opts* o);
spdinv_status cuda_fail(cudaError_t e);
// With SPDINV_LOG=1 in the environment, a call that returns an error status
// prints one line to stderr (SPDINV_LOG=2: every call); returns st.
spdinv_status log_status(const char* fn, const char* size_name, int64_t size, spdinv_status st);
// d_diag: STEPS_DIAG only, receives diag(A^{-1}).
spdinv_status run_fp64(int64_t n, double* dA, int64_t lda, int steps, const spdinv_opts* o, int* d_info,
                       cudaStream_t stream, double* d_diag = nullptr);
// FP32 backward on the tensor cores (backward_tc.cu); arguments already checked.
spdinv_status backward_f32_tc(int batch, int64_t n, const float* dX, int64_t ldx, int64_t sx, const float* dG,
                              int64_t ldg, int64_t sg, float* dGrad, int64_t ldr, int64_t sr, cudaStream_t stream);
spdinv_status run_mixed(int64_t n, double* dA, int64_t lda, const spdinv_opts* o, int* d_info,
                        cudaStream_t stream);

}  // namespace spdinv
