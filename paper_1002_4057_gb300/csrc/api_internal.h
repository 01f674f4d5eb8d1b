// Host-side state shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/spdinv.h"

namespace spdinv {

struct DevicePlan {
    uint32_t* d_tasks = nullptr;
    int ntasks = 0;
};

// One per CUDA device: the workspace (renamed stores, flags) and the plans.
struct DeviceState {
    std::mutex mu;
    int num_sms = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int last_grid = 0;
    std::map<std::pair<int, int>, DevicePlan> plans;  // (t, steps) -> plan
    cudaError_t ensure_workspace(size_t bytes);
    cudaError_t exec_plan(int t, int steps, const uint32_t** d_tasks, int* ntasks);
};

DeviceState& device_state(int dev);
void count_launches(int k);
spdinv_status cuda_fail(cudaError_t e);
// d_diag: STEPS_DIAG only, receives diag(A^{-1}).
spdinv_status run_fp64(int64_t n, double* dA, int64_t lda, int steps, const spdinv_opts* o, int* d_info,
                       cudaStream_t stream, double* d_diag = nullptr);
spdinv_status run_mixed(int64_t n, double* dA, int64_t lda, const spdinv_opts* o, int* d_info,
                        cudaStream_t stream);

}  // namespace spdinv
