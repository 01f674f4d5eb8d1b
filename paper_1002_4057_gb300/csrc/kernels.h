// Kernel entry points and their parameter blocks (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/spdinv.h"
#include "plan.h"

namespace spdinv {

struct KParamsF64 {
    int64_t n;            // matrix order
    int64_t lda;          // leading dimension of A
    int t;                // tiles per side, ceil(n / b)
    int b;                // tile order
    int steps;            // PlanSteps
    int ntasks;           // tasks in the plan
    double* A;            // column-major matrix (lower triangle used)
    double* Bw;           // renamed store of L: t(t-1)/2 tiles, tile-major
    double* Cw;           // renamed store of X = L^{-1}: t(t-1)/2 tiles
    double* Dw;           // inverted diagonal tiles X_jj: t tiles
    const uint32_t* tasks;  // plan order (device)
    int* flags;           // readiness flags: [t*t] L, [t*t] X, [t] D
    int* ctrl;            // [0] ticket, [1] abort, [2] error, [3] info
    long long timeout_ns; // limit of one dependency wait
    int drop_task;        // failure-injection hook (-1 = off)
    double* diag;         // STEPS_DIAG: receives diag(A^{-1}) (n entries); A is not written
    // Execution variants (PlanVariant flags; 0 = the renamed, pipelined plan).
    int variant;
    int* reads;             // read counters: [t*t] of L (B), [t*t] of X (C), [t] of D
    const PartTask* parts;  // VAR_SPLIT3: segments by part id
    const SplitInfo* split; // VAR_SPLIT3: per Step-3 tile, tri_index(i, j)
    double* Pw;             // VAR_SPLIT3: partial tiles by part id, tile-major
    int* fP;                // VAR_SPLIT3: their readiness flags
    spdinv_trace_record* trace;  // per-task trace, indexed by ticket (nullptr = off)
};

// Queues the FP64 persistent inversion (plus the stage-in copy for the
// standalone TRTRI / LAUUM and, with d_info, the status write).
cudaError_t launch_potri_fp64(const KParamsF64& p, int ctas_per_sm, int num_sms, int* d_info, cudaStream_t s,
                              int* grid_out);
// The b = 128 kernel (potri_fp64_b128.cu): the whole inversion only, one
// 256-thread CTA per SM.
cudaError_t launch_potri_fp64_b128(const KParamsF64& p, int num_sms, cudaStream_t s, int* grid_out);

}  // namespace spdinv
