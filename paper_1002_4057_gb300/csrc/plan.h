// Host-side planner: the paper's task DAG analysis and the execution plan of
// the persistent kernel.
#pragma once
#include <cstdint>
#include <vector>

namespace spdinv {

// Chain-task kinds of the execution plan (one task per output tile and step).
enum TaskKind : uint32_t {
    K_S1_DIAG = 0,  // Step 1, diagonal tile: SYRK chain, POTRF, then TRTRI of the factor
    K_S1_OFF = 1,   // Step 1, off-diagonal tile: GEMM chain, then TRSM as TRMM by X_jj^T
    K_S2_DIAG = 2,  // Step 2, diagonal tile (TRTRI alone: spdinv_trtri only)
    K_S2_OFF = 3,   // Step 2, off-diagonal tile: TRMM, GEMM chain, TRMM
    K_S3_DIAG = 4,  // Step 3, diagonal tile: LAUUM, SYRK chain
    K_S3_OFF = 5,   // Step 3, off-diagonal tile: TRMM, GEMM chain
};

#if defined(__CUDACC__)
#define SPDINV_HD __host__ __device__
#else
#define SPDINV_HD
#endif
SPDINV_HD inline uint32_t encode_task(uint32_t kind, uint32_t i, uint32_t j) { return (kind << 28) | (i << 14) | j; }
SPDINV_HD inline uint32_t task_kind(uint32_t e) { return e >> 28; }
SPDINV_HD inline uint32_t task_i(uint32_t e) { return (e >> 14) & 0x3FFFu; }
SPDINV_HD inline uint32_t task_j(uint32_t e) { return e & 0x3FFFu; }

// STEPS_DIAG: Steps 1 and 2 in full and, of Step 3, only the diagonal tiles
// (the selected inverse diag(A^{-1})).
enum PlanSteps { STEPS_ALL = 0, STEPS_POTRF = 1, STEPS_TRTRI = 2, STEPS_LAUUM = 3, STEPS_DIAG = 4 };

struct ExecPlan {
    int t = 0;
    int steps = 0;
    std::vector<uint32_t> order;  // tasks in the order CTAs take them
    double crit = 0.0;            // weighted critical path (tile-product units)
    double work = 0.0;            // total weight
};

// Ticket order of a plan (both are topological, so any grid is free of
// deadlock, and the result does not depend on the order: every output tile
// keeps its own accumulation order).
//   ORDER_BOTTOM_LEVEL  decreasing task-level bottom level (the default);
//   ORDER_ALAP          increasing latest finish time of each task in the
//                       element-pipelined schedule on unlimited CTAs (each
//                       chain element starts when its own inputs are final),
//                       raised to the largest key among the task's producers
//                       so that the order stays topological.  O(t^3).
enum PlanOrder { ORDER_BOTTOM_LEVEL = 0, ORDER_ALAP = 1 };

// The order the library plans with: ORDER_BOTTOM_LEVEL unless
// SPDINV_PLAN_ORDER=alap (or 1) in the environment or spdinv_set_plan_order.
int current_plan_order();
int set_plan_order(int order);  // returns the previous one

// Builds the chain-task plan for t x t tiles (t <= 16383).  The bottom
// levels that order it take O(t^2); exhaustive walks every dependency edge,
// O(t^3) -- the same result, kept to check the fast path.
ExecPlan build_exec_plan(int t, int steps, bool exhaustive = false, int order = ORDER_BOTTOM_LEVEL);

// Fine-grained DAG of Algorithm 1 / its Sec. 3 variants: critical paths.
void dag_critical_path(int t, int flags, int64_t out[4]);
void dag_task_counts(int t, int64_t out[12]);

}  // namespace spdinv
