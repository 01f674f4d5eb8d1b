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
    K_S3_PART = 6,  // Step 3, one segment of a split chain into a partial tile (word: kind, part id)
};

// Execution variants of the FP64 plan (Sec. 3's study, on the GPU; STEPS_ALL only).
enum PlanVariant : int {
    VAR_UUU = 1,       // Step 2's chains in increasing k (loop reversal: U, U, U instead of U, D, U)
    VAR_SHARE_BC = 2,  // C (X = L^{-1}) in B's slots (L): renaming under a memory budget (Sec. 4)
    VAR_INPLACE = 4,   // one store: L, X and A^{-1} overwrite each other tile by tile (no renaming)
    VAR_SPLIT3 = 8,    // Step 3 chains split into segments with partial sums (associative reduction, Sec. 4)
};
constexpr int kVariantMask = VAR_UUU | VAR_SHARE_BC | VAR_INPLACE | VAR_SPLIT3;

// A segment of a split Step-3 chain: sum over k0 <= k < k1 of X_ki^T X_kj.
struct PartTask {
    uint16_t i, j, k0, k1;
};
// Split of the Step-3 chain of tile (i, j): its task runs k < own_end itself,
// then adds the partial tiles first .. first + np - 1 (np = 0: not split).
struct SplitInfo {
    uint32_t first;
    uint16_t np, own_end;
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
SPDINV_HD inline uint32_t encode_part(uint32_t id) { return ((uint32_t)K_S3_PART << 28) | id; }
SPDINV_HD inline uint32_t part_id(uint32_t e) { return e & 0x0FFFFFFFu; }
SPDINV_HD inline int64_t tri_index(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }  // j <= i

// Number of readers of each stored tile in the chain-task plan (STEPS_ALL):
// a task that reads a tile twice counts twice.  With shared storage a tile's
// next version may be stored only after all of them have read it.
SPDINV_HD inline int readers_L(int t, int a, int b) { return 2 * t - a - b - 1; }  // L_ab, a > b
SPDINV_HD inline int readers_X(int t, int a, int b) { (void)t; return a + b + 1; }  // X_ab, a > b
SPDINV_HD inline int readers_D(int t, int j) { (void)j; return 2 * t - 1; }         // X_jj


// STEPS_DIAG: Steps 1 and 2 in full and, of Step 3, only the diagonal tiles
// (the selected inverse diag(A^{-1})).
enum PlanSteps { STEPS_ALL = 0, STEPS_POTRF = 1, STEPS_TRTRI = 2, STEPS_LAUUM = 3, STEPS_DIAG = 4 };

struct ExecPlan {
    int t = 0;
    int steps = 0;
    int variant = 0, seg = 0;
    std::vector<uint32_t> order;  // tasks in the order CTAs take them
    std::vector<PartTask> parts;  // VAR_SPLIT3: the segments, by part id
    std::vector<SplitInfo> split; // VAR_SPLIT3: per Step-3 tile, tri_index(i, j)
    double crit = 0.0;            // weighted critical path (tile-product units)
    double work = 0.0;            // total weight
};

// Ticket order of a plan (both are topological, so any grid is free of
// deadlock, and the result does not depend on the order: every output tile
// keeps its own accumulation order).
//   ORDER_BOTTOM_LEVEL  decreasing task-level bottom level;
//   ORDER_ALAP          increasing latest finish time of each task in the
//                       element-pipelined schedule on unlimited CTAs (each
//                       chain element starts when its own inputs are final),
//                       raised to the largest key among the task's producers
//                       so that the order stays topological.  O(t^3)
//                       chain elements, walked along rows and columns of
//                       the task grids (exhaustive: producer by producer).
enum PlanOrder { ORDER_BOTTOM_LEVEL = 0, ORDER_ALAP = 1 };

// The order the library plans with: ORDER_ALAP unless
// SPDINV_PLAN_ORDER=bottom_level (or 0) in the environment or
// spdinv_set_plan_order says otherwise.
int current_plan_order();
int set_plan_order(int order);  // returns the previous one

// Builds the chain-task plan for t x t tiles (t <= 16383).  The bottom
// levels that order it take O(t^2); exhaustive walks every dependency edge,
// O(t^3) -- the same result, kept to check the fast path.
ExecPlan build_exec_plan(int t, int steps, bool exhaustive = false, int order = ORDER_BOTTOM_LEVEL);

// The plan of an execution variant (PlanVariant flags, STEPS_ALL; 0 = the
// plan above), ordered by decreasing bottom level over every dependency --
// read after write and, with shared storage, write after read -- walked
// edge by edge (O(t^3)).  seg: VAR_SPLIT3's segment length (chains of more
// than seg elements are split into ceil(m / seg) segments).  Returns false
// for an unsupported combination (VAR_SPLIT3 with VAR_SHARE_BC or
// VAR_INPLACE, seg < 1 with VAR_SPLIT3).
bool build_variant_plan(int t, int variant, int seg, ExecPlan* out);

// Fine-grained DAG of Algorithm 1 / its Sec. 3 variants: critical paths.
void dag_critical_path(int t, int flags, int64_t out[4]);
void dag_task_counts(int t, int64_t out[12]);

}  // namespace spdinv
