// Host planner.
//
// (1) dag_critical_path: the fine-grained task DAG of Algorithm 1 (Sec. 2)
//     and of its variants studied in Sec. 3 -- array renaming (out-of-place,
//     Table 1), loop reversal (UDU vs UUU) and pipelining of the three steps.
//     Tasks are unfolded in their sequential order and the hazards on tiles
//     (read after write, write after read, write after write) become edges,
//     which is how the paper's dynamic scheduler builds its DAG (Sec. 1).
//     Every task weighs one unit; tile copies weigh zero.
//
// (2) build_exec_plan: the plan the persistent kernel runs.  Each task owns
//     one output tile of one step and carries that tile's whole commutative
//     update chain (Sec. 3, "loop reversal": the innermost GEMMs of each step
//     commute), in the loop orders U (Step 1), D (Step 2), U (Step 3) that the
//     paper chose because they shorten the critical path.  Renamed stores
//     B (L), C (L^{-1}) and D (inverted diagonal tiles) remove every
//     write-after-read hazard, so a task depends only on the tiles it reads.
//     Tasks are ordered by increasing latest finish time in the
//     element-pipelined schedule (ORDER_ALAP, the default; alap_order_grid)
//     or by decreasing bottom level (longest weighted path to the end;
//     ORDER_BOTTOM_LEVEL, also the order of the execution variants).  Both
//     are topological orders: a CTA only ever waits for tasks taken before
//     its own, so the persistent kernel cannot deadlock.
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/spdinv.h"

namespace spdinv {

// --------------------------------------------------------------------------
// (1) fine-grained DAG
// --------------------------------------------------------------------------
namespace {

struct HazardSim {
    // Per address: finish time of the last writer and the latest finish of
    // the readers since that write.
    std::vector<int64_t> last_write, last_reads;
    int64_t span = 0;
    explicit HazardSim(size_t naddr) : last_write(naddr, 0), last_reads(naddr, 0) {}
    void reset() {
        std::fill(last_write.begin(), last_write.end(), 0);
        std::fill(last_reads.begin(), last_reads.end(), 0);
        span = 0;
    }
    // One task: start when every RAW/WAW/WAR predecessor has finished.
    void task(std::initializer_list<int64_t> reads, std::initializer_list<int64_t> writes, int64_t w) {
        int64_t start = 0;
        for (int64_t a : reads) start = std::max(start, last_write[a]);
        for (int64_t a : writes) start = std::max({start, last_write[a], last_reads[a]});
        const int64_t fin = start + w;
        for (int64_t a : reads) last_reads[a] = std::max(last_reads[a], fin);
        for (int64_t a : writes) {
            last_write[a] = fin;
            last_reads[a] = 0;
        }
        span = std::max(span, fin);
    }
};

}  // namespace

void dag_critical_path(int t, int flags, int64_t out[4]) {
    const bool oop = flags & SPDINV_DAG_OUT_OF_PLACE;
    const bool rdiag = flags & SPDINV_DAG_RENAME_DIAG;
    const bool uuu = flags & SPDINV_DAG_UUU;
    const bool pipe = flags & SPDINV_DAG_PIPELINE;
    const bool tree_all = flags & SPDINV_DAG_TREE, tree3 = tree_all || (flags & SPDINV_DAG_TREE_STEP3);
    bool tree = false;  // the current step's chains are tree-reduced
    const int64_t T = t;
    // address spaces: A(i,j), B(i,j), C(i,j), D(j), then one fresh temporary
    // per product of a tree-reduced chain
    auto A = [&](int64_t i, int64_t j) { return i * T + j; };
    auto B = [&](int64_t i, int64_t j) { return T * T + i * T + j; };
    // SPDINV_DAG_SHARE_BC: C (the copy of L^{-1}) reuses B's storage (the
    // copy of L), the memory-constrained renaming of Sec. 4: half the extra
    // memory, at the price of the hazards between Step 2's reads of B and
    // Step 3's copies into C.
    const bool share = flags & SPDINV_DAG_SHARE_BC;
    auto C = [&](int64_t i, int64_t j) { return (share ? T * T : 2 * T * T) + i * T + j; };
    auto D = [&](int64_t j) { return 3 * T * T + j; };
    const int64_t base = 3 * T * T + T;
    // temporaries per pass: each chain of m products takes m + (m - 1); the
    // products per pass are 3 T(T-1)(T-2)/6 GEMMs + T(T-1) SYRKs < T^3/2 + T^2
    const int64_t ntmp = tree3 ? T * T * T + 2 * T * T + 8 : 0;
    HazardSim sim(base + ntmp);
    HazardSim whole(base + ntmp);
    int64_t step_cp[3] = {0, 0, 0};
    int64_t next_tmp = base;
    // One commutative update chain acc <- acc + sum_q P_q, P_q reading the
    // tiles ins[q] (Sec. 3: its order is free).  Without SPDINV_DAG_TREE it
    // is m sequential tasks on acc.  With it (the associative reduction the
    // paper names for shortening the critical path): m products into fresh
    // temporaries, a pairwise reduction tree, and one update of acc -- depth
    // 1 + ceil(log2 m) + 1 instead of m.
    auto chain = [&](HazardSim& s, int64_t acc, const std::vector<std::vector<int64_t>>& ins) {
        const size_t m = ins.size();
        if (!tree || m < 2) {
            for (const auto& r : ins) {
                if (r.size() == 1) s.task({acc, r[0]}, {acc}, 1);
                else s.task({acc, r[0], r[1]}, {acc}, 1);
            }
            return;
        }
        std::vector<int64_t> tmp(m);
        for (size_t q = 0; q < m; ++q) {
            tmp[q] = next_tmp++;
            if (ins[q].size() == 1) s.task({ins[q][0]}, {tmp[q]}, 1);
            else s.task({ins[q][0], ins[q][1]}, {tmp[q]}, 1);
        }
        while (tmp.size() > 1) {  // each level writes fresh temporaries: no false hazards
            std::vector<int64_t> up;
            for (size_t q = 0; q + 1 < tmp.size(); q += 2) {
                up.push_back(next_tmp++);
                s.task({tmp[q], tmp[q + 1]}, {up.back()}, 1);
            }
            if (tmp.size() % 2) up.push_back(tmp.back());
            tmp.swap(up);
        }
        s.task({acc, tmp[0]}, {acc}, 1);
    };

    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: each step's own DAG (state reset between steps);
        // pass 1: the whole inversion with one continuing state (pipelined).
        HazardSim& s = pass == 0 ? sim : whole;
        next_tmp = base;  // each pass has its own simulator, so its own temporaries
        // ---- Step 1: tile Cholesky (Algorithm 1, Step 1)
        if (pass == 0) s.reset();
        tree = tree_all;
        for (int64_t j = 0; j < T; ++j) {
            std::vector<std::vector<int64_t>> ins;
            for (int64_t k = 0; k < j; ++k) ins.push_back({A(j, k)});
            chain(s, A(j, j), ins);           // SYRK
            s.task({A(j, j)}, {A(j, j)}, 1);  // POTRF
            for (int64_t i = j + 1; i < T; ++i) {
                ins.clear();
                for (int64_t k = 0; k < j; ++k) ins.push_back({A(i, k), A(j, k)});
                chain(s, A(i, j), ins);  // GEMM
            }
            for (int64_t i = j + 1; i < T; ++i) s.task({A(i, j), A(j, j)}, {A(i, j)}, 1);  // TRSM
        }
        if (pass == 0) step_cp[0] = s.span;
        // ---- Step 2: tile triangular inversion (Algorithm 1, Step 2)
        if (pass == 0) s.reset();
        if (oop)
            for (int64_t i = 0; i < T; ++i)
                for (int64_t j = 0; j < i; ++j) s.task({A(i, j)}, {B(i, j)}, 0);  // B <- A
        for (int64_t j = T - 1; j >= 0; --j) {
            if (rdiag) s.task({A(j, j)}, {D(j)}, 1);  // TRTRI into D_j
            else s.task({A(j, j)}, {A(j, j)}, 1);     // TRTRI in place
            const int64_t Xj = rdiag ? D(j) : A(j, j);
            for (int64_t i = T - 1; i > j; --i) {
                const int64_t Xi = rdiag ? D(i) : A(i, i);
                s.task({Xi, A(i, j)}, {A(i, j)}, 1);  // TRMM: A_ij <- X_ii A_ij
                std::vector<std::vector<int64_t>> ins;
                for (int64_t m = 0; m < i - j - 1; ++m) {
                    const int64_t k = uuu ? j + 1 + m : i - 1 - m;  // U or D order
                    ins.push_back({A(i, k), oop ? B(k, j) : A(k, j)});
                }
                chain(s, A(i, j), ins);  // GEMM
                s.task({A(i, j), Xj}, {A(i, j)}, 1);  // TRMM: A_ij <- -A_ij X_jj
            }
        }
        if (pass == 0) step_cp[1] = s.span;
        // ---- Step 3: product X^T X (Algorithm 1, Step 3)
        if (pass == 0) s.reset();
        tree = tree3;
        if (oop)
            for (int64_t i = 0; i < T; ++i)
                for (int64_t j = 0; j <= i; ++j)
                    if (j < i || !rdiag) s.task({A(i, j)}, {C(i, j)}, 0);  // C <- A
        for (int64_t i = 0; i < T; ++i) {
            const int64_t Xii = rdiag ? D(i) : (oop ? C(i, i) : A(i, i));
            for (int64_t j = 0; j < i; ++j) s.task({Xii, A(i, j)}, {A(i, j)}, 1);  // TRMM
            if (rdiag) s.task({D(i)}, {A(i, i)}, 1);                                 // LAUUM from D_i
            else s.task({A(i, i)}, {A(i, i)}, 1);                                    // LAUUM in place
            std::vector<std::vector<int64_t>> ins;
            for (int64_t j = 0; j < i; ++j) {
                ins.clear();
                for (int64_t k = i + 1; k < T; ++k) ins.push_back({oop ? C(k, i) : A(k, i), oop ? C(k, j) : A(k, j)});
                chain(s, A(i, j), ins);  // GEMM
            }
            ins.clear();
            for (int64_t k = i + 1; k < T; ++k) ins.push_back({oop ? C(k, i) : A(k, i)});
            chain(s, A(i, i), ins);  // SYRK
        }
        if (pass == 0) step_cp[2] = s.span;
    }
    out[0] = step_cp[0];
    out[1] = step_cp[1];
    out[2] = step_cp[2];
    out[3] = pipe ? whole.span : step_cp[0] + step_cp[1] + step_cp[2];
}

void dag_task_counts(int t, int64_t out[12]) {
    const int64_t T = t;
    const int64_t tri = T * (T - 1) / 2;                // tiles strictly below the diagonal
    const int64_t tet = T * (T - 1) * (T - 2) / 6;      // triples i > j > k
    out[0] = T;    // POTRF
    out[1] = tri;  // TRSM
    out[2] = tri;  // SYRK (step 1)
    out[3] = tet;  // GEMM (step 1)
    out[4] = T;    // TRTRI
    out[5] = tri;  // TRMM (step 2, left)
    out[6] = tet;  // GEMM (step 2)
    out[7] = tri;  // TRMM (step 2, right)
    out[8] = tri;  // TRMM (step 3)
    out[9] = T;    // LAUUM
    out[10] = tet; // GEMM (step 3)
    out[11] = tri; // SYRK (step 3)
}

// --------------------------------------------------------------------------
// (2) execution plan of the persistent kernel
// --------------------------------------------------------------------------
namespace {

struct TaskIndex {
    int t;
    std::vector<int32_t> id;  // (kind, i, j) -> task id, -1 if absent
    explicit TaskIndex(int t_) : t(t_), id((size_t)6 * t_ * t_, -1) {}
    int32_t& at(uint32_t kind, int i, int j) { return id[((size_t)kind * t + i) * t + j]; }
};

// ALAP ticket order (ORDER_ALAP) by the same three passes as the element walk
// in build_exec_plan's exhaustive path -- earliest finish forward, latest
// finish backward, keys forward -- with the same operations in the same
// order, so the same doubles and the same order.  Each pass walks a task's
// chain over rows and columns of the L and X task grids; the grids are kept
// both row-major and column-major so that every walk is sequential in memory.
void alap_order_grid(int t, const std::vector<uint32_t>& seq, bool s1, bool s2, bool s2diag,
                     std::vector<uint32_t>& perm) {
    const size_t N = seq.size(), T = (size_t)t;
    const bool hasL = s1, hasX = s2, hasD = s1 || s2diag;
    std::vector<double> Lr(T * T), Lc(T * T), Xr(T * T), Xc(T * T), D(T);
    auto rm = [T](int i, int j) { return (size_t)i * T + (size_t)j; };  // row-major (i, j)
    auto cm = [T](int i, int j) { return (size_t)j * T + (size_t)i; };  // column-major (i, j)
    // One forward pass.  step(v, p) folds a producer's value into v; elem(v)
    // ends an element of cost c; store keeps a task's value for its readers.
    auto forward = [&](std::vector<double>& val, auto&& init, auto&& fold, auto&& end_elem) {
        std::fill(D.begin(), D.end(), 0.0);
        for (size_t r = 0; r < N; ++r) {
            const uint32_t e = seq[r];
            const int i = (int)task_i(e), j = (int)task_j(e);
            double v = init(r);
            switch (task_kind(e)) {
                case K_S1_DIAG:
                    for (int k = 0; k < j; ++k) {
                        if (hasL) v = fold(v, Lr[rm(j, k)]);
                        v = end_elem(v, 1.0);
                    }
                    v = end_elem(v, 0.7);
                    if (hasD) D[j] = v;
                    break;
                case K_S1_OFF:
                    for (int k = 0; k < j; ++k) {
                        if (hasL) v = fold(fold(v, Lr[rm(i, k)]), Lr[rm(j, k)]);
                        v = end_elem(v, 1.0);
                    }
                    if (hasD) v = fold(v, D[j]);
                    v = end_elem(v, 1.0);
                    Lr[rm(i, j)] = Lc[cm(i, j)] = v;
                    break;
                case K_S2_DIAG:
                    v = end_elem(v, 0.4);
                    if (!s1) D[j] = v;
                    break;
                case K_S2_OFF:
                    if (hasD) v = fold(v, D[i]);
                    if (hasL) v = fold(v, Lr[rm(i, j)]);
                    v = end_elem(v, 1.0);
                    for (int k = i - 1; k > j; --k) {
                        v = fold(v, Xr[rm(i, k)]);
                        if (hasL) v = fold(v, Lc[cm(k, j)]);
                        v = end_elem(v, 1.0);
                    }
                    if (hasD) v = fold(v, D[j]);
                    v = end_elem(v, 1.0);
                    Xr[rm(i, j)] = Xc[cm(i, j)] = v;
                    break;
                case K_S3_DIAG:
                    if (hasD) v = fold(v, D[i]);
                    v = end_elem(v, 1.0);
                    for (int k = i + 1; k < t; ++k) {
                        if (hasX) v = fold(v, Xc[cm(k, i)]);
                        v = end_elem(v, 1.0);
                    }
                    break;
                default:  // K_S3_OFF
                    if (hasD) v = fold(v, D[i]);
                    if (hasX) v = fold(v, Xr[rm(i, j)]);
                    v = end_elem(v, 1.0);
                    for (int k = i + 1; k < t; ++k) {
                        if (hasX) v = fold(fold(v, Xc[cm(k, i)]), Xc[cm(k, j)]);
                        v = end_elem(v, 1.0);
                    }
                    break;
            }
            val[r] = v;
        }
    };
    auto vmax = [](double a, double b) { return std::max(a, b); };
    // Earliest finish with unlimited CTAs (seq is topological).
    std::vector<double> fin(N);
    forward(
        fin, [](size_t) { return 0.0; }, vmax, [](double v, double c) { return v + c; });
    double span = 0.0;
    for (size_t r = 0; r < N; ++r) span = std::max(span, fin[r]);
    // Latest finish that keeps the span: the grids now hold, per produced
    // tile, the least latest start among the elements that read it (row walks
    // into the row-major copy, column walks into the column-major one).
    std::fill(Lr.begin(), Lr.end(), span);
    std::fill(Lc.begin(), Lc.end(), span);
    std::fill(Xr.begin(), Xr.end(), span);
    std::fill(Xc.begin(), Xc.end(), span);
    std::fill(D.begin(), D.end(), span);
    std::vector<double> late(N, span);
    auto lower = [](double& a, double v) { a = std::min(a, v); };
    for (size_t r = N; r-- > 0;) {
        const uint32_t e = seq[r];
        const int i = (int)task_i(e), j = (int)task_j(e);
        double tail = span;
        switch (task_kind(e)) {
            case K_S1_DIAG:
                if (hasD) tail = D[j];
                late[r] = tail;
                tail -= 0.7;
                for (int k = j - 1; k >= 0; --k) {
                    tail -= 1.0;
                    if (hasL) lower(Lr[rm(j, k)], tail);
                }
                break;
            case K_S1_OFF:
                tail = std::min(Lr[rm(i, j)], Lc[cm(i, j)]);
                late[r] = tail;
                tail -= 1.0;
                if (hasD) lower(D[j], tail);
                for (int k = j - 1; k >= 0; --k) {
                    tail -= 1.0;
                    if (hasL) {
                        lower(Lr[rm(i, k)], tail);
                        lower(Lr[rm(j, k)], tail);
                    }
                }
                break;
            case K_S2_DIAG:
                if (!s1) tail = D[j];
                late[r] = tail;
                break;
            case K_S2_OFF:
                tail = std::min(Xr[rm(i, j)], Xc[cm(i, j)]);
                late[r] = tail;
                tail -= 1.0;
                if (hasD) lower(D[j], tail);
                for (int k = j + 1; k < i; ++k) {
                    tail -= 1.0;
                    lower(Xr[rm(i, k)], tail);
                    if (hasL) lower(Lc[cm(k, j)], tail);
                }
                tail -= 1.0;
                if (hasD) lower(D[i], tail);
                if (hasL) lower(Lr[rm(i, j)], tail);
                break;
            case K_S3_DIAG:
                late[r] = tail;
                for (int k = t - 1; k > i; --k) {
                    tail -= 1.0;
                    if (hasX) lower(Xc[cm(k, i)], tail);
                }
                tail -= 1.0;
                if (hasD) lower(D[i], tail);
                break;
            default:  // K_S3_OFF
                late[r] = tail;
                for (int k = t - 1; k > i; --k) {
                    tail -= 1.0;
                    if (hasX) {
                        lower(Xc[cm(k, i)], tail);
                        lower(Xc[cm(k, j)], tail);
                    }
                }
                tail -= 1.0;
                if (hasD) lower(D[i], tail);
                if (hasX) lower(Xr[rm(i, j)], tail);
                break;
        }
    }
    // Keys raised to the producers' keys keep the sorted order topological
    // (ties go to the earlier task of Algorithm 1's order).
    std::vector<double> key(N);
    forward(
        key, [&](size_t r) { return late[r]; }, vmax, [](double v, double) { return v; });
    std::iota(perm.begin(), perm.end(), 0u);
    std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
}

}  // namespace

ExecPlan build_exec_plan(int t, int steps, bool exhaustive, int order) {
    ExecPlan p;
    p.t = t;
    p.steps = steps;
    const bool s1 = steps == STEPS_ALL || steps == STEPS_POTRF || steps == STEPS_DIAG;
    const bool s2 = steps == STEPS_ALL || steps == STEPS_TRTRI || steps == STEPS_DIAG;
    const bool s3 = steps == STEPS_ALL || steps == STEPS_LAUUM || steps == STEPS_DIAG;
    const bool s3off = steps != STEPS_DIAG;
    const bool s2diag = steps == STEPS_TRTRI;  // in potri the Step-1 diagonal task inverts

    // Sequential (topological) order: Algorithm 1's loop nest.
    std::vector<uint32_t> seq;
    if (s1)
        for (int j = 0; j < t; ++j) {
            seq.push_back(encode_task(K_S1_DIAG, j, j));
            for (int i = j + 1; i < t; ++i) seq.push_back(encode_task(K_S1_OFF, i, j));
        }
    if (s2)
        for (int j = t - 1; j >= 0; --j) {
            if (s2diag) seq.push_back(encode_task(K_S2_DIAG, j, j));
            for (int i = t - 1; i > j; --i) seq.push_back(encode_task(K_S2_OFF, i, j));
        }
    if (s3)
        for (int i = 0; i < t; ++i) {
            if (s3off)
                for (int j = 0; j < i; ++j) seq.push_back(encode_task(K_S3_OFF, i, j));
            seq.push_back(encode_task(K_S3_DIAG, i, i));
        }
    const size_t N = seq.size();
    TaskIndex ix(t);
    for (size_t m = 0; m < N; ++m) ix.at(task_kind(seq[m]), task_i(seq[m]), task_j(seq[m])) = (int32_t)m;

    // Producer of each renamed store, or -1 when the data is ready at launch.
    auto dprod = [&](int j) -> int32_t {  // D_j = X_jj
        if (s1) return ix.at(K_S1_DIAG, j, j);
        if (s2diag) return ix.at(K_S2_DIAG, j, j);
        return -1;
    };
    auto lprod = [&](int i, int j) -> int32_t { return s1 ? ix.at(K_S1_OFF, i, j) : -1; };  // B_ij = L_ij
    auto xprod = [&](int i, int j) -> int32_t { return s2 ? ix.at(K_S2_OFF, i, j) : -1; };  // C_ij = X_ij

    // Cost of each task in units of one b x b x b tile product (b^3 FMA).
    auto cost = [&](uint32_t e) -> double {
        const int i = task_i(e), j = task_j(e);
        switch (task_kind(e)) {
            case K_S1_DIAG: return j + 0.7;
            case K_S1_OFF: return j + 1.0;
            case K_S2_DIAG: return 0.4;
            case K_S2_OFF: return (i - j - 1) + 2.0;
            case K_S3_DIAG: return (t - 1 - i) + 1.0;
            default: return (t - 1 - i) + 1.0;
        }
    };
    // Visits every predecessor (task whose output this task reads).
    auto for_preds = [&](uint32_t e, auto&& f) {
        const int i = task_i(e), j = task_j(e);
        auto g = [&](int32_t p) { if (p >= 0) f(p); };
        switch (task_kind(e)) {
            case K_S1_DIAG:
                for (int k = 0; k < j; ++k) g(lprod(j, k));
                break;
            case K_S1_OFF:
                for (int k = 0; k < j; ++k) { g(lprod(i, k)); g(lprod(j, k)); }
                g(dprod(j));
                break;
            case K_S2_DIAG:
                break;
            case K_S2_OFF:
                g(dprod(i)); g(lprod(i, j));
                for (int k = i - 1; k > j; --k) { g(xprod(i, k)); g(lprod(k, j)); }
                g(dprod(j));
                break;
            case K_S3_DIAG:
                g(dprod(i));
                for (int k = i + 1; k < t; ++k) g(xprod(k, i));
                break;
            case K_S3_OFF:
                g(dprod(i)); g(xprod(i, j));
                for (int k = i + 1; k < t; ++k) { g(xprod(k, i)); g(xprod(k, j)); }
                break;
        }
    };
    // Bottom levels (cost plus the largest bottom level among the tasks that
    // read this task's output), in reverse sequential order.
    std::vector<double> bl(N, 0.0);
    double work = 0.0;
    if (exhaustive) {  // push each task's level to its predecessors: O(t^3) edges
        std::vector<double> succmax(N, 0.0);
        for (size_t r = N; r-- > 0;) {
            const double c = cost(seq[r]);
            work += c;
            bl[r] = c + succmax[r];
            for_preds(seq[r], [&](int32_t p) { succmax[p] = std::max(succmax[p], bl[r]); });
        }
    } else {
        // The same levels in O(t^2): the readers of each output form whole
        // rows, columns or prefixes/suffixes of them in the task grids, so
        // running maxima replace the edge walk (the max of the same values:
        // the same doubles, the same order).
        //   D(j)  <- S1off(., j), S2off(j, .), S2off(., j), S3diag(j), S3off(j, .)
        //   L(i,j) <- S1diag(i), S1off(i, j'>j), S1off(., i), S2off(i, j), S2off(i'>i, j)
        //   X(i,j) <- S2off(i, j'<j), S3off(i, j), S3diag(j), S3off(j, .), S3off(j<i'<i, j)
        // A step that is not in the plan leaves its grids at zero (its data
        // is ready at launch); D(j) comes from S2diag(j) in the TRTRI plan.
        const size_t T = (size_t)t;
        std::vector<double> c1d(T, 0.0), c2d(T, 0.0), c3d(T, 0.0), g1(T * T, 0.0), g2(T * T, 0.0),
            g3(T * T, 0.0);
        for (size_t r = N; r-- > 0;) work += cost(seq[r]);  // summed in the same order as above
        auto at = [&](int i, int j) { return (size_t)i * T + (size_t)j; };
        // Step 3 tasks have no readers: level = cost.
        for (int i = 0; i < t && s3; ++i) {
            c3d[i] = cost(encode_task(K_S3_DIAG, i, i));
            if (s3off)
                for (int j = 0; j < i; ++j) g3[at(i, j)] = cost(encode_task(K_S3_OFF, i, j));
        }
        std::vector<double> row3(T, 0.0), colpre3(T * T, 0.0);  // colpre3(i, j) = max g3(i', j), j < i' < i
        for (int j = 0; j < t; ++j) {
            for (int k = 0; k < j; ++k) row3[j] = std::max(row3[j], g3[at(j, k)]);
            double m = 0.0;
            for (int i = j + 1; i < t; ++i) {
                colpre3[at(i, j)] = m;
                m = std::max(m, g3[at(i, j)]);
            }
        }
        // Step 2, reverse sequential order: j ascending, i ascending.
        std::vector<double> rowpre2(T, 0.0);  // max g2(i, j') over the j' < j done so far
        for (int j = 0; j < t && s2; ++j)
            for (int i = j + 1; i < t; ++i) {
                double m = std::max({rowpre2[i], g3[at(i, j)], c3d[j], row3[j], colpre3[at(i, j)]});
                g2[at(i, j)] = cost(encode_task(K_S2_OFF, i, j)) + m;
                rowpre2[i] = std::max(rowpre2[i], g2[at(i, j)]);
            }
        std::vector<double> row2(T, 0.0), col2(T, 0.0), colsuf2(T * T, 0.0);  // colsuf2(i, j) = max g2(i', j), i' > i
        for (int j = 0; j < t; ++j) {
            for (int k = 0; k < j; ++k) row2[j] = std::max(row2[j], g2[at(j, k)]);
            double m = 0.0;
            for (int i = t - 1; i > j; --i) {
                colsuf2[at(i, j)] = m;
                m = std::max(m, g2[at(i, j)]);
            }
            col2[j] = m;
            if (s2diag) c2d[j] = cost(encode_task(K_S2_DIAG, j, j)) + std::max(row2[j], col2[j]);
        }
        // Step 1, reverse sequential order: j descending; S1off(i, j) for i
        // descending, then S1diag(j).
        std::vector<double> rowsuf1(T, 0.0), col1(T, 0.0);
        for (int j = t - 1; j >= 0 && s1; --j) {
            for (int i = t - 1; i > j; --i) {
                double m = std::max({c1d[i], rowsuf1[i], col1[i], g2[at(i, j)], colsuf2[at(i, j)]});
                g1[at(i, j)] = cost(encode_task(K_S1_OFF, i, j)) + m;
                rowsuf1[i] = std::max(rowsuf1[i], g1[at(i, j)]);
                col1[j] = std::max(col1[j], g1[at(i, j)]);
            }
            const double m = std::max({col1[j], row2[j], col2[j], c3d[j], row3[j]});
            c1d[j] = cost(encode_task(K_S1_DIAG, j, j)) + m;
        }
        for (size_t r = 0; r < N; ++r) {
            const uint32_t e = seq[r];
            const int i = (int)task_i(e), j = (int)task_j(e);
            switch (task_kind(e)) {
                case K_S1_DIAG: bl[r] = c1d[j]; break;
                case K_S1_OFF: bl[r] = g1[at(i, j)]; break;
                case K_S2_DIAG: bl[r] = c2d[j]; break;
                case K_S2_OFF: bl[r] = g2[at(i, j)]; break;
                case K_S3_DIAG: bl[r] = c3d[i]; break;
                default: bl[r] = g3[at(i, j)]; break;
            }
        }
    }
    std::vector<uint32_t> perm(N);
    std::iota(perm.begin(), perm.end(), 0u);
    std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return bl[a] > bl[b]; });
    p.crit = N ? bl[perm[0]] : 0.0;
    p.work = work;

    if (order == ORDER_ALAP && N && !exhaustive) {
        alap_order_grid(t, seq, s1, s2, s2diag, perm);
    } else if (order == ORDER_ALAP && N) {
        // Each task's chain elements in the kernel's order: up to two producer
        // tasks (-1: ready at launch) and a cost; the costs add up to cost().
        struct Elem {
            int32_t p0, p1;
            double c;
        };
        std::vector<Elem> el;
        auto elements = [&](uint32_t e) {
            const int i = task_i(e), j = task_j(e);
            el.clear();
            switch (task_kind(e)) {
                case K_S1_DIAG:
                    for (int k = 0; k < j; ++k) el.push_back({lprod(j, k), -1, 1.0});
                    el.push_back({-1, -1, 0.7});
                    break;
                case K_S1_OFF:
                    for (int k = 0; k < j; ++k) el.push_back({lprod(i, k), lprod(j, k), 1.0});
                    el.push_back({dprod(j), -1, 1.0});
                    break;
                case K_S2_DIAG:
                    el.push_back({-1, -1, 0.4});
                    break;
                case K_S2_OFF:
                    el.push_back({dprod(i), lprod(i, j), 1.0});
                    for (int k = i - 1; k > j; --k) el.push_back({xprod(i, k), lprod(k, j), 1.0});
                    el.push_back({dprod(j), -1, 1.0});
                    break;
                case K_S3_DIAG:
                    el.push_back({dprod(i), -1, 1.0});
                    for (int k = i + 1; k < t; ++k) el.push_back({xprod(k, i), -1, 1.0});
                    break;
                default:  // K_S3_OFF
                    el.push_back({dprod(i), xprod(i, j), 1.0});
                    for (int k = i + 1; k < t; ++k) el.push_back({xprod(k, i), xprod(k, j), 1.0});
                    break;
            }
        };
        // Earliest finish with unlimited CTAs (seq is topological).
        std::vector<double> fin(N, 0.0);
        double span = 0.0;
        for (size_t r = 0; r < N; ++r) {
            elements(seq[r]);
            double now = 0.0;
            for (const Elem& x : el) {
                if (x.p0 >= 0) now = std::max(now, fin[x.p0]);
                if (x.p1 >= 0) now = std::max(now, fin[x.p1]);
                now += x.c;
            }
            fin[r] = now;
            span = std::max(span, now);
        }
        // Latest finish that keeps the span: each element's latest start
        // bounds the finish of the tasks it reads.
        std::vector<double> late(N, span);
        for (size_t r = N; r-- > 0;) {
            elements(seq[r]);
            double tail = late[r];
            for (size_t q = el.size(); q-- > 0;) {
                tail -= el[q].c;
                if (el[q].p0 >= 0) late[el[q].p0] = std::min(late[el[q].p0], tail);
                if (el[q].p1 >= 0) late[el[q].p1] = std::min(late[el[q].p1], tail);
            }
        }
        // Keys raised to the producers' keys keep the sorted order topological
        // (ties go to the earlier task of Algorithm 1's order).
        std::vector<double> key(N, 0.0);
        for (size_t r = 0; r < N; ++r) {
            elements(seq[r]);
            double k = late[r];
            for (const Elem& x : el) {
                if (x.p0 >= 0) k = std::max(k, key[x.p0]);
                if (x.p1 >= 0) k = std::max(k, key[x.p1]);
            }
            key[r] = k;
        }
        std::iota(perm.begin(), perm.end(), 0u);
        std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
    }
    p.order.resize(N);
    for (size_t m = 0; m < N; ++m) p.order[m] = seq[perm[m]];
    return p;
}

bool build_variant_plan(int t, int variant, int seg, ExecPlan* out) {
    if (variant & ~kVariantMask) return false;
    const bool share = variant & (VAR_SHARE_BC | VAR_INPLACE), inplace = variant & VAR_INPLACE;
    const bool split = variant & VAR_SPLIT3;
    if (split && (share || seg < 1)) return false;
    if (variant == 0) {
        *out = build_exec_plan(t, STEPS_ALL, false);
        return true;
    }
    ExecPlan p;
    p.t = t;
    p.steps = STEPS_ALL;
    p.variant = variant;
    p.seg = split ? seg : 0;
    const size_t T = (size_t)t;
    // Sequential order: Algorithm 1's loop nest (Step 2: j and i decreasing),
    // each split chain's segments just before the task that adds them.  It is
    // a topological order of every edge below, write-after-read included: it
    // is the order of a correct sequential in-place program.
    std::vector<uint32_t> seq;
    for (int j = 0; j < t; ++j) {
        seq.push_back(encode_task(K_S1_DIAG, j, j));
        for (int i = j + 1; i < t; ++i) seq.push_back(encode_task(K_S1_OFF, i, j));
    }
    for (int j = t - 1; j >= 0; --j)
        for (int i = t - 1; i > j; --i) seq.push_back(encode_task(K_S2_OFF, i, j));
    if (split) p.split.assign(T * (T + 1) / 2, SplitInfo{0, 0, 0});
    for (int i = 0; i < t; ++i)
        for (int j = 0; j <= i; ++j) {
            const int m = t - 1 - i;  // chain length
            if (split && m > seg) {
                const int np = (m + seg - 1) / seg;
                SplitInfo& si = p.split[tri_index(i, j)];
                si.first = (uint32_t)p.parts.size();
                si.np = (uint16_t)(np - 1);
                si.own_end = (uint16_t)(i + 1 + seg);
                for (int q = 1; q < np; ++q) {
                    const int k0 = i + 1 + q * seg, k1 = std::min(t, k0 + seg);
                    seq.push_back(encode_part((uint32_t)p.parts.size()));
                    p.parts.push_back(PartTask{(uint16_t)i, (uint16_t)j, (uint16_t)k0, (uint16_t)k1});
                }
            }
            seq.push_back(j < i ? encode_task(K_S3_OFF, i, j) : encode_task(K_S3_DIAG, i, i));
        }
    const size_t N = seq.size();
    TaskIndex ix(t);
    std::vector<int32_t> part_pos(p.parts.size(), -1);
    for (size_t r = 0; r < N; ++r) {
        const uint32_t e = seq[r];
        if (task_kind(e) == K_S3_PART) part_pos[part_id(e)] = (int32_t)r;
        else ix.at(task_kind(e), task_i(e), task_j(e)) = (int32_t)r;
    }
    auto L = [&](int i, int j) { return ix.at(K_S1_OFF, i, j); };
    auto X = [&](int i, int j) { return ix.at(K_S2_OFF, i, j); };
    auto D = [&](int j) { return ix.at(K_S1_DIAG, j, j); };
    auto own_end = [&](int i, int j) -> int {
        if (!split) return t;
        const SplitInfo& si = p.split[tri_index(i, j)];
        return si.np ? si.own_end : t;
    };
    auto cost = [&](uint32_t e) -> double {
        const int i = task_i(e), j = task_j(e);
        switch (task_kind(e)) {
            case K_S1_DIAG: return j + 0.7;
            case K_S1_OFF: return j + 1.0;
            case K_S2_OFF: return (i - j - 1) + 2.0;
            case K_S3_PART: {
                const PartTask& q = p.parts[part_id(e)];
                return (double)(q.k1 - q.k0);
            }
            default: {  // K_S3_OFF, K_S3_DIAG: the own segment, the TRMM / LAUUM, the partial sums
                const int np = split ? p.split[tri_index(i, j)].np : 0;
                return (own_end(i, j) - i - 1) + 1.0 + 0.25 * np;
            }
        }
    };
    // Every task that must finish before task e: the producers of what it
    // reads and, when e stores over a tile that others still read, those
    // readers (write after read).
    auto for_preds = [&](uint32_t e, auto&& f) {
        const int i = task_i(e), j = task_j(e);
        switch (task_kind(e)) {
            case K_S1_DIAG:
                for (int k = 0; k < j; ++k) f(L(j, k));
                break;
            case K_S1_OFF:
                for (int k = 0; k < j; ++k) { f(L(i, k)); f(L(j, k)); }
                f(D(j));
                break;
            case K_S2_OFF:
                f(D(i)); f(L(i, j));
                for (int k = j + 1; k < i; ++k) { f(X(i, k)); f(L(k, j)); }
                f(D(j));
                if (share) {  // X_ij is stored over L_ij: every other reader of L_ij first
                    f(D(i));  // S1_DIAG(i) read L_ij (it is also D(i)'s producer)
                    for (int q = j + 1; q < i; ++q) f(L(i, q));
                    for (int q = i + 1; q < t; ++q) { f(L(q, i)); f(X(q, j)); }
                }
                break;
            case K_S3_PART: {
                const PartTask& q = p.parts[part_id(e)];
                for (int k = q.k0; k < q.k1; ++k) { f(X(k, q.i)); if (q.j != q.i) f(X(k, q.j)); }
                break;
            }
            case K_S3_OFF:
                f(D(i)); f(X(i, j));
                for (int k = i + 1; k < own_end(i, j); ++k) { f(X(k, i)); f(X(k, j)); }
                if (split)
                    for (uint32_t q = 0; q < p.split[tri_index(i, j)].np; ++q)
                        f(part_pos[p.split[tri_index(i, j)].first + q]);
                if (inplace) {  // A^{-1}_ij is stored over X_ij
                    for (int q = 0; q < j; ++q) f(X(i, q));             // S2(i, q) read X_ij
                    for (int q = 0; q < j; ++q) f(ix.at(K_S3_OFF, j, q));  // S3(j, q) read X_ij as X_kj
                    for (int q = j + 1; q < i; ++q) f(ix.at(K_S3_OFF, q, j));
                    f(ix.at(K_S3_DIAG, j, j));
                }
                break;
            case K_S3_DIAG:
                f(D(i));
                for (int k = i + 1; k < own_end(i, i); ++k) f(X(k, i));
                if (split)
                    for (uint32_t q = 0; q < p.split[tri_index(i, i)].np; ++q)
                        f(part_pos[p.split[tri_index(i, i)].first + q]);
                if (inplace) {  // A^{-1}_ii is stored over X_ii
                    for (int q = i + 1; q < t; ++q) { f(L(q, i)); f(X(q, i)); }
                    for (int q = 0; q < i; ++q) { f(X(i, q)); f(ix.at(K_S3_OFF, i, q)); }
                }
                break;
        }
    };
    std::vector<double> bl(N, 0.0), succmax(N, 0.0);
    double work = 0.0;
    for (size_t r = N; r-- > 0;) {
        const double c = cost(seq[r]);
        work += c;
        bl[r] = c + succmax[r];
        for_preds(seq[r], [&](int32_t q) {
            if (q >= 0 && (size_t)q != r) succmax[q] = std::max(succmax[q], bl[r]);
        });
    }
    std::vector<uint32_t> perm(N);
    std::iota(perm.begin(), perm.end(), 0u);
    std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return bl[a] > bl[b]; });
    p.crit = N ? bl[perm[0]] : 0.0;
    p.work = work;
    p.order.resize(N);
    for (size_t m = 0; m < N; ++m) p.order[m] = seq[perm[m]];
    *out = std::move(p);
    return true;
}

namespace {
std::atomic<int>& plan_order_setting() {
    static std::atomic<int> order{[] {
        const char* env = std::getenv("SPDINV_PLAN_ORDER");
        if (env && (std::strcmp(env, "bottom_level") == 0 || std::strcmp(env, "0") == 0))
            return (int)ORDER_BOTTOM_LEVEL;
        return (int)ORDER_ALAP;
    }()};
    return order;
}
}  // namespace

int current_plan_order() { return plan_order_setting().load(std::memory_order_relaxed); }

int set_plan_order(int order) { return plan_order_setting().exchange(order); }

}  // namespace spdinv
