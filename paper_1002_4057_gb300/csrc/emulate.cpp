// Host emulation of the persistent kernel's scheduling protocol (no GPU):
// worker threads stand in for the CTAs.  Each takes the next ticket of the
// execution plan (build_exec_plan, the order the kernel's CTAs take tasks),
// waits -- bounded, as the kernel does -- for the readiness flag of every
// input tile of its task in the order the kernel reads them, spends a
// seeded random time on each chain element and on its own tile kernel, stores
// its outputs and publishes its output flag.  Run with many worker counts and
// seeds, it covers the protocol's races and deadlock freedom on the CPU; a
// dropped completion (the kernel's fault_drop_task hook) must end every worker
// with a timeout, not a hang.
//
// Besides the flags, every tile location the kernel touches carries a writer
// word: the task that last stored it (0 = the caller's input, or a copy of it
// staged before the launch).  Every read checks that it sees the value
// Algorithm 1 needs there -- the input for A's tiles, the producing task for
// the renamed stores B = L, C = X, D = X_jj -- so a read before its producer
// stored (a missing wait) or after Step 3 overwrote A (a write-after-read
// hazard that renaming must remove) counts as a hazard.
//
// Inputs and outputs per task kind, as the kernel waits for, reads and
// writes them (the standalone steps wait only for what their own launch
// produces; their other inputs are staged):
//   Step 1, diagonal j      A(j,j); L(j,k), k < j;                  -> D(j) [A(j,j) in potrf]
//   Step 1, off-diagonal    A(i,j); (L(i,k), L(j,k)), k < j; D(j)   -> L(i,j) [A(i,j) in potrf]
//   Step 2, diagonal j      A(j,j) (trtri only)                     -> D(j), A(j,j)
//   Step 2, off-diagonal    (D(i), L(i,j)); (X(i,k), L(k,j)), k = i-1 .. j+1; D(j)
//                                                                   -> X(i,j) [A(i,j) in trtri]
//   Step 3, off-diagonal    (D(i), X(i,j)); (X(k,i), X(k,j)), k > i -> A(i,j)
//   Step 3, diagonal        D(i); X(k,i), k > i                     -> A(i,i) (diag(A^{-1}) alone
//                                                                      in the selected inverse)
#include <atomic>
#include <chrono>
#include <cstdint>
#include <algorithm>
#include <functional>
#include <memory>
#include <queue>
#include <random>
#include <thread>
#include <vector>

#include "../../include/spdinv.h"
#include "plan.h"

namespace spdinv {
namespace {

using Flags = std::unique_ptr<std::atomic<int>[]>;
using Words = std::unique_ptr<std::atomic<uint32_t>[]>;

struct Emu {
    int t = 0, steps = STEPS_ALL;
    bool s1 = true, s2 = true, from_A = true, wait_d = true, wait_x = true;
    const std::vector<uint32_t>* tasks = nullptr;
    Flags fL, fX, fD;      // readiness flags of B, C, D
    Words wA, wB, wC, wD;  // writer words: encoded task + 1, or 0 for input / staged data
    // Execution variants (PlanVariant): the kernel's read counters and
    // write-after-read waits, the split chains' partial tiles.
    int variant = 0;
    const ExecPlan* plan = nullptr;
    Flags rL, rX, rD, fP;  // reads of L (B), X (C), D; partials' flags
    Words wP;              // partial tiles' writer words
    bool uuu() const { return variant & VAR_UUU; }
    bool shared() const { return variant & (VAR_SHARE_BC | VAR_INPLACE); }
    bool inplace() const { return variant & VAR_INPLACE; }
    bool split() const { return variant & VAR_SPLIT3; }
    // The store that holds X: C, or B's slots when the variant shares them.
    std::atomic<uint32_t>& slotC(int i, int j) { return shared() ? wB[(size_t)i * t + j] : wC[(size_t)i * t + j]; }
    std::atomic<int> ticket{0}, abort{0}, completed{0}, protocol_errors{0}, hazards{0};
    std::atomic<int64_t> max_wait_us{0};
    int drop = -1, skip = -1;
    double limit_s = 1.0;
    int max_delay_us = 20;
    uint64_t seed = 0;

    // Bounded wait for one flag; false when the limit ran out or another
    // worker aborted (the kernel's flag wait with its timeout and abort word).
    bool wait(const std::atomic<int>* f) {
        if (!f || f->load(std::memory_order_acquire)) return true;
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            if (f->load(std::memory_order_acquire)) break;
            if (abort.load(std::memory_order_relaxed)) return false;
            const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (s > limit_s) {
                abort.store(1);
                return false;
            }
            std::this_thread::yield();
        }
        const int64_t us = std::chrono::duration_cast<std::chrono::microseconds>(
                               std::chrono::steady_clock::now() - t0).count();
        int64_t m = max_wait_us.load();
        while (us > m && !max_wait_us.compare_exchange_weak(m, us)) {
        }
        return true;
    }

    void work(std::mt19937_64& rng) {
        if (max_delay_us > 0)
            std::this_thread::sleep_for(std::chrono::microseconds(rng() % (uint64_t)(max_delay_us + 1)));
    }

    void publish(std::atomic<int>& f, int tk) {
        if (tk == drop) return;  // fault injection: the consumers never see this tile
        if (f.exchange(1, std::memory_order_release)) protocol_errors.fetch_add(1);  // published twice
    }

    static uint32_t code(uint32_t kind, int i, int j) { return encode_task(kind, (uint32_t)i, (uint32_t)j) + 1u; }

    // What a read must find in each location.
    uint32_t expect_B(int i, int j) const { return s1 ? code(K_S1_OFF, i, j) : 0u; }
    uint32_t expect_C(int i, int j) const { return s2 ? code(K_S2_OFF, i, j) : 0u; }
    uint32_t expect_D(int j) const {
        if (s1) return code(K_S1_DIAG, j, j);
        if (steps == STEPS_TRTRI) return code(K_S2_DIAG, j, j);
        return 0u;  // lauum: staged
    }

    void check(const std::atomic<uint32_t>& w, uint32_t want) {
        if (w.load(std::memory_order_acquire) != want) hazards.fetch_add(1);
    }
    // Each read also counts itself, as the kernel does once the copy is in
    // shared memory, where a later version overwrites the tile.
    void read_A(int i, int j) { check(wA[(size_t)i * t + j], 0u); }
    void read_B(int i, int j) {
        check(wB[(size_t)i * t + j], expect_B(i, j));
        if (shared()) rL[(size_t)i * t + j].fetch_add(1, std::memory_order_release);
    }
    void read_C(int i, int j) {
        check(slotC(i, j), expect_C(i, j));
        if (inplace()) rX[(size_t)i * t + j].fetch_add(1, std::memory_order_release);
    }
    void read_D(int j) {
        check(wD[j], expect_D(j));
        if (inplace()) rD[j].fetch_add(1, std::memory_order_release);
    }
    // Bounded wait until `expected` reads of a tile were counted (the
    // kernel's write-after-read wait); false on timeout or abort.
    bool wait_reads(const std::atomic<int>& r, int expected) {
        if (r.load(std::memory_order_acquire) >= expected) return true;
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            if (r.load(std::memory_order_acquire) >= expected) return true;
            if (abort.load(std::memory_order_relaxed)) return false;
            const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (s > limit_s) {
                abort.store(1);
                return false;
            }
            std::this_thread::yield();
        }
    }
    static void store(std::atomic<uint32_t>& w, uint32_t c) { w.store(c, std::memory_order_release); }

    std::atomic<int>* L(int i, int j) { return &fL[(size_t)i * t + j]; }
    std::atomic<int>* X(int i, int j) { return &fX[(size_t)i * t + j]; }
    std::atomic<int>* D(int j) { return &fD[j]; }

    void run_worker(int w) {
        std::mt19937_64 rng(seed * 1000003u + (uint64_t)w);
        const int n = (int)tasks->size();
        for (;;) {
            if (abort.load()) return;
            const int tk = ticket.fetch_add(1);
            if (tk >= n) return;
            const uint32_t e = (*tasks)[tk];
            const int kind = (int)task_kind(e), i = (int)task_i(e), j = (int)task_j(e);
            const uint32_t me = e + 1u;
            const bool waits = tk != skip;  // test hook: this task reads at once, without waiting
            bool ok = true;
            // Waits for up to two flags (either may be absent), then runs one
            // chain element.
            auto need = [&](std::atomic<int>* a, std::atomic<int>* b) {
                if (!waits) return;
                ok = ok && wait(a) && wait(b);
                if (ok) work(rng);
            };
            if (kind == K_S1_DIAG) {
                read_A(j, j);
                for (int k = 0; k < j && ok; ++k) {
                    need(L(j, k), nullptr);
                    if (ok) read_B(j, k);
                }
                if (!ok) return;
                work(rng);  // POTRF and TRTRI of the tile
                if (steps == STEPS_POTRF) store(wA[(size_t)j * t + j], me);
                store(wD[j], me);
                publish(*D(j), tk);
            } else if (kind == K_S1_OFF) {
                read_A(i, j);
                for (int k = 0; k < j && ok; ++k) {
                    need(L(i, k), L(j, k));
                    if (ok) { read_B(i, k); read_B(j, k); }
                }
                need(D(j), nullptr);
                if (!ok) return;
                read_D(j);
                store(wB[(size_t)i * t + j], me);
                if (steps == STEPS_POTRF) store(wA[(size_t)i * t + j], me);
                publish(*L(i, j), tk);
            } else if (kind == K_S2_DIAG) {
                read_A(j, j);
                work(rng);
                store(wD[j], me);
                store(wA[(size_t)j * t + j], me);
                publish(*D(j), tk);
            } else if (kind == K_S2_OFF) {
                need(D(i), from_A ? L(i, j) : nullptr);
                if (ok) { read_D(i); read_B(i, j); }
                for (int m = 0; m < i - j - 1 && ok; ++m) {
                    const int k = uuu() ? j + 1 + m : i - 1 - m;
                    need(X(i, k), from_A ? L(k, j) : nullptr);
                    if (ok) { read_C(i, k); read_B(k, j); }
                }
                need(D(j), nullptr);
                if (!ok) return;
                read_D(j);
                if (shared() && !wait_reads(rL[(size_t)i * t + j], readers_L(t, i, j))) return;
                store(slotC(i, j), me);
                if (steps == STEPS_TRTRI) store(wA[(size_t)i * t + j], me);
                publish(*X(i, j), tk);
            } else if (kind == K_S3_PART) {  // a segment of a split chain: X tiles only
                const PartTask q = plan->parts[part_id(e)];
                for (int k = q.k0; k < q.k1 && ok; ++k) {
                    need(X(k, q.i), q.j != q.i ? X(k, q.j) : nullptr);
                    if (ok) { read_C(k, q.i); if (q.j != q.i) read_C(k, q.j); }
                }
                if (!ok) return;
                store(wP[part_id(e)], me);
                publish(fP[part_id(e)], tk);
            } else if (kind == K_S3_OFF) {
                const SplitInfo si = split() ? plan->split[tri_index(i, j)] : SplitInfo{0, 0, 0};
                const int kend = si.np ? si.own_end : t;
                need(wait_d ? D(i) : nullptr, wait_x ? X(i, j) : nullptr);
                if (ok) { read_D(i); read_C(i, j); }
                for (int k = i + 1; k < kend && ok; ++k) {
                    need(wait_x ? X(k, i) : nullptr, wait_x ? X(k, j) : nullptr);
                    if (ok) { read_C(k, i); read_C(k, j); }
                }
                for (uint32_t q = si.first; q < si.first + si.np && ok; ++q) {
                    need(&fP[q], nullptr);
                    if (ok) check(wP[q], encode_part(q) + 1u);
                }
                if (!ok) return;
                if (inplace()) {  // A^{-1}_ij over X_ij, after every read of X_ij
                    if (!wait_reads(rX[(size_t)i * t + j], readers_X(t, i, j))) return;
                    store(slotC(i, j), me);
                } else {
                    store(wA[(size_t)i * t + j], me);
                }
            } else if (kind == K_S3_DIAG) {
                const SplitInfo si = split() ? plan->split[tri_index(i, i)] : SplitInfo{0, 0, 0};
                const int kend = si.np ? si.own_end : t;
                need(wait_d ? D(i) : nullptr, nullptr);
                if (ok) read_D(i);
                for (int k = i + 1; k < kend && ok; ++k) {
                    need(wait_x ? X(k, i) : nullptr, nullptr);
                    if (ok) read_C(k, i);
                }
                for (uint32_t q = si.first; q < si.first + si.np && ok; ++q) {
                    need(&fP[q], nullptr);
                    if (ok) check(wP[q], encode_part(q) + 1u);
                }
                if (!ok) return;
                if (inplace()) {  // A^{-1}_ii over X_ii, after every read of X_ii
                    if (!wait_reads(rD[i], readers_D(t, i))) return;
                    store(wD[i], me);
                } else if (steps != STEPS_DIAG) {
                    store(wA[(size_t)i * t + i], me);
                }
            } else {
                protocol_errors.fetch_add(1);  // no other kind exists
            }
            completed.fetch_add(1);
        }
    }
};

template <typename W>
W zeroed(size_t count) {
    W a(new typename W::element_type[count]);
    for (size_t q = 0; q < count; ++q) a[q].store(0);
    return a;
}

}  // namespace
}  // namespace spdinv

using namespace spdinv;

namespace spdinv {
namespace {

spdinv_status emulate(int t, int steps, int variant, int seg, int workers, uint64_t seed, int drop_task,
                      int skip_wait_task, double wait_limit_s, int max_delay_us, int64_t out[5]) {
    if (t < 1 || t > 256) return SPDINV_ERR_N;
    if (steps < STEPS_ALL || steps > STEPS_DIAG) return SPDINV_ERR_UNSUPPORTED;
    if (workers < 1 || workers > 1024 || wait_limit_s <= 0.0 || max_delay_us < 0) return SPDINV_ERR_UNSUPPORTED;
    if (!out) return SPDINV_ERR_NULL;
    if (variant != 0 && steps != STEPS_ALL) return SPDINV_ERR_UNSUPPORTED;
    ExecPlan plan;
    if (variant == 0) plan = build_exec_plan(t, steps, false, current_plan_order());
    else if (!build_variant_plan(t, variant, seg, &plan)) return SPDINV_ERR_UNSUPPORTED;
    Emu emu;
    emu.t = t;
    emu.steps = steps;
    emu.variant = variant;
    emu.plan = &plan;
    emu.s1 = steps == STEPS_ALL || steps == STEPS_POTRF || steps == STEPS_DIAG;
    emu.s2 = steps == STEPS_ALL || steps == STEPS_TRTRI || steps == STEPS_DIAG;
    emu.from_A = emu.s1;                   // else L is staged before the launch
    emu.wait_d = steps != STEPS_LAUUM;     // lauum stages D and C
    emu.wait_x = steps != STEPS_LAUUM;
    emu.tasks = &plan.order;
    const size_t tt = (size_t)t * t;
    emu.fL = zeroed<Flags>(tt);
    emu.fX = zeroed<Flags>(tt);
    emu.fD = zeroed<Flags>((size_t)t);
    emu.wA = zeroed<Words>(tt);
    emu.wB = zeroed<Words>(tt);
    emu.wC = zeroed<Words>(tt);
    emu.wD = zeroed<Words>((size_t)t);
    emu.rL = zeroed<Flags>(tt);
    emu.rX = zeroed<Flags>(tt);
    emu.rD = zeroed<Flags>((size_t)t);
    emu.fP = zeroed<Flags>(plan.parts.size() + 1);
    emu.wP = zeroed<Words>(plan.parts.size() + 1);
    emu.drop = drop_task;
    emu.skip = skip_wait_task;
    emu.limit_s = wait_limit_s;
    emu.max_delay_us = max_delay_us;
    emu.seed = seed;
    std::vector<std::thread> th;
    th.reserve(workers);
    for (int w = 0; w < workers; ++w) th.emplace_back([&emu, w] { emu.run_worker(w); });
    for (auto& x : th) x.join();
    // Every counted tile must have been read exactly as often as the kernel's
    // write-after-read waits assume (a wrong count would make them release a
    // tile early or wait forever).
    if (!emu.abort.load() && emu.completed.load() == (int)plan.order.size()) {
        for (int a = 0; a < t; ++a) {
            for (int b = 0; b < a; ++b) {
                if (emu.shared() && emu.rL[(size_t)a * t + b].load() != readers_L(t, a, b)) emu.protocol_errors++;
                if (emu.inplace() && emu.rX[(size_t)a * t + b].load() != readers_X(t, a, b)) emu.protocol_errors++;
            }
            if (emu.inplace() && emu.rD[a].load() != readers_D(t, a)) emu.protocol_errors++;
        }
    }
    out[0] = emu.completed.load();
    out[1] = (int64_t)plan.order.size();
    out[2] = emu.protocol_errors.load();
    out[3] = emu.hazards.load();
    out[4] = emu.max_wait_us.load();
    return emu.abort.load() ? SPDINV_ERR_TIMEOUT : SPDINV_OK;
}

}  // namespace
}  // namespace spdinv

extern "C" SPDINV_API spdinv_status spdinv_plan_emulate(int t, int steps, int workers, uint64_t seed, int drop_task,
                                                        int skip_wait_task, double wait_limit_s, int max_delay_us,
                                                        int64_t out[5]) {
    return emulate(t, steps, 0, 0, workers, seed, drop_task, skip_wait_task, wait_limit_s, max_delay_us, out);
}

extern "C" SPDINV_API spdinv_status spdinv_plan_emulate_variant(int t, int variant, int split_segment, int workers,
                                                                uint64_t seed, int drop_task, double wait_limit_s,
                                                                int max_delay_us, int64_t out[5]) {
    if (variant < 0) return SPDINV_ERR_UNSUPPORTED;
    return emulate(t, STEPS_ALL, variant, split_segment, workers, seed, drop_task, -1, wait_limit_s, max_delay_us,
                   out);
}

// Deterministic schedule of the same plan on `workers` CTAs (a list-scheduling
// model of the persistent kernel): the next ticket goes to the CTA that
// becomes free first, which then runs the task's chain elements in the
// kernel's order, each starting when the CTA is done with the previous one
// and the element's input tiles are final.  Costs in units of one b x b x b
// tile product, as in the plan: 1 per chain element and per TRMM, 0.7 for a
// diagonal POTRF + TRTRI, 0.4 for a TRTRI alone.
extern "C" SPDINV_API spdinv_status spdinv_plan_simulate(int t, int steps, int workers, double out[3]) {
    if (t < 1 || t > 4096) return SPDINV_ERR_N;
    if (steps < STEPS_ALL || steps > STEPS_DIAG || workers < 1) return SPDINV_ERR_UNSUPPORTED;
    if (!out) return SPDINV_ERR_NULL;
    const ExecPlan plan = build_exec_plan(t, steps, false, current_plan_order());
    const bool s1 = steps == STEPS_ALL || steps == STEPS_POTRF || steps == STEPS_DIAG;
    const bool from_A = s1, wait_d = steps != STEPS_LAUUM, wait_x = steps != STEPS_LAUUM;
    const size_t tt = (size_t)t * t;
    // Time at which each renamed tile is final (0: input or staged before the launch).
    std::vector<double> rL(tt, 0.0), rX(tt, 0.0), rD((size_t)t, 0.0);
    auto L = [&](int i, int j) -> double& { return rL[(size_t)i * t + j]; };
    auto X = [&](int i, int j) -> double& { return rX[(size_t)i * t + j]; };
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int w = 0; w < workers && w < (int)plan.order.size(); ++w) free_at.push(0.0);
    double makespan = 0.0, work = 0.0;
    for (const uint32_t e : plan.order) {
        const int kind = (int)task_kind(e), i = (int)task_i(e), j = (int)task_j(e);
        double now = free_at.top(), busy = 0.0;
        free_at.pop();
        auto elem = [&](double r0, double r1, double c) {
            now = std::max(now, std::max(r0, r1)) + c;
            busy += c;
        };
        switch (kind) {
            case K_S1_DIAG:
                for (int k = 0; k < j; ++k) elem(L(j, k), 0.0, 1.0);
                elem(0.0, 0.0, 0.7);
                rD[j] = now;
                break;
            case K_S1_OFF:
                for (int k = 0; k < j; ++k) elem(L(i, k), L(j, k), 1.0);
                elem(rD[j], 0.0, 1.0);
                L(i, j) = now;
                break;
            case K_S2_DIAG:
                elem(0.0, 0.0, 0.4);
                rD[j] = now;
                break;
            case K_S2_OFF:
                elem(rD[i], from_A ? L(i, j) : 0.0, 1.0);
                for (int k = i - 1; k > j; --k) elem(X(i, k), from_A ? L(k, j) : 0.0, 1.0);
                elem(rD[j], 0.0, 1.0);
                X(i, j) = now;
                break;
            case K_S3_OFF:
                elem(wait_d ? rD[i] : 0.0, wait_x ? X(i, j) : 0.0, 1.0);
                for (int k = i + 1; k < t; ++k) elem(wait_x ? X(k, i) : 0.0, wait_x ? X(k, j) : 0.0, 1.0);
                break;
            default:  // K_S3_DIAG
                elem(wait_d ? rD[i] : 0.0, 0.0, 1.0);
                for (int k = i + 1; k < t; ++k) elem(wait_x ? X(k, i) : 0.0, 0.0, 1.0);
                break;
        }
        work += busy;
        free_at.push(now);
        makespan = std::max(makespan, now);
    }
    out[0] = makespan;
    out[1] = work;
    out[2] = plan.crit;
    return SPDINV_OK;
}
