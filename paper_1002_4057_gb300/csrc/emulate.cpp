// Host emulation of the persistent kernel's scheduling protocol (no GPU):
// worker threads stand in for the CTAs.  Each takes the next ticket of the
// execution plan (build_exec_plan, the order the kernel's CTAs take tasks),
// waits -- bounded, as the kernel does -- for the readiness flag of every
// input tile of its task in the order the kernel reads them, spends a
// seeded random time on each chain element, and publishes its output flag.
// Run with many worker counts and seeds, it covers the protocol's races and
// deadlock freedom on the CPU; a dropped completion (the kernel's
// fault_drop_task hook) must end every worker with a timeout, not a hang.
//
// Inputs and outputs per task kind, as the kernel waits for and publishes
// them (Algorithm 1 with the renamed stores B = L, C = X, D = X_jj):
//   Step 1, diagonal j      waits L(j,k), k < j;                publishes D(j)
//   Step 1, off-diagonal    waits (L(i,k), L(j,k)), k < j; D(j); publishes L(i,j)
//   Step 2, off-diagonal    waits (D(i), L(i,j)); (X(i,k), L(k,j)), k = i-1 .. j+1;
//                           D(j);                                publishes X(i,j)
//   Step 3, off-diagonal    waits (D(i), X(i,j)); (X(k,i), X(k,j)), k > i
//   Step 3, diagonal        waits D(i); X(k,i), k > i
#include <atomic>
#include <chrono>
#include <cstdint>
#include <memory>
#include <random>
#include <thread>
#include <vector>

#include "../../include/spdinv.h"
#include "plan.h"

namespace spdinv {
namespace {

struct Emu {
    int t = 0;
    const std::vector<uint32_t>* tasks = nullptr;
    std::unique_ptr<std::atomic<int>[]> fL, fX, fD;  // readiness flags of B, C, D
    std::atomic<int> ticket{0}, abort{0}, completed{0}, order_errors{0};
    std::atomic<int64_t> max_wait_us{0};
    int drop = -1;
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
        if (f.exchange(1, std::memory_order_release)) order_errors.fetch_add(1);  // published twice
    }

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
            bool ok = true;
            auto need = [&](std::atomic<int>* a, std::atomic<int>* b) {
                ok = ok && wait(a) && wait(b);
                if (ok) work(rng);
            };
            if (kind == K_S1_DIAG) {
                for (int k = 0; k < j && ok; ++k) need(L(j, k), nullptr);
                if (!ok) return;
                publish(*D(j), tk);
            } else if (kind == K_S1_OFF) {
                for (int k = 0; k < j && ok; ++k) need(L(i, k), L(j, k));
                need(D(j), nullptr);
                if (!ok) return;
                publish(*L(i, j), tk);
            } else if (kind == K_S2_OFF) {
                need(D(i), L(i, j));
                for (int k = i - 1; k > j && ok; --k) need(X(i, k), L(k, j));
                need(D(j), nullptr);
                if (!ok) return;
                publish(*X(i, j), tk);
            } else if (kind == K_S3_OFF) {
                need(D(i), X(i, j));
                for (int k = i + 1; k < t && ok; ++k) need(X(k, i), X(k, j));
                if (!ok) return;
            } else if (kind == K_S3_DIAG) {
                need(D(i), nullptr);
                for (int k = i + 1; k < t && ok; ++k) need(X(k, i), nullptr);
                if (!ok) return;
            } else {
                order_errors.fetch_add(1);  // no other kind in the full inversion's plan
            }
            completed.fetch_add(1);
        }
    }
};

}  // namespace
}  // namespace spdinv

using namespace spdinv;

extern "C" SPDINV_API spdinv_status spdinv_plan_emulate(int t, int workers, uint64_t seed, int drop_task,
                                                        double wait_limit_s, int max_delay_us, int64_t out[4]) {
    if (t < 1 || t > 256) return SPDINV_ERR_N;
    if (workers < 1 || workers > 1024 || wait_limit_s <= 0.0 || max_delay_us < 0) return SPDINV_ERR_UNSUPPORTED;
    if (!out) return SPDINV_ERR_NULL;
    const ExecPlan plan = build_exec_plan(t, STEPS_ALL);
    Emu emu;
    emu.t = t;
    emu.tasks = &plan.order;
    const size_t tt = (size_t)t * t;
    emu.fL.reset(new std::atomic<int>[tt]);
    emu.fX.reset(new std::atomic<int>[tt]);
    emu.fD.reset(new std::atomic<int>[t]);
    for (size_t q = 0; q < tt; ++q) {
        emu.fL[q].store(0);
        emu.fX[q].store(0);
    }
    for (int q = 0; q < t; ++q) emu.fD[q].store(0);
    emu.drop = drop_task;
    emu.limit_s = wait_limit_s;
    emu.max_delay_us = max_delay_us;
    emu.seed = seed;
    std::vector<std::thread> th;
    th.reserve(workers);
    for (int w = 0; w < workers; ++w) th.emplace_back([&emu, w] { emu.run_worker(w); });
    for (auto& x : th) x.join();
    out[0] = emu.completed.load();
    out[1] = (int64_t)plan.order.size();
    out[2] = emu.order_errors.load();
    out[3] = emu.max_wait_us.load();
    if (emu.order_errors.load()) return SPDINV_ERR_UNSUPPORTED;
    return emu.abort.load() ? SPDINV_ERR_TIMEOUT : SPDINV_OK;
}
