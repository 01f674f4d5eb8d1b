// Device-side machinery shared by the persistent tile-DAG kernels: error and
// info words, bounded waits on readiness flags, bulk (TMA) tile fetches into
// shared memory and publication of finished tiles.  It takes the place of the
// paper's dynamic scheduler (Sec. 3): a task starts as soon as the tiles it
// reads are final, across the boundaries of the three steps.
//
// Protocol.  A producer CTA writes a tile with ordinary stores; every thread
// then fences its stores for the async proxy and the GPU scope, the CTA
// synchronises, and thread 0 raises the tile's flag with st.release.gpu.  A
// consumer's thread 0 spins with ld.acquire.gpu on the flag (bounded),
// fences, and issues the bulk copy; before that every thread has fenced its
// own generic accesses of the destination buffer (fence.proxy.async is per
// thread).  The other threads wait at a barrier and then on the mbarrier
// that counts the copied bytes.
#pragma once
#include <cstdint>

#include "../../include/spdinv.h"
#include "ptx.cuh"

namespace spdinv {

struct PCtx {
    void* T0;          // shared tile buffers
    void* T1;
    uint64_t* bar;     // mbarrier of the CTA's copies
    int* s_flag;       // shared: thread 0's verdict
    uint32_t phase;
    int* ctrl;         // [0] ticket, [1] abort, [2] error, [3] info
    long long timeout_ns;
    int drop_task;
    uint64_t* wait_ns;  // tracing: thread 0 adds the time it waits on flags here (nullptr = off)
};

__device__ __forceinline__ void raise_error(int* ctrl, int code) {
    atomicCAS(&ctrl[2], 0, code);
    atomicExch(&ctrl[1], 1);
}

// First failing column wins (0 = none).
__device__ __forceinline__ void record_info(int* ctrl, int v) {
    int cur = atomicCAS(&ctrl[3], 0, v);
    while (cur != 0 && v < cur) {
        const int prev = atomicCAS(&ctrl[3], cur, v);
        if (prev == cur) break;
        cur = prev;
    }
    atomicExch(&ctrl[1], 1);
}

// Bounded spin on a readiness flag (thread 0 only).  false = give up (abort
// raised elsewhere, or this wait hit its limit, which raises the error).
__device__ __forceinline__ bool wait_flag(const int* flag, int* ctrl, long long timeout_ns) {
    if (flag == nullptr) return true;
    if (ld_acquire_gpu(flag) != 0) return true;
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
        if (ld_acquire_gpu(flag) != 0) return true;
        if (ld_relaxed_gpu(&ctrl[1]) != 0) return false;
        if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
            raise_error(ctrl, SPDINV_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

// Bounded wait on the CTA's mbarrier for the current phase (copies only).
__device__ __forceinline__ bool mbar_wait_bounded(PCtx& c) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(c.bar, c.phase)) {
        if ((long long)(globaltimer_ns() - t0) > 2000000000LL) {
            if (threadIdx.x == 0) raise_error(c.ctrl, SPDINV_ERR_TIMEOUT);
            return false;
        }
    }
    c.phase ^= 1u;
    return true;
}

// Bulk copies need 16-byte aligned addresses and sizes: checked once per CTA
// for the shared buffers and the stores' bases (tile sizes are multiples of
// 16 bytes), so a wrong layout ends the run with an error instead of a fault.
__device__ __forceinline__ bool layout_ok(const void* T0, const void* T1, const void* b0, const void* b1,
                                          const void* b2, int* ctrl) {
    const uintptr_t g = reinterpret_cast<uintptr_t>(b0) | reinterpret_cast<uintptr_t>(b1) |
                        reinterpret_cast<uintptr_t>(b2);
    const uint32_t s = smem_u32(T0) | smem_u32(T1);
    if ((g & 15u) == 0 && (s & 15u) == 0) return true;
    if (threadIdx.x == 0) raise_error(ctrl, SPDINV_ERR_UNSUPPORTED);
    return false;
}

// Wait for up to two readiness flags, then copy up to two tiles of `bytes`
// each into T0 / T1.  Called by all threads; false = stop (abort or timeout).
__device__ __forceinline__ bool fetch(PCtx& c, const int* f0, const int* f1, const void* g0, const void* g1,
                                      uint32_t bytes) {
    // Each thread orders its own generic reads and writes of T0 / T1 before
    // the async-proxy (bulk copy) writes that follow the barrier: the proxy
    // fence is per thread, so thread 0 fencing alone would leave the others'
    // stores free to land on top of the copied tile.
    fence_proxy_async_shared();
    cta_sync();  // every thread is done with T0 / T1
    if (threadIdx.x == 0) {
        const uintptr_t ga = reinterpret_cast<uintptr_t>(g0) | reinterpret_cast<uintptr_t>(g1);
        if ((ga & 15u) != 0 || (bytes & 15u) != 0) raise_error(c.ctrl, SPDINV_ERR_UNSUPPORTED);
        const uint64_t w0 = c.wait_ns ? globaltimer_ns() : 0;
        const bool ok = (ga & 15u) == 0 && (bytes & 15u) == 0 && wait_flag(f0, c.ctrl, c.timeout_ns) &&
                        wait_flag(f1, c.ctrl, c.timeout_ns);
        if (c.wait_ns) *c.wait_ns += globaltimer_ns() - w0;
        *c.s_flag = ok ? 0 : 1;
        if (ok) {
            fence_proxy_async_global();
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(c.bar, (g0 ? bytes : 0u) + (g1 ? bytes : 0u));
            if (g0) bulk_g2s(c.T0, g0, bytes, c.bar);
            if (g1) bulk_g2s(c.T1, g1, bytes, c.bar);
        }
    }
    // The others wait here while thread 0 waits on the dependency flags (its
    // own limit); the mbarrier wait below then covers only the copy itself.
    cta_sync();
    if (*c.s_flag != 0) return false;
    return mbar_wait_bounded(c);
}

// Double-buffered update chains.  Two sets of tile buffers, each with its own
// mbarrier; element e of a chain lands in set e & 1.  While element e is
// multiplied, the copy of element e + 1 is already in flight when its input
// flags were raised by the time element e started (thread 0 checks them once,
// without waiting); otherwise thread 0 waits for them (bounded) after element
// e, as the single-buffered fetch does.  Every issued copy is waited exactly
// once, also on the abort path, so no copy lands after the CTA has left.
struct Chain2 {
    unsigned char* base;  // set s, operand o at base + (2 s + o) * stride
    uint32_t stride;      // bytes per tile buffer
    uint64_t* bar;        // [2] mbarriers
    uint32_t phase;       // bit s: the parity set s waits for next
    int* s_state;         // shared [3]: [0] thread 0's verdict, [1..2] copy issued into set 0 / 1
    __device__ __forceinline__ void* buf(int s, int o) const { return base + (2 * s + o) * stride; }
};

struct ChainElem {
    const int* f0;
    const int* f1;
    const void* g0;
    const void* g1;
};

// Thread 0: copy element x into set s (flags already final).
__device__ __forceinline__ void chain_issue(Chain2& ch, int s, const ChainElem& x, uint32_t bytes) {
    fence_proxy_async_global();
    fence_proxy_async_shared();
    mbar_arrive_expect_tx(&ch.bar[s], (x.g0 ? bytes : 0u) + (x.g1 ? bytes : 0u));
    if (x.g0) bulk_g2s(ch.buf(s, 0), x.g0, bytes, &ch.bar[s]);
    if (x.g1) bulk_g2s(ch.buf(s, 1), x.g1, bytes, &ch.bar[s]);
}

// All threads: wait (bounded) for the copy into set s.
__device__ __forceinline__ bool chain_wait(Chain2& ch, int s, int* ctrl) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(&ch.bar[s], (ch.phase >> s) & 1u)) {
        if ((long long)(globaltimer_ns() - t0) > 2000000000LL) {
            if (threadIdx.x == 0) raise_error(ctrl, SPDINV_ERR_TIMEOUT);
            return false;
        }
    }
    ch.phase ^= 1u << s;
    return true;
}

// Runs a chain of m >= 1 elements: elem(e) names element e's flags and
// tiles, mul(e, Ta, Tb) consumes it from shared memory (all threads).  The
// buffers of both sets may be written by generic stores before the call
// (each thread fences them here).  false = stop (abort or timeout), with no
// copy in flight.
template <class Elem, class Mul>
__device__ __forceinline__ bool run_chain(Chain2& ch, PCtx& c, int m, uint32_t bytes, Elem&& elem, Mul&& mul) {
    fence_proxy_async_shared();
    cta_sync();
    if (threadIdx.x == 0) {
        const ChainElem x = elem(0);
        const uint64_t w0 = c.wait_ns ? globaltimer_ns() : 0;
        const bool ok = wait_flag(x.f0, c.ctrl, c.timeout_ns) && wait_flag(x.f1, c.ctrl, c.timeout_ns);
        if (c.wait_ns) *c.wait_ns += globaltimer_ns() - w0;
        if (ok) chain_issue(ch, 0, x, bytes);
        ch.s_state[0] = ok ? 0 : 1;
        ch.s_state[1] = ok ? 1 : 0;
        ch.s_state[2] = 0;
    }
    cta_sync();
    if (ch.s_state[0] != 0) return false;
    for (int e = 0; e < m; ++e) {
        const int s = e & 1;
        bool prefetched = false;  // thread 0 only
        if (threadIdx.x == 0 && e + 1 < m) {  // prefetch e + 1 if its inputs are final
            const ChainElem x = elem(e + 1);
            prefetched = (x.f0 == nullptr || ld_acquire_gpu(x.f0) != 0) &&
                         (x.f1 == nullptr || ld_acquire_gpu(x.f1) != 0);
            if (prefetched) chain_issue(ch, s ^ 1, x, bytes);
            ch.s_state[1 + (s ^ 1)] = prefetched ? 1 : 0;
        }
        if (!chain_wait(ch, s, c.ctrl)) {  // (2 s on one copy: the error is raised)
            if (prefetched) chain_wait(ch, s ^ 1, c.ctrl);  // drain the prefetch, bounded
            return false;
        }
        mul(e, ch.buf(s, 0), ch.buf(s, 1));
        fence_proxy_async_shared();  // this thread's reads of set s before the next copy into it
        cta_sync();
        if (e + 1 < m && ch.s_state[1 + (s ^ 1)] == 0) {
            if (threadIdx.x == 0) {
                const ChainElem x = elem(e + 1);
                const uint64_t w0 = c.wait_ns ? globaltimer_ns() : 0;
                const bool ok = wait_flag(x.f0, c.ctrl, c.timeout_ns) && wait_flag(x.f1, c.ctrl, c.timeout_ns);
                if (c.wait_ns) *c.wait_ns += globaltimer_ns() - w0;
                if (ok) chain_issue(ch, s ^ 1, x, bytes);
                ch.s_state[0] = ok ? 0 : 1;
            }
            cta_sync();
            if (ch.s_state[0] != 0) return false;  // nothing in flight: e + 1 was not issued
        }
    }
    return true;
}

// All threads: make the CTA's global writes visible -- to the generic proxy
// and to the async proxy of the consumers' bulk copies -- then raise the flag.
__device__ __forceinline__ void publish(PCtx& c, int* flag, int ticket) {
    fence_proxy_async_global();  // per thread, for its own stores
    __threadfence();
    cta_sync();
    if (threadIdx.x == 0 && flag != nullptr && ticket != c.drop_task) {
        __threadfence();
        st_release_gpu(flag, 1);
    }
}

// Takes the next ticket (thread 0) unless the run was aborted; -1 = done.
__device__ __forceinline__ int next_ticket(int* ctrl, int ntasks, int* s_task) {
    cta_sync();
    if (threadIdx.x == 0) {
        int m = -1;
        if (ld_relaxed_gpu(&ctrl[1]) == 0) {
            m = atomicAdd(&ctrl[0], 1);
            if (m >= ntasks) m = -1;
        }
        *s_task = m;
    }
    cta_sync();
    return *s_task;
}

}  // namespace spdinv
