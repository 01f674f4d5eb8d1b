// Persistent FP64 kernel for the tiled SPD inversion (Algorithm 1 of Agullo
// et al., with the array renaming and pipelining of Sec. 3).
//
// One launch runs the whole tile DAG.  CTAs take tasks from a global ticket
// counter in the planner's order (a topological order), so every task a CTA
// waits for was taken earlier by a running CTA: no deadlock, for any grid.
// Each task owns one output tile of one step and runs its whole commutative
// update chain with the accumulator in registers, waiting on the device-side
// readiness flag of each input tile just before it needs it:
//
//   Step 1, diagonal j      A_jj - sum_k L_jk L_jk^T, POTRF -> L_jj, TRTRI -> X_jj (store D_j)
//   Step 1, tile (i,j)      (A_ij - sum_k L_ik L_jk^T) X_jj^T = L_ij            (store B_ij)
//   Step 2, tile (i,j)      -(X_ii L_ij + sum_{k=i-1..j+1} X_ik L_kj) X_jj = X_ij (store C_ij)
//   Step 3, tile (i,j)      X_ii^T X_ij + sum_{k=i+1..t-1} X_ki^T X_kj          (into A)
//   Step 3, diagonal i      X_ii^T X_ii + sum_{k>i} X_ki^T X_ki  (lower part)   (into A)
//
// The renamed stores B (L), C (X = L^{-1}) and D (X_jj) are written once and
// never overwritten, so no task has a write-after-read hazard and the three
// steps overlap freely.  A is read once (Step 1) and written once (Step 3).
// Step 2's right TRMM uses X_jj rather than the A_jj printed in Algorithm 1:
// X L = I gives X_ij L_jj = -sum_{k=j+1..i} X_ik L_kj.  Step 1's TRSM is done
// as a product with X_jj^T, the inverse Step 2 needs anyway.
//
// Tiles of the stores are b x b, column-major, contiguous ("tile-major") and
// move between global and shared memory as single bulk (TMA) copies.  Ragged
// edges (n not a multiple of b) are padded with zeros and, on the diagonal,
// with the identity, which every step carries through unchanged.
#include <climits>

#include "kernels.h"
#include "persist.cuh"
#include "tile_fp64.cuh"

namespace spdinv {

namespace {

template <int B>
__device__ __forceinline__ bool fetch(PCtx& c, const int* f0, const int* f1, const double* g0, const double* g1) {
    return spdinv::fetch(c, f0, f1, g0, g1, (uint32_t)(B * B * sizeof(double)));
}

template <int B>
__device__ __forceinline__ const double* tileB(const KParamsF64& p, int i, int j) {
    return p.Bw + ((int64_t)i * (i - 1) / 2 + j) * (int64_t)(B * B);
}
template <int B>
__device__ __forceinline__ const double* tileC(const KParamsF64& p, int i, int j) {
    return p.Cw + ((int64_t)i * (i - 1) / 2 + j) * (int64_t)(B * B);
}
template <int B>
__device__ __forceinline__ const double* tileD(const KParamsF64& p, int j) {
    return p.Dw + (int64_t)j * (B * B);
}

// Tile (ti, tj) of the column-major A into T (padded: zeros, identity on the
// diagonal past n).  lower_only: diagonal tile, strictly upper part of A not read.
template <int B>
__device__ void load_A_tile(const KParamsF64& p, int ti, int tj, double* T, bool lower_only) {
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + c;
        double v;
        if (gr < p.n && gc < p.n) v = (lower_only && r < c) ? 0.0 : p.A[gr + gc * p.lda];
        else v = (ti == tj && r == c) ? 1.0 : 0.0;
        T[idx] = v;
    }
}

// T into tile (ti, tj) of A, clipped to n; lower_only keeps the upper part of A.
template <int B>
__device__ void store_A_tile(const KParamsF64& p, int ti, int tj, const double* T, bool lower_only) {
    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int r = idx % B, c = idx / B;
        const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + c;
        if (gr < p.n && gc < p.n && !(lower_only && r < c)) p.A[gr + gc * p.lda] = T[idx];
    }
}

template <int B>
__device__ void store_ws_tile(double* g, const double* T) {
    const double2* s = reinterpret_cast<const double2*>(T);
    double2* d = reinterpret_cast<double2*>(g);
    for (int idx = threadIdx.x; idx < B * B / 2; idx += kThreads) d[idx] = s[idx];
}

// Write-after-read wait of the shared-storage variants: thread 0 waits
// (bounded) until `expected` readers have counted their reads of the tile the
// CTA is about to overwrite.  false = stop (abort or timeout).
__device__ __forceinline__ bool wait_reads(PCtx& c, const int* r, int expected) {
    if (threadIdx.x == 0) {
        bool ok = true;
        if (ld_acquire_gpu(r) < expected) {
            const uint64_t t0 = globaltimer_ns();
            unsigned ns = 32;
            for (;;) {
                if (ld_acquire_gpu(r) >= expected) break;
                if (ld_relaxed_gpu(&c.ctrl[1]) != 0) {
                    ok = false;
                    break;
                }
                if ((long long)(globaltimer_ns() - t0) > c.timeout_ns) {
                    raise_error(c.ctrl, SPDINV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
            }
        }
        *c.s_flag = ok ? 0 : 1;
    }
    cta_sync();
    return *c.s_flag == 0;
}

// Thread 0 counts one completed read of each given tile (the copies are in
// shared memory when fetch returns, so the tile may be overwritten after it).
__device__ __forceinline__ void count_reads(int* r0, int* r1) {
    if (threadIdx.x == 0) {
        if (r0) red_release_add_gpu(r0, 1);
        if (r1) red_release_add_gpu(r1, 1);
    }
}

// VAR = false: the renamed, pipelined plan (the library's default).  VAR =
// true also runs the execution variants of p.variant: Step 2's chains in U
// order, C sharing B's storage, a single in-place store, split Step-3
// chains.  The variant code is compiled only into the VAR = true kernel.
template <int B, bool VAR>
__global__ void __launch_bounds__(kThreads) potri_fp64_persistent(const KParamsF64 prm) {
    unsigned char* const smem_raw = dynamic_smem();
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_task, s_flag, s_fail;
    const KParamsF64& p = prm;
    double* const T0 = reinterpret_cast<double*>(smem_raw);
    double* const T1 = T0 + B * B;
    double* const tmp = T1 + B * B;
    PCtx c;
    c.T0 = T0;
    c.T1 = T1;
    c.bar = &bar;
    c.s_flag = &s_flag;
    c.phase = 0;
    c.ctrl = p.ctrl;
    c.timeout_ns = p.timeout_ns;
    c.drop_task = p.drop_task;
    uint64_t wait_acc = 0;  // tracing: flag-wait time of the current task (thread 0)
    c.wait_ns = (VAR && p.trace) ? &wait_acc : nullptr;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async_shared();
    }
    cta_sync();
    if (!layout_ok(T0, T1, p.Bw, p.Cw, p.Dw, p.ctrl)) return;
    const int t = p.t;
    int* const fL = p.flags;                  // [t*t]  B_ij holds L_ij
    int* const fX = p.flags + (int64_t)t * t; // [t*t]  C_ij holds X_ij
    int* const fD = p.flags + 2 * (int64_t)t * t;  // [t]  D_j holds X_jj
    const bool from_A = p.steps == STEPS_ALL || p.steps == STEPS_POTRF || p.steps == STEPS_DIAG;
    // D_i is staged before the launch for spdinv_lauum: nothing to wait for.
    auto dflag = [&](int q) -> const int* { return p.steps == STEPS_LAUUM ? nullptr : &fD[q]; };
    // Variants: which reads are counted (the tiles a later version overwrites).
    const int var = VAR ? p.variant : 0;
    const bool uuu = VAR && (var & VAR_UUU);
    const bool cnt_l = VAR && (var & (VAR_SHARE_BC | VAR_INPLACE));
    const bool inplace = VAR && (var & VAR_INPLACE);
    const bool split = VAR && (var & VAR_SPLIT3);
    int* const rL = VAR ? p.reads : nullptr;
    auto cL = [&](int a, int b) -> int* { return cnt_l ? rL + (int64_t)a * t + b : nullptr; };
    auto cX = [&](int a, int b) -> int* { return inplace ? rL + (int64_t)t * t + (int64_t)a * t + b : nullptr; };
    auto cD = [&](int j) -> int* { return inplace ? rL + 2 * (int64_t)t * t + j : nullptr; };

    int prev_ticket = -1;  // tracing: the task this CTA ran last, and when it started
    uint64_t prev_t0 = 0;
    for (;;) {
        if constexpr (VAR) {
            if (p.trace && threadIdx.x == 0 && prev_ticket >= 0) {
                uint32_t smid;
                asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
                spdinv_trace_record r;
                r.task = p.tasks[prev_ticket];
                r.sm = smid;
                r.ticket = (uint32_t)prev_ticket;
                r.cta = blockIdx.x;
                r.t_start_ns = prev_t0;
                r.t_end_ns = globaltimer_ns();
                r.t_wait_ns = wait_acc;
                r.reserved = 0;
                p.trace[prev_ticket] = r;
            }
        }
        const int ticket = next_ticket(p.ctrl, p.ntasks, &s_task);
        if (ticket < 0) return;
        const uint32_t e = p.tasks[ticket];
        const int kind = (int)task_kind(e), i = (int)task_i(e), j = (int)task_j(e);
        Acc<B> acc;
        if constexpr (VAR) {
            prev_ticket = ticket;
            prev_t0 = globaltimer_ns();
            wait_acc = 0;
        }

        if (kind == K_S1_DIAG) {
            load_A_tile<B>(p, j, j, T0, true);
            cta_sync();
            acc_load<B>(acc, T0);
            for (int k = 0; k < j; ++k) {  // SYRK chain, U order
                if (!fetch<B>(c, &fL[j * t + k], nullptr, tileB<B>(p, j, k), nullptr)) return;
                if constexpr (VAR) count_reads(cL(j, k), nullptr);
                tile_mma<B, false, true, true, FULL, FULL>(acc, T0, T0);
            }
            cta_sync();
            acc_store<B>(acc, T0);
            const int fail = tile_potrf<B>(T0, &s_fail);
            if (fail) {
                if (threadIdx.x == 0) record_info(p.ctrl, j * B + fail);
                return;
            }
            tile_zero_upper<B>(T0);
            cta_sync();
            if (p.steps == STEPS_POTRF) store_A_tile<B>(p, j, j, T0, true);
            tile_trtri<B>(T0, tmp);
            store_ws_tile<B>(const_cast<double*>(tileD<B>(p, j)), T0);
            publish(c, &fD[j], ticket);
        } else if (kind == K_S1_OFF) {
            load_A_tile<B>(p, i, j, T0, false);
            cta_sync();
            acc_load<B>(acc, T0);
            for (int k = 0; k < j; ++k) {  // GEMM chain, U order
                if (!fetch<B>(c, &fL[i * t + k], &fL[j * t + k], tileB<B>(p, i, k), tileB<B>(p, j, k))) return;
                if constexpr (VAR) count_reads(cL(i, k), cL(j, k));
                tile_mma<B, false, true, true, FULL, FULL>(acc, T0, T1);
            }
            // TRSM: L_ij = A'_ij L_jj^{-T} = A'_ij X_jj^T
            if (!fetch<B>(c, &fD[j], nullptr, nullptr, tileD<B>(p, j))) return;
            if constexpr (VAR) count_reads(cD(j), nullptr);
            acc_store<B>(acc, T0);
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, false, true, false, FULL, LOWER>(acc, T0, T1);
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            store_ws_tile<B>(const_cast<double*>(tileB<B>(p, i, j)), T0);
            if (p.steps == STEPS_POTRF) store_A_tile<B>(p, i, j, T0, false);
            publish(c, &fL[i * t + j], ticket);
        } else if (kind == K_S2_DIAG) {  // spdinv_trtri: X_jj = TRTRI(A_jj)
            load_A_tile<B>(p, j, j, T0, true);
            tile_trtri<B>(T0, tmp);
            store_ws_tile<B>(const_cast<double*>(tileD<B>(p, j)), T0);
            store_A_tile<B>(p, j, j, T0, true);
            publish(c, &fD[j], ticket);
        } else if (kind == K_S2_OFF) {
            // X_ii L_ij
            if (!fetch<B>(c, &fD[i], from_A ? &fL[i * t + j] : nullptr, tileD<B>(p, i), tileB<B>(p, i, j))) return;
            if constexpr (VAR) count_reads(cD(i), cL(i, j));
            acc_zero<B>(acc);
            tile_mma<B, false, false, false, LOWER, FULL>(acc, T0, T1);
            if (!uuu) {
                for (int k = i - 1; k > j; --k) {  // GEMM chain, D order
                    if (!fetch<B>(c, &fX[i * t + k], from_A ? &fL[k * t + j] : nullptr, tileC<B>(p, i, k),
                                  tileB<B>(p, k, j)))
                        return;
                    if constexpr (VAR) count_reads(cX(i, k), cL(k, j));
                    tile_mma<B, false, false, false, FULL, FULL>(acc, T0, T1);
                }
            } else if constexpr (VAR) {
                for (int k = j + 1; k < i; ++k) {  // GEMM chain, U order (the UUU variant)
                    if (!fetch<B>(c, &fX[i * t + k], &fL[k * t + j], tileC<B>(p, i, k), tileB<B>(p, k, j))) return;
                    count_reads(cX(i, k), cL(k, j));
                    tile_mma<B, false, false, false, FULL, FULL>(acc, T0, T1);
                }
            }
            // X_ij = -(...) X_jj
            if (!fetch<B>(c, &fD[j], nullptr, nullptr, tileD<B>(p, j))) return;
            if constexpr (VAR) count_reads(cD(j), nullptr);
            acc_store<B>(acc, T0);
            cta_sync();
            acc_zero<B>(acc);
            tile_mma<B, false, false, true, FULL, LOWER>(acc, T0, T1);
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            if constexpr (VAR) {  // X_ij goes over L_ij: every reader of L_ij first
                if (cnt_l && !wait_reads(c, cL(i, j), readers_L(t, i, j))) return;
            }
            store_ws_tile<B>(const_cast<double*>(tileC<B>(p, i, j)), T0);
            if (p.steps == STEPS_TRTRI) store_A_tile<B>(p, i, j, T0, false);
            publish(c, &fX[i * t + j], ticket);
        } else if (VAR && kind == K_S3_PART) {  // one segment of a split Step-3 chain
            if constexpr (VAR) {
                const int q = (int)part_id(e);
                const PartTask pt = p.parts[q];
                acc_zero<B>(acc);
                for (int k = pt.k0; k < pt.k1; ++k) {
                    if (pt.i == pt.j) {
                        if (!fetch<B>(c, &fX[k * t + pt.i], nullptr, tileC<B>(p, k, pt.i), nullptr)) return;
                        tile_mma<B, true, false, false, FULL, FULL>(acc, T0, T0);
                    } else {
                        if (!fetch<B>(c, &fX[k * t + pt.i], &fX[k * t + pt.j], tileC<B>(p, k, pt.i),
                                      tileC<B>(p, k, pt.j)))
                            return;
                        tile_mma<B, true, false, false, FULL, FULL>(acc, T0, T1);
                    }
                }
                cta_sync();
                acc_store<B>(acc, T0);
                cta_sync();
                store_ws_tile<B>(p.Pw + (int64_t)q * (B * B), T0);
                publish(c, &p.fP[q], ticket);
            }
        } else if (kind == K_S3_OFF) {
            const bool wait_x = p.steps != STEPS_LAUUM;
            int kend = t;
            if constexpr (VAR) {
                if (split && p.split[tri_index(i, j)].np) kend = p.split[tri_index(i, j)].own_end;
            }
            // X_ii^T X_ij
            if (!fetch<B>(c, dflag(i), wait_x ? &fX[i * t + j] : nullptr, tileD<B>(p, i), tileC<B>(p, i, j))) return;
            if constexpr (VAR) count_reads(cD(i), cX(i, j));
            acc_zero<B>(acc);
            tile_mma<B, true, false, false, LOWER, FULL>(acc, T0, T1);
            for (int k = i + 1; k < kend; ++k) {  // GEMM chain, U order
                if (!fetch<B>(c, wait_x ? &fX[k * t + i] : nullptr, wait_x ? &fX[k * t + j] : nullptr,
                              tileC<B>(p, k, i), tileC<B>(p, k, j)))
                    return;
                if constexpr (VAR) count_reads(cX(k, i), cX(k, j));
                tile_mma<B, true, false, false, FULL, FULL>(acc, T0, T1);
            }
            if constexpr (VAR) {  // the partial sums of the chain's other segments, in order
                if (split) {
                    const SplitInfo si = p.split[tri_index(i, j)];
                    for (uint32_t q = si.first; q < si.first + si.np; ++q) {
                        if (!fetch<B>(c, &p.fP[q], nullptr, p.Pw + (int64_t)q * (B * B), nullptr)) return;
                        acc_add<B>(acc, T0);
                    }
                }
            }
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            if constexpr (VAR) {
                if (inplace) {  // A^{-1}_ij goes over X_ij: every reader of X_ij first
                    if (!wait_reads(c, cX(i, j), readers_X(t, i, j))) return;
                    store_ws_tile<B>(const_cast<double*>(tileC<B>(p, i, j)), T0);
                    continue;
                }
            }
            store_A_tile<B>(p, i, j, T0, false);
        } else {  // K_S3_DIAG
            const bool wait_x = p.steps != STEPS_LAUUM;
            int kend = t;
            if constexpr (VAR) {
                if (split && p.split[tri_index(i, i)].np) kend = p.split[tri_index(i, i)].own_end;
            }
            // LAUUM: X_ii^T X_ii
            if (!fetch<B>(c, dflag(i), nullptr, tileD<B>(p, i), nullptr)) return;
            if constexpr (VAR) count_reads(cD(i), nullptr);
            acc_zero<B>(acc);
            tile_mma<B, true, false, false, LOWER, LOWER>(acc, T0, T0);
            for (int k = i + 1; k < kend; ++k) {  // SYRK chain, U order
                if (!fetch<B>(c, wait_x ? &fX[k * t + i] : nullptr, nullptr, tileC<B>(p, k, i), nullptr)) return;
                if constexpr (VAR) count_reads(cX(k, i), nullptr);
                tile_mma<B, true, false, false, FULL, FULL>(acc, T0, T0);
            }
            if constexpr (VAR) {
                if (split) {
                    const SplitInfo si = p.split[tri_index(i, i)];
                    for (uint32_t q = si.first; q < si.first + si.np; ++q) {
                        if (!fetch<B>(c, &p.fP[q], nullptr, p.Pw + (int64_t)q * (B * B), nullptr)) return;
                        acc_add<B>(acc, T0);
                    }
                }
            }
            cta_sync();
            acc_store<B>(acc, T0);
            cta_sync();
            if constexpr (VAR) {
                if (inplace) {  // A^{-1}_ii goes over X_ii: every reader of X_ii first
                    if (!wait_reads(c, cD(i), readers_D(t, i))) return;
                    store_ws_tile<B>(const_cast<double*>(tileD<B>(p, i)), T0);
                    continue;
                }
            }
            if (p.steps == STEPS_DIAG) {
                for (int r = threadIdx.x; r < B; r += kThreads) {
                    const int64_t g = (int64_t)i * B + r;
                    if (g < p.n) p.diag[g] = T0[r * B + r];
                }
            } else {
                store_A_tile<B>(p, i, i, T0, true);
            }
        }
    }
}

// The in-place variant's result: the lower tiles of its single store (which
// hold A^{-1} after Step 3) into A, clipped to n; diagonal tiles' lower part.
template <int B>
__global__ void __launch_bounds__(kThreads) stage_out_fp64(const KParamsF64 p) {
    const int t = p.t;
    const int64_t ntri = (int64_t)t * (t - 1) / 2;
    for (int64_t tile = blockIdx.x; tile < ntri + t; tile += gridDim.x) {
        int ti, tj;
        const bool is_diag = tile >= ntri;
        if (is_diag) {
            ti = tj = (int)(tile - ntri);
        } else {
            ti = (int)((1.0 + sqrt(1.0 + 8.0 * (double)tile)) / 2.0);
            while ((int64_t)ti * (ti - 1) / 2 > tile) --ti;
            while ((int64_t)(ti + 1) * ti / 2 <= tile) ++ti;
            tj = (int)(tile - (int64_t)ti * (ti - 1) / 2);
        }
        const double* src = is_diag ? p.Dw + (int64_t)ti * B * B : p.Cw + tile * (int64_t)(B * B);
        for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
            const int r = idx % B, cc = idx / B;
            const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + cc;
            if (gr < p.n && gc < p.n && !(is_diag && r < cc)) p.A[gr + gc * p.lda] = src[idx];
        }
    }
}

// Copies A's tiles into the renamed stores for the standalone steps:
// lower-triangular tiles below the diagonal into dst (B or C), diagonal tiles
// (lower part, identity padding) into D when diag != nullptr.  For TRTRI it
// also records the first exactly-zero diagonal entry (LAPACK dtrtri), which
// makes the main kernel leave A untouched.
template <int B>
__global__ void __launch_bounds__(kThreads) stage_in_fp64(const KParamsF64 p, double* dst, double* diag,
                                                          int check_zero_diag) {
    const int t = p.t;
    const int64_t ntri = (int64_t)t * (t - 1) / 2;
    for (int64_t tile = blockIdx.x; tile < ntri + t; tile += gridDim.x) {
        int ti, tj;
        bool is_diag = tile >= ntri;
        if (is_diag) {
            ti = tj = (int)(tile - ntri);
            if (diag == nullptr && !check_zero_diag) continue;
        } else {
            // tile = ti*(ti-1)/2 + tj
            ti = (int)((1.0 + sqrt(1.0 + 8.0 * (double)tile)) / 2.0);
            while ((int64_t)ti * (ti - 1) / 2 > tile) --ti;
            while ((int64_t)(ti + 1) * ti / 2 <= tile) ++ti;
            tj = (int)(tile - (int64_t)ti * (ti - 1) / 2);
        }
        double* out = is_diag ? (diag ? diag + (int64_t)ti * B * B : nullptr) : dst + tile * (int64_t)(B * B);
        for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
            const int r = idx % B, cc = idx / B;
            const int64_t gr = (int64_t)ti * B + r, gc = (int64_t)tj * B + cc;
            double v;
            if (gr < p.n && gc < p.n) v = (is_diag && r < cc) ? 0.0 : p.A[gr + gc * p.lda];
            else v = (is_diag && r == cc) ? 1.0 : 0.0;
            if (is_diag && check_zero_diag && r == cc && gr < p.n && v == 0.0) record_info(p.ctrl, (int)gr + 1);
            if (out) out[idx] = v;
        }
    }
}

__global__ void finalize_info(const int* ctrl, int* d_info) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int err = ctrl[2], info = ctrl[3];
        *d_info = err != 0 ? err : info;
    }
}

template <int B>
int smem_bytes() {
    return (2 * B * B + kThreads) * (int)sizeof(double);
}

template <int B, bool VAR>
cudaError_t launch_impl(const KParamsF64& p, int ctas_per_sm, int num_sms, cudaStream_t s, int* grid_out) {
    auto kern = potri_fp64_persistent<B, VAR>;
    const int sm = smem_bytes<B>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // 3 resident CTAs per SM at either tile: with the DFMA tile products the
    // FP64 pipe stays full, and fewer CTAs wait less on the DAG (tile 32,
    // 3 against 6: 1126 vs 1026 Gflop/s at n = 4096, 1210 vs 1165 at 8192,
    // 1237 vs 1201 at 16384).
    int per = ctas_per_sm > 0 ? ctas_per_sm : 3;
    per = per < occ ? per : occ;
    int grid = num_sms * per;
    if (grid > p.ntasks) grid = p.ntasks > 0 ? p.ntasks : 1;
    *grid_out = grid;
    if (p.steps == STEPS_TRTRI || p.steps == STEPS_LAUUM) {
        const int64_t ntiles = (int64_t)p.t * (p.t + 1) / 2;
        const int g2 = (int)(ntiles < 4096 ? ntiles : 4096);
        if (p.steps == STEPS_TRTRI)
            stage_in_fp64<B><<<g2, kThreads, 0, s>>>(p, p.Bw, nullptr, 1);
        else
            stage_in_fp64<B><<<g2, kThreads, 0, s>>>(p, p.Cw, p.Dw, 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kThreads, sm, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (VAR && (p.variant & VAR_INPLACE)) {
        const int64_t ntiles = (int64_t)p.t * (p.t + 1) / 2;
        const int g2 = (int)(ntiles < 4096 ? ntiles : 4096);
        stage_out_fp64<B><<<g2, kThreads, 0, s>>>(p);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

cudaError_t launch_potri_fp64(const KParamsF64& p, int ctas_per_sm, int num_sms, int* d_info, cudaStream_t s,
                              int* grid_out) {
    cudaError_t e;
    const bool var = p.variant != 0 || p.trace != nullptr;
    switch (p.b) {
        case 32:
            e = var ? launch_impl<32, true>(p, ctas_per_sm, num_sms, s, grid_out)
                    : launch_impl<32, false>(p, ctas_per_sm, num_sms, s, grid_out);
            break;
        case 64:
            e = var ? launch_impl<64, true>(p, ctas_per_sm, num_sms, s, grid_out)
                    : launch_impl<64, false>(p, ctas_per_sm, num_sms, s, grid_out);
            break;
        case 128:
            if (var) return cudaErrorInvalidValue;
            e = launch_potri_fp64_b128(p, num_sms, s, grid_out);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (d_info) {
        finalize_info<<<1, 32, 0, s>>>(p.ctrl, d_info);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace spdinv
