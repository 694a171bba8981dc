// Persistent multi-batch kernel of the grid schedule (sm_103a).
//
// One cooperative launch runs every batch of a bc_compute call.  Up to W
// batches (kMaxPSlots at most) are in flight, each on a batch slot of its
// own (bc_internal.cuh), and the whole level loop of Brandes' two phases
// (Sec. II, Algorithm 1) runs on the device: nothing is read back between
// levels.  The kernel advances in ticks; in one tick every batch in flight
// takes one step:
//   INIT    clear the slot's per-vertex words over the batch's graph
//   DISC    discovery of level l+1 (top-down from the level-l entries, or
//           bottom-up over the graph's vertices, as decided for the step)
//   GATHER  sigma of the new level's entries from their predecessors
//   BWD     backward step of level l (Eq. 2), dependencies added into BC
// A tick has four phases, separated by grid-wide barriers:
//   A  row items, a warp each (all batches' items in one index space)
//   B  chunk tasks of heavy rows and deferred pull rows, a block each
//   C  finish of heavy rows, a warp each
//   D  bookkeeping, a warp per batch slot (block 0): direction decision,
//      level advance, end of a batch, next batch from the work list.
// BC is added with exact 128-bit integer atomics, so batches in flight at the
// same time may add into the same vertex, and the bits do not depend on
// which slot ran which batch or in which tick.
//
// The grid barrier is bounded: a block whose spin_limit-th poll still finds
// the barrier closed sets the error word and returns, and every other block returns at its next
// poll; the host reports GBBC_ERR_TIMEOUT.  Only the narrow (64-bit sigma)
// format runs here: a batch whose counts reach 2^64 is listed in wide_list
// with its BC untouched, and the host reruns it in the wide format.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bc_internal.cuh"
#include "bc_policy.cuh"
#include "bc_rows.cuh"

namespace gbbc {

namespace {

constexpr int kPWarps = kPBlock / kWarp;
constexpr int kClearPerWarp = 256;  // vertices a warp clears per INIT item

// ---- bounded grid barrier --------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks of the (co-resident, cooperative) grid meet here.  Returns false
// when the wait gave up or another block reported an error: the caller
// returns at once.
__device__ __forceinline__ bool grid_barrier(PGlobal* G, long long spin_limit, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_gpu(&G->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&G->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&G->bar_count, 0u);
            __threadfence();
            atomicAdd(&G->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_gpu(&G->bar_gen) == gen) {
                if (ld_acquire_gpu(&G->err) & 1u) {
                    ok = 0;
                    break;
                }
                if (++spins >= spin_limit) {
                    atomicOr(&G->err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ok && (ld_acquire_gpu(&G->err) & 1u)) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---- per-slot view of the shared state ---------------------------------------

struct TickView {  // what every block needs of a slot in one tick
    int phase, dir, level;
    int32_t lo, hi;
    long long q_lo, q_hi, items;
    u64 lanes;
};

__device__ __forceinline__ int locate(const long long* pre, int W, long long i) {
    int s = 0;
    while (s + 1 < W && pre[s + 1] <= i) ++s;
    return s;
}

// Flush the per-warp statistics of one slot's discovery items.
__device__ __forceinline__ void flush_slot_stats(const Slot& S, StepStats& st, unsigned long long& lsum,
                                                 unsigned long long& lesum) {
    flush_stats(S, st);
    if ((threadIdx.x & 31) == 0 && lsum) {
        atomicAdd(&S.ctr->lane_sum, lsum);
        atomicAdd(&S.ctr->lane_esum, lesum);
    }
    st.esum = st.scanned = 0ull;
    st.lanes = 0ull;
    lsum = lesum = 0ull;
}

// Seed of a new batch by one warp: lane j (j and j+32 per thread) starts at
// its source; repeated sources share one queue entry (first occurrence).
// Returns the number of level-0 entries; sets the counters for level 0.
__device__ __forceinline__ long long seed_warp(const Csr& g, const Slot& S, const int32_t* src, int nsrc) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    bool first[2] = {false, false};
    u64 mask[2] = {0ull, 0ull};
    int32_t v[2] = {-1, -1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j < nsrc) {
            v[h] = src[j];
            first[h] = true;
            for (int i = 0; i < nsrc; ++i)
                if (src[i] == v[h]) {
                    mask[h] |= 1ull << i;
                    if (i < j) first[h] = false;
                }
        }
    }
    const unsigned f0 = __ballot_sync(FULL, first[0]), f1 = __ballot_sync(FULL, first[1]);
    long long deg = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j < nsrc) {
            atomicOr(&S.vis[v[h]], 1ull << j);
            S.sigma[(size_t)v[h] * kLanes + j] = 1ull;
            if (first[h]) {
                const int pos = h == 0 ? __popc(f0 & below) : __popc(f0) + __popc(f1 & below);
                S.qv[pos] = v[h];
                S.qm[pos] = mask[h];
                MaskTag t;
                t.mask = mask[h];
                t.tag = 0;
                t.pad = 0;
                S.F[v[h]] = t;
                deg += __ldg(g.row_ptr + v[h] + 1) - __ldg(g.row_ptr + v[h]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) deg += __shfl_xor_sync(FULL, deg, o);
    const long long nq0 = __popc(f0) + __popc(f1);
    if (lane == 0) {
        S.ctr->qtail = (unsigned long long)nq0;
        S.ctr->edge_sum = (unsigned long long)deg;
        S.ctr->lane_sum = (unsigned long long)nsrc;
        S.ctr->lanes = nsrc == 64 ? ~0ull : ((1ull << nsrc) - 1ull);
    }
    __syncwarp();
    return nq0;
}

__device__ __forceinline__ void zero_counters(Counters* c) {
    const int lane = threadIdx.x & 31;
    constexpr int words = (int)(sizeof(Counters) / sizeof(unsigned));
    for (int i = lane; i < words; i += 32) ((unsigned*)c)[i] = 0u;
    __syncwarp();
}

// Counters a discovery step accumulates.
__device__ __forceinline__ void zero_disc(Counters* c) {
    c->heavy = c->tasks = c->medium = 0ull;
    c->edge_sum = c->scanned = 0ull;
    c->lanes = 0ull;
}

__device__ __forceinline__ long long pull_items(int32_t lo, int32_t hi) { return ((long long)hi - lo + 31) / 32; }

// Next batch of the work list for slot `w` (lane 0 of its bookkeeping warp).
__device__ __forceinline__ void take_batch(PCtl& c, PGlobal* G, const BlockBatch* batches, int nb) {
    const unsigned b = atomicAdd(&G->next, 1u);
    if ((int)b >= nb) {
        c.phase = PH_DONE;
        c.items = 0;
        return;
    }
    const BlockBatch bb = batches[b];
    c.batch = (int)b;
    c.lo = bb.lo;
    c.hi = bb.hi;
    c.phase = PH_INIT;
    c.level = 0;
    c.npull = 0;
    c.items = ((long long)bb.hi - bb.lo + kClearPerWarp - 1) / kClearPerWarp;
}

// Bookkeeping of slot w by one warp of block 0 (phase D).
__device__ void bookkeep(const Csr& g, const Slot& S, PCtl* ctl_w, long long* lev, const BlockBatch* batches, int nb,
                         const int32_t* srcs, int policy, const __half* wts, const long long* gmaxdeg,
                         PGlobal* G, int32_t* wide_list) {
    const int lane = threadIdx.x & 31;
    PCtl c = *ctl_w;  // every lane holds a copy; lane 0 writes it back
    Counters* ctr = S.ctr;
    const bool active = c.phase != PH_IDLE && c.phase != PH_DONE;  // the counters hold this batch's step
    bool finished = false;  // batch over: take the next one
    bool counted = true;    // the batch's work counts in the stats (not when rerun wide)
    if (c.phase == PH_IDLE) {
        finished = true;
    } else if (c.phase == PH_INIT) {
        const BlockBatch bb = batches[c.batch];
        zero_counters(ctr);
        const long long nq0 = seed_warp(g, S, srcs + bb.src_off, bb.nsrc);
        const float n_range = (float)(bb.hi - bb.lo);
        const float nnz_range = (float)(__ldg(g.row_ptr + bb.hi) - __ldg(g.row_ptr + bb.lo));
        __threadfence_block();
        decide_step(ctr, 0, 0, policy, wts, n_range, nnz_range, (float)gmaxdeg[bb.gi]);
        if (lane == 0) {
            lev[0] = 0;
            lev[1] = nq0;
        }
        c.level = 0;
        c.q_lo = 0;
        c.q_hi = nq0;
        c.dir = ctr->dir;
        c.lanes = ctr->lanes;
        c.npull += c.dir;
        __syncwarp();
        if (lane == 0) zero_disc(ctr);
        c.phase = PH_DISC;
        c.items = c.dir ? pull_items(c.lo, c.hi) : c.q_hi - c.q_lo;
    } else if (c.phase == PH_DISC) {
        const long long new_hi = (long long)ctr->qtail;
        if (new_hi == c.q_hi) {  // the forward phase is over: levels 0 .. level
            c.nlev = c.level + 1;
            if (c.nlev >= 2) {
                c.phase = PH_BWD;
                c.level = c.nlev - 1;
                c.q_lo = lev[c.level];
                c.q_hi = lev[c.level + 1];
                if (lane == 0) ctr->heavy = ctr->tasks = 0ull;
                c.items = c.q_hi - c.q_lo;
            } else {
                finished = true;
            }
        } else {
            if (lane == 0) {
                lev[c.level + 2] = new_hi;
                ctr->lane_sum = ctr->lane_esum = 0ull;
                ctr->heavy = ctr->tasks = 0ull;
            }
            c.new_hi = new_hi;
            c.phase = PH_GATHER;
            c.items = new_hi - c.q_hi;
        }
    } else if (c.phase == PH_GATHER) {
        if (ctr->carry) {  // a count reached 2^64: rerun wide on the host
            if (lane == 0) {
                const unsigned k = atomicAdd(&G->wide, 1u);
                wide_list[k] = c.batch;
            }
            counted = false;  // the host reruns it: its levels so far count, the batch does not
            c.nlev = c.level + 1;
            finished = true;
        } else {
            const BlockBatch bb = batches[c.batch];
            decide_step(ctr, c.q_hi, c.level + 1, policy, wts, (float)(bb.hi - bb.lo),
                        (float)(__ldg(g.row_ptr + bb.hi) - __ldg(g.row_ptr + bb.lo)), (float)gmaxdeg[bb.gi]);
            c.level += 1;
            c.q_lo = c.q_hi;
            c.q_hi = c.new_hi;
            c.dir = ctr->dir;
            c.lanes = ctr->lanes;
            c.npull += c.dir;
            __syncwarp();
            if (lane == 0) zero_disc(ctr);
            c.phase = PH_DISC;
            c.items = c.dir ? pull_items(c.lo, c.hi) : c.q_hi - c.q_lo;
        }
    } else if (c.phase == PH_BWD) {
        if (c.level - 1 >= 1) {
            c.level -= 1;
            c.q_lo = lev[c.level];
            c.q_hi = lev[c.level + 1];
            if (lane == 0) ctr->heavy = ctr->tasks = 0ull;
            c.items = c.q_hi - c.q_lo;
        } else {
            finished = true;
        }
    }
    if (active && ctr->err) {  // queue capacity: stop the launch
        if (lane == 0) {
            atomicOr(&G->err, 2u);
            G->err_info = ctr->err | ((unsigned)c.phase << 4) | ((unsigned)c.dir << 7) |
                          ((unsigned)(c.level & 0xffff) << 8);
        }
        c.phase = PH_DONE;
        c.items = 0;
        finished = false;
    }
    if (finished) {
        if (lane == 0 && c.phase != PH_IDLE) {
            if (counted) atomicAdd(&G->batches, 1ull);
            atomicAdd(&G->levels_fwd, (unsigned long long)c.nlev);
            atomicAdd(&G->levels_pull, (unsigned long long)c.npull);
        }
        if (lane == 0) take_batch(c, G, batches, nb);
    }
    __syncwarp();
    if (lane == 0) *ctl_w = c;
}

}  // namespace

#ifndef GBBC_PERSIST_MINB
#define GBBC_PERSIST_MINB 4
#endif
__global__ void __launch_bounds__(kPBlock, GBBC_PERSIST_MINB) k_persist(Csr g, const Slot* slots, int W, PCtl* ctl, long long* lev,
                                                     long long lev_stride, const BlockBatch* batches, int nb,
                                                     const int32_t* srcs, u64* bc, int policy, const __half* wts,
                                                     const long long* gmaxdeg, int heavy_deg, long long spin_limit,
                                                     PGlobal* G, int32_t* wide_list) {
    __shared__ __align__(16) unsigned char sl_raw[kMaxPSlots * sizeof(Slot)];
    __shared__ TickView tv[kMaxPSlots];
    __shared__ long long pre[kMaxPSlots + 1];
    extern __shared__ __align__(16) unsigned char dyn[];  // BwdWarpSmem per warp
    BwdWarpSmem* bsm = reinterpret_cast<BwdWarpSmem*>(dyn);
    __shared__ union {
        u128 b[kPWarps][kLanes];  // backward chunk partials
        struct {
            u64 ps[kPWarps][kLanes];
            unsigned pc[kPWarps][kLanes];
        } f;                      // gather chunk partials
        u64 part[kPWarps];        // bottom-up heavy row
    } tsm;
    __shared__ int s_ok, s_live;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Slot* sl = reinterpret_cast<Slot*>(sl_raw);
    {
        const unsigned* src = reinterpret_cast<const unsigned*>(slots);
        unsigned* dst = reinterpret_cast<unsigned*>(sl_raw);
        for (int i = threadIdx.x; i < (int)(W * sizeof(Slot) / sizeof(unsigned)); i += blockDim.x) dst[i] = src[i];
    }
    bwd_smem_zero(bsm[wid]);
    __syncthreads();
    BwdWarpSmem& sm = bsm[wid];
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (;;) {
        // ---- the tick's view of every slot (written by phase D of the last tick)
        if (threadIdx.x < W) {  // L2 reads: block 0 rewrote them before the barrier
            const PCtl* c = ctl + threadIdx.x;
            TickView& t = tv[threadIdx.x];
            t.phase = __ldcg(&c->phase);
            t.dir = __ldcg(&c->dir);
            t.level = __ldcg(&c->level);
            t.lo = __ldcg(&c->lo);
            t.hi = __ldcg(&c->hi);
            t.q_lo = __ldcg(&c->q_lo);
            t.q_hi = __ldcg(&c->q_hi);
            t.items = (t.phase == PH_IDLE || t.phase == PH_DONE) ? 0 : __ldcg(&c->items);
            t.lanes = __ldcg(&c->lanes);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int live = 0;
            pre[0] = 0;
            for (int s = 0; s < W; ++s) {
                pre[s + 1] = pre[s] + tv[s].items;
                live |= tv[s].phase != PH_DONE;
            }
            s_live = live;
        }
        __syncthreads();
        if (!s_live) return;  // every slot has run out of batches
        // ---- phase A: row items, a warp each
        {
            const long long total = pre[W];
            int cur = -1;
            StepStats st = {0ull, 0ull, 0ull};
            unsigned long long lsum = 0, lesum = 0;
            for (long long i = gw; i < total; i += nw) {
                const int s = locate(pre, W, i);
                if (s != cur) {
                    if (cur >= 0) flush_slot_stats(sl[cur], st, lsum, lesum);
                    cur = s;
                }
                const long long j = i - pre[s];
                const TickView& t = tv[s];
                const Slot& S = sl[s];
                if (t.phase == PH_INIT) {
                    const long long v0 = (long long)t.lo + j * kClearPerWarp;
                    MaskTag none;
                    none.mask = 0ull;
                    none.tag = -1;
                    none.pad = 0;
                    for (long long v = v0 + lane; v < v0 + kClearPerWarp && v < t.hi; v += 32) {
                        S.vis[v] = 0ull;
                        S.nx[v] = 0ull;
                        S.ovf[v] = 0ull;
                        S.F[v] = none;
                        S.F[S.n + v] = none;
                    }
                } else if (t.phase == PH_DISC) {
                    if (t.dir) pull_vertices(g, S, (long long)t.lo + j * 32, t.hi, t.lanes, t.level, heavy_deg, st);
                    else push_entry(g, S, t.q_lo + j, heavy_deg, st);
                } else if (t.phase == PH_GATHER) {
                    const MaskTag* F = S.F + (size_t)(t.level & 1) * S.n;
                    MaskTag* Fn = S.F + (size_t)((t.level + 1) & 1) * S.n;
                    gather_entry<false, false>(g, S, F, Fn, t.level, t.q_hi + j, heavy_deg, lsum, lesum);
                } else if (t.phase == PH_BWD) {
                    const MaskTag* Fs = S.F + (size_t)((t.level + 1) & 1) * S.n;
                    MaskTag* Fo = S.F + (size_t)(t.level & 1) * S.n;
                    bwd_entry<false, false, true>(g, S, bc, Fs, Fo, t.level, t.q_lo + j, heavy_deg, sm);
                }
            }
            if (cur >= 0) flush_slot_stats(sl[cur], st, lsum, lesum);
        }
        if (!grid_barrier(G, spin_limit, &s_ok)) return;
        // ---- phase B: chunk tasks and deferred bottom-up rows, a block each
        if (threadIdx.x == 0) {
            pre[0] = 0;
            for (int s = 0; s < W; ++s) {
                const TickView& t = tv[s];
                const Counters* c = sl[s].ctr;
                long long n = 0;
                if (t.phase == PH_DISC && t.dir) {
                    const long long med = (long long)__ldcg(&c->medium), hv = (long long)__ldcg(&c->heavy);
                    n = (med + kPWarps - 1) / kPWarps + hv;
                } else if (t.phase == PH_DISC || t.phase == PH_GATHER || t.phase == PH_BWD) {
                    const long long tk = (long long)__ldcg(&c->tasks);
                    n = tk < sl[s].tcap ? tk : sl[s].tcap;
                }
                pre[s + 1] = pre[s] + n;
            }
        }
        __syncthreads();
        {
            const long long total = pre[W];
            int cur = -1;
            StepStats st = {0ull, 0ull, 0ull};
            unsigned long long lsum = 0, lesum = 0;
            for (long long b = blockIdx.x; b < total; b += gridDim.x) {
                const int s = locate(pre, W, b);
                if (s != cur) {
                    if (cur >= 0) flush_slot_stats(sl[cur], st, lsum, lesum);
                    cur = s;
                }
                const long long j = b - pre[s];
                const TickView& t = tv[s];
                const Slot& S = sl[s];
                if (t.phase == PH_DISC && t.dir) {
                    const long long med = (long long)__ldcg(&S.ctr->medium);
                    const long long nmb = (med + kPWarps - 1) / kPWarps;
                    if (j < nmb) {
                        const long long r = j * kPWarps + wid;
                        if (r < med) pull_medium_row(g, S, t.lanes, t.level, S.medium[r], st);
                    } else {
                        pull_heavy_row(g, S, t.lanes, t.level, S.heavy[j - nmb], tsm.part, st);
                    }
                } else if (t.phase == PH_DISC) {
                    push_task(g, S, j, st);
                } else if (t.phase == PH_GATHER) {
                    const MaskTag* F = S.F + (size_t)(t.level & 1) * S.n;
                    gather_task<kPWarps, false>(g, S, F, t.level, j, tsm.f.ps, tsm.f.pc);
                } else {
                    const MaskTag* Fs = S.F + (size_t)((t.level + 1) & 1) * S.n;
                    bwd_task<kPWarps, false, false>(g, S, Fs, t.level, j, sm, tsm.b);
                }
            }
            if (cur >= 0) flush_slot_stats(sl[cur], st, lsum, lesum);
        }
        if (!grid_barrier(G, spin_limit, &s_ok)) return;
        // ---- phase C: finish of heavy rows, a warp each
        if (threadIdx.x == 0) {
            pre[0] = 0;
            for (int s = 0; s < W; ++s) {
                const TickView& t = tv[s];
                long long n = 0;
                if (t.phase == PH_GATHER || t.phase == PH_BWD) {
                    const long long hv = (long long)__ldcg(&sl[s].ctr->heavy);
                    n = hv < sl[s].hcap ? hv : sl[s].hcap;
                }
                pre[s + 1] = pre[s] + n;
            }
        }
        __syncthreads();
        {
            const long long total = pre[W];
            for (long long i = gw; i < total; i += nw) {
                const int s = locate(pre, W, i);
                const long long h = i - pre[s];
                if (tv[s].phase == PH_GATHER) gather_finish(sl[s], h);
                else bwd_finish<false, true>(sl[s], bc, h);
            }
        }
        if (!grid_barrier(G, spin_limit, &s_ok)) return;
        // ---- phase D: bookkeeping, a warp of block 0 per slot
        if (blockIdx.x == 0 && wid < W) {
            for (int s = wid; s < W; s += kPWarps)
                bookkeep(g, sl[s], ctl + s, lev + (long long)s * lev_stride, batches, nb, srcs, policy, wts, gmaxdeg,
                         G, wide_list);
        }
        if (!grid_barrier(G, spin_limit, &s_ok)) return;
    }
}

static size_t persist_dyn_smem() { return (size_t)kPWarps * sizeof(BwdWarpSmem); }

int persist_blocks_per_sm() {
    int n = 0;
    if (cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)persist_dyn_smem()) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist, kPBlock, persist_dyn_smem()) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_persist(const Csr& g, const Slot* slots, int W, PCtl* ctl, long long* lev, long long lev_stride,
                           const BlockBatch* batches, int nb, const int32_t* srcs, u64* bc, int policy,
                           const void* weights_fp16, const long long* graph_max_deg, int heavy_deg,
                           long long spin_limit, PGlobal* G, int32_t* wide_list, int blocks, cudaStream_t st) {
    if (W < 1 || W > kMaxPSlots || blocks < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)persist_dyn_smem());
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(kPBlock, 1, 1);
    cfg.dynamicSmemBytes = persist_dyn_smem();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persist, g, slots, W, ctl, lev, lev_stride, batches, nb, srcs, bc, policy,
                              (const __half*)weights_fp16, graph_max_deg, heavy_deg, spin_limit, G, wide_list);
}

}  // namespace gbbc
