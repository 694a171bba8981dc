// Per-row device functions of the batched Brandes kernels (64 sources per
// bitset word), shared by the per-step kernels (bc_kernels.cu) and the
// persistent multi-batch kernel (bc_persist.cu).  See bc_internal.cuh for the
// slot layout.  Every sum is an integer sum, so results do not depend on
// which thread, block or launch adds a term.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "bc_fixed.cuh"
#include "bc_internal.cuh"

namespace gbbc {

#define FULL 0xffffffffu

__device__ __forceinline__ u64 warp_or64(u64 x) {
    unsigned lo = __reduce_or_sync(FULL, (unsigned)x);
    unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
    return ((u64)hi << 32) | lo;
}

__device__ __forceinline__ u64 shfl64(u64 x, int src) {
    return __shfl_sync(FULL, x, src);
}

// Append `item` for the threads with pred set, one atomic per warp.  All
// 32 threads of the warp must call this.  Returns false on overflow.
__device__ __forceinline__ void warp_append(bool pred, int32_t item, unsigned long long* counter, int32_t* list,
                                            long long cap, unsigned* err, unsigned errbit) {
    const int lane = threadIdx.x & 31;
    unsigned bal = __ballot_sync(FULL, pred);
    if (!bal) return;
    int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (pred) {
        unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
        if ((long long)pos < cap) list[pos] = item;
        else atomicOr(err, errbit);
    }
}

// Loads of slot data: NC = the data is read-only for the whole kernel (one
// kernel per step), so the non-coherent path may serve it.  The persistent
// kernels rewrite slot data between their own steps, which are separated by
// barriers with acquire semantics (cluster or grid scope); their loads are
// then either L2-coherent (ld.cg) or ordinary loads, which the acquire makes
// see every write released before the barrier (GBBC_COHERENT_LOAD 1).
#ifndef GBBC_COHERENT_LOAD
#define GBBC_COHERENT_LOAD 0
#endif
template <bool NC>
__device__ __forceinline__ u64 ldv(const u64* p) {
    if (NC) return __ldg(p);
    return GBBC_COHERENT_LOAD ? *p : __ldcg(p);
}
template <bool NC>
__device__ __forceinline__ int ldi(const int* p) {
    if (NC) return __ldg(p);
    return GBBC_COHERENT_LOAD ? *p : __ldcg(p);
}

__device__ __forceinline__ long long gwarp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long nwarps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

// ---------------------------------------------------------------------------
// Heavy rows: a warp that meets entry e with more than heavy_deg neighbours
// reserves an accumulator slot h and ceil(deg / kChunk) chunk tasks.  All 32
// threads of the warp call this.
__device__ __forceinline__ void enqueue_heavy(const Slot& s, long long e, int32_t beg, int32_t end) {
    const int lane = threadIdx.x & 31;
    const int nch = (end - beg + kChunk - 1) / kChunk;
    unsigned long long h = 0, t0 = 0;
    if (lane == 0) {
        h = atomicAdd(&s.ctr->heavy, 1ull);
        t0 = atomicAdd(&s.ctr->tasks, (unsigned long long)nch);
    }
    h = __shfl_sync(FULL, h, 0);
    t0 = __shfl_sync(FULL, t0, 0);
    if ((long long)h >= s.hcap || (long long)(t0 + nch) > s.tcap) {
        if (lane == 0) atomicOr(&s.ctr->err, 2u);
        return;
    }
    if (lane == 0) s.hentry[h] = (int32_t)e;
    for (int i = lane; i < nch; i += 32) s.tasks[t0 + i] = make_int2((int)h, beg + i * kChunk);
}

// Task t of this step, validated against the capacities (a task slot that
// an overflowing reservation left unwritten is skipped).
__device__ __forceinline__ bool load_task(const Slot& s, const Csr& g, long long t, int& h, long long& e,
                                          int32_t& v, u64& m, int32_t& p0, int32_t& p1) {
    int2 tk = s.tasks[t];
    h = tk.x;
    if (h < 0 || h >= s.hcap) return false;
    e = s.hentry[h];
    if (e < 0 || e >= s.qcap) return false;
    v = s.qv[e];
    if (v < 0 || v >= g.n) return false;
    m = s.qm[e];
    int32_t beg = g.row_ptr[v], end = g.row_ptr[v + 1];
    p0 = tk.y;
    if (p0 < beg || p0 >= end) return false;
    p1 = p0 + kChunk < end ? p0 + kChunk : end;
    return true;
}

__device__ __forceinline__ long long task_count(const Slot& s) {
    long long c = (long long)s.ctr->tasks;
    return c < s.tcap ? c : s.tcap;
}

__device__ __forceinline__ long long heavy_count(const Slot& s) {
    long long c = (long long)s.ctr->heavy;
    return c < s.hcap ? c : s.hcap;
}

// ---------------------------------------------------------------------------
// Top-down discovery: for each frontier entry (v, m) and neighbour w, the
// lanes m & ~vis[w] reach w at the next level.  atomicOr collects them in
// nx[w]; the thread that turns nx[w] from 0 to non-zero queues w.
// Statistics of the next frontier gathered by the discovery kernels: the sum
// of degrees of newly queued vertices and the OR of the lanes reaching them.
struct StepStats {
    unsigned long long esum;
    unsigned long long scanned;
    u64 lanes;
};

__device__ __forceinline__ void flush_stats(const Slot& s, StepStats st) {
    // all 32 threads of the warp call this
    unsigned long long e = st.esum, c = st.scanned;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        e += __shfl_xor_sync(FULL, e, o);
        c += __shfl_xor_sync(FULL, c, o);
    }
    u64 l = warp_or64(st.lanes);
    if ((threadIdx.x & 31) == 0 && (e | l | c)) {
        atomicAdd(&s.ctr->edge_sum, e);
        atomicAdd(&s.ctr->scanned, c);
        atomicOr(&s.ctr->lanes, l);
    }
}

__device__ __forceinline__ void push_row(const Csr& g, const Slot& s, u64 m, int32_t beg, int32_t end, int t,
                                         int nthreads, StepStats& stats) {
    for (int32_t base = beg; base < end; base += nthreads) {
        int32_t p = base + t;
        bool newq = false;
        int32_t w = 0;
        if (p < end) {
            w = __ldg(g.col + p);
            u64 nm = m & ~s.vis[w];
            if (nm) {
                u64 old = atomicOr(&s.nx[w], nm);
                newq = (old == 0);
                stats.lanes |= nm;
                if (newq) stats.esum += (unsigned long long)(__ldg(g.row_ptr + w + 1) - __ldg(g.row_ptr + w));
            }
        }
        warp_append(newq, w, &s.ctr->qtail, s.qv, s.qcap, &s.ctr->err, 1u);
    }
}

// ---------------------------------------------------------------------------
// Forward gather + finalize for the entries queued at level `level`+1.
// Finalize: the entry's mask is nx[w] (then cleared), vis[w] gains it, and
// the dense frontier word of parity (level+1) is set.  Gather: for each lane
// j of the mask, sigma[w][j] = sum over neighbours v whose level-`level`
// mask has bit j of sigma[v][j], in CSR order, mod 2^64; a carry marks the
// lane in ovf[w].  Thread t owns lanes t and t+32.
//
// WIDE additionally keeps sigma of overflowed lanes as N * 2^X (N a
// normalised 64-bit mantissa, X an int32 exponent): terms are aligned to the
// largest exponent seen and summed in a u128, so the mantissa keeps 64 bits.
struct WideAcc {
    u128 a;   // sum, units of 2^x
    int x;    // exponent of a's unit; INT_MIN while empty
    bool ovf; // a predecessor overflowed
};

__device__ __forceinline__ u128 shr128(u128 a, int r) {
    u128 t;
    if (r <= 0) return a;
    if (r >= 128) { t.lo = t.hi = 0ull; return t; }
    if (r >= 64) { t.lo = a.hi >> (r - 64); t.hi = 0ull; return t; }
    t.lo = (a.lo >> r) | (a.hi << (64 - r));
    t.hi = a.hi >> r;
    return t;
}

__device__ __forceinline__ void wide_add(WideAcc& w, u128 v, int x) {
    if (v.lo == 0ull && v.hi == 0ull) return;
    if (w.x == INT_MIN) { w.a = v; w.x = x; return; }
    if (x > w.x) { w.a = shr128(w.a, x - w.x); w.x = x; }
    else v = shr128(v, w.x - x);
    w.a = add128(w.a, v);
}

struct GatherAcc {
    u64 a0, a1;
    unsigned c0, c1;
    WideAcc w0, w1;
};

__device__ __forceinline__ void gather_init(GatherAcc& acc) {
    acc.a0 = acc.a1 = 0ull;
    acc.c0 = acc.c1 = 0u;
    acc.w0.a.lo = acc.w0.a.hi = acc.w1.a.lo = acc.w1.a.hi = 0ull;
    acc.w0.x = acc.w1.x = INT_MIN;
    acc.w0.ovf = acc.w1.ovf = false;
}

// sigma of predecessor (v, lane) as mantissa/exponent
template <bool WIDE>
__device__ __forceinline__ void pred_term(const Slot& s, int32_t v, int lane_id, u64 x, u64 ovf_v, WideAcc& w) {
    if (!WIDE) return;
    u128 t;
    int X;
    if ((ovf_v >> lane_id) & 1ull) {
        t.lo = s.sN[(size_t)v * kLanes + lane_id];
        X = s.sX[(size_t)v * kLanes + lane_id];
        w.ovf = true;
    } else {
        t.lo = x;  // exact: x * 2^0
        X = 0;
    }
    t.hi = 0ull;
    wide_add(w, t, X);
}

// Up to four contributing neighbours per round: their (vertex, mask) pairs
// are broadcast from the ballot, then all loads are issued before any is
// used, so a warp keeps several independent loads in flight.
#ifndef GBBC_GATHER_ROUND
#define GBBC_GATHER_ROUND 4
#endif
// Backward: psi loads each thread issues before accumulating any of them
// (the terms of a flush, lane-compacted).  4 measured fastest with 5 blocks
// per SM (R-MAT 18 and 22: 2-4% faster backward than one at a time).
#ifndef GBBC_BWD_Q
#define GBBC_BWD_Q 4
#endif
// Occupancy hints: an explicit minimum of blocks per SM changes ptxas's
// register allocation.  The gather measured fastest without one; the
// backward keeps 5 blocks per SM (48 registers with four psi loads in flight
// per thread, no spills; its per-warp shared memory is 2.9 KB).
#ifdef GBBC_GATHER_MIN_BLOCKS
#define GBBC_GATHER_BOUNDS __launch_bounds__(kBlock, GBBC_GATHER_MIN_BLOCKS)
#else
#define GBBC_GATHER_BOUNDS
#endif
#ifndef GBBC_BWD_MIN_BLOCKS
#define GBBC_BWD_MIN_BLOCKS 5
#endif
#define GBBC_BWD_BOUNDS __launch_bounds__(kBlock, GBBC_BWD_MIN_BLOCKS)

template <int R>
struct RoundR {
    int32_t v[R];
    u64 f[R];
};
typedef RoundR<4> Round4;

template <int R>
__device__ __forceinline__ void take_round(unsigned& bal, int32_t v, u64 f, RoundR<R>& r) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
        int src = bal ? __ffs(bal) - 1 : -1;
        if (bal) bal &= bal - 1;
        int sl = src < 0 ? 0 : src;
        r.v[u] = __shfl_sync(FULL, v, sl);
        u64 ff = shfl64(f, sl);
        r.f[u] = src < 0 ? 0ull : ff;
    }
}

template <int NT, bool WIDE, bool NC = true>
__device__ __forceinline__ void fwd_gather_row(const Csr& g, const Slot& s, const MaskTag* F, int level, u64 m,
                                               int32_t beg, int32_t end, int first, GatherAcc& acc) {
    // this warp handles chunks starting at beg + first*32, stepping NT*32
    const int lane = threadIdx.x & 31;
    for (int32_t base = beg + first * kWarp; base < end; base += NT * kWarp) {
        int32_t p = base + lane;
        int32_t v = 0;
        u64 f = 0;
        if (p < end) {
            v = __ldg(g.col + p);
            MaskTag t = F[v];
            if (t.tag == level) f = t.mask & m;
        }
        unsigned bal = __ballot_sync(FULL, f != 0);
        if (WIDE) {
            while (bal) {
                int src = __ffs(bal) - 1;
                bal &= bal - 1;
                int32_t vv = __shfl_sync(FULL, v, src);
                u64 ff = shfl64(f, src);
                const u64* row = s.sigma + (size_t)vv * kLanes;
                u64 ov = s.ovf[vv];
                if ((ff >> lane) & 1ull) {
                    u64 x = ldv<NC>(row + lane);
                    acc.a0 += x;
                    acc.c0 |= acc.a0 < x;
                    pred_term<WIDE>(s, vv, lane, x, ov, acc.w0);
                }
                if ((ff >> (lane + 32)) & 1ull) {
                    u64 x = ldv<NC>(row + lane + 32);
                    acc.a1 += x;
                    acc.c1 |= acc.a1 < x;
                    pred_term<WIDE>(s, vv, lane + 32, x, ov, acc.w1);
                }
            }
        } else {
            while (bal) {
                constexpr int R = GBBC_GATHER_ROUND;
                RoundR<R> r;
                take_round<R>(bal, v, f, r);
                u64 x0[R], x1[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const u64* row = s.sigma + (size_t)r.v[u] * kLanes;
                    x0[u] = ((r.f[u] >> lane) & 1ull) ? ldv<NC>(row + lane) : 0ull;
                    x1[u] = ((r.f[u] >> (lane + 32)) & 1ull) ? ldv<NC>(row + lane + 32) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    acc.a0 += x0[u];
                    acc.c0 |= acc.a0 < x0[u];
                    acc.a1 += x1[u];
                    acc.c1 |= acc.a1 < x1[u];
                }
            }
        }
    }
}

template <bool WIDE>
__device__ __forceinline__ void wide_store(const Slot& s, int32_t w, int lane_id, const WideAcc& a) {
    // normalise to a 64-bit mantissa (truncating) and exponent
    int lz = clz128(a.a);
    int bits = 128 - lz;
    u64 N;
    if (bits > 64) N = shr128(a.a, bits - 64).lo;
    else N = a.a.lo << (64 - bits);
    s.sN[(size_t)w * kLanes + lane_id] = N;
    s.sX[(size_t)w * kLanes + lane_id] = a.x + bits - 64;
}

template <bool WIDE>
__device__ __forceinline__ void fwd_store(const Slot& s, int32_t w, u64 m, const GatherAcc& acc) {
    const int lane = threadIdx.x & 31;
    u64* row = s.sigma + (size_t)w * kLanes;
    const bool l0 = (m >> lane) & 1ull, l1 = (m >> (lane + 32)) & 1ull;
    if (l0) row[lane] = acc.a0;
    if (l1) row[lane + 32] = acc.a1;
    bool o0 = l0 && (acc.c0 || (WIDE && acc.w0.ovf));
    bool o1 = l1 && (acc.c1 || (WIDE && acc.w1.ovf));
    if (WIDE) {
        if (o0) wide_store<WIDE>(s, w, lane, acc.w0);
        if (o1) wide_store<WIDE>(s, w, lane + 32, acc.w1);
    }
    unsigned b0 = __ballot_sync(FULL, o0);
    unsigned b1 = __ballot_sync(FULL, o1);
    if (lane == 0 && (b0 | b1)) {
        s.ovf[w] |= ((u64)b1 << 32) | b0;
        atomicOr(&s.ctr->carry, 1u);
    }
}

// ---------------------------------------------------------------------------
// Backward step for the entries of level `level` (>= 1), in the integer
// fixed-point form of bc_fixed.cuh.  Successors of (v, lane j) are the
// neighbours w whose level-(level+1) mask has bit j.  Per (v, j):
//   A     = sum over successors of psi_w * 2^(E_v + 64)       (u128)
//   delta = N_v * A / 2^63                                    (units 2^-64)
//   psi_v = (floor(2^127 / N_v) + A) * 2^(-64 - E_v)         (stored rounded)
//   BC[v] += sum over lanes of delta                          (u128)
// The entry's own mask is published with tag `level` for the next step.

// sigma of (v, lane) as normalised mantissa N and exponent E = floor(log2)
template <bool WIDE>
__device__ __forceinline__ void sigma_norm(const Slot& s, int32_t v, int lane_id, u64 ovf_v, u64& N, int& E) {
    if (WIDE && ((ovf_v >> lane_id) & 1ull)) {
        N = s.sN[(size_t)v * kLanes + lane_id];
        E = s.sX[(size_t)v * kLanes + lane_id] + 63;
    } else {
        u64 x = s.sigma[(size_t)v * kLanes + lane_id];
        int lz = __clzll(x);
        N = x << lz;
        E = 63 - lz;
    }
}

template <bool WIDE>
__device__ __forceinline__ u128 psi_term(u64 bits, int eoff, int Ev) {
    int e = (int)((bits >> 52) & 0x7FFull) - 1023 + (WIDE ? eoff : 0);
    u64 M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return shl_term(M, e + Ev + 12);
}

// Lane-compacted accumulation over a whole row chunk.  The chunk's
// contributing successors (at most 32) get slots 0..S-1 in ballot order;
// their (slot, lane) terms are listed slot by slot, and each thread of the
// warp takes one term at a time: it loads psi[w_slot][lane], shifts it to
// the lane's fixed point and adds it into the lane's accumulator in shared
// memory.  Two terms of one flush may share a lane, so the adds are shared-
// memory atomics; the 128-bit term is split into three parts (bits 0-31,
// 32-63 and 64-127), each summed in its own 64-bit word, which cannot wrap
// for fewer than 2^32 terms, and recombined when the row is done.  Integer
// adds commute, so the sums do not depend on the order of the terms.
constexpr int kBwdListCap = 256;  // terms per flush (at most 64 per successor)
struct BwdWarpSmem {
    u64 acc[kLanes][3];
    u64 N[kLanes];
    int E[kLanes];
    int32_t w[kWarp];
    unsigned short list[kBwdListCap];
};

template <bool WIDE, bool NC>
__device__ __forceinline__ void bwd_flush(const Slot& s, BwdWarpSmem& sm, int K) {
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < K; i0 += GBBC_BWD_Q * kWarp) {
        u64 bits[GBBC_BWD_Q];
        int xo[GBBC_BWD_Q], jj[GBBC_BWD_Q];
        // every psi load of the round is issued before any is used
#pragma unroll
        for (int q = 0; q < GBBC_BWD_Q; ++q) {
            const int i = i0 + q * kWarp + lane;
            bits[q] = 0ull;
            xo[q] = 0;
            jj[q] = -1;
            if (i < K) {
                const unsigned code = sm.list[i];
                const int j = (int)(code & 63u);
                const size_t at = (size_t)sm.w[code >> 6] * kLanes + j;
                jj[q] = j;
                bits[q] = ldv<NC>(s.psi + at);
                if (WIDE) xo[q] = ldi<NC>(s.psi_e + at);
            }
        }
#pragma unroll
        for (int q = 0; q < GBBC_BWD_Q; ++q) {
            if (jj[q] >= 0) {
                const u128 t = psi_term<WIDE>(bits[q], xo[q], sm.E[jj[q]]);
                u64* a = sm.acc[jj[q]];
                atomicAdd(a, t.lo & 0xFFFFFFFFull);
                atomicAdd(a + 1, t.lo >> 32);
                if (t.hi) atomicAdd(a + 2, t.hi);
            }
        }
    }
}

template <int NT, bool WIDE, bool NC = true>
__device__ __forceinline__ void bwd_gather_row(const Csr& g, const Slot& s, const MaskTag* Fs, int level, u64 m,
                                               int32_t beg, int32_t end, int first, BwdWarpSmem& sm) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int32_t base = beg + first * kWarp; base < end; base += NT * kWarp) {
        int32_t p = base + lane;
        int32_t w = 0;
        u64 f = 0;
        if (p < end) {
            w = __ldg(g.col + p);
            MaskTag t = Fs[w];
            if (t.tag == level + 1) f = t.mask & m;
        }
        unsigned bal = __ballot_sync(FULL, f != 0);
        if (!bal) continue;
        if (f) sm.w[__popc(bal & below)] = w;
        int K = 0, slot = 0;
        while (bal) {
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const u64 ff = shfl64(f, src);
            const unsigned lo = (unsigned)ff, hi = (unsigned)(ff >> 32);
            const int clo = __popc(lo);
            if ((lo >> lane) & 1u) sm.list[K + __popc(lo & below)] = (unsigned short)((slot << 6) | lane);
            if ((hi >> lane) & 1u)
                sm.list[K + clo + __popc(hi & below)] = (unsigned short)((slot << 6) | (lane + 32));
            K += clo + __popc(hi);
            ++slot;
            if (bal == 0 || K > kBwdListCap - kLanes) {
                __syncwarp();
                bwd_flush<WIDE, NC>(s, sm, K);
                __syncwarp();
                K = 0;
            }
        }
    }
}

// Before a row: publish the lanes' exponents.  After it: the lanes' sums
// for this thread's two lanes, leaving the accumulators at zero.
__device__ __forceinline__ void bwd_row_begin(BwdWarpSmem& sm, int E0, int E1) {
    const int lane = threadIdx.x & 31;
    sm.E[lane] = E0;
    sm.E[lane + 32] = E1;
    __syncwarp();
}

__device__ __forceinline__ void bwd_row_begin_n(BwdWarpSmem& sm, u64 N0, int E0, u64 N1, int E1) {
    const int lane = threadIdx.x & 31;
    sm.N[lane] = N0;
    sm.N[lane + 32] = N1;
    bwd_row_begin(sm, E0, E1);
}

__device__ __forceinline__ u128 bwd_take(u64* a) {
    // a[0] + a[1] * 2^32 + a[2] * 2^64, mod 2^128
    u128 r;
    r.lo = a[0] + (a[1] << 32);
    r.hi = a[2] + (a[1] >> 32) + (r.lo < a[0] ? 1ull : 0ull);
    a[0] = a[1] = a[2] = 0ull;
    return r;
}

__device__ __forceinline__ void bwd_row_end(BwdWarpSmem& sm, u128& a0, u128& a1) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    a0 = bwd_take(sm.acc[lane]);
    a1 = bwd_take(sm.acc[lane + 32]);
    __syncwarp();
}

__device__ __forceinline__ void bwd_smem_zero(BwdWarpSmem& sm) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        sm.acc[lane][c] = 0ull;
        sm.acc[lane + 32][c] = 0ull;
    }
    __syncwarp();
}

// per-lane finish: delta (returned, units 2^-64) and psi_v (stored)
template <bool WIDE>
__device__ __forceinline__ u128 bwd_lane(const Slot& s, int32_t v, int lane_id, u64 N, int E, u128 A) {
    u128 d = mul_shift63(N, A);
    u128 psi = add128(recip127(N), A);
    u64 M;
    int e;
    round128(psi, -64 - E, M, e);
    size_t at = (size_t)v * kLanes + lane_id;
    if (WIDE) {
        s.psi[at] = unit_bits(M);
        s.psi_e[at] = e;
    } else {
        s.psi[at] = double_bits(M, e);
    }
    return d;
}

__device__ __forceinline__ u128 shfl_xor128(u128 a, int o) {
    u128 r;
    r.lo = __shfl_xor_sync(FULL, a.lo, o);
    r.hi = __shfl_xor_sync(FULL, a.hi, o);
    return r;
}

// Exact 128-bit add into a (low, high) pair with two 64-bit atomics (the low
// word's carry goes into the high word): the total is exact whatever the
// order of the adds.
__device__ __forceinline__ void atomic_add128(u64* a, u128 t) {
    if ((t.lo | t.hi) == 0ull) return;
    u64 old = atomicAdd(a, t.lo);
    u64 carry = (old + t.lo) < old ? 1ull : 0ull;
    if (t.hi + carry) atomicAdd(a + 1, t.hi + carry);
}

template <bool WIDE, bool ATOMIC_BC = false>
__device__ __forceinline__ void bwd_store(const Slot& s, u64* bc, int32_t v, u64 m, int E0, int E1, u64 N0, u64 N1,
                                          u128 a0, u128 a1) {
    const int lane = threadIdx.x & 31;
    u128 c;
    c.lo = c.hi = 0ull;
    if ((m >> lane) & 1ull) c = add128(c, bwd_lane<WIDE>(s, v, lane, N0, E0, a0));
    if ((m >> (lane + 32)) & 1ull) c = add128(c, bwd_lane<WIDE>(s, v, lane + 32, N1, E1, a1));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c = add128(c, shfl_xor128(c, o));
    if (lane == 0) {
        if (ATOMIC_BC) {  // several batches of one graph may run at once
            atomic_add128(bc + 2 * (size_t)v, c);
        } else {
            u128 b;
            b.lo = bc[2 * (size_t)v];
            b.hi = bc[2 * (size_t)v + 1];
            b = add128(b, c);
            bc[2 * (size_t)v] = b.lo;
            bc[2 * (size_t)v + 1] = b.hi;
        }
    }
}

// Finish a row (after bwd_row_begin_n and bwd_gather_row): the lanes of m
// are compacted, so a thread finishes one lane (two past 32 lanes) instead
// of two mostly idle ones; each lane's sum is taken from shared memory,
// delta and psi_v computed (bwd_lane), and the lanes' deltas summed into
// BC[v].
template <bool WIDE, bool ATOMIC_BC>
__device__ __forceinline__ void bwd_row_finish(const Slot& s, u64* bc, int32_t v, u64 m, BwdWarpSmem& sm) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const unsigned lo = (unsigned)m, hi = (unsigned)(m >> 32);
    const int clo = __popc(lo), cnt = clo + __popc(hi);
    __syncwarp();
    if ((lo >> lane) & 1u) sm.list[__popc(lo & below)] = (unsigned short)lane;
    if ((hi >> lane) & 1u) sm.list[clo + __popc(hi & below)] = (unsigned short)(lane + 32);
    __syncwarp();
    u128 c;
    c.lo = c.hi = 0ull;
    for (int i = lane; i < cnt; i += kWarp) {
        const int j = sm.list[i];
        const u128 A = bwd_take(sm.acc[j]);
        c = add128(c, bwd_lane<WIDE>(s, v, j, sm.N[j], sm.E[j], A));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c = add128(c, shfl_xor128(c, o));
    if (lane == 0) {
        if (ATOMIC_BC) {
            atomic_add128(bc + 2 * (size_t)v, c);
        } else {
            u128 b;
            b.lo = bc[2 * (size_t)v];
            b.hi = bc[2 * (size_t)v + 1];
            b = add128(b, c);
            bc[2 * (size_t)v] = b.lo;
            bc[2 * (size_t)v + 1] = b.hi;
        }
    }
    __syncwarp();
}

template <bool WIDE>
__device__ __forceinline__ void lane_norms(const Slot& s, int32_t v, u64 m, u64& N0, int& E0, u64& N1, int& E1) {
    const int lane = threadIdx.x & 31;
    u64 ov = WIDE ? s.ovf[v] : 0ull;
    N0 = N1 = 1ull << 63;
    E0 = E1 = 0;
    if ((m >> lane) & 1ull) sigma_norm<WIDE>(s, v, lane, ov, N0, E0);
    if ((m >> (lane + 32)) & 1ull) sigma_norm<WIDE>(s, v, lane + 32, ov, N1, E1);
}

// ---------------------------------------------------------------------------
// One work item of each step kind.  The per-step kernels (bc_kernels.cu) run
// them in grid-stride loops over one batch; the persistent kernel
// (bc_persist.cu) runs them over the combined items of all batches in flight.
// NC selects the read-only load path for slot data, valid only when no
// thread of the same launch writes that data.

// Top-down discovery of frontier entry e (a warp): rows longer than
// heavy_deg become chunk tasks.
__device__ __forceinline__ void push_entry(const Csr& g, const Slot& s, long long e, int heavy_deg,
                                           StepStats& stats) {
    int32_t v = s.qv[e];
    u64 m = s.qm[e];
    int32_t beg = __ldg(g.row_ptr + v), end = __ldg(g.row_ptr + v + 1);
    if (end - beg > heavy_deg) {
        enqueue_heavy(s, e, beg, end);
        return;
    }
    push_row(g, s, m, beg, end, threadIdx.x & 31, kWarp, stats);
}

// Top-down discovery of chunk task t of a heavy frontier row (a block).
__device__ __forceinline__ void push_task(const Csr& g, const Slot& s, long long t, StepStats& stats) {
    int h;
    long long e;
    int32_t v, p0, p1;
    u64 m;
    if (!load_task(s, g, t, h, e, v, m, p0, p1)) return;
    push_row(g, s, m, p0, p1, threadIdx.x, blockDim.x, stats);
}

// Bottom-up discovery of vertices base + lane, lane = 0..31, below hi (a
// warp): w collects the OR of its neighbours' level-`level` frontier masks,
// restricted to the active lanes that still miss w, and stops once every
// such lane is found.  Rows up to 32 entries are scanned by their thread;
// longer ones go to the medium (warp per row) or heavy (block per row) list.
__device__ __forceinline__ void pull_vertices(const Csr& g, const Slot& s, long long base, int32_t hi, u64 lanes,
                                              int level, int heavy_deg, StepStats& stats) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    const int32_t w = (int32_t)(base + (threadIdx.x & 31));
    u64 u = 0;
    int32_t beg = 0, end = 0;
    bool defer_med = false, defer_heavy = false;
    if (w < hi) {
        u = ~s.vis[w] & lanes;
        if (u) {
            beg = __ldg(g.row_ptr + w);
            end = __ldg(g.row_ptr + w + 1);
            if (end - beg > heavy_deg) {
                defer_heavy = true;
                u = 0;
            } else if (end - beg > kWarp) {
                defer_med = true;
                u = 0;
            }
        }
    }
    u64 f = 0;
    if (u) {
        for (int32_t p = beg; p < end; ++p) {
            ++stats.scanned;
            int32_t v = __ldg(g.col + p);
            MaskTag t = F[v];
            if (t.tag == level) {
                f |= t.mask;
                if ((f & u) == u) break;
            }
        }
    }
    u64 nm = f & u;
    if (nm) {
        s.nx[w] = nm;
        stats.lanes |= nm;
        stats.esum += (unsigned long long)(end - beg);
    }
    warp_append(nm != 0, w, &s.ctr->qtail, s.qv, s.qcap, &s.ctr->err, 1u);
    warp_append(defer_med, w, &s.ctr->medium, s.medium, s.n, &s.ctr->err, 2u);
    warp_append(defer_heavy, w, &s.ctr->heavy, s.heavy, s.n, &s.ctr->err, 2u);
}

// Bottom-up discovery of a deferred medium row w (a warp).
__device__ __forceinline__ void pull_medium_row(const Csr& g, const Slot& s, u64 lanes, int level, int32_t w,
                                                StepStats& stats) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    const int lane = threadIdx.x & 31;
    u64 u = ~s.vis[w] & lanes;
    int32_t beg = g.row_ptr[w], end = g.row_ptr[w + 1];
    u64 f = 0;
    for (int32_t base = beg; base < end; base += kWarp) {
        int32_t p = base + lane;
        if (p < end) {
            ++stats.scanned;
            MaskTag t = F[__ldg(g.col + p)];
            if (t.tag == level) f |= t.mask;
        }
        f = warp_or64(f);
        if ((f & u) == u) break;
    }
    u64 nm = f & u;
    if (nm && lane == 0) {
        s.nx[w] = nm;
        stats.lanes |= nm;
        stats.esum += (unsigned long long)(end - beg);
    }
    warp_append(nm != 0 && lane == 0, w, &s.ctr->qtail, s.qv, s.qcap, &s.ctr->err, 1u);
}

// Bottom-up discovery of a deferred heavy row w (a block, no early exit);
// part holds blockDim.x / 32 words of shared memory.
__device__ __forceinline__ void pull_heavy_row(const Csr& g, const Slot& s, u64 lanes, int level, int32_t w,
                                               u64* part, StepStats& stats) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 u = ~s.vis[w] & lanes;
    int32_t beg = g.row_ptr[w], end = g.row_ptr[w + 1];
    u64 f = 0;
    for (int32_t p = beg + threadIdx.x; p < end; p += blockDim.x) {
        ++stats.scanned;
        MaskTag t = F[__ldg(g.col + p)];
        if (t.tag == level) f |= t.mask;
    }
    f = warp_or64(f);
    if (lane == 0) part[wid] = f;
    __syncthreads();
    if (wid == 0) {
        u64 x = lane < nw ? part[lane] : 0;
        x = warp_or64(x);
        u64 nm = x & u;
        if (nm && lane == 0) {
            s.nx[w] = nm;
            stats.lanes |= nm;
            stats.esum += (unsigned long long)(end - beg);
        }
        warp_append(nm != 0 && lane == 0, w, &s.ctr->qtail, s.qv, s.qcap, &s.ctr->err, 1u);
    }
    __syncthreads();
}

// Gather of entry e of the new level `level`+1 (a warp): finalise its mask
// (from nx, then cleared), publish it in vis and in the frontier words of
// parity level+1, and sum sigma over its predecessors; heavy rows become
// chunk tasks (narrow) or block-per-row work (wide).
template <bool WIDE, bool NC>
__device__ __forceinline__ void gather_entry(const Csr& g, const Slot& s, const MaskTag* F, MaskTag* Fn, int level,
                                             long long e, int heavy_deg, unsigned long long& lsum,
                                             unsigned long long& lesum) {
    const int lane = threadIdx.x & 31;
    int32_t w = s.qv[e];
    u64 m = s.nx[w];
    int32_t beg = __ldg(g.row_ptr + w), end = __ldg(g.row_ptr + w + 1);
    __syncwarp();
    if (lane == 0) {
        s.qm[e] = m;
        s.nx[w] = 0;
        s.vis[w] |= m;
        MaskTag t;
        t.mask = m;
        t.tag = level + 1;
        t.pad = 0;
        Fn[w] = t;
        unsigned pc = (unsigned)__popcll(m);
        lsum += pc;
        lesum += (unsigned long long)pc * (unsigned long long)(end - beg);
    }
    if (end - beg > heavy_deg) {
        if (WIDE) {  // block per row (the wide sum is not order-free)
            if (lane == 0) {
                unsigned long long pos = atomicAdd(&s.ctr->heavy, 1ull);
                if ((long long)pos < s.n) s.heavy[pos] = (int32_t)e;
                else atomicOr(&s.ctr->err, 2u);
            }
        } else {
            __syncwarp();
            enqueue_heavy(s, e, beg, end);
        }
        return;
    }
    GatherAcc acc;
    gather_init(acc);
    fwd_gather_row<1, WIDE, NC>(g, s, F, level, m, beg, end, 0, acc);
    fwd_store<WIDE>(s, w, m, acc);
}

// Narrow gather of chunk task t of a heavy row (a block of NW warps): per-lane
// partial sums go into hacc[h][lane] with 64-bit atomics; a carry of any add
// (or inside a partial) marks the lane in hcarry[h].
template <int NW, bool NC>
__device__ __forceinline__ void gather_task(const Csr& g, const Slot& s, const MaskTag* F, int level, long long t,
                                            u64 (*ps)[kLanes], unsigned (*pc)[kLanes]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int h;
    long long e;
    int32_t v, p0, p1;
    u64 m;
    bool ok = load_task(s, g, t, h, e, v, m, p0, p1);
    GatherAcc acc;
    gather_init(acc);
    if (ok) fwd_gather_row<NW, false, NC>(g, s, F, level, m, p0, p1, wid, acc);
    ps[wid][lane] = acc.a0;
    ps[wid][lane + 32] = acc.a1;
    pc[wid][lane] = acc.c0;
    pc[wid][lane + 32] = acc.c1;
    __syncthreads();
    if (wid == 0 && ok) {
        u64 carry = 0;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            int j = lane + 32 * half;
            u64 sum = 0;
            unsigned c = 0;
            for (int i = 0; i < NW; ++i) {
                u64 x = ps[i][j];
                sum += x;
                c |= (sum < x) | pc[i][j];
            }
            if ((m >> j) & 1ull) {
                u64 old = atomicAdd(s.hacc + ((size_t)h * kLanes + j) * 2, sum);
                c |= (old + sum) < old;
                if (c) carry |= 1ull << j;
            }
        }
        u64 cw = warp_or64(carry);
        if (lane == 0 && cw) atomicOr(s.hcarry + h, cw);
    }
    __syncthreads();
}

// Narrow gather: finish heavy row h (a warp), reading and clearing its
// accumulators.
__device__ __forceinline__ void gather_finish(const Slot& s, long long h) {
    const int lane = threadIdx.x & 31;
    long long e = s.hentry[h];
    int32_t w = s.qv[e];
    u64 m = s.qm[e];
    u64* a = s.hacc + (size_t)h * kLanes * 2;
    GatherAcc acc;
    gather_init(acc);
    u64 cw = s.hcarry[h];
    acc.a0 = a[2 * lane];
    acc.a1 = a[2 * (lane + 32)];
    acc.c0 = (unsigned)((cw >> lane) & 1ull);
    acc.c1 = (unsigned)((cw >> (lane + 32)) & 1ull);
    a[2 * lane] = 0ull;
    a[2 * (lane + 32)] = 0ull;
    __syncwarp();
    if (lane == 0) s.hcarry[h] = 0ull;
    fwd_store<false>(s, w, m, acc);
}

// Backward step of entry e at level `level` (a warp): publish the entry's
// mask with tag `level` for the next (lower) step, then accumulate its
// lanes' dependencies from the successors at level+1; heavy rows become
// chunk tasks.  ATOMIC_BC: several batches may add into bc at once.
template <bool WIDE, bool NC, bool ATOMIC_BC>
__device__ __forceinline__ void bwd_entry(const Csr& g, const Slot& s, u64* bc, const MaskTag* Fs, MaskTag* Fo,
                                          int level, long long e, int heavy_deg, BwdWarpSmem& sm) {
    const int lane = threadIdx.x & 31;
    int32_t v = s.qv[e];
    u64 m = s.qm[e];
    int32_t beg = __ldg(g.row_ptr + v), end = __ldg(g.row_ptr + v + 1);
    if (lane == 0) {
        MaskTag t;
        t.mask = m;
        t.tag = level;
        t.pad = 0;
        Fo[v] = t;
    }
    if (end - beg > heavy_deg) {
        enqueue_heavy(s, e, beg, end);
        return;
    }
    u64 N0, N1;
    int E0, E1;
    lane_norms<WIDE>(s, v, m, N0, E0, N1, E1);
    bwd_row_begin_n(sm, N0, E0, N1, E1);
    bwd_gather_row<1, WIDE, NC>(g, s, Fs, level, m, beg, end, 0, sm);
    bwd_row_finish<WIDE, ATOMIC_BC>(s, bc, v, m, sm);
}

// Backward chunk task t of a heavy row (a block of NW warps): per-lane u128
// partial sums into hacc[h][lane] with exact 128-bit atomics.
template <int NW, bool WIDE, bool NC>
__device__ __forceinline__ void bwd_task(const Csr& g, const Slot& s, const MaskTag* Fs, int level, long long t,
                                         BwdWarpSmem& sm, u128 (*ps)[kLanes]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int h;
    long long e;
    int32_t v, p0, p1;
    u64 m;
    bool ok = load_task(s, g, t, h, e, v, m, p0, p1);
    u128 a0 = {0ull, 0ull}, a1 = {0ull, 0ull};
    if (ok) {
        u64 N0, N1;
        int E0, E1;
        lane_norms<WIDE>(s, v, m, N0, E0, N1, E1);
        bwd_row_begin(sm, E0, E1);
        bwd_gather_row<NW, WIDE, NC>(g, s, Fs, level, m, p0, p1, wid, sm);
        bwd_row_end(sm, a0, a1);
    }
    ps[wid][lane] = a0;
    ps[wid][lane + 32] = a1;
    __syncthreads();
    if (wid == 0 && ok) {
        u128 t0 = {0ull, 0ull}, t1 = {0ull, 0ull};
        for (int i = 0; i < NW; ++i) {
            t0 = add128(t0, ps[i][lane]);
            t1 = add128(t1, ps[i][lane + 32]);
        }
        u64* a = s.hacc + (size_t)h * kLanes * 2;
        atomic_add128(a + 2 * lane, t0);
        atomic_add128(a + 2 * (lane + 32), t1);
    }
    __syncthreads();
}

// Backward: finish heavy row h (a warp), reading and clearing its
// accumulators.
template <bool WIDE, bool ATOMIC_BC>
__device__ __forceinline__ void bwd_finish(const Slot& s, u64* bc, long long h) {
    const int lane = threadIdx.x & 31;
    long long e = s.hentry[h];
    int32_t v = s.qv[e];
    u64 m = s.qm[e];
    u64* a = s.hacc + (size_t)h * kLanes * 2;
    u128 a0 = {a[2 * lane], a[2 * lane + 1]};
    u128 a1 = {a[2 * (lane + 32)], a[2 * (lane + 32) + 1]};
    a[2 * lane] = a[2 * lane + 1] = 0ull;
    a[2 * (lane + 32)] = a[2 * (lane + 32) + 1] = 0ull;
    u64 N0, N1;
    int E0, E1;
    lane_norms<WIDE>(s, v, m, N0, E0, N1, E1);
    bwd_store<WIDE, ATOMIC_BC>(s, bc, v, m, E0, E1, N0, N1, a0, a1);
}

}  // namespace gbbc
