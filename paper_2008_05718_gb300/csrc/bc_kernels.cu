// Batched Brandes kernels (64 sources per bitset word) for sm_103a.
//
// Every kernel works on one batch slot (bc_internal.cuh).  Entries of the
// frontier queue are (vertex, lane mask) pairs; the queue holds the levels
// back to back, so the backward phase walks the same entries in reverse.
// Rows are processed by a warp each; rows longer than `heavy_deg` are
// deferred to a list that a second kernel processes with a whole block per
// row.  All floating-point sums run in CSR order within a row, and across
// warps of a block in warp order, so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

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

__device__ __forceinline__ long long gwarp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long nwarps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

static int grid_for(long long warps_needed, int nsm, int per_sm = 8) {
    long long blocks = (warps_needed * kWarp + kBlock - 1) / kBlock;
    long long cap = (long long)nsm * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// ---------------------------------------------------------------------------
// Seed: lane j starts at source d_src[j]; sources repeated within a batch
// share one queue entry.  One block of 64 threads.
__global__ void k_seed(Slot s, int nsrc) {
    const int j = threadIdx.x;
    __shared__ int32_t src[kLanes];
    if (j < nsrc) src[j] = s.d_src[j];
    __syncthreads();
    if (j < nsrc) {
        int32_t v = src[j];
        atomicOr(&s.vis[v], 1ull << j);
        s.sigma[(size_t)v * kLanes + j] = 1ull;
        bool first = true;
        u64 mask = 0;
        for (int i = 0; i < nsrc; ++i)
            if (src[i] == v) {
                mask |= 1ull << i;
                if (i < j) first = false;
            }
        if (first) {
            int pos = 0;  // distinct sources among lanes < j
            for (int i = 0; i < j; ++i) {
                bool fi = true;
                for (int h = 0; h < i; ++h)
                    if (src[h] == src[i]) { fi = false; break; }
                pos += fi;
            }
            s.qv[pos] = v;
            s.qm[pos] = mask;
            MaskTag t;
            t.mask = mask;
            t.tag = 0;
            t.pad = 0;
            s.F[v] = t;  // parity 0
        }
    }
}

void launch_seed(const Slot& s, int nsrc, cudaStream_t st) { k_seed<<<1, kLanes, 0, st>>>(s, nsrc); }

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

__global__ void k_push(Csr g, Slot s, long long q_lo, long long q_hi, int heavy_deg) {
    const int lane = threadIdx.x & 31;
    StepStats stats = {0ull, 0ull, 0ull};
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
        int32_t v = s.qv[e];
        u64 m = s.qm[e];
        int32_t beg = __ldg(g.row_ptr + v), end = __ldg(g.row_ptr + v + 1);
        if (end - beg > heavy_deg) {
            if (lane == 0) {
                unsigned long long pos = atomicAdd(&s.ctr->heavy, 1ull);
                if ((long long)pos < s.n) s.heavy[pos] = (int32_t)e;
                else atomicOr(&s.ctr->err, 2u);
            }
            continue;
        }
        push_row(g, s, m, beg, end, lane, kWarp, stats);
    }
    flush_stats(s, stats);
}

__global__ void k_push_heavy(Csr g, Slot s) {
    const long long cnt = (long long)s.ctr->heavy;
    StepStats stats = {0ull, 0ull, 0ull};
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        long long e = s.heavy[h];
        int32_t v = s.qv[e];
        u64 m = s.qm[e];
        push_row(g, s, m, g.row_ptr[v], g.row_ptr[v + 1], threadIdx.x, blockDim.x, stats);
    }
    flush_stats(s, stats);
}

void launch_push(const Csr& g, const Slot& s, long long q_lo, long long q_hi, int level, int heavy_deg, int nsm,
                 cudaStream_t st) {
    (void)level;
    long long cnt = q_hi - q_lo;
    if (cnt <= 0) return;
    k_push<<<grid_for(cnt, nsm), kBlock, 0, st>>>(g, s, q_lo, q_hi, heavy_deg);
    k_push_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, s);
}

// ---------------------------------------------------------------------------
// Bottom-up discovery over the vertex range [lo, hi): w collects the OR of
// its neighbours' level-`level` frontier masks, restricted to the lanes that
// still miss w; the scan stops once every such lane is found.
// Rows up to 32 entries: one thread per row.  Longer rows go to a list that
// k_pull_medium (a warp per row) or k_pull_heavy (a block per row) handles.
__global__ void k_pull_thread(Csr g, Slot s, int32_t lo, int32_t hi, u64 lanes, int level, int heavy_deg,
                              int32_t* medium, unsigned long long* n_medium) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    StepStats stats = {0ull, 0ull, 0ull};
    for (long long base = (long long)lo + (long long)blockIdx.x * blockDim.x; base < hi; base += stride) {
        int32_t w = (int32_t)(base + threadIdx.x);
        u64 u = 0;
        int32_t beg = 0, end = 0;
        bool defer_med = false, defer_heavy = false;
        if (w < hi) {
            u = ~s.vis[w] & lanes;
            if (u) {
                beg = __ldg(g.row_ptr + w);
                end = __ldg(g.row_ptr + w + 1);
                if (end - beg > heavy_deg) { defer_heavy = true; u = 0; }
                else if (end - beg > kWarp) { defer_med = true; u = 0; }
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
        warp_append(defer_med, w, n_medium, medium, s.n, &s.ctr->err, 2u);
        warp_append(defer_heavy, w, &s.ctr->heavy, s.heavy, s.n, &s.ctr->err, 2u);
    }
    flush_stats(s, stats);
}

// Warp per row (medium rows).
__global__ void k_pull_medium(Csr g, Slot s, u64 lanes, int level, const int32_t* medium,
                              const unsigned long long* n_medium) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    const int lane = threadIdx.x & 31;
    const long long cnt = (long long)*n_medium;
    StepStats stats = {0ull, 0ull, 0ull};
    for (long long i = gwarp(); i < cnt; i += nwarps()) {
        int32_t w = medium[i];
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
    flush_stats(s, stats);
}

// Block per row (heavy rows).  No early exit: a block-wide OR per row.
__global__ void k_pull_heavy(Csr g, Slot s, u64 lanes, int level) {
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    __shared__ u64 part[kHeavyBlock / kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long cnt = (long long)s.ctr->heavy;
    StepStats stats = {0ull, 0ull, 0ull};
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        int32_t w = s.heavy[h];
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
    flush_stats(s, stats);
}

void launch_pull(const Csr& g, const Slot& s, int32_t lo, int32_t hi, u64 lanes, int level, int heavy_deg, int nsm,
                 cudaStream_t st) {
    if (hi <= lo) return;
    int32_t* medium = s.medium;
    unsigned long long* n_medium = &s.ctr->medium;
    long long range = (long long)hi - lo;
    long long blocks = (range + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    k_pull_thread<<<(int)blocks, kBlock, 0, st>>>(g, s, lo, hi, lanes, level, heavy_deg, medium, n_medium);
    k_pull_medium<<<nsm * 8, kBlock, 0, st>>>(g, s, lanes, level, medium, n_medium);
    k_pull_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, s, lanes, level);
}

// ---------------------------------------------------------------------------
// Forward gather + finalize for the entries queued at level `level`+1.
// Finalize: the entry's mask is nx[w] (then cleared), vis[w] gains it, and
// the dense frontier word of parity (level+1) is set.  Gather: for each lane
// j of the mask, sigma[w][j] = sum over neighbours v whose level-`level`
// mask has bit j of sigma[v][j], in CSR order, mod 2^64; a carry marks the
// lane in ovf[w].  Thread t owns lanes t and t+32.
struct GatherAcc {
    u64 a0, a1;
    unsigned c0, c1;
};

template <int NT>
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
        while (bal) {
            int src = __ffs(bal) - 1;
            bal &= bal - 1;
            int32_t vv = __shfl_sync(FULL, v, src);
            u64 ff = shfl64(f, src);
            const u64* row = s.sigma + (size_t)vv * kLanes;
            if ((ff >> lane) & 1ull) {
                u64 x = __ldg(row + lane);
                acc.a0 += x;
                acc.c0 |= acc.a0 < x;
            }
            if ((ff >> (lane + 32)) & 1ull) {
                u64 x = __ldg(row + lane + 32);
                acc.a1 += x;
                acc.c1 |= acc.a1 < x;
            }
        }
    }
}

__device__ __forceinline__ void fwd_store(const Slot& s, int32_t w, u64 m, const GatherAcc& acc) {
    const int lane = threadIdx.x & 31;
    u64* row = s.sigma + (size_t)w * kLanes;
    if ((m >> lane) & 1ull) row[lane] = acc.a0;
    if ((m >> (lane + 32)) & 1ull) row[lane + 32] = acc.a1;
    unsigned b0 = __ballot_sync(FULL, acc.c0 && ((m >> lane) & 1ull));
    unsigned b1 = __ballot_sync(FULL, acc.c1 && ((m >> (lane + 32)) & 1ull));
    if (lane == 0 && (b0 | b1)) {
        s.ovf[w] |= ((u64)b1 << 32) | b0;
        atomicOr(&s.ctr->carry, 1u);
    }
}

__global__ void k_fwd_gather(Csr g, Slot s, long long q_lo, long long q_hi, int level, int heavy_deg) {
    const int lane = threadIdx.x & 31;
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    MaskTag* Fn = s.F + (size_t)((level + 1) & 1) * s.n;
    unsigned long long lsum = 0, lesum = 0;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
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
            if (lane == 0) {
                unsigned long long pos = atomicAdd(&s.ctr->heavy, 1ull);
                if ((long long)pos < s.n) s.heavy[pos] = (int32_t)e;
                else atomicOr(&s.ctr->err, 2u);
            }
            continue;
        }
        GatherAcc acc = {0ull, 0ull, 0u, 0u};
        fwd_gather_row<1>(g, s, F, level, m, beg, end, 0, acc);
        fwd_store(s, w, m, acc);
    }
    if (lane == 0 && lsum) {
        atomicAdd(&s.ctr->lane_sum, lsum);
        atomicAdd(&s.ctr->lane_esum, lesum);
    }
}

// Block per heavy row: warps take interleaved 32-entry chunks; partial sums
// are combined in warp order (integer sums: order-free; carries OR-ed, and
// a carry in the combination counts too).
__global__ void k_fwd_gather_heavy(Csr g, Slot s, int level) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = kHeavyBlock / kWarp;
    const MaskTag* F = s.F + (size_t)(level & 1) * s.n;
    __shared__ u64 ps[NW][kLanes];
    __shared__ unsigned pc[NW][kLanes];
    const long long cnt = (long long)s.ctr->heavy;
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        long long e = s.heavy[h];
        int32_t w = s.qv[e];
        u64 m = s.qm[e];
        GatherAcc acc = {0ull, 0ull, 0u, 0u};
        fwd_gather_row<NW>(g, s, F, level, m, g.row_ptr[w], g.row_ptr[w + 1], wid, acc);
        ps[wid][lane] = acc.a0;
        ps[wid][lane + 32] = acc.a1;
        pc[wid][lane] = acc.c0;
        pc[wid][lane + 32] = acc.c1;
        __syncthreads();
        if (wid == 0) {
            GatherAcc tot = {0ull, 0ull, 0u, 0u};
            for (int i = 0; i < NW; ++i) {
                u64 x0 = ps[i][lane], x1 = ps[i][lane + 32];
                tot.a0 += x0;
                tot.c0 |= (tot.a0 < x0) | pc[i][lane];
                tot.a1 += x1;
                tot.c1 |= (tot.a1 < x1) | pc[i][lane + 32];
            }
            fwd_store(s, w, m, tot);
        }
        __syncthreads();
    }
}

void launch_fwd_gather(const Csr& g, const Slot& s, long long q_lo, long long q_hi, int level, int heavy_deg,
                       int nsm, cudaStream_t st) {
    long long cnt = q_hi - q_lo;
    if (cnt <= 0) return;
    k_fwd_gather<<<grid_for(cnt, nsm), kBlock, 0, st>>>(g, s, q_lo, q_hi, level, heavy_deg);
    k_fwd_gather_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, s, level);
}

// ---------------------------------------------------------------------------
// Backward step for the entries of level `level` (>= 1): successors of
// (v, lane j) are the neighbours w whose level-(level+1) mask has bit j.
//   acc_j   = sum over successors of coef[w][j]          (CSR order, FP64)
//   delta_j = sigma_v * acc_j                              (Eq. 2)
//   coef[v][j] = 1/sigma_v + acc_j  = (1 + delta_j) / sigma_v
//   BC[v]  += sum over lanes of delta_j                    (fixed tree order)
// The entry's own mask is published with tag `level` for the next step.
template <int NT>
__device__ __forceinline__ void bwd_gather_row(const Csr& g, const Slot& s, const MaskTag* Fs, int level, u64 m,
                                               int32_t beg, int32_t end, int first, double& a0, double& a1) {
    const int lane = threadIdx.x & 31;
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
        while (bal) {
            int src = __ffs(bal) - 1;
            bal &= bal - 1;
            int32_t ww = __shfl_sync(FULL, w, src);
            u64 ff = shfl64(f, src);
            const double* row = s.coef + (size_t)ww * kLanes;
            if ((ff >> lane) & 1ull) a0 += __ldg(row + lane);
            if ((ff >> (lane + 32)) & 1ull) a1 += __ldg(row + lane + 32);
        }
    }
}

__device__ __forceinline__ void bwd_store(const Slot& s, double* bc, int32_t v, u64 m, double a0, double a1) {
    const int lane = threadIdx.x & 31;
    const u64* srow = s.sigma + (size_t)v * kLanes;
    double* crow = s.coef + (size_t)v * kLanes;
    double d0 = 0.0, d1 = 0.0;
    if ((m >> lane) & 1ull) {
        double sg = (double)srow[lane];
        d0 = sg * a0;
        crow[lane] = 1.0 / sg + a0;
    }
    if ((m >> (lane + 32)) & 1ull) {
        double sg = (double)srow[lane + 32];
        d1 = sg * a1;
        crow[lane + 32] = 1.0 / sg + a1;
    }
    double c = d0 + d1;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) bc[v] += c;
}

__global__ void k_bwd(Csr g, Slot s, double* bc, long long q_lo, long long q_hi, int level, int heavy_deg) {
    const int lane = threadIdx.x & 31;
    const MaskTag* Fs = s.F + (size_t)((level + 1) & 1) * s.n;
    MaskTag* Fo = s.F + (size_t)(level & 1) * s.n;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
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
            if (lane == 0) {
                unsigned long long pos = atomicAdd(&s.ctr->heavy, 1ull);
                if ((long long)pos < s.n) s.heavy[pos] = (int32_t)e;
                else atomicOr(&s.ctr->err, 2u);
            }
            continue;
        }
        double a0 = 0.0, a1 = 0.0;
        bwd_gather_row<1>(g, s, Fs, level, m, beg, end, 0, a0, a1);
        bwd_store(s, bc, v, m, a0, a1);
    }
}

__global__ void k_bwd_heavy(Csr g, Slot s, double* bc, int level) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = kHeavyBlock / kWarp;
    const MaskTag* Fs = s.F + (size_t)((level + 1) & 1) * s.n;
    __shared__ double ps[NW][kLanes];
    const long long cnt = (long long)s.ctr->heavy;
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        long long e = s.heavy[h];
        int32_t v = s.qv[e];
        u64 m = s.qm[e];
        double a0 = 0.0, a1 = 0.0;
        bwd_gather_row<NW>(g, s, Fs, level, m, g.row_ptr[v], g.row_ptr[v + 1], wid, a0, a1);
        ps[wid][lane] = a0;
        ps[wid][lane + 32] = a1;
        __syncthreads();
        if (wid == 0) {
            double t0 = 0.0, t1 = 0.0;
            for (int i = 0; i < NW; ++i) {
                t0 += ps[i][lane];
                t1 += ps[i][lane + 32];
            }
            bwd_store(s, bc, v, m, t0, t1);
        }
        __syncthreads();
    }
}

void launch_bwd(const Csr& g, const Slot& s, double* bc, long long q_lo, long long q_hi, int level, int heavy_deg,
                int nsm, cudaStream_t st) {
    long long cnt = q_hi - q_lo;
    if (cnt <= 0) return;
    k_bwd<<<grid_for(cnt, nsm), kBlock, 0, st>>>(g, s, bc, q_lo, q_hi, level, heavy_deg);
    k_bwd_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, s, bc, level);
}

// ---------------------------------------------------------------------------
// Per-source state for parity checks (only with GBBC_KEEP_STATE).
__global__ void k_keep_dist(Slot s, long long q_lo, long long q_hi, int level, int32_t* dist, long long n_total,
                            long long first_src, int nsrc) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
        int32_t v = s.qv[e];
        u64 m = s.qm[e];
        for (int j = lane; j < nsrc; j += 32)
            if ((m >> j) & 1ull) dist[(first_src + j) * n_total + v] = level;
    }
}

void launch_keep_dist(const Slot& s, long long q_lo, long long q_hi, int level, int32_t* dist, long long n_total,
                      long long first_src, int nsrc, cudaStream_t st) {
    long long cnt = q_hi - q_lo;
    if (cnt <= 0) return;
    k_keep_dist<<<grid_for(cnt, 152, 8), kBlock, 0, st>>>(s, q_lo, q_hi, level, dist, n_total, first_src, nsrc);
}

__global__ void k_keep_sigma(Slot s, int32_t lo, int32_t hi, uint64_t* sigma, uint8_t* ovf, long long n_total,
                             long long first_src, int nsrc) {
    long long total = ((long long)hi - lo) * nsrc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int32_t v = lo + (int32_t)(i / nsrc);
        int j = (int)(i % nsrc);
        if ((s.vis[v] >> j) & 1ull) {
            sigma[(first_src + j) * n_total + v] = s.sigma[(size_t)v * kLanes + j];
            ovf[(first_src + j) * n_total + v] = (uint8_t)((s.ovf[v] >> j) & 1ull);
        }
    }
}

void launch_keep_sigma(const Slot& s, int32_t lo, int32_t hi, uint64_t* sigma, uint8_t* ovf, long long n_total,
                       long long first_src, int nsrc, cudaStream_t st) {
    if (hi <= lo || nsrc <= 0) return;
    k_keep_sigma<<<1216, 256, 0, st>>>(s, lo, hi, sigma, ovf, n_total, first_src, nsrc);
}

// ---------------------------------------------------------------------------
// Undo a discovery step (used to time both directions at one level): the
// vertices queued in [q_lo, q_hi) get nx cleared; the host rewinds qtail.
__global__ void k_undo(Slot s, long long q_lo, long long q_hi) {
    for (long long e = q_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < q_hi;
         e += (long long)gridDim.x * blockDim.x)
        s.nx[s.qv[e]] = 0ull;
}

void launch_undo(const Slot& s, long long q_lo, long long q_hi, cudaStream_t st) {
    if (q_hi <= q_lo) return;
    k_undo<<<1216, 256, 0, st>>>(s, q_lo, q_hi);
}

// ---------------------------------------------------------------------------
// CSR validation.  flags bits: 1 row_ptr decreasing, 2 col out of range,
// 4 self-loop, 8 row not strictly increasing (unsorted or duplicate),
// 16 asymmetric (u in row v but v not in row u).
__global__ void k_validate(Csr g, int32_t* flags) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (long long)gridDim.x * blockDim.x) {
        int32_t beg = g.row_ptr[v], end = g.row_ptr[v + 1];
        int f = 0;
        if (end < beg || beg < 0 || end > g.nnz) { atomicOr(flags, 1); continue; }
        int32_t prev = -1;
        for (int32_t p = beg; p < end; ++p) {
            int32_t u = g.col[p];
            if (u < 0 || u >= g.n) { f |= 2; continue; }
            if (u == v) f |= 4;
            if (u <= prev) f |= 8;
            prev = u;
            int32_t lo = g.row_ptr[u], hi = g.row_ptr[u + 1];
            bool found = false;
            if (lo >= 0 && hi <= g.nnz && lo <= hi) {
                // rows are checked sorted separately; binary search assumes it
                while (lo < hi) {
                    int32_t mid = lo + (hi - lo) / 2;
                    int32_t x = g.col[mid];
                    if (x == (int32_t)v) { found = true; break; }
                    if (x < (int32_t)v) lo = mid + 1; else hi = mid;
                }
            }
            if (!found) f |= 16;
        }
        if (f) atomicOr(flags, f);
    }
}

void launch_validate(const Csr& g, int32_t* flags, cudaStream_t st) {
    if (g.n <= 0) return;
    k_validate<<<1216, 256, 0, st>>>(g, flags);
}

__global__ void k_fill_i32(int32_t* p, long long count, int32_t value) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = value;
}

void launch_fill_i32(int32_t* p, long long count, int32_t value, cudaStream_t st) {
    if (count <= 0) return;
    k_fill_i32<<<1216, 256, 0, st>>>(p, count, value);
}

__global__ void k_offset_copy(const int32_t* src, int32_t* dst, long long count, int32_t add) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}

void launch_offset_copy(const int32_t* src, int32_t* dst, long long count, int32_t add, cudaStream_t st) {
    if (count <= 0) return;
    k_offset_copy<<<1216, 256, 0, st>>>(src, dst, count, add);
}

}  // namespace gbbc
