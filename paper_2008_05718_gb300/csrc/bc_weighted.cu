// Pair-granular betweenness centrality: Brandes with shortest paths measured
// by positive integer edge weights (the SSSP case of the paper's forward
// phase, Sec. IV-C, which names BFS and SSSP side by side), and the same
// kernel with all weights 1 for unweighted graphs whose sources rarely share
// a level (high-diameter graphs).  A batch holds L sources (lanes) and one
// CTA runs one batch; the host picks L so that every resident CTA gets one.
// Work items are (vertex, lane) pairs: when the lanes of a vertex rarely
// share a distance, rows of all lanes would be mostly idle.
//
// Forward (Dial's bucketed Dijkstra over all lanes at once).  dist[v][lane] is
// the tentative distance (int32, INT_MAX unreached).  Distances settle in
// increasing order D = 0, 1, 2, ...: every pending tentative value lies in
// (D, D + W] for weights in [1, W], so W + 1 circular buckets, one per
// residue, list the pairs improved to a value of that residue.  For the
// current D:
//   settle  - a listed pair with dist == D settles (others are stale: lowered
//             since) and joins the queue; sigma[w][lane] = sum of
//             sigma[v][lane] over neighbours v with dist[v][lane] +
//             weight(v, w) == D, all settled earlier, mod 2^64 with carry;
//   relax   - from each settled pair, dist[u][lane] = min(dist[u][lane],
//             D + weight) by atomicMin; a success lists (u, lane) in bucket
//             (D + weight) mod (W + 1).
// A pair succeeds at most once per value, so it is listed once per value and
// settles exactly once.
// Wide format: a batch whose counts pass 2^64 is rerun with, per pair, a flag
// and sigma = N 2^X (64-bit normalised mantissa N), summed aligned to the
// largest exponent in 128 bits, as in the unweighted path.
// Backward (Eq. 2).  Walking the queue's distance steps in reverse, (v, lane)
// at distance D sums psi[u][lane] = (1 + delta_u) / sigma_u over neighbours u
// with dist[u][lane] == D + weight(v, u), in the same 128-bit fixed point as
// the unweighted path, so BC is exact and independent of the order.  psi
// overwrites sigma in place (in the wide format its exponent overwrites X):
// once (v, lane) has its delta only its predecessors read it, and they read
// psi.  Rows longer than kWHeavy are scanned by a whole warp (lanes stride the
// neighbours), shorter ones by one thread.
#include <climits>
#include <cstdint>

#include "bc_fixed.cuh"
#include "bc_internal.cuh"

namespace gbbc {
namespace {

constexpr unsigned FULLW = 0xffffffffu;

__device__ __forceinline__ int32_t ld_dist(const int32_t* p) { return __ldcg(p); }

__device__ __forceinline__ u128 u128_add64(u128 a, u64 x) {
    u128 r;
    r.lo = a.lo + x;
    r.hi = a.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ u128 shfl128(u128 a, int o) {
    u128 x;
    x.lo = __shfl_xor_sync(FULLW, a.lo, o);
    x.hi = __shfl_xor_sync(FULLW, a.hi, o);
    return x;
}

__device__ __forceinline__ u128 warp_sum128(u128 a) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) a = add128(a, shfl128(a, o));
    return a;
}

__device__ __forceinline__ u128 shr128w(u128 a, int r) {
    u128 t;
    if (r <= 0) return a;
    if (r >= 128) {
        t.lo = t.hi = 0ull;
        return t;
    }
    if (r >= 64) {
        t.lo = a.hi >> (r - 64);
        t.hi = 0ull;
        return t;
    }
    t.lo = (a.lo >> r) | (a.hi << (64 - r));
    t.hi = a.hi >> r;
    return t;
}

// wide sum: a in units of 2^x (x = INT_MIN while empty)
struct WSum {
    u128 a;
    int x;
    bool big;  // a term was itself >= 2^64
};

__device__ __forceinline__ void wsum_init(WSum& w) {
    w.a.lo = w.a.hi = 0ull;
    w.x = INT_MIN;
    w.big = false;
}

__device__ __forceinline__ void wsum_add(WSum& w, u128 v, int x) {
    if (v.lo == 0ull && v.hi == 0ull) return;
    if (w.x == INT_MIN) {
        w.a = v;
        w.x = x;
        return;
    }
    if (x > w.x) {
        w.a = shr128w(w.a, x - w.x);
        w.x = x;
    } else {
        v = shr128w(v, w.x - x);
    }
    w.a = add128(w.a, v);
}

__device__ __forceinline__ WSum warp_wsum(WSum w) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        WSum t;
        t.a = shfl128(w.a, o);
        t.x = __shfl_xor_sync(FULLW, w.x, o);
        t.big = __shfl_xor_sync(FULLW, w.big ? 1 : 0, o) != 0;
        wsum_add(w, t.a, t.x);
        w.big = w.big || t.big;
    }
    return w;
}

// psi (double bits, plus an exponent offset in the wide format) times
// 2^(Ev + 64), truncated below 2^0
__device__ __forceinline__ u128 w_psi_term(u64 bits, int eoff, int Ev) {
    const int e = (int)((bits >> 52) & 0x7FFull) - 1023 + eoff;
    const u64 M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return shl_term(M, e + Ev + 12);
}

__device__ __forceinline__ void w_atomic_add128(u64* a, u128 t) {
    if ((t.lo | t.hi) == 0ull) return;
    const u64 old = atomicAdd(a, t.lo);
    const u64 carry = (old + t.lo) < old ? 1ull : 0ull;
    if (t.hi + carry) atomicAdd(a + 1, t.hi + carry);
}

__device__ __forceinline__ void norm(u64 x, u64& N, int& E) {
    const int lz = __clzll((long long)x);
    N = x << lz;
    E = 63 - lz;
}

// One batch's arrays and the CTA's shared scalars.
struct WView {
    int32_t* dist;
    u64* sp;
    u64* sN;
    int32_t* sX;
    uint8_t* wf;
    uint32_t* blist;
    uint32_t* qv;
    int32_t* levD;
    long long* levOff;
    const int32_t* wt;
    int* cnt;
    unsigned* err;
    unsigned long long* tail;
    int* steps;
    long long bcap, qcap, levcap;
    int L, B;
};

__device__ __forceinline__ int wgt(const WView& w, int32_t p) { return w.wt ? __ldg(w.wt + p) : 1; }

__device__ __forceinline__ void relax_edge(const WView& w, long long D, int32_t u, int j, int c) {
    const int32_t t = (int32_t)(D + c);
    int32_t* du = w.dist + (long long)u * w.L + j;
    if (t < ld_dist(du) && t < atomicMin(du, t)) {
        const int b = (int)((D + c) % w.B);
        const int pos = atomicAdd(w.cnt + b, 1);
        if (pos < w.bcap) w.blist[(long long)b * w.bcap + pos] = (uint32_t)((long long)u * w.L + j);
        else atomicOr(w.err, 8u);
    }
}

// sigma of a predecessor pair as a wide term
template <bool WIDE>
__device__ __forceinline__ void pred_wide(const WView& w, long long q, u64 x, WSum& s) {
    if (!WIDE) return;
    u128 t;
    t.hi = 0ull;
    if (w.wf[q]) {
        t.lo = w.sN[q];
        wsum_add(s, t, w.sX[q]);
        s.big = true;
    } else {
        t.lo = x;
        wsum_add(s, t, 0);
    }
}

// store a pair's sigma: exact low 64 bits, and the wide value when it is >= 2^64
template <bool WIDE>
__device__ __forceinline__ void store_sigma(const WView& w, long long pr, u128 a, const WSum& s) {
    w.sp[pr] = a.lo;
    if (WIDE) {
        const bool big = a.hi != 0ull || s.big;
        w.wf[pr] = big ? 1 : 0;
        if (big) {
            const int lz = (s.a.hi ? __clzll((long long)s.a.hi) : 64 + __clzll((long long)s.a.lo));
            const int bits = 128 - lz;
            w.sN[pr] = bits > 64 ? shr128w(s.a, bits - 64).lo : s.a.lo << (64 - bits);
            w.sX[pr] = s.x + bits - 64;
        }
    } else if (a.hi) {
        atomicOr(w.err, 1u);
    }
}

// delta of one pair in units of 2^-64 from sigma = N 2^(E-63) and the
// successor sum A; psi = (1 + delta) / sigma replaces sigma
template <bool WIDE>
__device__ __forceinline__ u128 w_lane(const WView& w, long long pr, u64 N, int E, u128 A) {
    const u128 d = mul_shift63(N, A);
    const u128 psi = add128(recip127(N), A);
    u64 M;
    int e;
    round128(psi, -64 - E, M, e);
    if (WIDE) {
        w.sp[pr] = unit_bits(M);
        w.sX[pr] = e;
    } else {
        w.sp[pr] = double_bits(M, e);
    }
    return d;
}

template <bool WIDE>
__device__ __forceinline__ void pair_norm(const WView& w, long long pr, u64& N, int& E) {
    if (WIDE && w.wf[pr]) {
        N = w.sN[pr];
        E = w.sX[pr] + 63;
    } else {
        norm(w.sp[pr], N, E);
    }
}

// One batch.  Returns false when a count passed 2^64 in the narrow format
// (the caller reruns it wide; BC untouched).
template <bool WIDE>
__device__ bool w_batch(const Csr& g, const WView& v, const WBatch& bb, const int32_t* srcs, u64* bc,
                        int32_t* k_dist, u64* k_sigma, uint8_t* k_ovf, long long n_total,
                        unsigned long long* stats) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int L = v.L, B = v.B;
    const int32_t lo = bb.lo;
    const int32_t* rp = g.row_ptr + lo;
    const long long nr = (long long)bb.hi - bb.lo;
    int32_t* dist = v.dist;
    u64* sp = v.sp;
    for (long long i = tid; i < nr * L; i += blockDim.x) {
        dist[i] = INT_MAX;
        sp[i] = 0ull;
        if (WIDE) v.wf[i] = 0;
    }
    if (tid < B) v.cnt[tid] = 0;
    if (tid == 0) {
        *v.tail = 0ull;
        *v.steps = 0;
        *v.err = 0u;
    }
    __syncthreads();
    if (tid < bb.nsrc) {
        const long long pr = (long long)(srcs[bb.src_off + tid] - lo) * L + tid;
        dist[pr] = 0;
        sp[pr] = 1ull;
        const int pos = atomicAdd(v.cnt, 1);
        v.blist[pos] = (uint32_t)pr;  // bucket 0 holds at most L <= bcap pairs here
    }
    __syncthreads();
    // ---- forward: settle distances D = 0, 1, ... in bucket order ----
    // Two block barriers per distance: after the settle, and after the relax.
    // Every thread finds the next non-empty bucket itself (the counts do not
    // change between the relax barrier and the next settle), and the queue
    // does not grow during the relax, so the step's first entry is the
    // previous step's end.
    long long D = 0;
    unsigned long long qprev = 0ull;
    for (;;) {
        int found = -1;
        for (int i = 0; i < B; ++i)
            if (v.cnt[(int)((D + i) % B)] > 0) {
                found = i;
                break;
            }
        if (found < 0 || *v.err) break;
        D += found;
        const int bi = (int)(D % B);
        const int cnt = min(v.cnt[bi], (int)v.bcap);
        const unsigned long long q0 = qprev;
        // settle; sigma of pairs with short rows
        for (int i = tid; i < cnt; i += blockDim.x) {
            const uint32_t pr = v.blist[(long long)bi * v.bcap + i];
            if (ld_dist(dist + pr) != D) continue;
            const unsigned long long pos = atomicAdd(v.tail, 1ull);
            if ((long long)pos < v.qcap) v.qv[pos] = pr;
            else atomicOr(v.err, 4u);
            if (D == 0) continue;  // sources: sigma = 1 already
            const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
            const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
            if (end - beg > kWHeavy) continue;
            u128 a = {0ull, 0ull};
            WSum s;
            wsum_init(s);
            for (int32_t p = beg; p < end; ++p) {
                const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                if (ld_dist(dist + q) == D - wgt(v, p)) {
                    const u64 x = sp[q];
                    a = u128_add64(a, x);
                    pred_wide<WIDE>(v, q, x, s);
                }
            }
            store_sigma<WIDE>(v, pr, a, s);
        }
        __syncthreads();
        const unsigned long long q1 = min((unsigned long long)v.qcap, *v.tail);
        // sigma of pairs with long rows: a warp each
        if (D > 0)
            for (long long e = (long long)q0 + wid; e < (long long)q1; e += nw) {
                const uint32_t pr = v.qv[e];
                const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
                if (end - beg <= kWHeavy) continue;
                u128 a = {0ull, 0ull};
                WSum s;
                wsum_init(s);
                for (int32_t p = beg + lane; p < end; p += 32) {
                    const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                    if (ld_dist(dist + q) == D - wgt(v, p)) {
                        const u64 x = sp[q];
                        a = u128_add64(a, x);
                        pred_wide<WIDE>(v, q, x, s);
                    }
                }
                a = warp_sum128(a);
                if (WIDE) s = warp_wsum(s);
                if (lane == 0) store_sigma<WIDE>(v, pr, a, s);
            }
        if (tid == 0) {  // bucket bi is consumed; the relax never adds to it
            v.cnt[bi] = 0;
            if (*v.steps < v.levcap) {
                v.levD[*v.steps] = (int32_t)D;
                v.levOff[*v.steps] = (long long)q0;
                ++*v.steps;
            } else {
                atomicOr(v.err, 2u);
            }
        }
        // relax (alongside the long rows' sigma above, which reads only
        // settled pairs, while the relax lowers only distances above D):
        // short rows by a thread, long rows by a warp
        for (long long e = (long long)q0 + tid; e < (long long)q1; e += blockDim.x) {
            const uint32_t pr = v.qv[e];
            const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
            const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
            if (end - beg > kWHeavy) continue;
            for (int32_t p = beg; p < end; ++p) relax_edge(v, D, __ldg(g.col + p) - lo, j, wgt(v, p));
        }
        for (long long e = (long long)q0 + wid; e < (long long)q1; e += nw) {
            const uint32_t pr = v.qv[e];
            const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
            const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
            if (end - beg <= kWHeavy) continue;
            for (int32_t p = beg + lane; p < end; p += 32) relax_edge(v, D, __ldg(g.col + p) - lo, j, wgt(v, p));
        }
        __syncthreads();
        qprev = q1;
        D += 1;
    }
    if (tid == 0) v.levOff[*v.steps] = (long long)min((unsigned long long)v.qcap, *v.tail);
    __syncthreads();
    const int nsteps = *v.steps;
    const unsigned err = *v.err;
    __syncthreads();
    if (tid == 0) atomicAdd(stats + 1, (unsigned long long)nsteps);
    if (!WIDE && (err & 1u)) return false;
    if (err) {  // reported by the host; BC is not trusted
        if (tid == 0) atomicOr((unsigned*)(stats + 3), err);
        return true;
    }
    // ---- kept per-source state (parity checks) ----
    if (k_dist) {
        for (long long i = tid; i < nr * bb.nsrc; i += blockDim.x) {
            const long long vv = i / bb.nsrc;
            const int j = (int)(i % bb.nsrc);
            const int32_t d = ld_dist(dist + vv * L + j);
            const long long at = (bb.first + j) * n_total + lo + vv;
            k_dist[at] = d == INT_MAX ? -1 : d;
            k_sigma[at] = d == INT_MAX ? 0ull : sp[vv * L + j];
            k_ovf[at] = WIDE && d != INT_MAX ? v.wf[vv * L + j] : 0;
        }
        __syncthreads();
    }
    // ---- backward: distances in decreasing order, step 0 (sources) excluded ----
    for (int st = nsteps - 1; st >= 1; --st) {
        const long long Dv = v.levD[st];
        const long long e0 = v.levOff[st], e1 = v.levOff[st + 1];
        for (long long e = e0 + tid; e < e1; e += blockDim.x) {
            const uint32_t pr = v.qv[e];
            const int32_t x = (int32_t)(pr / L), j = (int32_t)(pr % L);
            const int32_t beg = __ldg(rp + x), end = __ldg(rp + x + 1);
            if (end - beg > kWHeavy) continue;
            u64 N;
            int E;
            pair_norm<WIDE>(v, pr, N, E);
            u128 A = {0ull, 0ull};
            for (int32_t p = beg; p < end; ++p) {
                const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                if (ld_dist(dist + q) == Dv + wgt(v, p)) A = add128(A, w_psi_term(sp[q], WIDE ? v.sX[q] : 0, E));
            }
            w_atomic_add128(bc + 2 * ((long long)lo + x), w_lane<WIDE>(v, pr, N, E, A));
        }
        for (long long e = e0 + wid; e < e1; e += nw) {
            const uint32_t pr = v.qv[e];
            const int32_t x = (int32_t)(pr / L), j = (int32_t)(pr % L);
            const int32_t beg = __ldg(rp + x), end = __ldg(rp + x + 1);
            if (end - beg <= kWHeavy) continue;
            u64 N;
            int E;
            pair_norm<WIDE>(v, pr, N, E);
            u128 A = {0ull, 0ull};
            for (int32_t p = beg + lane; p < end; p += 32) {
                const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                if (ld_dist(dist + q) == Dv + wgt(v, p)) A = add128(A, w_psi_term(sp[q], WIDE ? v.sX[q] : 0, E));
            }
            A = warp_sum128(A);
            if (lane == 0) w_atomic_add128(bc + 2 * ((long long)lo + x), w_lane<WIDE>(v, pr, N, E, A));
        }
        __syncthreads();
    }
    return true;
}

}  // namespace

__global__ void __launch_bounds__(kWThreads) k_weighted_batches(Csr g, const int32_t* wt, WSlots S,
                                                                const WBatch* batches, int nb, const int32_t* srcs,
                                                                unsigned* next, u64* bc, int W, int32_t* k_dist,
                                                                u64* k_sigma, uint8_t* k_ovf, long long n_total,
                                                                int* gwide, unsigned long long* stats) {
    __shared__ int s_cnt[kMaxBuckets];
    __shared__ int s_b, s_steps;
    __shared__ unsigned s_err;
    __shared__ unsigned long long s_tail;
    const int tid = threadIdx.x;
    const long long ns = S.nslot, slot = blockIdx.x;
    const int L = S.L;
    WView v;
    v.dist = S.dist + slot * ns * L;
    v.sp = S.sp + slot * ns * L;
    v.sN = S.sN + slot * ns * L;
    v.sX = S.sX + slot * ns * L;
    v.wf = S.wf + slot * ns * L;
    v.blist = S.blist + slot * (long long)S.B * S.bcap;
    v.qv = S.qv + slot * S.qcap;
    v.levD = S.levD + slot * S.levcap;
    v.levOff = S.levOff + slot * (S.levcap + 1);
    v.wt = wt;
    v.cnt = s_cnt;
    v.err = &s_err;
    v.tail = &s_tail;
    v.steps = &s_steps;
    v.bcap = S.bcap;
    v.qcap = S.qcap;
    v.levcap = S.levcap;
    v.L = L;
    v.B = W + 1;
    for (;;) {
        if (tid == 0) s_b = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int b = s_b;
        if (b >= nb) break;
        const WBatch bb = batches[b];
        const bool wide = bb.wide || __ldcg(gwide + bb.gi) != 0;
        if (wide || !w_batch<false>(g, v, bb, srcs, bc, k_dist, k_sigma, k_ovf, n_total, stats)) {
            if (!wide && tid == 0) {
                atomicAdd(stats + 2, 1ull);
                atomicExch(gwide + bb.gi, 1);
            }
            __syncthreads();
            w_batch<true>(g, v, bb, srcs, bc, k_dist, k_sigma, k_ovf, n_total, stats);
        }
        if (tid == 0) atomicAdd(stats, 1ull);
        __syncthreads();
    }
}

int weighted_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_weighted_batches, kWThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return b < 1 ? 1 : b;
}

cudaError_t launch_weighted_batches(const Csr& g, const int32_t* wt, const WSlots& S, const WBatch* batches, int nb,
                                    const int32_t* srcs, unsigned* next, u64* bc, int W, int32_t* k_dist,
                                    u64* k_sigma, uint8_t* k_ovf, long long n_total, int* gwide,
                                    unsigned long long* stats, cudaStream_t st) {
    if (W < 1 || W + 1 > kMaxBuckets || S.B != W + 1 || S.L < 1 || S.L > kLanes) return cudaErrorInvalidValue;
    k_weighted_batches<<<S.count, kWThreads, 0, st>>>(g, wt, S, batches, nb, srcs, next, bc, W, k_dist, k_sigma,
                                                       k_ovf, n_total, gwide, stats);
    return cudaGetLastError();
}

}  // namespace gbbc
