// Weighted betweenness centrality: Brandes with shortest paths measured by
// positive integer edge weights (the SSSP case of the paper's forward phase,
// Sec. IV-C, which names BFS and SSSP side by side).  A batch holds L sources
// (lanes) and one CTA runs one batch; the host picks L so that the batches
// cover every SM.  Work items are (vertex, lane) pairs: with weights, the
// lanes of a vertex rarely share a distance, so rows of all lanes would be
// mostly idle.
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
//             weight(v, w) == D, all settled earlier (mod 2^64, a carry fails
//             the call: there is no wide format here);
//   relax   - from each settled pair, dist[u][lane] = min(dist[u][lane],
//             D + weight) by atomicMin; a success lists (u, lane) in bucket
//             (D + weight) mod (W + 1).
// A pair succeeds at most once per value, so it is listed once per value and
// settles exactly once.
// Backward (Eq. 2).  Walking the queue's distance steps in reverse, (v, lane)
// at distance D sums psi[u][lane] = (1 + delta_u) / sigma_u over neighbours u
// with dist[u][lane] == D + weight(v, u), in the same 128-bit fixed point as
// the unweighted path, so BC is exact and independent of the order.  psi
// overwrites sigma in place: once (v, lane) has its delta only its
// predecessors read it, and they read psi.
// Rows longer than kWHeavy are scanned by a whole warp (lanes stride the
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

__device__ __forceinline__ u128 warp_sum128(u128 a) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        u128 x;
        x.lo = __shfl_xor_sync(FULLW, a.lo, o);
        x.hi = __shfl_xor_sync(FULLW, a.hi, o);
        a = add128(a, x);
    }
    return a;
}

// psi (a double, read as integers) times 2^(Ev + 64), truncated below 2^0
__device__ __forceinline__ u128 w_psi_term(u64 bits, int Ev) {
    const int e = (int)((bits >> 52) & 0x7FFull) - 1023;
    const u64 M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return shl_term(M, e + Ev + 12);
}

// delta of one pair in units of 2^-64 from sigma = N 2^(E-63) and the
// successor sum A; psi = (1 + delta) / sigma replaces sigma at *slot
__device__ __forceinline__ u128 w_lane(u64* slot, u64 N, int E, u128 A) {
    const u128 d = mul_shift63(N, A);
    const u128 psi = add128(recip127(N), A);
    u64 M;
    int e;
    round128(psi, -64 - E, M, e);
    *slot = double_bits(M, e);
    return d;
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

struct WView {
    int32_t* dist;
    u64* sp;
    uint32_t* blist;
    int* cnt;
    unsigned* err;
    long long bcap;
    int L, B;
};

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

}  // namespace

__global__ void __launch_bounds__(kWThreads) k_weighted_batches(Csr g, const int32_t* wt, WSlots S,
                                                                const WBatch* batches, int nb, const int32_t* srcs,
                                                                unsigned* next, u64* bc, int W, int32_t* k_dist,
                                                                u64* k_sigma, long long n_total,
                                                                unsigned long long* stats) {
    __shared__ int s_cnt[kMaxBuckets];
    __shared__ int s_b, s_done, s_steps;
    __shared__ long long s_D;
    __shared__ unsigned s_err;
    __shared__ unsigned long long s_tail;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int B = W + 1, L = S.L;
    const long long ns = S.nslot;
    const long long slot = blockIdx.x;
    WView v;
    v.dist = S.dist + slot * ns * L;
    v.sp = S.sp + slot * ns * L;
    v.blist = S.blist + slot * (long long)S.B * S.bcap;
    v.cnt = s_cnt;
    v.err = &s_err;
    v.bcap = S.bcap;
    v.L = L;
    v.B = B;
    int32_t* dist = v.dist;
    u64* sp = v.sp;
    uint32_t* qv = S.qv + slot * S.qcap;
    int32_t* levD = S.levD + slot * S.levcap;
    long long* levOff = S.levOff + slot * (S.levcap + 1);
    for (;;) {
        if (tid == 0) s_b = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int b = s_b;
        if (b >= nb) break;
        const WBatch bb = batches[b];
        const int32_t lo = bb.lo;
        const int32_t* rp = g.row_ptr + lo;
        const long long nr = (long long)bb.hi - bb.lo;
        for (long long i = tid; i < nr * L; i += blockDim.x) {
            dist[i] = INT_MAX;
            sp[i] = 0ull;
        }
        if (tid < B) s_cnt[tid] = 0;
        if (tid == 0) {
            s_tail = 0ull;
            s_steps = 0;
            s_err = 0u;
        }
        __syncthreads();
        if (tid < bb.nsrc) {
            const long long pr = (long long)(srcs[bb.src_off + tid] - lo) * L + tid;
            dist[pr] = 0;
            sp[pr] = 1ull;
            const int pos = atomicAdd(&s_cnt[0], 1);
            v.blist[pos] = (uint32_t)pr;  // bucket 0 holds at most L <= bcap pairs here
        }
        __syncthreads();
        // ---- forward: settle distances D = 0, 1, ... in bucket order ----
        long long D = 0;
        for (;;) {
            if (tid == 0) {
                int found = -1;
                for (int i = 0; i < B; ++i)
                    if (s_cnt[(int)((D + i) % B)] > 0) {
                        found = i;
                        break;
                    }
                s_done = found < 0;
                s_D = D + (found < 0 ? 0 : found);
            }
            __syncthreads();
            if (s_done) break;
            D = s_D;
            const int bi = (int)(D % B);
            const int cnt = min(s_cnt[bi], (int)S.bcap);
            const unsigned long long q0 = s_tail;
            // settle; sigma of pairs with short rows
            for (int i = tid; i < cnt; i += blockDim.x) {
                const uint32_t pr = v.blist[(long long)bi * S.bcap + i];
                if (ld_dist(dist + pr) != D) continue;
                const unsigned long long pos = atomicAdd(&s_tail, 1ull);
                if ((long long)pos < S.qcap) qv[pos] = pr;
                else atomicOr(&s_err, 4u);
                if (D == 0) continue;  // sources: sigma = 1 already
                const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
                if (end - beg > kWHeavy) continue;
                u128 a = {0ull, 0ull};
                for (int32_t p = beg; p < end; ++p) {
                    const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                    if (ld_dist(dist + q) == D - __ldg(wt + p)) a = u128_add64(a, sp[q]);
                }
                sp[pr] = a.lo;
                if (a.hi) atomicOr(&s_err, 1u);
            }
            __syncthreads();
            const unsigned long long q1 = min((unsigned long long)S.qcap, s_tail);
            // sigma of pairs with long rows: a warp each
            if (D > 0)
                for (long long e = (long long)q0 + wid; e < (long long)q1; e += nw) {
                    const uint32_t pr = qv[e];
                    const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
                    const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
                    if (end - beg <= kWHeavy) continue;
                    u128 a = {0ull, 0ull};
                    for (int32_t p = beg + lane; p < end; p += 32) {
                        const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                        if (ld_dist(dist + q) == D - __ldg(wt + p)) a = u128_add64(a, sp[q]);
                    }
                    a = warp_sum128(a);
                    if (lane == 0) {
                        sp[pr] = a.lo;
                        if (a.hi) atomicOr(&s_err, 1u);
                    }
                }
            if (tid == 0) {
                s_cnt[bi] = 0;
                if (s_steps < S.levcap) {
                    levD[s_steps] = (int32_t)D;
                    levOff[s_steps] = (long long)q0;
                    ++s_steps;
                } else {
                    s_err |= 2u;
                }
            }
            __syncthreads();
            if (s_err) break;
            // relax: short rows by a thread, long rows by a warp
            for (long long e = (long long)q0 + tid; e < (long long)q1; e += blockDim.x) {
                const uint32_t pr = qv[e];
                const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
                if (end - beg > kWHeavy) continue;
                for (int32_t p = beg; p < end; ++p) relax_edge(v, D, __ldg(g.col + p) - lo, j, __ldg(wt + p));
            }
            for (long long e = (long long)q0 + wid; e < (long long)q1; e += nw) {
                const uint32_t pr = qv[e];
                const int32_t w = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + w), end = __ldg(rp + w + 1);
                if (end - beg <= kWHeavy) continue;
                for (int32_t p = beg + lane; p < end; p += 32) relax_edge(v, D, __ldg(g.col + p) - lo, j, __ldg(wt + p));
            }
            __syncthreads();
            D += 1;
        }
        if (tid == 0) levOff[s_steps] = (long long)min((unsigned long long)S.qcap, s_tail);
        __syncthreads();
        const int nsteps = s_steps;
        const unsigned err = s_err;
        if (tid == 0) {
            atomicAdd(stats + 1, (unsigned long long)nsteps);
            if (err) atomicOr((unsigned*)(stats + 3), err);
        }
        if (err) {  // reported by the host; BC is not trusted
            __syncthreads();
            continue;
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
            }
            __syncthreads();
        }
        // ---- backward: distances in decreasing order, step 0 (sources) excluded ----
        for (int st = nsteps - 1; st >= 1; --st) {
            const long long Dv = levD[st];
            const long long e0 = levOff[st], e1 = levOff[st + 1];
            for (long long e = e0 + tid; e < e1; e += blockDim.x) {
                const uint32_t pr = qv[e];
                const int32_t x = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + x), end = __ldg(rp + x + 1);
                if (end - beg > kWHeavy) continue;
                u64 N;
                int E;
                norm(sp[pr], N, E);
                u128 A = {0ull, 0ull};
                for (int32_t p = beg; p < end; ++p) {
                    const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                    if (ld_dist(dist + q) == Dv + __ldg(wt + p)) A = add128(A, w_psi_term(sp[q], E));
                }
                w_atomic_add128(bc + 2 * ((long long)lo + x), w_lane(sp + pr, N, E, A));
            }
            for (long long e = e0 + wid; e < e1; e += nw) {
                const uint32_t pr = qv[e];
                const int32_t x = (int32_t)(pr / L), j = (int32_t)(pr % L);
                const int32_t beg = __ldg(rp + x), end = __ldg(rp + x + 1);
                if (end - beg <= kWHeavy) continue;
                u64 N;
                int E;
                norm(sp[pr], N, E);
                u128 A = {0ull, 0ull};
                for (int32_t p = beg + lane; p < end; p += 32) {
                    const long long q = (long long)(__ldg(g.col + p) - lo) * L + j;
                    if (ld_dist(dist + q) == Dv + __ldg(wt + p)) A = add128(A, w_psi_term(sp[q], E));
                }
                A = warp_sum128(A);
                if (lane == 0) w_atomic_add128(bc + 2 * ((long long)lo + x), w_lane(sp + pr, N, E, A));
            }
            __syncthreads();
        }
        if (tid == 0) atomicAdd(stats, 1ull);
        __syncthreads();
    }
}

cudaError_t launch_weighted_batches(const Csr& g, const int32_t* wt, const WSlots& S, const WBatch* batches, int nb,
                                    const int32_t* srcs, unsigned* next, u64* bc, int W, int32_t* k_dist,
                                    u64* k_sigma, long long n_total, unsigned long long* stats, cudaStream_t st) {
    if (W < 1 || W + 1 > kMaxBuckets || S.B != W + 1 || S.L < 1 || S.L > kLanes) return cudaErrorInvalidValue;
    k_weighted_batches<<<S.count, kWThreads, 0, st>>>(g, wt, S, batches, nb, srcs, next, bc, W, k_dist, k_sigma,
                                                       n_total, stats);
    return cudaGetLastError();
}

}  // namespace gbbc
