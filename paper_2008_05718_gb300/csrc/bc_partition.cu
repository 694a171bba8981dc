// Kernels of the partitioned method (Sec. IV and Sec. V-A of the paper) on
// one GPU: the graph's vertices are split into P parts; a border edge joins
// two parts and its end points are border nodes.  The host code (bc_api.cu)
// runs, per batch of up to 64 sources (lanes):
//   Step 1     BFS from each source inside its own part (the intra-part
//              graph: border edges removed), with sigma
//   Steps 2-5  iterative refinement of the border nodes' distances over the
//              border edges (Steps 2, 4) and the border matrices BM (Steps
//              3, 5) until no distance changes
//   sigma      of the border nodes, in increasing distance order, from the
//              sigma matrix sigmaM (Sec. V-A)
//   Step 6     relaxation: BFS inside every part seeded by the source and by
//              the border nodes at their refined distances
// and then the backward phase over the whole graph.
//
// Border arrays of a batch are lane-minor: entry [b * 64 + j] is border node
// b (global border index) in lane j.  Distances are int32 with kInf for
// unreached; path counts are kept as WNum: the count mod 2^64 (always exact),
// a flag for counts >= 2^64, and then an approximation N * 2^X with a
// normalised 64-bit mantissa N (the slots' wide sigma format).
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "bc_fixed.cuh"
#include "bc_internal.cuh"
#include "bc_rows.cuh"

namespace gbbc {

namespace {

struct WNum {
    u64 mod;  // value mod 2^64
    u64 N;    // normalised mantissa (big only)
    int X;    // exponent: value ~ N * 2^X (big only)
    int big;  // value >= 2^64
};

__device__ __forceinline__ WNum wn_zero() {
    WNum z;
    z.mod = 0ull;
    z.N = 0ull;
    z.X = 0;
    z.big = 0;
    return z;
}

__device__ __forceinline__ bool wn_nonzero(const WNum& a) { return a.big || a.mod != 0ull; }

// mantissa and exponent of a (exact for small values)
__device__ __forceinline__ void wn_parts(const WNum& a, u64& m, int& x) {
    if (a.big) {
        m = a.N;
        x = a.X;
    } else {
        m = a.mod;
        x = 0;
    }
}

// Normalise a 128-bit magnitude times 2^x to a 64-bit mantissa (truncating).
__device__ __forceinline__ void wn_norm(u128 v, int x, u64& N, int& X) {
    const int lz = clz128(v);
    const int bits = 128 - lz;
    if (bits > 64) {
        u128 t;
        const int r = bits - 64;
        if (r >= 64) {
            t.lo = v.hi >> (r - 64);
        } else {
            t.lo = (v.lo >> r) | (v.hi << (64 - r));
        }
        N = t.lo;
    } else {
        N = v.lo << (64 - bits);
    }
    X = x + bits - 64;
}

__device__ __forceinline__ WNum wn_mul(const WNum& a, const WNum& b) {
    WNum r = wn_zero();
    if (!wn_nonzero(a) || !wn_nonzero(b)) return r;
    r.mod = a.mod * b.mod;
    const u64 hi = __umul64hi(a.mod, b.mod);
    r.big = a.big || b.big || hi != 0ull;
    if (r.big) {
        u64 ma, mb;
        int xa, xb;
        wn_parts(a, ma, xa);
        wn_parts(b, mb, xb);
        u128 p;
        p.lo = ma * mb;
        p.hi = __umul64hi(ma, mb);
        wn_norm(p, xa + xb, r.N, r.X);
    }
    return r;
}

// Accumulator of a sum of WNum terms: exact mod 2^64, the flag, and the
// approximate magnitude summed in a u128 aligned to the largest exponent.
struct WSum {
    u64 mod;
    int big;
    u128 a;
    int x;  // INT_MIN while empty
};

__device__ __forceinline__ void ws_init(WSum& s) {
    s.mod = 0ull;
    s.big = 0;
    s.a.lo = s.a.hi = 0ull;
    s.x = INT_MIN;
}

__device__ __forceinline__ u128 shr128p(u128 a, int r) {
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

__device__ __forceinline__ void ws_add(WSum& s, const WNum& t) {
    if (!wn_nonzero(t)) return;
    const u64 old = s.mod;
    s.mod += t.mod;
    s.big |= t.big | (s.mod < old ? 1 : 0);
    u64 m;
    int x;
    wn_parts(t, m, x);
    u128 v;
    v.lo = m;
    v.hi = 0ull;
    if (s.x == INT_MIN) {
        s.a = v;
        s.x = x;
        return;
    }
    if (x > s.x) {
        s.a = shr128p(s.a, x - s.x);
        s.x = x;
    } else {
        v = shr128p(v, s.x - x);
    }
    s.a = add128(s.a, v);
}

__device__ __forceinline__ WNum ws_value(const WSum& s) {
    WNum r = wn_zero();
    r.mod = s.mod;
    r.big = s.big;
    if (s.big && s.x != INT_MIN) wn_norm(s.a, s.x, r.N, r.X);
    return r;
}

struct WArr {  // lane-minor arrays of WNum fields
    u64* mod;
    u64* N;
    int32_t* X;
    uint8_t* big;
};

__device__ __forceinline__ WNum wa_load(const WArr& a, long long i) {
    WNum r;
    r.mod = a.mod[i];
    r.big = a.big[i];
    r.N = r.big ? a.N[i] : 0ull;
    r.X = r.big ? a.X[i] : 0;
    return r;
}

__device__ __forceinline__ void wa_store(const WArr& a, long long i, const WNum& v) {
    a.mod[i] = v.mod;
    a.big[i] = (uint8_t)v.big;
    if (v.big) {
        a.N[i] = v.N;
        a.X[i] = v.X;
    }
}

// sigma of (v, lane j) from a slot as a WNum
__device__ __forceinline__ WNum slot_sigma(const Slot& s, int32_t v, int j, bool wide) {
    WNum r = wn_zero();
    const size_t at = (size_t)v * kLanes + j;
    r.mod = s.sigma[at];
    r.big = wide && ((s.ovf[v] >> j) & 1ull) ? 1 : 0;
    if (!wide && ((s.ovf[v] >> j) & 1ull)) r.big = 1;  // narrow pass: flagged, no mantissa
    if (r.big && wide) {
        r.N = s.sN[at];
        r.X = s.sX[at];
    }
    return r;
}

}  // namespace

// ---- extraction of a finished BFS at the border nodes ----------------------
// Entries [q_lo, q_hi) of level `level`.  Mode 0 (border matrices): lane j's
// source is border node lane_b[j]; where the entry's vertex v is a border
// node of the same part, write BM = level and sigmaM = sigma into the part's
// matrix block (row: the source's index in the part, column: v's).  Mode 1
// (Step 1 of a batch): write dist and sigma of border node bidx[v] in lane j.
__global__ void k_part_extract(Slot s, long long q_lo, long long q_hi, int level, bool wide, int mode,
                               const int32_t* bidx, const int32_t* bpart, const long long* boff,
                               const long long* moff, const int32_t* lane_b, int32_t* dist_out, WArr sig_out) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
        const int32_t v = s.qv[e];
        const u64 m = s.qm[e];
        const int32_t iv = bidx[v];
        if (iv < 0) continue;
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (!((m >> j) & 1ull)) continue;
            const WNum val = slot_sigma(s, v, j, wide);
            long long at;
            if (mode == 0) {
                const int32_t ib = lane_b[j];
                if (ib < 0) continue;
                const int p = bpart[ib];
                if (bpart[iv] != p) continue;
                const long long B = boff[p + 1] - boff[p];
                at = moff[p] + (ib - boff[p]) * B + (iv - boff[p]);
            } else {
                at = (long long)iv * kLanes + j;
            }
            dist_out[at] = level;
            wa_store(sig_out, at, val);
        }
    }
}

void launch_part_extract(const Slot& s, long long q_lo, long long q_hi, int level, bool wide, int mode,
                         const int32_t* bidx, const int32_t* bpart, const long long* boff, const long long* moff,
                         const int32_t* lane_b, int32_t* dist_out, u64* mod, u64* N, int32_t* X, uint8_t* big,
                         int nsm, cudaStream_t st) {
    if (q_hi <= q_lo) return;
    long long blocks = ((q_hi - q_lo) * kWarp + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    WArr w{mod, N, X, big};
    k_part_extract<<<(int)blocks, kBlock, 0, st>>>(s, q_lo, q_hi, level, wide, mode, bidx, bpart, boff, moff, lane_b,
                                                  dist_out, w);
}

// ---- Steps 2-5: iterative refinement of the border distances -------------
// Steps 2 and 4: over the border edges, D[b] = min(D[b], D[c] + 1) for the
// border neighbours c of b in other parts.  Thread per (border node, lane).
// Updates only lower distances, so the sweep's order does not change the
// fixed point.
__global__ void k_refine_cut(const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border,
                             const int32_t* bidx, long long nbt, int32_t* D, int* changed) {
    const long long total = nbt * kLanes;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / kLanes;
        const int j = (int)(i % kLanes);
        const int32_t v = border[b];
        int32_t best = D[i];
        for (int32_t p = cut_rp[v]; p < cut_rp[v + 1]; ++p) {
            const int32_t c = bidx[cut_col[p]];
            const int32_t dc = D[(long long)c * kLanes + j];
            if (dc < kPartInf && dc + 1 < best) best = dc + 1;
        }
        if (best < D[i]) {
            D[i] = best;
            *changed = 1;
        }
    }
}

// Steps 3 and 5: over the border matrices, D[b] = min over border nodes b'
// of the same part of D[b'] + BM[b'][b].
__global__ void k_refine_bm(const int32_t* bpart, const long long* boff, const long long* moff, const int32_t* BM,
                            long long nbt, int32_t* D, int* changed) {
    const long long total = nbt * kLanes;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / kLanes;
        const int j = (int)(i % kLanes);
        const int p = bpart[b];
        const long long b0 = boff[p], B = boff[p + 1] - b0;
        const int32_t* col = BM + moff[p] + (b - b0);  // BM[b'][b] at col[(b' - b0) * B]
        int32_t best = D[i];
        for (long long q = 0; q < B; ++q) {
            const int32_t len = col[q * B];
            if (len < 0) continue;
            const int32_t dq = D[(b0 + q) * kLanes + j];
            if (dq < kPartInf && dq + len < best) best = dq + len;
        }
        if (best < D[i]) {
            D[i] = best;
            *changed = 1;
        }
    }
}

// ---- sigma of the border nodes (Sec. V-A) ----------------------------------
// A shortest path from s to border node b of part p either stays in p from s
// (Step 1 counted it: S1[b] when d1[b] = D[b]) or enters p for the last time
// over a border edge (c, b') into a border node b' of p, then runs inside p
// from b' to b (sigmaM[b'][b] such runs when D[b'] + BM[b'][b] = D[b]).
// With A[b'] = sum of sigma[c] over the border neighbours c of b' at
// distance D[b'] - 1 (the paths arriving at b' over a border edge):
//   sigma[b] = [d1[b] = D[b]] S1[b] + sum over b' of A[b'] sigmaM[b'][b].
// Every term has D[b'] <= D[b] and every A[b'] uses sigma at D[b'] - 1, so
// the border nodes are done level by level: arrivals, then sigma.
__global__ void k_border_arrivals(int level, const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border,
                                  const int32_t* bidx, long long nbt, const int32_t* D, WArr Sig, WArr A) {
    const long long total = nbt * kLanes;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (D[i] != level) continue;
        const int j = (int)(i % kLanes);
        const int32_t v = border[i / kLanes];
        WSum acc;
        ws_init(acc);
        for (int32_t p = cut_rp[v]; p < cut_rp[v + 1]; ++p) {
            const long long c = (long long)bidx[cut_col[p]] * kLanes + j;
            if (D[c] == level - 1) ws_add(acc, wa_load(Sig, c));
        }
        wa_store(A, i, ws_value(acc));
    }
}

__global__ void k_border_sigma(int level, const int32_t* bpart, const long long* boff, const long long* moff,
                               const int32_t* BM, WArr SM, long long nbt, const int32_t* D, const int32_t* D1,
                               WArr S1, WArr A, WArr Sig) {
    const long long total = nbt * kLanes;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (D[i] != level) continue;
        const long long b = i / kLanes;
        const int j = (int)(i % kLanes);
        const int p = bpart[b];
        const long long b0 = boff[p], B = boff[p + 1] - b0;
        WSum acc;
        ws_init(acc);
        if (D1[i] == level) ws_add(acc, wa_load(S1, i));
        for (long long q = 0; q < B; ++q) {
            const long long at = moff[p] + q * B + (b - b0);  // BM[b'][b]
            const int32_t len = BM[at];
            if (len < 0) continue;
            const long long iq = (b0 + q) * kLanes + j;
            if (D[iq] >= kPartInf || D[iq] + len != level) continue;
            const WNum a = wa_load(A, iq);
            if (!wn_nonzero(a)) continue;
            ws_add(acc, wn_mul(a, wa_load(SM, at)));
        }
        wa_store(Sig, i, ws_value(acc));
    }
}

// ---- Step 6: the seeds of the relaxation --------------------------------
// After the discovery of level `level`: border node b enters the level in
// the lanes where D[b] = level and A[b] is non-zero (paths arriving over a
// border edge); a vertex no lane reached yet is appended to the queue.
// Warp per border node.
__global__ void k_seed_inject(Slot s, int level, const int32_t* border, long long nbt, const int32_t* D, WArr A,
                              const int32_t* row_ptr) {
    const int lane = threadIdx.x & 31;
    unsigned long long esum = 0;
    u64 lanes_or = 0ull;
    for (long long b = gwarp(); b < nbt; b += nwarps()) {
        bool on[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long i = b * kLanes + lane + 32 * h;
            on[h] = D[i] == level && (A.big[i] || A.mod[i] != 0ull);
        }
        const u64 m = ((u64)__ballot_sync(FULL, on[1]) << 32) | __ballot_sync(FULL, on[0]);
        bool newq = false;
        const int32_t v = border[b];
        if (m && lane == 0) {
            const u64 old = atomicOr(&s.nx[v], m);
            newq = old == 0ull;
            lanes_or |= m;
            if (newq) esum += (unsigned long long)(row_ptr[v + 1] - row_ptr[v]);
        }
        warp_append(newq, v, &s.ctr->qtail, s.qv, s.qcap, &s.ctr->err, 1u);
    }
    if (lane == 0 && (esum | lanes_or)) {
        atomicAdd(&s.ctr->edge_sum, esum);
        atomicOr(&s.ctr->lanes, lanes_or);
    }
}

// After the gather of level `level`: the seeds' arrivals are added to the
// sigma the gather found inside the part.  A count reaching 2^64 sets the
// lane's overflow flag (and, in the narrow pass, the batch's carry flag: the
// batch is rerun in the wide format).
__global__ void k_seed_add(Slot s, int level, const int32_t* border, long long nbt, const int32_t* D, WArr A,
                           bool wide) {
    const long long total = nbt * kLanes;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (D[i] != level) continue;
        const WNum a = wa_load(A, i);
        if (!wn_nonzero(a)) continue;
        const int j = (int)(i % kLanes);
        const int32_t v = border[i / kLanes];
        const WNum cur = slot_sigma(s, v, j, wide);
        WSum acc;
        ws_init(acc);
        ws_add(acc, cur);
        ws_add(acc, a);
        const WNum r = ws_value(acc);
        const size_t at = (size_t)v * kLanes + j;
        s.sigma[at] = r.mod;
        if (r.big) {
            if (wide) {
                s.sN[at] = r.N;
                s.sX[at] = r.X;
            }
            atomicOr(&s.ovf[v], 1ull << j);
            atomicOr(&s.ctr->carry, 1u);
        }
    }
}

static int grid_of(long long items, int nsm) {
    long long blocks = (items + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    return (int)(blocks < 1 ? 1 : blocks);
}

void launch_refine_cut(const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border, const int32_t* bidx,
                       long long nbt, int32_t* D, int* changed, int nsm, cudaStream_t st) {
    if (nbt <= 0) return;
    k_refine_cut<<<grid_of(nbt * kLanes, nsm), kBlock, 0, st>>>(cut_rp, cut_col, border, bidx, nbt, D, changed);
}

void launch_refine_bm(const int32_t* bpart, const long long* boff, const long long* moff, const int32_t* BM,
                      long long nbt, int32_t* D, int* changed, int nsm, cudaStream_t st) {
    if (nbt <= 0) return;
    k_refine_bm<<<grid_of(nbt * kLanes, nsm), kBlock, 0, st>>>(bpart, boff, moff, BM, nbt, D, changed);
}

void launch_border_sigma_level(int level, const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border,
                               const int32_t* bidx, const int32_t* bpart, const long long* boff,
                               const long long* moff, const int32_t* BM, const PartWide& SM, long long nbt,
                               const int32_t* D, const int32_t* D1, const PartWide& S1, const PartWide& A,
                               const PartWide& Sig, int nsm, cudaStream_t st) {
    if (nbt <= 0) return;
    WArr a{A.mod, A.N, A.X, A.big}, sg{Sig.mod, Sig.N, Sig.X, Sig.big};
    WArr sm{SM.mod, SM.N, SM.X, SM.big}, s1{S1.mod, S1.N, S1.X, S1.big};
    k_border_arrivals<<<grid_of(nbt * kLanes, nsm), kBlock, 0, st>>>(level, cut_rp, cut_col, border, bidx, nbt, D,
                                                                     sg, a);
    k_border_sigma<<<grid_of(nbt * kLanes, nsm), kBlock, 0, st>>>(level, bpart, boff, moff, BM, sm, nbt, D, D1, s1,
                                                                  a, sg);
}

void launch_seed_inject(const Slot& s, int level, const int32_t* border, long long nbt, const int32_t* D,
                        const PartWide& A, const int32_t* row_ptr, int nsm, cudaStream_t st) {
    if (nbt <= 0) return;
    WArr a{A.mod, A.N, A.X, A.big};
    long long blocks = (nbt * kWarp + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    k_seed_inject<<<(int)blocks, kBlock, 0, st>>>(s, level, border, nbt, D, a, row_ptr);
}

void launch_seed_add(const Slot& s, int level, const int32_t* border, long long nbt, const int32_t* D,
                     const PartWide& A, bool wide, int nsm, cudaStream_t st) {
    if (nbt <= 0) return;
    WArr a{A.mod, A.N, A.X, A.big};
    k_seed_add<<<grid_of(nbt * kLanes, nsm), kBlock, 0, st>>>(s, level, border, nbt, D, a, wide);
}

// ---- the asynchronous backward phase (Sec. V-B) ------------------------------
// After Step 6 every part walks its own levels from the deepest one up, on its
// own group of blocks, and waits for another part only at a level where one of
// its border nodes has a successor in that part one level deeper
// (need[p][l], a bit per other part): the wait ends once that part has
// finished the deeper level (done[q] <= l + 1).  The part with the deepest
// pending level never waits, so the waits always end; each is bounded by
// spin_limit polls all the same (error bit 0, GBBC_ERR_TIMEOUT).
// Successors are found from per-(vertex, lane) distances: parts run at
// different levels, so the level-parity frontier words cannot serve them.

// dist[v][j] = level for the entries of one level (lane-minor rows of 64).
__global__ void k_part_dist(Slot s, long long q_lo, long long q_hi, int level, int32_t* dist) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
        const int32_t v = s.qv[e];
        const u64 m = s.qm[e];
        if ((m >> lane) & 1ull) dist[(size_t)v * kLanes + lane] = level;
        if ((m >> (lane + 32)) & 1ull) dist[(size_t)v * kLanes + lane + 32] = level;
    }
}

// need[part(v) * nlev + level] |= 1 << part(w) for border entries (v, m) at
// `level` with a border neighbour w at level + 1 in one of m's lanes.
__global__ void k_part_need(Slot s, long long q_lo, long long q_hi, int level, int nlev, const int32_t* dist,
                            const int32_t* part, const int32_t* bidx, const int32_t* cut_rp, const int32_t* cut_col,
                            unsigned* need) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + gwarp(); e < q_hi; e += nwarps()) {
        const int32_t v = s.qv[e];
        if (bidx[v] < 0) continue;
        const u64 m = s.qm[e];
        unsigned bits = 0u;
        for (int32_t p = cut_rp[v]; p < cut_rp[v + 1]; ++p) {
            const int32_t w = cut_col[p];
            const int32_t* dw = dist + (size_t)w * kLanes;
            const bool hit = (((m >> lane) & 1ull) && dw[lane] == level + 1) ||
                             (((m >> (lane + 32)) & 1ull) && dw[lane + 32] == level + 1);
            if (__any_sync(FULL, hit)) bits |= 1u << part[w];
        }
        if (lane == 0 && bits) atomicOr(need + (size_t)part[v] * nlev + level, bits);
    }
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acq_i(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel_i(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the G blocks of one part's group (bar[0] arrivals, bar[1]
// generation); false when it gave up or an error was reported.
__device__ __forceinline__ bool group_barrier(unsigned* bar, unsigned G, unsigned* err, long long spin_limit,
                                              int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acq(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == G - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (ld_acq(bar + 1) == gen) {
                if (ld_acq(err) & 1u) {
                    ok = 0;
                    break;
                }
                if (++spins >= spin_limit) {
                    atomicOr(err, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Backward step of entry e at `level` from the distance rows: for each lane
// j of the entry, the successors are the neighbours w (any part) with
// dist[w][j] = level + 1; the same fixed-point sums as the level-synchronous
// backward (bc_fixed.cuh), BC added without atomics (each vertex belongs to
// one part, whose group runs its levels one after the other).
template <bool WIDE>
__device__ __forceinline__ void bwd_entry_dist(const Csr& g, const Slot& s, const int32_t* dist, u64* bc, int level,
                                               long long e) {
    const int lane = threadIdx.x & 31;
    const int32_t v = s.qv[e];
    const u64 m = s.qm[e];
    u64 N0, N1;
    int E0, E1;
    lane_norms<WIDE>(s, v, m, N0, E0, N1, E1);
    const bool l0 = (m >> lane) & 1ull, l1 = (m >> (lane + 32)) & 1ull;
    u128 a0 = {0ull, 0ull}, a1 = {0ull, 0ull};
    for (int32_t p = __ldg(g.row_ptr + v); p < __ldg(g.row_ptr + v + 1); ++p) {
        const int32_t w = __ldg(g.col + p);
        const size_t at0 = (size_t)w * kLanes + lane, at1 = at0 + 32;
        if (l0 && __ldcg(dist + at0) == level + 1)
            a0 = add128(a0, psi_term<WIDE>(__ldcg(s.psi + at0), WIDE ? __ldcg(s.psi_e + at0) : 0, E0));
        if (l1 && __ldcg(dist + at1) == level + 1)
            a1 = add128(a1, psi_term<WIDE>(__ldcg(s.psi + at1), WIDE ? __ldcg(s.psi_e + at1) : 0, E1));
    }
    bwd_store<WIDE, false>(s, bc, v, m, E0, E1, N0, N1, a0, a1);
}

// One cooperative launch: part p runs on blocks [p * G, (p + 1) * G).
// ctl: [0] error bits, [1] waits performed, [2 + 2p], [3 + 2p] part p's group
// barrier; done[p] = the last level part p finished (nlev before any).
template <bool WIDE>
__global__ void __launch_bounds__(kBlock) k_part_backward(Csr g, Slot s, const int32_t* dist, const int32_t* part,
                                                          int P, const long long* off, int nlev,
                                                          const unsigned* need, int* done, unsigned* ctl, u64* bc,
                                                          long long spin_limit) {
    __shared__ int s_ok;
    const unsigned G = gridDim.x / (unsigned)P;
    const int p = (int)(blockIdx.x / G);
    if (p >= P) return;
    const unsigned r = blockIdx.x % G;
    const long long gw = ((long long)r * blockDim.x + threadIdx.x) >> 5;
    const long long gnw = ((long long)G * blockDim.x) >> 5;
    unsigned* err = ctl;
    unsigned* bar = ctl + 2 + 2 * p;
    for (int l = nlev - 1; l >= 1; --l) {
        const unsigned mask = need[(size_t)p * nlev + l] & ~(1u << p);
        if (mask && threadIdx.x == 0) {  // wait for the parts holding successors one level deeper
            int ok = 1;
            long long spins = 0;
            for (int q = 0; q < P && ok; ++q) {
                if (!((mask >> q) & 1u)) continue;
                while (ld_acq_i(done + q) > l + 1) {
                    if (ld_acq(err) & 1u) {
                        ok = 0;
                        break;
                    }
                    if (++spins >= spin_limit) {
                        atomicOr(err, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (r == 0 && ok) atomicAdd(ctl + 1, 1u);
            s_ok = ok;
        }
        if (mask) {
            __syncthreads();
            if (!s_ok) return;
        }
        const long long q_lo = off[l], q_hi = off[l + 1];
        for (long long e = q_lo + gw; e < q_hi; e += gnw)
            if (part[s.qv[e]] == p) bwd_entry_dist<WIDE>(g, s, dist, bc, l, e);
        if (!group_barrier(bar, G, err, spin_limit, &s_ok)) return;
        if (r == 0 && threadIdx.x == 0) st_rel_i(done + p, l);
    }
}

int part_backward_blocks_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_part_backward<false>, kBlock, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_part_backward<true>, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return a < b ? a : b;
}

void launch_part_dist(const Slot& s, long long q_lo, long long q_hi, int level, int32_t* dist, int nsm,
                      cudaStream_t st) {
    if (q_hi <= q_lo) return;
    long long blocks = ((q_hi - q_lo) * kWarp + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    k_part_dist<<<(int)blocks, kBlock, 0, st>>>(s, q_lo, q_hi, level, dist);
}

void launch_part_need(const Slot& s, long long q_lo, long long q_hi, int level, int nlev, const int32_t* dist,
                      const int32_t* part, const int32_t* bidx, const int32_t* cut_rp, const int32_t* cut_col,
                      unsigned* need, int nsm, cudaStream_t st) {
    if (q_hi <= q_lo) return;
    long long blocks = ((q_hi - q_lo) * kWarp + kBlock - 1) / kBlock;
    if (blocks > (long long)nsm * 8) blocks = (long long)nsm * 8;
    k_part_need<<<(int)blocks, kBlock, 0, st>>>(s, q_lo, q_hi, level, nlev, dist, part, bidx, cut_rp, cut_col, need);
}

cudaError_t launch_part_backward(const Csr& g, const Slot& s, const int32_t* dist, const int32_t* part, int P,
                                 const long long* off, int nlev, const unsigned* need, int* done, unsigned* ctl,
                                 u64* bc, long long spin_limit, bool wide, int blocks, cudaStream_t st) {
    if (P < 1 || blocks < P) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(blocks / P * P), 1, 1);
    cfg.blockDim = dim3(kBlock, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (wide)
        return cudaLaunchKernelEx(&cfg, k_part_backward<true>, g, s, dist, part, P, off, nlev, need, done, ctl, bc,
                                  spin_limit);
    return cudaLaunchKernelEx(&cfg, k_part_backward<false>, g, s, dist, part, P, off, nlev, need, done, ctl, bc,
                              spin_limit);
}

}  // namespace gbbc
