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

}  // namespace gbbc
