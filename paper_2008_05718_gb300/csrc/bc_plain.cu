// Plain one-source-at-a-time Brandes on the GPU (batch width 1): the
// baseline the bitset-batched path is measured against.
//
// Per source, level by level (Sec. II, Algorithm 1):
//   forward  - a warp per frontier vertex v (a block for rows longer than
//              the heavy degree) claims each undiscovered neighbour w with
//              atomicCAS(dist[w], -1, l+1), queues it, and adds sigma[v]
//              into sigma[w] with a 64-bit atomic when dist[w] == l+1 (the
//              work-efficient queue form of McLaughlin and Bader, SC'14);
//   backward - a warp per vertex of level l pulls from the neighbours at
//              level l+1 with the same 128-bit fixed-point sums as the
//              batched path (bc_fixed.cuh), so both give identical BC bits.
// Counts of 2^64 or more are not supported here (GBBC_ERR_CAPACITY); the
// batched path handles them.
//
// The same steps also run with coarse-grained source parallelism (the block
// schedule with batch width 1, McLaughlin and Bader's design): every thread
// block runs whole sources one after another, taken from a work list, on
// its own per-source arrays; many blocks run at once.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bc_fixed.cuh"
#include "bc_internal.cuh"
#include "bc_plain.cuh"
#include "bc_rows.cuh"

namespace gbbc {

#define PFULL 0xffffffffu

__device__ __forceinline__ long long pw_gwarp() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long pw_nwarps() { return ((long long)gridDim.x * blockDim.x) >> 5; }

__global__ void k_plain_seed(PlainState p, int32_t src) {
    p.dist[src] = 0;
    p.sigma[src] = 1ull;
    p.queue[0] = src;
}

// Scan neighbours [beg, end) of v with `nt` threads starting at `t`.
__device__ __forceinline__ void plain_push_row(const Csr& g, const PlainState& p, int32_t v, int level,
                                               int32_t beg, int32_t end, int t, int nt) {
    const int lane = threadIdx.x & 31;
    const u64 sv = p.sigma[v];
    unsigned carry = 0;
    for (int32_t base = beg; base < end; base += nt) {
        int32_t q = base + t;
        bool newq = false;
        int32_t w = 0;
        if (q < end) {
            w = __ldg(g.col + q);
            int old = atomicCAS(p.dist + w, -1, level + 1);
            newq = old == -1;
            if (old == -1 || old == level + 1) {
                u64 o = atomicAdd(p.sigma + w, sv);
                carry |= (o + sv) < o;
            }
        }
        unsigned bal = __ballot_sync(PFULL, newq);
        if (bal) {
            int leader = __ffs(bal) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(&p.ctr->qtail, (unsigned long long)__popc(bal));
            b = __shfl_sync(PFULL, b, leader);
            if (newq) p.queue[b + __popc(bal & ((1u << lane) - 1u))] = w;
        }
    }
    if (carry) atomicOr(&p.ctr->carry, 1u);
}

__global__ void k_plain_fwd(Csr g, PlainState p, long long q_lo, long long q_hi, int level, int heavy_deg) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + pw_gwarp(); e < q_hi; e += pw_nwarps()) {
        int32_t v = p.queue[e];
        int32_t beg = __ldg(g.row_ptr + v), end = __ldg(g.row_ptr + v + 1);
        if (end - beg > heavy_deg) {
            if (lane == 0) {
                unsigned long long h = atomicAdd(&p.ctr->heavy, 1ull);
                p.heavy[h] = v;
            }
            continue;
        }
        plain_push_row(g, p, v, level, beg, end, lane, kWarp);
    }
}

__global__ void k_plain_fwd_heavy(Csr g, PlainState p, int level) {
    const long long cnt = (long long)p.ctr->heavy;
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        int32_t v = p.heavy[h];
        plain_push_row(g, p, v, level, g.row_ptr[v], g.row_ptr[v + 1], threadIdx.x, blockDim.x);
    }
}

// Backward: sum over successors of psi_w * 2^(E_v + 64) in a u128.
__device__ __forceinline__ u128 plain_bwd_row(const Csr& g, const PlainState& p, int level, int Ev, int32_t beg,
                                              int32_t end, int t, int nt) {
    u128 a = {0ull, 0ull};
    for (int32_t q = beg + t; q < end; q += nt) {
        int32_t w = __ldg(g.col + q);
        if (p.dist[w] == level + 1) {
            u64 bits = p.psi[w];
            int e = (int)((bits >> 52) & 0x7FFull) - 1023;
            u64 M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
            a = add128(a, shl_term(M, e + Ev + 12));
        }
    }
    return a;
}

__device__ __forceinline__ void plain_bwd_finish(const PlainState& p, u64* bc, int32_t v, u128 A) {
    u64 x = p.sigma[v];
    int lz = __clzll(x);
    u64 N = x << lz;
    int E = 63 - lz;
    u128 d = mul_shift63(N, A);
    u128 psi = add128(recip127(N), A);
    u64 M;
    int e;
    round128(psi, -64 - E, M, e);
    p.psi[v] = double_bits(M, e);
    u128 b = {bc[2 * (size_t)v], bc[2 * (size_t)v + 1]};
    b = add128(b, d);
    bc[2 * (size_t)v] = b.lo;
    bc[2 * (size_t)v + 1] = b.hi;
}

__global__ void k_plain_bwd(Csr g, PlainState p, u64* bc, long long q_lo, long long q_hi, int level, int heavy_deg) {
    const int lane = threadIdx.x & 31;
    for (long long e = q_lo + pw_gwarp(); e < q_hi; e += pw_nwarps()) {
        int32_t v = p.queue[e];
        int32_t beg = __ldg(g.row_ptr + v), end = __ldg(g.row_ptr + v + 1);
        if (end - beg > heavy_deg) {
            if (lane == 0) {
                unsigned long long h = atomicAdd(&p.ctr->heavy, 1ull);
                p.heavy[h] = v;
            }
            continue;
        }
        int Ev = 63 - __clzll(p.sigma[v]);
        u128 a = plain_bwd_row(g, p, level, Ev, beg, end, lane, kWarp);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            u128 x = {__shfl_xor_sync(PFULL, a.lo, o), __shfl_xor_sync(PFULL, a.hi, o)};
            a = add128(a, x);
        }
        if (lane == 0) plain_bwd_finish(p, bc, v, a);
    }
}

__global__ void k_plain_bwd_heavy(Csr g, PlainState p, u64* bc, int level) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ u128 part[kHeavyBlock / kWarp];
    const long long cnt = (long long)p.ctr->heavy;
    for (long long h = blockIdx.x; h < cnt; h += gridDim.x) {
        int32_t v = p.heavy[h];
        int Ev = 63 - __clzll(p.sigma[v]);
        u128 a = plain_bwd_row(g, p, level, Ev, g.row_ptr[v], g.row_ptr[v + 1], threadIdx.x, blockDim.x);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            u128 x = {__shfl_xor_sync(PFULL, a.lo, o), __shfl_xor_sync(PFULL, a.hi, o)};
            a = add128(a, x);
        }
        if (lane == 0) part[wid] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            u128 t = {0ull, 0ull};
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = add128(t, part[i]);
            plain_bwd_finish(p, bc, v, t);
        }
        __syncthreads();
    }
}

static int plain_grid(long long warps, int nsm) {
    long long b = (warps * kWarp + kBlock - 1) / kBlock;
    if (b > (long long)nsm * 8) b = (long long)nsm * 8;
    return b < 1 ? 1 : (int)b;
}

void launch_plain_seed(const PlainState& p, int32_t src, cudaStream_t st) { k_plain_seed<<<1, 1, 0, st>>>(p, src); }

void launch_plain_fwd(const Csr& g, const PlainState& p, long long q_lo, long long q_hi, int level, int heavy_deg,
                      int nsm, cudaStream_t st) {
    if (q_hi <= q_lo) return;
    k_plain_fwd<<<plain_grid(q_hi - q_lo, nsm), kBlock, 0, st>>>(g, p, q_lo, q_hi, level, heavy_deg);
    k_plain_fwd_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, p, level);
}

void launch_plain_bwd(const Csr& g, const PlainState& p, u64* bc, long long q_lo, long long q_hi, int level,
                      int heavy_deg, int nsm, cudaStream_t st) {
    if (q_hi <= q_lo) return;
    k_plain_bwd<<<plain_grid(q_hi - q_lo, nsm), kBlock, 0, st>>>(g, p, bc, q_lo, q_hi, level, heavy_deg);
    k_plain_bwd_heavy<<<nsm * 2, kHeavyBlock, 0, st>>>(g, p, bc, level);
}

// ---- one source per thread block, many blocks at once -------------------
// Block b owns dist/sigma/psi/queue rows b of the PlainBlocks arrays (clean
// between sources: dist -1 and sigma 0 everywhere), and level boundaries.
// Inside the block a warp takes each frontier vertex (whole rows, however
// long); the levels are separated by block barriers.  After the backward the
// block resets dist and sigma of the vertices it reached.  BC is added with
// exact 128-bit atomics: blocks may add into one vertex at the same time.
__global__ void __launch_bounds__(kPlainBlock) k_plain_blocks(Csr g, PlainBlocks B, const int32_t* src, long long k,
                                                             unsigned long long* next, u64* bc,
                                                             unsigned long long* stats) {
    __shared__ long long s_i;
    __shared__ long long s_hi;
    __shared__ unsigned s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t n = (size_t)B.n;
    PlainState p;
    p.n = B.n;
    p.dist = B.dist + blockIdx.x * n;
    p.sigma = B.sigma + blockIdx.x * n;
    p.psi = B.psi + blockIdx.x * n;
    p.queue = B.queue + blockIdx.x * n;
    p.heavy = nullptr;
    p.ctr = B.ctr + blockIdx.x;
    int32_t* lev = B.lev + blockIdx.x * (n + 2);
    for (;;) {
        if (threadIdx.x == 0) s_i = (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long i = s_i;
        if (i >= k) break;
        const int32_t s0 = src[i];
        if (threadIdx.x == 0) {
            p.dist[s0] = 0;
            p.sigma[s0] = 1ull;
            p.queue[0] = s0;
            p.ctr->qtail = 1ull;
            lev[0] = 0;
            lev[1] = 1;
        }
        __syncthreads();
        int level = 0;
        for (;;) {  // forward, level by level
            const long long q_lo = lev[level], q_hi = lev[level + 1];
            for (long long e = q_lo + wid; e < q_hi; e += nw) {
                const int32_t v = p.queue[e];
                plain_push_row(g, p, v, level, __ldg(g.row_ptr + v), __ldg(g.row_ptr + v + 1), lane, kWarp);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_hi = (long long)(*(volatile unsigned long long*)&p.ctr->qtail);
                lev[level + 2] = (int32_t)s_hi;
                s_carry = *(volatile unsigned*)&p.ctr->carry;
            }
            __syncthreads();
            if (s_hi == q_hi) break;
            ++level;
        }
        const int nlev = level + 1;
        // backward, levels nlev-1 .. 1; skipped for a source whose counts
        // reached 2^64 (the call then fails with nothing of it added)
        for (int l = s_carry ? 0 : nlev - 1; l >= 1; --l) {
            for (long long e = lev[l] + wid; e < lev[l + 1]; e += nw) {
                const int32_t v = p.queue[e];
                const int Ev = 63 - __clzll(p.sigma[v]);
                u128 a = plain_bwd_row(g, p, l, Ev, __ldg(g.row_ptr + v), __ldg(g.row_ptr + v + 1), lane, kWarp);
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    u128 x = {__shfl_xor_sync(PFULL, a.lo, o), __shfl_xor_sync(PFULL, a.hi, o)};
                    a = add128(a, x);
                }
                if (lane == 0) {
                    const u64 x = p.sigma[v];
                    const int lz = __clzll(x);
                    const u64 N = x << lz;
                    const u128 d = mul_shift63(N, a);
                    u128 psi = add128(recip127(N), a);
                    u64 M;
                    int ex;
                    round128(psi, -64 - (63 - lz), M, ex);
                    p.psi[v] = double_bits(M, ex);
                    atomic_add128(bc + 2 * (size_t)v, d);
                }
            }
            __syncthreads();
        }
        // reset what this source touched; report counts of 2^64 or more
        const long long reached = lev[nlev];
        for (long long e = threadIdx.x; e < reached; e += blockDim.x) {
            const int32_t v = p.queue[e];
            p.dist[v] = -1;
            p.sigma[v] = 0ull;
        }
        if (threadIdx.x == 0) {
            atomicAdd(stats, 1ull);
            atomicAdd(stats + 1, (unsigned long long)nlev);
            if (s_carry) atomicOr((unsigned*)(stats + 2), 1u);
            p.ctr->carry = 0u;
        }
        __syncthreads();
    }
}

int plain_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_plain_blocks, kPlainBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_plain_blocks(const Csr& g, const PlainBlocks& B, const int32_t* src, long long k,
                                unsigned long long* next, u64* bc, unsigned long long* stats, cudaStream_t st) {
    if (k <= 0 || B.count < 1) return cudaSuccess;
    k_plain_blocks<<<B.count, kPlainBlock, 0, st>>>(g, B, src, k, next, bc, stats);
    return cudaGetLastError();
}

}  // namespace gbbc
