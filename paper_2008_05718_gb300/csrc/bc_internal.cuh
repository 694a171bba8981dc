// Internal declarations of libgbbc: device data layout of one batch "slot"
// and the launch wrappers of the kernels.  Not part of the public ABI.
//
// A batch packs up to 64 sources, one per bit ("lane") of a 64-bit word, and
// runs Brandes' two phases (Sec. II, Algorithm 1) for all of them at once:
//   forward  - level-synchronous BFS; per level a discovery step (top-down
//              push from the frontier queue, or bottom-up pull over the
//              vertex range) finds next[w] = (OR of frontier masks of w's
//              neighbours) & ~visited[w], then a gather step computes sigma
//              of each newly reached (vertex, lane) from its predecessors in
//              CSR order (integer adds mod 2^64 with carry detection).
//   backward - levels in reverse; for each (v, lane) at level l, the
//              successors are the neighbours at level l+1 in that lane, and
//              delta_s(v) = sigma_v * sum_w (1 + delta_w) / sigma_w  (Eq. 2),
//              accumulated in 128-bit fixed point (bc_fixed.cuh) and written
//              back as psi_v = (1 + delta_v) / sigma_v; BC[v] += sum over
//              lanes of delta, also in 128-bit fixed point (units 2^-64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbbc.h"

namespace gbbc {

constexpr int kLanes = 64;         // sources per batch word
constexpr int kWarp = 32;
constexpr int kBlock = 256;        // threads per block of the warp-per-row kernels
constexpr int kHeavyBlock = 512;   // threads per block of the block-per-row kernels
constexpr int kChunk = 1024;       // CSR entries per chunk task of a heavy row
constexpr int kChunkBlock = 256;   // threads per block of the chunk-task kernels

typedef unsigned long long u64;

// Dense per-vertex frontier word with the level it belongs to: the mask is
// valid for level `tag` only, so stale entries never need clearing.
struct __align__(16) MaskTag {
    u64 mask;
    int32_t tag;
    int32_t pad;
};

// Counters of one batch, written by kernels, read back by the host once per
// level.  Field order matters: the host zeroes [lane_sum, heavy] before a
// gather step and [heavy, lanes] before a discovery step.
struct __align__(16) Counters {
    unsigned long long qtail;     // next free position in the entry queue
    unsigned long long lane_sum;  // gather: sum of popc(mask) of its entries
    unsigned long long lane_esum; // gather: sum of popc(mask) * degree
    unsigned long long heavy;     // heavy rows of this step (accumulator slots)
    unsigned long long tasks;     // chunk tasks of the heavy rows
    unsigned long long medium;    // rows deferred to the warp-per-row pull kernel
    unsigned long long edge_sum;  // discovery: sum of degrees of new vertices
    unsigned long long scanned;   // discovery: CSR entries read by a pull step
    u64 lanes;                    // discovery: OR of the lanes reaching them
    unsigned err;                 // bit 0: queue overflow, bit 1: row list overflow
    unsigned carry;               // some sigma reached 2^64 in this batch
    // direction decision (k_decide), state kept across the levels of a batch
    unsigned long long visited;   // (vertex, lane) pairs reached so far
    unsigned long long explored;  // frontier edges already expanded (threshold rule)
    int dir;                      // decision for the next step: 0 push, 1 pull
    int pull_state;               // threshold rule hysteresis
    float feat[6];                // policy features of the decided step
    float logit[2];               // MLP outputs (push, pull) when learned
};

// Device state of one batch slot (sized for n vertices, 64 lanes).
struct Slot {
    int32_t n = 0;
    u64* vis = nullptr;      // [n] lanes that have reached v
    u64* nx = nullptr;       // [n] lanes reaching v at the next level (scratch)
    u64* ovf = nullptr;      // [n] lanes whose sigma(v) >= 2^64
    MaskTag* F = nullptr;    // [2][n] frontier masks by level parity
    u64* sigma = nullptr;    // [n][64] sigma mod 2^64, lane-minor
    u64* psi = nullptr;      // [n][64] (1 + delta) / sigma as double bits, lane-minor
    // wide sigma format (lanes whose sigma reached 2^64), allocated on demand
    u64* sN = nullptr;       // [n][64] normalised 64-bit mantissa of sigma
    int32_t* sX = nullptr;   // [n][64] exponent: sigma ~ sN * 2^sX
    int32_t* psi_e = nullptr;// [n][64] exponent of psi (psi bits hold [1, 2))
    int32_t* qv = nullptr;   // [qcap] queued vertex per entry, levels back to back
    u64* qm = nullptr;       // [qcap] lanes of the entry
    int32_t* heavy = nullptr;// [n] deferred entries/rows of the current step
    // heavy rows are split into chunk tasks of kChunk entries whose partial
    // sums meet in per-row accumulators (exact integer atomics)
    long long hcap = 0;      // heavy rows per step (vertices of degree > heavy_deg)
    long long tcap = 0;      // chunk tasks per step
    int32_t* hentry = nullptr; // [hcap] queue entry of heavy slot h
    u64* hacc = nullptr;     // [hcap][64][2] per-lane accumulators (zero between steps)
    u64* hcarry = nullptr;   // [hcap] lanes whose sigma sum carried
    int2* tasks = nullptr;   // [tcap] (heavy slot, first CSR position)
    int32_t* medium = nullptr;// [n] rows deferred by the thread-per-row pull
    long long qcap = 0;
    Counters* ctr = nullptr; // device
    Counters* hctr = nullptr;// pinned host mirror
    int32_t* d_src = nullptr;// [64] sources of the batch
};

// Device state of the plain one-source-at-a-time path (batch width 1).
struct PlainState {
    int32_t n = 0;
    int32_t* dist = nullptr;   // [n]
    u64* sigma = nullptr;      // [n]
    u64* psi = nullptr;        // [n] (1 + delta) / sigma as double bits
    int32_t* queue = nullptr;  // [n] vertices by level
    int32_t* heavy = nullptr;  // [n] rows deferred to the block-per-row kernels
    Counters* ctr = nullptr;
};

struct Csr {
    int32_t n;
    long long nnz;
    const int32_t* row_ptr;
    const int32_t* col;
};

// ---- block-per-batch mode ----
// One thread-block cluster (csize CTAs, csize = 1 is a single block) runs a
// whole batch, forward and backward, separated by cluster barriers only;
// clusters take batches from a work list.  Slot k holds the state of the
// batch that cluster k is running, indexed by vertex - lo of the batch's
// graph, so slots are sized for the largest graph of the handle.
constexpr int kBlockThreads = 512;

struct BlockBatch {
    int32_t gi, lo, hi, nsrc;
    long long src_off;   // first source of the batch in the source array
    int32_t wide;        // start in the wide sigma format
    int32_t pad;
};

struct BlockSlots {
    long long nslot = 0;  // vertices per slot
    long long qcap = 0;   // queue entries per slot
    int count = 0;        // slots (= clusters of the launch)
    int csize = 1;        // thread blocks per cluster (per batch)
    int* slot_batch = nullptr;  // [count] batch each slot is running
    void* lsp = nullptr;  // [slot][nslot + 2] per-level "thread-per-entry" flags
    u64* vis = nullptr;
    u64* nx = nullptr;
    u64* ovf = nullptr;
    MaskTag* F = nullptr;     // [slot][2][nslot]
    u64* sigma = nullptr;     // [slot][nslot][64]
    u64* psi = nullptr;
    u64* sN = nullptr;
    int32_t* sX = nullptr;
    int32_t* psi_e = nullptr;
    int32_t* qv = nullptr;    // [slot][qcap]
    u64* qm = nullptr;
    long long* lev = nullptr; // [slot][nslot + 2] level boundaries
    Counters* ctr = nullptr;  // [slot]
};

// ---- persistent multi-batch kernel of the grid schedule (bc_persist.cu) ----
// One cooperative launch runs every batch of a call: up to kMaxPSlots batches
// are in flight at once, each on a batch slot of its own, and the level loop
// runs on the device.  A "tick" is one level step of every batch in flight
// (batch init, top-down or bottom-up discovery, sigma gather, or backward
// step), in four phases separated by grid-wide barriers: rows (a warp per
// item), heavy-row chunk tasks (a block per item), heavy-row finish (a warp
// per item), and the bookkeeping of each batch (a warp per batch: direction
// decision, level advance, next batch).
constexpr int kMaxPSlots = 16;
constexpr int kPBlock = 256;  // threads per block of the persistent kernel

enum PPhase { PH_IDLE = 0, PH_INIT = 1, PH_DISC = 2, PH_GATHER = 3, PH_BWD = 4, PH_DONE = 5 };

// State of one batch slot between ticks (device memory, written by the
// slot's bookkeeping warp, read by every block after the barrier).
struct __align__(16) PCtl {
    int32_t phase;       // PPhase
    int32_t batch;       // batch index
    int32_t level;       // forward: level whose discovery / gather runs; backward: level
    int32_t dir;         // direction of the discovery step (0 push, 1 pull)
    int32_t lo, hi;      // vertex range of the batch's graph
    int32_t nlev;        // forward levels of the batch (set when the forward ends)
    int32_t npull;       // bottom-up steps of the batch
    long long q_lo, q_hi;// entry range of the step (gather: new entries [q_hi, new_hi))
    long long new_hi;    // end of the entries the discovery queued
    long long items;     // warp items of the step's first phase
    u64 lanes;           // active lanes (bottom-up steps)
};

// Whole-launch control: grid barrier, error bits, batch work list, stats.
struct __align__(16) PGlobal {
    unsigned bar_count;  // blocks arrived at the current barrier
    unsigned bar_gen;    // barrier generation
    unsigned err;        // bit 0: a barrier wait gave up; bit 1: queue capacity
    unsigned next;       // next batch of the work list
    unsigned long long batches, levels_fwd, levels_pull;
    unsigned wide;       // batches whose counts reached 2^64 (listed in wide_list)
    unsigned err_info;   // with err bit 1: the slot's error bits, step kind, direction and level
};

// Resident blocks of the persistent kernel per SM (0 if the query fails).
int persist_blocks_per_sm();
// Launch it cooperatively on `blocks` blocks (at most SMs x resident blocks).
// slots: W device Slot structs; ctl: W PCtl (zeroed: idle); lev: W rows of
// lev_stride level boundaries; bc: the handle's BC (exact atomic adds).
cudaError_t launch_persist(const Csr& g, const Slot* slots, int W, PCtl* ctl, long long* lev, long long lev_stride,
                           const BlockBatch* batches, int nb, const int32_t* srcs, u64* bc, int policy,
                           const void* weights_fp16, const long long* graph_max_deg, int heavy_deg,
                           long long spin_limit, PGlobal* G, int32_t* wide_list, int blocks, cudaStream_t st);

// ---- the partitioned method (bc_partition.cu) ----
constexpr int32_t kPartInf = 0x7f7f7f7f;  // an unreached border distance (memset 0x7f)
// Path counts of border nodes (lane-minor, [border][64]) or of a border
// matrix: value mod 2^64, a flag for values >= 2^64, and then an
// approximation N * 2^X with a normalised 64-bit mantissa.
struct PartWide {
    u64* mod = nullptr;
    u64* N = nullptr;
    int32_t* X = nullptr;
    uint8_t* big = nullptr;
};
void launch_part_extract(const Slot& s, long long q_lo, long long q_hi, int level, bool wide, int mode,
                         const int32_t* bidx, const int32_t* bpart, const long long* boff, const long long* moff,
                         const int32_t* lane_b, int32_t* dist_out, u64* mod, u64* N, int32_t* X, uint8_t* big,
                         int nsm, cudaStream_t st);
void launch_refine_cut(const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border, const int32_t* bidx,
                       long long nbt, int32_t* D, int* changed, int nsm, cudaStream_t st);
void launch_refine_bm(const int32_t* bpart, const long long* boff, const long long* moff, const int32_t* BM,
                      long long nbt, int32_t* D, int* changed, int nsm, cudaStream_t st);
void launch_border_sigma_level(int level, const int32_t* cut_rp, const int32_t* cut_col, const int32_t* border,
                               const int32_t* bidx, const int32_t* bpart, const long long* boff,
                               const long long* moff, const int32_t* BM, const PartWide& SM, long long nbt,
                               const int32_t* D, const int32_t* D1, const PartWide& S1, const PartWide& A,
                               const PartWide& Sig, int nsm, cudaStream_t st);
void launch_seed_inject(const Slot& s, int level, const int32_t* border, long long nbt, const int32_t* D,
                        const PartWide& A, const int32_t* row_ptr, int nsm, cudaStream_t st);
void launch_seed_add(const Slot& s, int level, const int32_t* border, long long nbt, const int32_t* D,
                     const PartWide& A, bool wide, int nsm, cudaStream_t st);

// the asynchronous backward of the partitioned method (at most 32 parts)
constexpr int kMaxParts = 32;
int part_backward_blocks_per_sm();
void launch_part_dist(const Slot& s, long long q_lo, long long q_hi, int level, int32_t* dist, int nsm,
                      cudaStream_t st);
void launch_part_need(const Slot& s, long long q_lo, long long q_hi, int level, int nlev, const int32_t* dist,
                      const int32_t* part, const int32_t* bidx, const int32_t* cut_rp, const int32_t* cut_col,
                      unsigned* need, int nsm, cudaStream_t st);
cudaError_t launch_part_backward(const Csr& g, const Slot& s, const int32_t* dist, const int32_t* part, int P,
                                 const long long* off, int nlev, const unsigned* need, int* done, unsigned* ctl,
                                 u64* bc, long long spin_limit, bool wide, int blocks, cudaStream_t st);

// ---- launch wrappers (bc_kernels.cu) ----
void launch_seed(const Slot& s, int nsrc, cudaStream_t st);
void launch_push(const Csr& g, const Slot& s, long long q_lo, long long q_hi, int level, int heavy_deg,
                 int nsm, cudaStream_t st);
void launch_pull(const Csr& g, const Slot& s, int32_t lo, int32_t hi, u64 lanes, int level, int heavy_deg,
                 int nsm, cudaStream_t st);
void launch_fwd_gather(const Csr& g, const Slot& s, long long q_lo, int level, int heavy_deg, int nsm,
                       cudaStream_t st, bool wide);
void launch_bwd(const Csr& g, const Slot& s, u64* bc_fixed, long long q_lo, long long q_hi, int level,
                int heavy_deg, int nsm, cudaStream_t st, bool wide);
void launch_bc_to_double(const u64* bc_fixed, double* out, long long n, bool add, cudaStream_t st);
void launch_keep_dist(const Slot& s, long long q_lo, long long q_hi, int level, int32_t* dist, long long n_total,
                      long long first_src, int nsrc, cudaStream_t st);
void launch_keep_sigma(const Slot& s, int32_t lo, int32_t hi, uint64_t* sigma, uint8_t* ovf, long long n_total,
                       long long first_src, int nsrc, cudaStream_t st);
void launch_undo(const Slot& s, long long q_lo, long long q_hi, cudaStream_t st);
// Block-per-batch persistent kernel over `nb` batches; stats[0..3]: batches,
// forward levels, bottom-up levels, wide reruns (device, accumulated).
// ---- weighted graphs (bc_weighted.cu) ----
#ifndef GBBC_WTHREADS
#define GBBC_WTHREADS 512
#endif
constexpr int kWThreads = GBBC_WTHREADS;  // one CTA per batch
constexpr int kMaxWeight = 64;   // weights in [1, kMaxWeight]
constexpr int kMaxBuckets = kMaxWeight + 1;
#ifndef GBBC_WHEAVY
#define GBBC_WHEAVY 64
#endif
constexpr int kWHeavy = GBBC_WHEAVY;  // rows longer than this are scanned by a whole warp

struct WBatch {
    int32_t lo, hi, nsrc, gi;
    int32_t wide, pad;  // wide = 1: start in the wide sigma format
    long long first;    // position of the batch's first source in the call's list
    long long src_off;  // first source of the batch in the uploaded source array
};

// Per-CTA state of the weighted path: `count` slots of nslot vertices with L
// lanes (sources) each; a (vertex, lane) pair has id v * L + lane.
struct WSlots {
    long long nslot = 0, qcap = 0, levcap = 0, bcap = 0;
    int count = 0, B = 0, L = 0;  // slots; buckets (max weight + 1); lanes per batch
    int32_t* dist = nullptr;      // [count][nslot][L]
    u64* sp = nullptr;            // [count][nslot][L] sigma, then psi
    uint32_t* blist = nullptr;    // [count][B][bcap] pair ids pending per bucket
    uint32_t* qv = nullptr;       // [count][qcap] settled pairs in distance order
    int32_t* levD = nullptr;      // [count][levcap] distance of each settle step
    long long* levOff = nullptr;  // [count][levcap + 1] queue offset of each step
    u64* sN = nullptr;            // [count][nslot][L] wide sigma mantissa (sigma >= 2^64)
    int32_t* sX = nullptr;        // [count][nslot][L] wide sigma exponent, then psi exponent
    uint8_t* wf = nullptr;        // [count][nslot][L] 1 where sigma >= 2^64
};

// Resident blocks of the pair-granular kernel per SM.
int weighted_blocks_per_sm();
// Every batch of a weighted graph (weights in [1, W]; wt null: all weights 1,
// W = 1, an unweighted graph run pair by pair).  A batch whose path counts
// pass 2^64 is rerun in the wide format and sets gwide[its graph]; batches
// with .wide set, or of a graph with gwide set, start wide.  stats[0] +=
// batches done, stats[1] += settle steps, stats[2] += batches rerun wide, low
// word of stats[3] |= error bits (2: too many distinct distances, 4: queue
// full, 8: a bucket list full).  k_dist/k_sigma/k_ovf (may be null) receive
// the per-source state, rows by source position, n_total columns.
cudaError_t launch_weighted_batches(const Csr& g, const int32_t* wt, const WSlots& S, const WBatch* batches, int nb,
                                    const int32_t* srcs, unsigned* next, u64* bc, int W, int32_t* k_dist,
                                    u64* k_sigma, uint8_t* k_ovf, long long n_total, int* gwide,
                                    unsigned long long* stats, cudaStream_t st);

// Clusters of csize CTAs of k_block_batches that fit on the device at once
// (0 if the query fails).
int block_max_clusters(int csize);
// A batch with .wide set starts in the wide sigma format; one that has to be
// rerun wide sets gwide[its graph] = 1.
cudaError_t launch_block_batches(const Csr& g, const BlockSlots& S, const BlockBatch* batches, int nb,
                                 const int32_t* srcs, unsigned* next, u64* bc, int policy, const void* weights_fp16,
                                 const long long* graph_max_deg, unsigned long long* stats, int* gwide,
                                 cudaStream_t st);
// Source grouping: features [k][6] and the network's score per source.
cudaError_t launch_source_features(const Csr& g, const int32_t* src, const int32_t* gid, long long k,
                                   const long long* goff, const long long* gmaxdeg, float* x, cudaStream_t st);
cudaError_t launch_group_score(const void* w_half, const float* x, long long k, float* score, cudaStream_t st);
cudaError_t mlp_to_half(const float* params_dev, void* half_dev, int count, cudaStream_t st);
// Direction of the step at `level`, whose entries start at q_lo (end: qtail).
void launch_decide(const Slot& s, long long q_lo, int level, int policy, const void* weights_fp16, long long n_range,
                   long long nnz_range, long long max_deg, cudaStream_t st);
void launch_plain_seed(const PlainState& p, int32_t src, cudaStream_t st);
void launch_plain_fwd(const Csr& g, const PlainState& p, long long q_lo, long long q_hi, int level, int heavy_deg,
                      int nsm, cudaStream_t st);
void launch_plain_bwd(const Csr& g, const PlainState& p, u64* bc, long long q_lo, long long q_hi, int level,
                      int heavy_deg, int nsm, cudaStream_t st);
void launch_validate(const Csr& g, int32_t* flags, cudaStream_t st);
void launch_fill_i32(int32_t* p, long long count, int32_t value, cudaStream_t st);
void launch_offset_copy(const int32_t* src, int32_t* dst, long long count, int32_t add, cudaStream_t st);

}  // namespace gbbc
