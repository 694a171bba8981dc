// Host side of libgbbc: the C ABI declared in include/gbbc.h.
//
// Handle = the CSR in device memory (one graph, or a disjoint union of many),
// the accumulated BC vector, and one batch slot of device state.  bc_compute
// splits the source list into batches of up to 64 sources (sources of one
// graph only, in list order), and drives each batch through Brandes' forward
// and backward phases (Sec. II, Algorithm 1) level by level.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <climits>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bc_fixed.cuh"
#include "bc_internal.cuh"
#include "bc_plain.cuh"

using namespace gbbc;

// Default bound on a device-side wait, in polls (options.timeout_spins = 0).
#ifndef GBBC_DEFAULT_SPINS
#define GBBC_DEFAULT_SPINS 100000000LL
#endif

extern "C" const char* bc_status_string(gbbc_status s);
extern "C" void bc_graph_destroy(gbbc_graph* g);
extern "C" gbbc_status bc_clear_trace(gbbc_graph* g);
extern "C" int64_t bc_mlp_param_count(int32_t k_out);
namespace gbbc {
cudaError_t policy_to_half(const float* params_dev, void* half_dev, cudaStream_t st);
}

struct gbbc_graph {
    int device = 0;
    cudaStream_t ast = nullptr;      // stream of the library's pool allocations and frees
    int nsm = 152;
    int32_t n = 0;
    long long nnz = 0;
    int32_t* d_row_ptr = nullptr;
    int32_t* d_col = nullptr;
    std::vector<int32_t> h_row_ptr;  // host copy for scheduling decisions
    std::vector<long long> goff;     // graph vertex offsets (count + 1)
    u64* d_bc = nullptr;             // [2n] BC in 128-bit fixed point (units 2^-64)
    double* d_bc_out = nullptr;      // [n] staging for bc_read into host memory
    int32_t* d_w = nullptr;          // edge weights (weighted graphs), aligned with d_col
    int32_t max_w = 0;               // largest weight (0: unweighted)
    WSlots wsl;                      // weighted path's per-CTA state
    WBatch* d_wb = nullptr;
    long long d_wb_cap = 0;
    std::vector<char> wide_graph;    // per graph: its batches start in the wide sigma format
    int max_clusters[4] = {0, 0, 0, 0};  // resident block-schedule clusters of 1, 2, 4, 8 CTAs
    int w_bps = 0;                   // resident pair-kernel blocks per SM (0: not yet asked)
    std::vector<signed char> pair_graph;  // per graph: the auto schedule takes pair (1), not (0), undecided (-1)
    int* d_gwide = nullptr;          // per graph: set by the block schedule when a batch went wide
    Slot slot;
    bool slot_ready = false;
    PlainState plain;            // batch width 1
    bool plain_ready = false;
    PlainBlocks pblk;            // batch width 1 on the block schedule: a source per thread block
    unsigned long long* d_pnext = nullptr;   // [4] work-list counter, then the kernel's stats
    gbbc_options opt;
    std::string err;
    std::vector<std::pair<void*, size_t>> allocs;
    size_t bytes = 0;
    gbbc_stats stats;
    cudaStream_t last_stream = nullptr;
    // learned direction policy (FP16 copy of the network) and per-graph stats
    void* d_policy = nullptr;
    std::vector<long long> graph_max_deg;
    long long* d_graph_max_deg = nullptr;
    long long* d_goff = nullptr;
    void* d_grouping = nullptr;      // FP16 copy of the source-grouping network
    // block-per-batch schedule
    BlockSlots blk;
    BlockBatch* d_bb = nullptr;
    long long d_bb_cap = 0;
    int32_t* d_bsrc = nullptr;
    long long d_bsrc_cap = 0;
    unsigned* d_next = nullptr;
    unsigned long long* d_bstats = nullptr;
    int tuned_schedule = 0;  // autotuner's choice (0: not tuned yet)
    // autotuning of the grid schedule's batch width, heavy-row threshold and
    // level loop (options left automatic)
    bool auto_width = false, auto_heavy = false;
    bool tuned_device = false;       // the persistent kernel runs the grid schedule
    bool tuned = false;              // the trials have run
    int cap_heavy_degree = 1024;     // the slots' heavy-row capacities are sized for this threshold
    // tracing (GBBC_TRACE)
    std::vector<gbbc_level_trace> trace;
    gbbc_kernel_profile prof[5];
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::atomic<long long> batch_counter{0};
    std::recursive_mutex mtx;        // allocation, error text and shared flags under concurrent batches
    // extra workers of the grid schedule: concurrent batches, each on its own
    // stream with its own slot and fixed-point BC accumulator
    struct Worker {
        Slot slot;
        u64* bc = nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        gbbc_stats stats;
    };
    std::vector<Worker> workers;
    cudaEvent_t ev_start = nullptr;
    // persistent grid schedule: device copies of the slots, their control
    // words and level boundaries, the launch's control block and wide list
    Slot* p_slots = nullptr;
    PCtl* p_ctl = nullptr;
    long long* p_lev = nullptr;
    int p_lev_rows = 0;
    PGlobal* p_glob = nullptr;
    int32_t* p_wide = nullptr;
    long long p_wide_cap = 0;
    int p_blocks = 0;                // cooperative grid (0: not yet asked)
    bool p_dirty = false;            // a launch stopped early: heavy-row accumulators may hold partial sums
    cudaEvent_t p_ev[2] = {nullptr, nullptr};  // around each persistent launch
    // kept per-source state of the last bc_compute
    int32_t* k_dist = nullptr;
    uint64_t* k_sigma = nullptr;
    uint8_t* k_ovf = nullptr;
    long long k_count = 0;
    // partitioned method (bc_partition): the parts, the intra-part and the
    // border-edge CSRs, the border nodes and their matrices, and the border
    // arrays of one batch
    struct Part {
        int32_t P = 0;                  // parts (0: not partitioned)
        int32_t* part = nullptr;        // [n] part of each vertex
        int32_t* in_rp = nullptr;       // [n + 1] intra-part CSR (border edges removed)
        int32_t* in_col = nullptr;
        long long in_nnz = 0;
        int32_t* cut_rp = nullptr;      // [n + 1] border edges only
        int32_t* cut_col = nullptr;
        long long cut_nnz = 0;
        long long nbt = 0;              // border nodes
        int32_t* border = nullptr;      // [nbt] vertex of each border node (by part, then id)
        int32_t* bidx = nullptr;        // [n] border index of each vertex, or -1
        int32_t* bpart = nullptr;       // [nbt] part of each border node
        long long* boff = nullptr;      // [P + 1] first border index of each part
        long long* moff = nullptr;      // [P + 1] first entry of each part's matrix block
        std::vector<long long> h_boff, h_moff;
        int32_t* BM = nullptr;          // border matrices: shortest distances inside the part
        PartWide SM;                    // sigma matrices: shortest-path counts inside the part
        int32_t* D = nullptr;           // [nbt][64] refined distances of a batch
        int32_t* D1 = nullptr;          // [nbt][64] Step 1 distances
        PartWide S1, A, Sig;            // [nbt][64] Step 1 sigma, arrivals, sigma
        int* changed = nullptr;
        int32_t* lane_b = nullptr;      // [64] border index of each lane's source
        long long sweeps = 0;           // refinement sweeps of the last bc_compute_partitioned
        // asynchronous backward: per-(vertex, lane) distances, the per-(part,
        // level) waits, the parts' progress, error word and group barriers
        int32_t* dist = nullptr;        // [n][64]
        unsigned* need = nullptr;       // [P][n + 1]
        int* done = nullptr;            // [P]
        unsigned* ctl = nullptr;        // [2 + 2P]
        long long* off = nullptr;       // [n + 2] level boundaries of the batch
        int blocks = 0;                 // cooperative grid of the backward
        long long waits = 0;            // cross-part waits of the last bc_compute_partitioned
    } pt;
};

namespace {

// Detail of the last error of a create call on this thread (the handle of
// a failed create is released, so its message is kept here).
thread_local std::string tl_create_err;

gbbc_status fail(gbbc_graph* g, gbbc_status st, const char* fmt, ...) {
    if (g) {
        std::lock_guard<std::recursive_mutex> lk(g->mtx);
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        g->err = buf;
    }
    return st;
}

void release_failed(gbbc_graph* g, gbbc_status r) {
    tl_create_err = g->err.empty() ? bc_status_string(r) : g->err;
    bc_graph_destroy(g);
}

#define CK(g, call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail((g), GBBC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                         \
    } while (0)

#define CKS(call)                          \
    do {                                   \
        gbbc_status s_ = (call);           \
        if (s_ != GBBC_OK) return s_;      \
    } while (0)

// Device memory comes from one stream-ordered pool per device, shared by the
// library's handles and never shrunk by itself (release threshold: all), so a
// handle created after another was destroyed finds its slots' memory ready;
// bc_release_memory gives the unused part back.  A pool allocation is made on
// the handle's allocation stream and synchronised, so every stream may use it;
// a free first synchronises the device (as cudaFree does).
std::mutex g_pool_mtx;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mtx);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

// Free device memory plus what the library's pool holds unused.
size_t avail_bytes(int dev) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaMemPool_t pool = device_pool(dev);
    if (pool) {
        uint64_t reserved = 0, used = 0;
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
        if (reserved > used) free_b += (size_t)(reserved - used);
    }
    return free_b;
}

gbbc_status dalloc(gbbc_graph* g, void** p, size_t bytes) {
    std::lock_guard<std::recursive_mutex> lk(g->mtx);
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (g->opt.mem_limit_bytes > 0 && g->bytes + bytes > (size_t)g->opt.mem_limit_bytes)
        return fail(g, GBBC_ERR_OOM, "allocation of %zu bytes exceeds mem_limit_bytes=%lld (held %zu)", bytes,
                    (long long)g->opt.mem_limit_bytes, g->bytes);
    cudaMemPool_t pool = g->ast ? device_pool(g->device) : nullptr;
    cudaError_t e;
    if (pool) {
        e = cudaMallocFromPoolAsync(p, bytes, pool, g->ast);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->ast);
    } else {
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(g, GBBC_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    g->allocs.push_back({*p, bytes});
    g->bytes += bytes;
    return GBBC_OK;
}

template <class T>
gbbc_status dalloc_t(gbbc_graph* g, T** p, size_t count) {
    return dalloc(g, (void**)p, count * sizeof(T));
}

void dfree(gbbc_graph* g, void* p) {
    if (!p) return;
    std::lock_guard<std::recursive_mutex> lk(g->mtx);
    for (size_t i = 0; i < g->allocs.size(); ++i)
        if (g->allocs[i].first == p) {
            g->bytes -= g->allocs[i].second;
            g->allocs.erase(g->allocs.begin() + i);
            break;
        }
    if (g->ast && device_pool(g->device)) {
        cudaDeviceSynchronize();
        cudaFreeAsync(p, g->ast);
    } else {
        cudaFree(p);
    }
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from a host or device pointer to device memory.
gbbc_status to_device(gbbc_graph* g, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return GBBC_OK;
    CK(g, cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          st));
    return GBBC_OK;
}

// Copy `bytes` of a host or device pointer into a host vector.
template <class T>
gbbc_status to_host(gbbc_graph* g, std::vector<T>& out, const T* src, size_t count, cudaStream_t st) {
    out.resize(count);
    if (count == 0) return GBBC_OK;
    if (is_device_ptr(src)) {
        CK(g, cudaMemcpyAsync(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, st));
        CK(g, cudaStreamSynchronize(st));
    } else {
        std::memcpy(out.data(), src, count * sizeof(T));
    }
    return GBBC_OK;
}

gbbc_options default_options() {
    gbbc_options o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(gbbc_options);
    o.batch_width = 0;
    o.policy = GBBC_POLICY_AUTO;
    o.validate = 0;
    o.timeout_spins = 0;
    o.flags = 0;
    o.heavy_degree = 0;
    o.mem_limit_bytes = 0;
    return o;
}

gbbc_status read_options(gbbc_graph* g, const gbbc_options* opt) {
    g->opt = default_options();
    if (opt) {
        if (opt->struct_size < offsetof(gbbc_options, heavy_degree) || opt->struct_size > sizeof(gbbc_options))
            return fail(g, GBBC_ERR_INVALID, "gbbc_options.struct_size %u not supported", opt->struct_size);
        std::memcpy(&g->opt, opt, opt->struct_size);
        g->opt.struct_size = sizeof(gbbc_options);
    }
    const gbbc_options& o = g->opt;
    if (!(o.batch_width == 0 || o.batch_width == 1 || o.batch_width == 32 || o.batch_width == 64))
        return fail(g, GBBC_ERR_INVALID, "batch_width must be 0, 1, 32 or 64 (got %d)", o.batch_width);
    if (o.policy < GBBC_POLICY_AUTO || o.policy > GBBC_POLICY_PULL)
        return fail(g, GBBC_ERR_INVALID, "unknown policy %d", o.policy);
    if (o.heavy_degree < 0) return fail(g, GBBC_ERR_INVALID, "heavy_degree must be >= 0");
    if (o.schedule < GBBC_SCHEDULE_AUTO || o.schedule > GBBC_SCHEDULE_PAIR)
        return fail(g, GBBC_ERR_INVALID, "unknown schedule %d", o.schedule);
    if (o.streams < 0 || o.streams > 16) return fail(g, GBBC_ERR_INVALID, "streams must be in [0, 16]");
    g->auto_width = g->opt.batch_width == 0;
    g->auto_heavy = g->opt.heavy_degree == 0;
    if (g->opt.heavy_degree == 0) g->opt.heavy_degree = 1024;
    if (g->opt.heavy_degree < 32) g->opt.heavy_degree = 32;
    // the smallest threshold the autotuner may try sizes the heavy-row lists
    g->cap_heavy_degree = g->auto_heavy ? 512 : g->opt.heavy_degree;
    return GBBC_OK;
}

gbbc_status init_device(gbbc_graph* g) {
    CK(g, cudaGetDevice(&g->device));
    CK(g, cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device));
    CK(g, cudaStreamCreateWithFlags(&g->ast, cudaStreamNonBlocking));
    return GBBC_OK;
}

// CSR bounds on the host copy of row_ptr (before col is read).
gbbc_status check_row_ptr(gbbc_graph* g) {
    const std::vector<int32_t>& rp = g->h_row_ptr;
    if (rp[0] != 0) return fail(g, GBBC_ERR_INVALID, "row_ptr[0] = %d, expected 0", rp[0]);
    if ((long long)rp[g->n] != g->nnz)
        return fail(g, GBBC_ERR_INVALID, "row_ptr[n] = %d differs from nnz = %lld", rp[g->n], g->nnz);
    for (int32_t v = 0; v < g->n; ++v)
        if (rp[v + 1] < rp[v]) return fail(g, GBBC_ERR_INVALID, "row_ptr decreases at vertex %d", v);
    return GBBC_OK;
}

// Optional full structure check on the device.
gbbc_status check_graph(gbbc_graph* g, cudaStream_t st) {
    if (!g->opt.validate || g->n == 0) return GBBC_OK;
    int32_t* d_flags = nullptr;
    CKS(dalloc_t(g, &d_flags, 1));
    CK(g, cudaMemsetAsync(d_flags, 0, sizeof(int32_t), st));
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    launch_validate(c, d_flags, st);
    g->stats.kernel_launches++;
    CK(g, cudaGetLastError());
    int32_t flags = 0;
    CK(g, cudaMemcpyAsync(&flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    dfree(g, d_flags);
    if (flags) {
        std::string why;
        if (flags & 1) why += " row_ptr-out-of-range";
        if (flags & 2) why += " col-out-of-range";
        if (flags & 4) why += " self-loop";
        if (flags & 8) why += " unsorted-or-duplicate-row";
        if (flags & 16) why += " asymmetric";
        return fail(g, GBBC_ERR_INVALID, "CSR validation failed:%s", why.c_str());
    }
    return GBBC_OK;
}

gbbc_status alloc_slot_into(gbbc_graph* g, Slot& s) {
    size_t n = (size_t)std::max<int32_t>(g->n, 1);
    s.n = g->n;
    long long qcap = (long long)n * kLanes + kLanes;
    if (qcap > 0x7fffffffLL) qcap = 0x7fffffffLL;
    s.qcap = qcap;
    CKS(dalloc_t(g, &s.vis, n));
    CKS(dalloc_t(g, &s.nx, n));
    CKS(dalloc_t(g, &s.ovf, n));
    CKS(dalloc_t(g, &s.F, 2 * n));
    CKS(dalloc_t(g, &s.sigma, n * kLanes));
    CKS(dalloc_t(g, &s.psi, n * kLanes));
    CKS(dalloc_t(g, &s.qv, (size_t)qcap));
    CKS(dalloc_t(g, &s.qm, (size_t)qcap));
    CKS(dalloc_t(g, &s.heavy, n));
    CKS(dalloc_t(g, &s.medium, n));
    // heavy rows: exact bounds from the degrees (a row appears at most once per step)
    long long hcap = 1, tcap = 1;
    for (int32_t v = 0; v < g->n; ++v) {
        long long d = (long long)g->h_row_ptr[v + 1] - g->h_row_ptr[v];
        if (d > g->cap_heavy_degree) {
            hcap += 1;
            tcap += (d + kChunk - 1) / kChunk;
        }
    }
    s.hcap = hcap;
    s.tcap = tcap;
    CKS(dalloc_t(g, &s.hentry, (size_t)hcap));
    CKS(dalloc_t(g, &s.hacc, (size_t)hcap * kLanes * 2));
    CKS(dalloc_t(g, &s.hcarry, (size_t)hcap));
    CKS(dalloc_t(g, &s.tasks, (size_t)tcap));
    CK(g, cudaMemset(s.hacc, 0, (size_t)hcap * kLanes * 2 * sizeof(u64)));
    CK(g, cudaMemset(s.hcarry, 0, (size_t)hcap * sizeof(u64)));
    CKS(dalloc_t(g, &s.ctr, 1));
    CKS(dalloc_t(g, &s.d_src, kLanes));
    if (!s.hctr) CK(g, cudaMallocHost((void**)&s.hctr, sizeof(Counters)));
    CK(g, cudaMemset(s.nx, 0, n * sizeof(u64)));
    return GBBC_OK;
}

gbbc_status alloc_slot(gbbc_graph* g) {
    if (g->slot_ready) return GBBC_OK;
    CKS(alloc_slot_into(g, g->slot));
    g->slot_ready = true;
    return GBBC_OK;
}

gbbc_status alloc_wide(gbbc_graph* g, Slot& s) {
    if (s.sN) return GBBC_OK;
    size_t n = (size_t)std::max<int32_t>(g->n, 1);
    CKS(dalloc_t(g, &s.sN, n * kLanes));
    CKS(dalloc_t(g, &s.sX, n * kLanes));
    CKS(dalloc_t(g, &s.psi_e, n * kLanes));
    return GBBC_OK;
}

int effective_policy(const gbbc_graph* g) {
    int p = g->opt.policy;
    if (p == GBBC_POLICY_AUTO) return g->d_policy ? GBBC_POLICY_LEARNED : GBBC_POLICY_BEAMER;
    return p;
}

struct BatchDesc {
    int32_t gi;         // graph index
    int32_t lo, hi;     // vertex range of the graph the sources belong to
    long long first;    // position of the first source in the call's list
    int nsrc;
    int32_t src[kLanes];
};

enum ProfKind { PK_PUSH = 0, PK_PULL = 1, PK_GATHER = 2, PK_BWD = 3, PK_INIT = 4, PK_COUNT = 5 };
const char* kProfNames[PK_COUNT] = {"push", "pull", "gather", "backward", "init"};

// CUDA events around traced steps, resolved at the next host sync.
struct Timed {
    int kind;
    cudaEvent_t a, b;
    long long rec;   // trace record index, or -1
    int field;       // 0 push, 1 pull, 2 gather, 3 backward, -1 none
    double bytes;
    bool count;      // counts in the profile (an undone probe step does not)
};

cudaEvent_t ev_get(gbbc_graph* g) {
    if (g->ev_used == g->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g->ev_pool.push_back(e);
    }
    return g->ev_pool[g->ev_used++];
}

gbbc_status resolve(gbbc_graph* g, std::vector<Timed>& pend) {
    for (const Timed& t : pend) {
        float ms = 0.f;
        CK(g, cudaEventElapsedTime(&ms, t.a, t.b));
        if (t.count) {
            g->prof[t.kind].launches += 1;
            g->prof[t.kind].ms += ms;
            g->prof[t.kind].bytes += t.bytes;
        }
        if (t.rec >= 0 && t.rec < (long long)g->trace.size()) {
            gbbc_level_trace& r = g->trace[t.rec];
            if (t.field == 0) r.ms_push = ms;
            if (t.field == 1) r.ms_pull = ms;
            if (t.field == 2) r.ms_gather = ms;
            if (t.field == 3) r.ms_backward = ms;
        }
    }
    pend.clear();
    g->ev_used = 0;
    return GBBC_OK;
}

inline double dmin(double a, double b) { return a < b ? a : b; }

gbbc_status run_batch_once(gbbc_graph* g, const BatchDesc& b, cudaStream_t st, bool wide, bool* need_wide, Slot& s,
                           u64* bc, gbbc_stats& stats);

// A batch runs in the narrow sigma format unless the handle has met a count
// >= 2^64 before; if the narrow forward meets one, the batch is rerun in the
// wide format (which keeps sigma mod 2^64 as well) and later batches start
// wide.  The backward only runs once, on the final forward.
// One batch in the grid schedule on slot s and stream st, BC added into bc
// (the handle's, or a worker's accumulator), counters into stats.
gbbc_status run_batch(gbbc_graph* g, const BatchDesc& b, cudaStream_t st, Slot& s, u64* bc, gbbc_stats& stats) {
    bool wide;
    {
        std::lock_guard<std::recursive_mutex> lk(g->mtx);
        wide = g->wide_graph[b.gi] != 0;
    }
    if (wide) CKS(alloc_wide(g, s));
    bool need_wide = false;
    CKS(run_batch_once(g, b, st, wide, &need_wide, s, bc, stats));
    if (need_wide) {
        CKS(alloc_wide(g, s));
        {
            std::lock_guard<std::recursive_mutex> lk(g->mtx);
            g->wide_graph[b.gi] = 1;  // later batches of this graph start wide
        }
        wide = true;
        CKS(run_batch_once(g, b, st, true, &need_wide, s, bc, stats));
    }
    if (wide) stats.wide_batches++;
    return GBBC_OK;
}

gbbc_status run_batch(gbbc_graph* g, const BatchDesc& b, cudaStream_t st) {
    return run_batch(g, b, st, g->slot, g->d_bc, g->stats);
}

gbbc_status run_batch_once(gbbc_graph* g, const BatchDesc& b, cudaStream_t st, bool wide, bool* need_wide, Slot& s,
                           u64* bc, gbbc_stats& stats) {
    *need_wide = false;
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    const int32_t lo = b.lo, hi = b.hi;
    const size_t rn = (size_t)(hi - lo);
    const int hd = g->opt.heavy_degree;
    const bool tr = (g->opt.flags & GBBC_TRACE) != 0;
    const bool both = tr && (g->opt.flags & GBBC_TRACE_BOTH) != 0;
    const int policy = effective_policy(g);
    std::vector<Timed> pend;
    const long long batch_id = g->batch_counter++;
    auto mark = [&](cudaEvent_t* e) -> gbbc_status {
        *e = nullptr;
        if (!tr) return GBBC_OK;
        *e = ev_get(g);
        if (!*e) return fail(g, GBBC_ERR_CUDA, "cudaEventCreate failed");
        CK(g, cudaEventRecord(*e, st));
        return GBBC_OK;
    };
    cudaEvent_t e0, e1;
    CKS(mark(&e0));
    // ---- batch init (vertex range only) ----
    CK(g, cudaMemsetAsync(s.vis + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.nx + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.ovf + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.F + lo, 0xff, rn * sizeof(MaskTag), st));
    CK(g, cudaMemsetAsync(s.F + s.n + lo, 0xff, rn * sizeof(MaskTag), st));
    CK(g, cudaMemcpyAsync(s.d_src, b.src, b.nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // distinct sources form the level-0 queue
    std::vector<int32_t> distinct(b.src, b.src + b.nsrc);
    std::sort(distinct.begin(), distinct.end());
    distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
    const long long nq0 = (long long)distinct.size();
    long long deg0 = 0, lane_deg0 = 0;
    for (int32_t v : distinct) deg0 += g->h_row_ptr[v + 1] - g->h_row_ptr[v];
    for (int j = 0; j < b.nsrc; ++j) lane_deg0 += g->h_row_ptr[b.src[j] + 1] - g->h_row_ptr[b.src[j]];
    const u64 lanes0 = (b.nsrc == 64) ? ~0ull : ((1ull << b.nsrc) - 1ull);
    // the counters describe level 0 for the first decision
    std::memset(s.hctr, 0, sizeof(Counters));
    s.hctr->qtail = (unsigned long long)nq0;
    s.hctr->edge_sum = (unsigned long long)deg0;
    s.hctr->lane_sum = (unsigned long long)b.nsrc;
    s.hctr->lanes = lanes0;
    CK(g, cudaMemcpyAsync(s.ctr, s.hctr, sizeof(Counters), cudaMemcpyHostToDevice, st));
    launch_seed(s, b.nsrc, st);
    const long long nnz_range = (long long)g->h_row_ptr[hi] - g->h_row_ptr[lo];
    const long long n_range = hi - lo;
    const double nr = (double)n_range;
    const long long max_deg = g->graph_max_deg[b.gi];
    launch_decide(s, 0, 0, policy, g->d_policy, n_range, nnz_range, max_deg, st);
    stats.kernel_launches += 2;
    CK(g, cudaGetLastError());
    CKS(mark(&e1));
    if (tr) pend.push_back({PK_INIT, e0, e1, -1, -1, (double)rn * (8 * 3 + 32), true});
    CK(g, cudaMemcpyAsync(s.hctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));

    // per-level sizes: entries, degree sum, (vertex, lane) pairs, pairs * degree
    std::vector<long long> off = {0, nq0}, nv = {nq0}, ne = {deg0}, nl = {b.nsrc}, nle = {lane_deg0};
    std::vector<long long> trace_rec;  // trace record of each level's step
    u64 lanes = lanes0;
    int level = 0;
    const size_t disc_off = offsetof(Counters, heavy), disc_bytes = offsetof(Counters, err) - disc_off;
    const size_t gath_off = offsetof(Counters, lane_sum), gath_bytes = offsetof(Counters, medium) - gath_off;
    for (;;) {
        const long long q_lo = off[level], q_hi = off[level + 1];
        const long long m_f = ne[level];
        const bool pull = s.hctr->dir != 0;
        long long rec = -1;
        if (tr) {
            gbbc_level_trace r;
            std::memset(&r, 0, sizeof(r));
            r.batch = (int32_t)batch_id;
            r.level = level;
            r.direction = pull ? 1 : 0;
            r.active_lanes = __builtin_popcountll(lanes);
            r.n_range = n_range;
            r.nnz_range = nnz_range;
            r.frontier_vertices = nv[level];
            r.frontier_edges = ne[level];
            r.frontier_lanes = nl[level];
            long long vl = 0, vle = 0;
            for (int i = 0; i <= level; ++i) {
                vl += nl[i];
                vle += nle[i];
            }
            r.visited_lanes = vl;
            r.visited_lane_edges = vle;
            r.max_degree = max_deg;
            for (int i = 0; i < 6; ++i) r.features[i] = s.hctr->feat[i];
            r.ms_push = r.ms_pull = r.ms_gather = r.ms_backward = -1.f;
            rec = (long long)g->trace.size();
            g->trace.push_back(r);
            trace_rec.push_back(rec);
        }
        // probe the direction not taken, then undo it (GBBC_TRACE_BOTH)
        if (both) {
            CK(g, cudaMemsetAsync((char*)s.ctr + disc_off, 0, disc_bytes, st));
            CKS(mark(&e0));
            if (!pull) launch_pull(c, s, lo, hi, lanes, level, hd, g->nsm, st);
            else launch_push(c, s, q_lo, q_hi, level, hd, g->nsm, st);
            CKS(mark(&e1));
            pend.push_back({pull ? PK_PUSH : PK_PULL, e0, e1, rec, pull ? 0 : 1, 0.0, false});
            CK(g, cudaGetLastError());
            Counters probe;
            CK(g, cudaMemcpyAsync(&probe, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            CK(g, cudaStreamSynchronize(st));
            launch_undo(s, q_hi, (long long)probe.qtail, st);
            unsigned long long rewind = (unsigned long long)q_hi;
            CK(g, cudaMemcpyAsync(&s.ctr->qtail, &rewind, sizeof(rewind), cudaMemcpyHostToDevice, st));
            CK(g, cudaStreamSynchronize(st));
        }
        CK(g, cudaMemsetAsync((char*)s.ctr + disc_off, 0, disc_bytes, st));
        CKS(mark(&e0));
        if (pull) {
            launch_pull(c, s, lo, hi, lanes, level, hd, g->nsm, st);
            stats.levels_pull++;
            stats.kernel_launches += 3;
        } else {
            launch_push(c, s, q_lo, q_hi, level, hd, g->nsm, st);
            stats.levels_push++;
            stats.kernel_launches += 2;
        }
        cudaEvent_t d1;
        CKS(mark(&d1));
        // gather of the new level: its range ends at the device's qtail
        CK(g, cudaMemsetAsync((char*)s.ctr + gath_off, 0, gath_bytes, st));
        launch_fwd_gather(c, s, q_hi, level, hd, g->nsm, st, wide);
        cudaEvent_t g1;
        CKS(mark(&g1));
        launch_decide(s, q_hi, level + 1, policy, g->d_policy, n_range, nnz_range, max_deg, st);
        stats.kernel_launches += wide ? 3 : 4;
        CK(g, cudaGetLastError());
        CK(g, cudaMemcpyAsync(s.hctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(g, cudaStreamSynchronize(st));
        if (s.hctr->err)
            return fail(g, GBBC_ERR_CAPACITY, "queue capacity exceeded in the forward phase (flags %u)",
                        s.hctr->err);
        const long long new_hi = (long long)s.hctr->qtail;
        const long long new_n = new_hi - q_hi, new_e = (long long)s.hctr->edge_sum;
        const long long new_l = (long long)s.hctr->lane_sum, new_le = (long long)s.hctr->lane_esum;
        if (tr) {
            gbbc_level_trace& r = g->trace[rec];
            r.next_vertices = new_n;
            r.next_edges = new_e;
            r.scanned_edges = pull ? (long long)s.hctr->scanned : 0;
            double dbytes = pull ? 8.0 * nr + 4.0 * (double)s.hctr->scanned +
                                       16.0 * dmin((double)s.hctr->scanned, nr) + 20.0 * (double)new_n
                                 : 20.0 * (double)nv[level] + 4.0 * (double)m_f + 8.0 * dmin((double)m_f, nr) +
                                       20.0 * (double)new_n;
            pend.push_back({pull ? PK_PULL : PK_PUSH, e0, d1, rec, pull ? 1 : 0, dbytes, true});
            double gbytes = 68.0 * (double)new_n + 4.0 * (double)new_e + 16.0 * dmin((double)new_e, nr) +
                            8.0 * (double)nl[level] + 8.0 * (double)new_l;
            if (new_n > 0) pend.push_back({PK_GATHER, d1, g1, rec, 2, gbytes, true});
            CKS(resolve(g, pend));
        }
        if (new_n == 0) break;  // no vertex reached at level+1
        if (s.hctr->carry && !wide) break;  // a lane passed 2^64: stop here, rerun wide
        off.push_back(new_hi);
        nv.push_back(new_n);
        ne.push_back(new_e);
        nl.push_back(new_l);
        nle.push_back(new_le);
        lanes = s.hctr->lanes;
        ++level;
    }
    const int nlev = level + 1;  // levels 0 .. level
    stats.levels_fwd += nlev;
    if (s.hctr->carry && !wide) {  // rerun this batch in the wide format
        if (tr) CKS(resolve(g, pend));
        *need_wide = true;
        g->batch_counter--;
        return GBBC_OK;
    }
    // ---- kept state for parity checks ----
    if (g->k_dist) {
        for (int l = 0; l < nlev; ++l)
            launch_keep_dist(s, off[l], off[l + 1], l, g->k_dist, g->n, b.first, b.nsrc, st);
        launch_keep_sigma(s, lo, hi, g->k_sigma, g->k_ovf, g->n, b.first, b.nsrc, st);
        stats.kernel_launches += nlev + 1;
        CK(g, cudaGetLastError());
    }
    // ---- backward phase: levels nlev-1 .. 1 ----
    for (int l = nlev - 1; l >= 1; --l) {
        CK(g, cudaMemsetAsync(&s.ctr->heavy, 0, 2 * sizeof(unsigned long long), st));  // heavy, tasks
        CKS(mark(&e0));
        launch_bwd(c, s, bc, off[l], off[l + 1], l, hd, g->nsm, st, wide);
        CKS(mark(&e1));
        stats.kernel_launches += 3;
        if (tr) {
            double succ_lanes = (l + 1 < nlev) ? (double)nl[l + 1] : 0.0;
            double bytes = 68.0 * (double)nv[l] + 4.0 * (double)ne[l] + 16.0 * dmin((double)ne[l], nr) +
                           8.0 * succ_lanes + 16.0 * (double)nl[l];
            long long rec = (l - 1 < (int)trace_rec.size()) ? trace_rec[l - 1] : -1;
            pend.push_back({PK_BWD, e0, e1, rec, 3, bytes, true});
        }
    }
    CK(g, cudaGetLastError());
    if (tr) {
        CK(g, cudaStreamSynchronize(st));
        CKS(resolve(g, pend));
    }
    stats.batches++;
    stats.sources += b.nsrc;
    return GBBC_OK;
}

gbbc_status alloc_plain(gbbc_graph* g) {
    if (g->plain_ready) return GBBC_OK;
    PlainState& p = g->plain;
    size_t n = (size_t)std::max<int32_t>(g->n, 1);
    p.n = g->n;
    CKS(dalloc_t(g, &p.dist, n));
    CKS(dalloc_t(g, &p.sigma, n));
    CKS(dalloc_t(g, &p.psi, n));
    CKS(dalloc_t(g, &p.queue, n));
    CKS(dalloc_t(g, &p.heavy, n));
    CKS(dalloc_t(g, &p.ctr, 1));
    if (!g->slot.hctr) CK(g, cudaMallocHost((void**)&g->slot.hctr, sizeof(Counters)));
    g->plain_ready = true;
    return GBBC_OK;
}

// One source through the plain path (level-synchronous, per-level kernels).
gbbc_status run_plain(gbbc_graph* g, int32_t src, int32_t lo, int32_t hi, long long index, cudaStream_t st) {
    PlainState& p = g->plain;
    Counters* hc = g->slot.hctr;
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    const size_t rn = (size_t)(hi - lo);
    const int hd = g->opt.heavy_degree;
    CK(g, cudaMemsetAsync(p.dist + lo, 0xff, rn * sizeof(int32_t), st));
    CK(g, cudaMemsetAsync(p.sigma + lo, 0, rn * sizeof(u64), st));
    std::memset(hc, 0, sizeof(Counters));
    hc->qtail = 1;
    CK(g, cudaMemcpyAsync(p.ctr, hc, sizeof(Counters), cudaMemcpyHostToDevice, st));
    launch_plain_seed(p, src, st);
    g->stats.kernel_launches++;
    std::vector<long long> off = {0, 1};
    int level = 0;
    for (;;) {
        CK(g, cudaMemsetAsync(&p.ctr->heavy, 0, sizeof(unsigned long long), st));
        launch_plain_fwd(c, p, off[level], off[level + 1], level, hd, g->nsm, st);
        g->stats.kernel_launches += 2;
        g->stats.levels_push++;
        CK(g, cudaGetLastError());
        CK(g, cudaMemcpyAsync(hc, p.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(g, cudaStreamSynchronize(st));
        long long nh = (long long)hc->qtail;
        if (nh == off[level + 1]) break;
        off.push_back(nh);
        ++level;
    }
    const int nlev = level + 1;
    g->stats.levels_fwd += nlev;
    if (hc->carry)
        return fail(g, GBBC_ERR_CAPACITY,
                    "plain path (batch width 1): a shortest-path count reached 2^64; use batch width 32 or 64");
    if (g->k_dist) {
        size_t at = (size_t)index * (size_t)g->n + (size_t)lo;
        CK(g, cudaMemcpyAsync(g->k_dist + at, p.dist + lo, rn * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
        CK(g, cudaMemcpyAsync(g->k_sigma + at, p.sigma + lo, rn * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    }
    for (int l = nlev - 1; l >= 1; --l) {
        CK(g, cudaMemsetAsync(&p.ctr->heavy, 0, sizeof(unsigned long long), st));
        launch_plain_bwd(c, p, g->d_bc, off[l], off[l + 1], l, hd, g->nsm, st);
        g->stats.kernel_launches += 2;
    }
    CK(g, cudaGetLastError());
    g->stats.batches++;
    g->stats.sources++;
    return GBBC_OK;
}

// Batch width 1 on the block schedule: up to `want` thread blocks, each with
// its own per-source arrays (28n + 8 bytes per block), as many as fit in half
// of the free memory (and mem_limit_bytes).
gbbc_status alloc_plain_blocks(gbbc_graph* g, int want) {
    PlainBlocks& B = g->pblk;
    if (B.count >= want) return GBBC_OK;
    for (void* q : {(void*)B.dist, (void*)B.sigma, (void*)B.psi, (void*)B.queue, (void*)B.lev, (void*)B.ctr})
        dfree(g, q);
    B = PlainBlocks();
    const size_t n = (size_t)std::max<int32_t>(g->n, 1);
    if (!g->d_pnext) CKS(dalloc_t(g, &g->d_pnext, 4));
    const double per_block = (double)n * 28.0 + 8.0 + sizeof(Counters);
    double budget = 0.5 * (double)avail_bytes(g->device);
    if (g->opt.mem_limit_bytes > 0) budget = std::min(budget, (double)g->opt.mem_limit_bytes - (double)g->bytes);
    const int count = (int)std::min<double>((double)want, std::floor(budget / per_block));
    if (count < 1) return fail(g, GBBC_ERR_OOM, "no room for one plain-path block state (%.0f bytes)", per_block);
    const size_t c = (size_t)count;
    B.n = g->n;
    CKS(dalloc_t(g, &B.dist, c * n));
    CKS(dalloc_t(g, &B.sigma, c * n));
    CKS(dalloc_t(g, &B.psi, c * n));
    CKS(dalloc_t(g, &B.queue, c * n));
    CKS(dalloc_t(g, &B.lev, c * (n + 2)));
    CKS(dalloc_t(g, &B.ctr, c));
    B.count = count;
    return GBBC_OK;
}

// Batch width 1, block schedule: every source runs whole on one thread block
// (McLaughlin and Bader's coarse-grained source parallelism), many blocks at
// once, one launch per call.  BC bits equal those of the other paths.
gbbc_status run_plain_blocks(gbbc_graph* g, const std::vector<int32_t>& gsrc, cudaStream_t st) {
    const long long k = (long long)gsrc.size();
    if (k == 0) return GBBC_OK;
    const int bps = plain_blocks_per_sm();
    if (bps < 1) return fail(g, GBBC_ERR_CUDA, "plain block kernel: no resident block");
    if (g->d_bsrc_cap < k) {
        dfree(g, g->d_bsrc);
        CKS(dalloc_t(g, &g->d_bsrc, (size_t)k));
        g->d_bsrc_cap = k;
    }
    CKS(alloc_plain_blocks(g, (int)std::min<long long>(k, (long long)g->nsm * bps)));
    PlainBlocks& B = g->pblk;
    const size_t n = (size_t)std::max<int32_t>(g->n, 1), c = (size_t)B.count;
    CK(g, cudaMemcpyAsync(g->d_bsrc, gsrc.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemsetAsync(B.dist, 0xff, c * n * sizeof(int32_t), st));
    CK(g, cudaMemsetAsync(B.sigma, 0, c * n * sizeof(u64), st));
    CK(g, cudaMemsetAsync(B.ctr, 0, c * sizeof(Counters), st));
    CK(g, cudaMemsetAsync(g->d_pnext, 0, 4 * sizeof(unsigned long long), st));
    Csr cs{g->n, g->nnz, g->d_row_ptr, g->d_col};
    CK(g, launch_plain_blocks(cs, B, g->d_bsrc, k, g->d_pnext, g->d_bc, g->d_pnext + 1, st));
    g->stats.kernel_launches++;
    unsigned long long h[4];
    CK(g, cudaMemcpyAsync(h, g->d_pnext, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    if ((long long)h[1] != k) return fail(g, GBBC_ERR_CUDA, "plain block kernel ran %llu of %lld sources", h[1], k);
    g->stats.batches += k;
    g->stats.sources += k;
    g->stats.levels_fwd += (long long)h[2];
    g->stats.levels_push += (long long)h[2];
    g->stats.schedule = GBBC_SCHEDULE_BLOCK;
    if (h[3] & 0xffffffffull)
        return fail(g, GBBC_ERR_CAPACITY,
                    "plain path (batch width 1): a shortest-path count reached 2^64; use batch width 32 or 64");
    return GBBC_OK;
}

gbbc_status alloc_keep(gbbc_graph* g, long long k, cudaStream_t st) {
    dfree(g, g->k_dist);
    dfree(g, g->k_sigma);
    dfree(g, g->k_ovf);
    g->k_dist = nullptr;
    g->k_sigma = nullptr;
    g->k_ovf = nullptr;
    g->k_count = 0;
    if (!(g->opt.flags & GBBC_KEEP_STATE) || k == 0) return GBBC_OK;
    size_t cells = (size_t)k * (size_t)g->n;
    CKS(dalloc_t(g, &g->k_dist, cells));
    CKS(dalloc_t(g, &g->k_sigma, cells));
    CKS(dalloc_t(g, &g->k_ovf, cells));
    launch_fill_i32(g->k_dist, (long long)cells, -1, st);
    CK(g, cudaMemsetAsync(g->k_sigma, 0, cells * sizeof(uint64_t), st));
    CK(g, cudaMemsetAsync(g->k_ovf, 0, cells, st));
    g->k_count = k;
    return GBBC_OK;
}

// ---- host-driven forward and backward of one batch over a given CSR -------
// (the partitioned method runs its BFS steps on the intra-part graph and its
// backward phase on the whole graph)

// Called by run_forward after the discovery and after the gather of each new
// level (the partitioned method injects its border seeds there).
struct FwdHooks {
    virtual gbbc_status after_discovery(int level, const Slot& s, bool wide, cudaStream_t st) = 0;
    virtual gbbc_status after_gather(int level, const Slot& s, bool wide, cudaStream_t st) = 0;
    virtual ~FwdHooks() {}
};

// Forward phase of batch b over CSR c on slot s: level l's entries end up in
// [off[l], off[l + 1]).  *carry: a count reached 2^64 in the narrow format
// (the pass stopped there; rerun wide).
gbbc_status run_forward(gbbc_graph* g, const Csr& c, const BatchDesc& b, cudaStream_t st, bool wide, Slot& s,
                        gbbc_stats& stats, std::vector<long long>& off, bool* carry, FwdHooks* hooks) {
    *carry = false;
    const int32_t lo = b.lo, hi = b.hi;
    const size_t rn = (size_t)(hi - lo);
    const int hd = g->opt.heavy_degree;
    const int policy = effective_policy(g);
    CK(g, cudaMemsetAsync(s.vis + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.nx + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.ovf + lo, 0, rn * sizeof(u64), st));
    CK(g, cudaMemsetAsync(s.F + lo, 0xff, rn * sizeof(MaskTag), st));
    CK(g, cudaMemsetAsync(s.F + s.n + lo, 0xff, rn * sizeof(MaskTag), st));
    CK(g, cudaMemcpyAsync(s.d_src, b.src, b.nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    std::vector<int32_t> distinct(b.src, b.src + b.nsrc);
    std::sort(distinct.begin(), distinct.end());
    distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
    const long long nq0 = (long long)distinct.size();
    std::memset(s.hctr, 0, sizeof(Counters));
    s.hctr->qtail = (unsigned long long)nq0;
    s.hctr->lane_sum = (unsigned long long)b.nsrc;
    s.hctr->lanes = (b.nsrc == 64) ? ~0ull : ((1ull << b.nsrc) - 1ull);
    CK(g, cudaMemcpyAsync(s.ctr, s.hctr, sizeof(Counters), cudaMemcpyHostToDevice, st));
    launch_seed(s, b.nsrc, st);
    const long long n_range = hi - lo;
    const long long nnz_range = (long long)g->h_row_ptr[hi] - g->h_row_ptr[lo];
    const long long max_deg = g->graph_max_deg[b.gi];
    launch_decide(s, 0, 0, policy, g->d_policy, n_range, nnz_range, max_deg, st);
    stats.kernel_launches += 2;
    CK(g, cudaGetLastError());
    CK(g, cudaMemcpyAsync(s.hctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    off.assign({0, nq0});
    u64 lanes = s.hctr->lanes;
    int level = 0;
    const size_t disc_off = offsetof(Counters, heavy), disc_bytes = offsetof(Counters, err) - disc_off;
    const size_t gath_off = offsetof(Counters, lane_sum), gath_bytes = offsetof(Counters, medium) - gath_off;
    for (;;) {
        const long long q_lo = off[level], q_hi = off[level + 1];
        const bool pull = s.hctr->dir != 0;
        CK(g, cudaMemsetAsync((char*)s.ctr + disc_off, 0, disc_bytes, st));
        if (pull) {
            launch_pull(c, s, lo, hi, lanes, level, hd, g->nsm, st);
            stats.levels_pull++;
        } else {
            launch_push(c, s, q_lo, q_hi, level, hd, g->nsm, st);
            stats.levels_push++;
        }
        if (hooks) CKS(hooks->after_discovery(level + 1, s, wide, st));
        CK(g, cudaMemsetAsync((char*)s.ctr + gath_off, 0, gath_bytes, st));
        launch_fwd_gather(c, s, q_hi, level, hd, g->nsm, st, wide);
        if (hooks) CKS(hooks->after_gather(level + 1, s, wide, st));
        launch_decide(s, q_hi, level + 1, policy, g->d_policy, n_range, nnz_range, max_deg, st);
        stats.kernel_launches += 7;
        CK(g, cudaGetLastError());
        CK(g, cudaMemcpyAsync(s.hctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        CK(g, cudaStreamSynchronize(st));
        if (s.hctr->err)
            return fail(g, GBBC_ERR_CAPACITY, "queue capacity exceeded in the forward phase (flags %u)", s.hctr->err);
        const long long new_hi = (long long)s.hctr->qtail;
        if (new_hi == q_hi) break;
        if (s.hctr->carry && !wide) {
            *carry = true;
            break;
        }
        off.push_back(new_hi);
        lanes = s.hctr->lanes;
        ++level;
    }
    stats.levels_fwd += level + 1;
    return GBBC_OK;
}

// Backward phase over CSR c for the levels of off (deepest first), BC into bc.
gbbc_status run_backward(gbbc_graph* g, const Csr& c, Slot& s, const std::vector<long long>& off, bool wide, u64* bc,
                         gbbc_stats& stats, cudaStream_t st) {
    const int nlev = (int)off.size() - 1;
    for (int l = nlev - 1; l >= 1; --l) {
        CK(g, cudaMemsetAsync(&s.ctr->heavy, 0, 2 * sizeof(unsigned long long), st));  // heavy, tasks
        launch_bwd(c, s, bc, off[l], off[l + 1], l, g->opt.heavy_degree, g->nsm, st, wide);
        stats.kernel_launches += 3;
    }
    CK(g, cudaGetLastError());
    return GBBC_OK;
}

// ---- the partitioned method (Sec. IV and Sec. V-A of the paper) -------------

void free_partition(gbbc_graph* g) {
    gbbc_graph::Part& q = g->pt;
    for (void* p : {(void*)q.part, (void*)q.in_rp, (void*)q.in_col, (void*)q.cut_rp, (void*)q.cut_col,
                    (void*)q.border, (void*)q.bidx, (void*)q.bpart, (void*)q.boff, (void*)q.moff, (void*)q.BM,
                    (void*)q.SM.mod, (void*)q.SM.N, (void*)q.SM.X, (void*)q.SM.big, (void*)q.D, (void*)q.D1,
                    (void*)q.S1.mod, (void*)q.S1.N, (void*)q.S1.X, (void*)q.S1.big, (void*)q.A.mod, (void*)q.A.N,
                    (void*)q.A.X, (void*)q.A.big, (void*)q.Sig.mod, (void*)q.Sig.N, (void*)q.Sig.X,
                    (void*)q.Sig.big, (void*)q.changed, (void*)q.lane_b, (void*)q.dist, (void*)q.need,
                    (void*)q.done, (void*)q.ctl, (void*)q.off})
        dfree(g, p);
    q = gbbc_graph::Part();
}

gbbc_status alloc_wide_arr(gbbc_graph* g, PartWide& w, size_t count) {
    CKS(dalloc_t(g, &w.mod, count));
    CKS(dalloc_t(g, &w.N, count));
    CKS(dalloc_t(g, &w.X, count));
    CKS(dalloc_t(g, &w.big, count));
    return GBBC_OK;
}

gbbc_status clear_wide_arr(gbbc_graph* g, const PartWide& w, size_t count, cudaStream_t st) {
    CK(g, cudaMemsetAsync(w.mod, 0, count * sizeof(u64), st));
    CK(g, cudaMemsetAsync(w.big, 0, count, st));
    return GBBC_OK;
}

// Forward of one batch over the intra-part graph, rerun wide when a count
// reaches 2^64 (later batches of the handle then start wide).
gbbc_status part_forward(gbbc_graph* g, const Csr& cin, const BatchDesc& b, cudaStream_t st, bool& wide,
                         std::vector<long long>& off, FwdHooks* hooks) {
    bool carry = false;
    if (wide) CKS(alloc_wide(g, g->slot));
    CKS(run_forward(g, cin, b, st, wide, g->slot, g->stats, off, &carry, hooks));
    if (carry) {
        CKS(alloc_wide(g, g->slot));
        wide = true;
        g->wide_graph[0] = 1;
        g->stats.wide_batches++;
        CKS(run_forward(g, cin, b, st, true, g->slot, g->stats, off, &carry, hooks));
    }
    return GBBC_OK;
}

// Step 6 seeds: inject the border nodes at their refined distances.
struct SeedHooks : FwdHooks {
    gbbc_graph* g;
    explicit SeedHooks(gbbc_graph* h) : g(h) {}
    gbbc_status after_discovery(int level, const Slot& s, bool wide, cudaStream_t st) override {
        (void)wide;
        launch_seed_inject(s, level, g->pt.border, g->pt.nbt, g->pt.D, g->pt.A, g->pt.in_rp, g->nsm, st);
        g->stats.kernel_launches++;
        return GBBC_OK;
    }
    gbbc_status after_gather(int level, const Slot& s, bool wide, cudaStream_t st) override {
        launch_seed_add(s, level, g->pt.border, g->pt.nbt, g->pt.D, g->pt.A, wide, g->nsm, st);
        g->stats.kernel_launches++;
        return GBBC_OK;
    }
};

// The asynchronous backward phase (Sec. V-B): every part walks its own
// levels on its own group of blocks and waits only where a border node's
// successor lies in another part one level deeper (bc_partition.cu).
gbbc_status part_backward_async(gbbc_graph* g, const Csr& call, const std::vector<long long>& off, bool wide,
                                cudaStream_t st) {
    gbbc_graph::Part& q = g->pt;
    const int nlev = (int)off.size() - 1;
    if (nlev < 2) return GBBC_OK;
    const int P = q.P;
    if (q.blocks == 0) {
        const int per_sm = part_backward_blocks_per_sm();
        if (per_sm < 1) return fail(g, GBBC_ERR_CUDA, "partitioned backward: occupancy query failed");
        q.blocks = per_sm * g->nsm;
        if (q.blocks < P) return fail(g, GBBC_ERR_INVALID, "partitioned backward: %d parts need %d blocks", P, P);
    }
    const size_t n = (size_t)std::max<int32_t>(g->n, 1);
    CK(g, cudaMemsetAsync(q.dist, 0xff, n * kLanes * sizeof(int32_t), st));
    for (int l = 0; l < nlev; ++l) launch_part_dist(g->slot, off[l], off[l + 1], l, q.dist, g->nsm, st);
    CK(g, cudaMemsetAsync(q.need, 0, (size_t)P * nlev * sizeof(unsigned), st));
    for (int l = 1; l < nlev; ++l)
        launch_part_need(g->slot, off[l], off[l + 1], l, nlev, q.dist, q.part, q.bidx, q.cut_rp, q.cut_col, q.need,
                         g->nsm, st);
    CK(g, cudaMemcpyAsync(q.off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st));
    launch_fill_i32(q.done, P, nlev, st);
    CK(g, cudaMemsetAsync(q.ctl, 0, (size_t)(2 + 2 * P) * sizeof(unsigned), st));
    const long long spins = g->opt.timeout_spins > 0 ? (long long)g->opt.timeout_spins : GBBC_DEFAULT_SPINS;
    CK(g, launch_part_backward(call, g->slot, q.dist, q.part, P, q.off, nlev, q.need, q.done, q.ctl, g->d_bc, spins,
                               wide, q.blocks, st));
    g->stats.kernel_launches += 2 * nlev + 1;
    unsigned hc[2] = {0u, 0u};
    CK(g, cudaMemcpyAsync(hc, q.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    if (hc[0] & 1u)
        return fail(g, GBBC_ERR_TIMEOUT,
                    "partitioned backward: a wait passed timeout_spins=%lld polls; the handle's BC is undefined until "
                    "bc_reset", spins);
    q.waits += hc[1];
    return GBBC_OK;
}

// One batch by the partitioned method: Step 1, Steps 2-5, border sigma,
// Step 6, kept state, backward over the whole graph.
gbbc_status part_batch(gbbc_graph* g, const BatchDesc& b, cudaStream_t st) {
    gbbc_graph::Part& q = g->pt;
    Csr cin{g->n, q.in_nnz, q.in_rp, q.in_col};
    Csr call{g->n, g->nnz, g->d_row_ptr, g->d_col};
    const size_t cells = (size_t)std::max<long long>(q.nbt, 1) * kLanes;
    bool wide = g->wide_graph[0] != 0;
    std::vector<long long> off;
    // Step 1: BFS inside each source's part; its border nodes' dist and sigma
    CKS(part_forward(g, cin, b, st, wide, off, nullptr));
    CK(g, cudaMemsetAsync(q.D1, 0x7f, cells * sizeof(int32_t), st));
    CKS(clear_wide_arr(g, q.S1, cells, st));
    CKS(clear_wide_arr(g, q.A, cells, st));
    CKS(clear_wide_arr(g, q.Sig, cells, st));
    for (size_t l = 0; l + 1 < off.size(); ++l)
        launch_part_extract(g->slot, off[l], off[l + 1], (int)l, wide, 1, q.bidx, q.bpart, q.boff, q.moff, nullptr,
                            q.D1, q.S1.mod, q.S1.N, q.S1.X, q.S1.big, g->nsm, st);
    CK(g, cudaMemcpyAsync(q.D, q.D1, cells * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    // Steps 2-5: sweeps over the border edges and the border matrices until
    // no border distance changes
    long long sweeps = 0;
    for (;;) {
        int changed = 0;
        CK(g, cudaMemsetAsync(q.changed, 0, sizeof(int), st));
        launch_refine_cut(q.cut_rp, q.cut_col, q.border, q.bidx, q.nbt, q.D, q.changed, g->nsm, st);
        launch_refine_bm(q.bpart, q.boff, q.moff, q.BM, q.nbt, q.D, q.changed, g->nsm, st);
        g->stats.kernel_launches += 2;
        CK(g, cudaMemcpyAsync(&changed, q.changed, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(g, cudaStreamSynchronize(st));
        ++sweeps;
        if (!changed) break;
        if (sweeps > q.nbt + 2) return fail(g, GBBC_ERR_CAPACITY, "partitioned method: refinement did not settle");
    }
    q.sweeps += sweeps;
    // sigma of the border nodes, level by level
    std::vector<int32_t> hD(cells);
    CK(g, cudaMemcpyAsync(hD.data(), q.D, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    int32_t maxD = -1;
    for (int32_t d : hD)
        if (d < kPartInf) maxD = std::max(maxD, d);
    for (int32_t l = 0; l <= maxD; ++l) {
        launch_border_sigma_level(l, q.cut_rp, q.cut_col, q.border, q.bidx, q.bpart, q.boff, q.moff, q.BM, q.SM, q.nbt,
                                  q.D, q.D1, q.S1, q.A, q.Sig, g->nsm, st);
        g->stats.kernel_launches += 2;
    }
    // Step 6: relaxation inside every part, seeded at the border nodes
    SeedHooks hooks(g);
    CKS(part_forward(g, cin, b, st, wide, off, &hooks));
    const int nlev = (int)off.size() - 1;
    if (g->k_dist) {
        for (int l = 0; l < nlev; ++l)
            launch_keep_dist(g->slot, off[l], off[l + 1], l, g->k_dist, g->n, b.first, b.nsrc, st);
        launch_keep_sigma(g->slot, b.lo, b.hi, g->k_sigma, g->k_ovf, g->n, b.first, b.nsrc, st);
        g->stats.kernel_launches += nlev + 1;
    }
    if (g->opt.flags & GBBC_SYNC_BACKWARD) {
        // level-synchronous backward over the whole graph
        CKS(run_backward(g, call, g->slot, off, wide, g->d_bc, g->stats, st));
    } else {
        CKS(part_backward_async(g, call, off, wide, st));
    }
    if (wide) g->stats.wide_batches++;
    g->stats.batches++;
    g->stats.sources += b.nsrc;
    return GBBC_OK;
}

gbbc_status dispatch(gbbc_graph* g, const std::vector<BatchDesc>& bs, cudaStream_t st);
gbbc_status grouping_scores(gbbc_graph* g, const std::vector<int32_t>& src, const std::vector<int32_t>& gid,
                            std::vector<float>& score, cudaStream_t st);

// Shared by bc_compute and bc_compute_multi: `gsrc` are whole-handle vertex
// ids, `gid` their graph index.
gbbc_status compute_weighted(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<int32_t>& gid,
                             cudaStream_t st);
gbbc_status compute_batched(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<int32_t>& gid,
                            cudaStream_t st, bool mixed);

// Under GBBC_SCHEDULE_AUTO, a large sparse graph of high diameter with few
// sources runs in the pair schedule: its sources rarely share a BFS level, so
// 64-lane rows are mostly idle (measured with 1024 sources: 1024^2
// triangulation 1.54x, 2^20-point random geometric graph 1.52x, 1024^2 grid
// 1.13x faster; the 100^3 mesh, degree 26, and small or low-diameter graphs
// are faster in the bitset schedules).  The
// test, per graph of the handle, once: above 65,536 vertices, average degree
// at most 12, and a BFS eccentricity of at least 64 from a vertex of its
// largest row (host BFS over a host copy of the columns).
bool pair_auto(gbbc_graph* g, int gi) {
    if (g->pair_graph.size() != g->goff.size() - 1) g->pair_graph.assign(g->goff.size() - 1, -1);
    if (g->pair_graph[gi] >= 0) return g->pair_graph[gi] == 1;
    g->pair_graph[gi] = 0;
    const long long lo = g->goff[gi], hi = g->goff[gi + 1], n = hi - lo;
    const long long e0 = g->h_row_ptr[lo], e1 = g->h_row_ptr[hi];
    if (n <= 65536 || (double)(e1 - e0) > 12.0 * (double)n) return false;
    std::vector<int32_t> col((size_t)(e1 - e0));
    if (cudaMemcpy(col.data(), g->d_col + e0, (size_t)(e1 - e0) * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    long long s = lo;
    for (long long v = lo + 1; v < hi; ++v)
        if (g->h_row_ptr[v + 1] - g->h_row_ptr[v] > g->h_row_ptr[s + 1] - g->h_row_ptr[s]) s = v;
    std::vector<int32_t> dist((size_t)n, -1), queue;
    queue.reserve((size_t)n);
    dist[s - lo] = 0;
    queue.push_back((int32_t)(s - lo));
    int32_t ecc = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
        const int32_t v = queue[h];
        for (int32_t p = g->h_row_ptr[lo + v]; p < g->h_row_ptr[lo + v + 1]; ++p) {
            const int32_t u = col[p - e0] - (int32_t)lo;
            if (dist[u] < 0) {
                dist[u] = dist[v] + 1;
                ecc = std::max(ecc, dist[u]);
                queue.push_back(u);
            }
        }
    }
    g->pair_graph[gi] = ecc >= 64 ? 1 : 0;
    return g->pair_graph[gi] == 1;
}

gbbc_status compute_impl(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<int32_t>& gid,
                         cudaStream_t st) {
    long long k = (long long)gsrc.size();
    if (g->opt.policy == GBBC_POLICY_LEARNED && !g->d_policy && g->opt.batch_width != 1)
        return fail(g, GBBC_ERR_STATE, "GBBC_POLICY_LEARNED needs weights (bc_policy_load)");
    CKS(alloc_keep(g, k, st));
    g->last_stream = st;
    if (g->d_w || g->opt.schedule == GBBC_SCHEDULE_PAIR) return compute_weighted(g, gsrc, gid, st);
    if (g->opt.schedule == GBBC_SCHEDULE_AUTO && g->opt.batch_width != 1 && !(g->opt.flags & GBBC_TRACE)) {
        const int ngraphs = (int)g->goff.size() - 1;
        // the pair kernel gains by spreading few sources over every SM; with
        // more than 8 sources per SM its batches are as wide as the bitset
        // words and the words' shared rows win (256-graph mix: 13.2 s bitset,
        // 19.4 s with its large grids in the pair kernel)
#ifndef GBBC_PAIR_MAX_PER_SM
#define GBBC_PAIR_MAX_PER_SM 8
#endif
        const long long pair_max = (long long)GBBC_PAIR_MAX_PER_SM * g->nsm;
        if (ngraphs == 1) {
            if (k <= pair_max && pair_auto(g, 0)) return compute_weighted(g, gsrc, gid, st);
        } else if (!g->k_dist) {  // kept state follows list order: no split then
            // the sources of graphs the pair schedule takes go there, the rest below
            std::vector<int32_t> ps, pg, rs, rg;
            for (long long i = 0; i < k; ++i) {
                const bool pr = pair_auto(g, gid[i]);
                (pr ? ps : rs).push_back(gsrc[i]);
                (pr ? pg : rg).push_back(gid[i]);
            }
            if (!ps.empty() && (long long)ps.size() <= pair_max) {
                CKS(compute_weighted(g, ps, pg, st));
                if (rs.empty()) return GBBC_OK;
                return compute_batched(g, rs, rg, st, true);
            }
        }
    }
    return compute_batched(g, gsrc, gid, st, false);
}

bool grid_graph(const gbbc_graph* g, const BatchDesc& b);
gbbc_status run_grid_batches(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st);
gbbc_status persist_prepare(gbbc_graph* g, int W);
double now_s();
int grid_workers(gbbc_graph* g, size_t nb);
gbbc_status ensure_workers(gbbc_graph* g, int count);

// Autotuning of the grid schedule (a handle's first call with at least
// kTuneMinSources sources on one large graph, width and heavy-row threshold
// left automatic): five configurations -- width 64 with heavy-row thresholds
// 1024, 512 and 2048, width 32 with 1024, and width 64 with 1024 on the
// persistent kernel (the device loop) -- each run kTuneBlocks blocks of 64
// consecutive sources of the call's ordered list (grouped and sorted by the
// grouping network when it is loaded).  The 5 x kTuneBlocks blocks sit at
// evenly spaced positions of the list and are dealt to the configurations
// in turn, so every configuration sees sources from the whole range; the
// one with the most sources per second is kept for the handle (the default,
// width 64 with threshold 1024 on the host loop, unless another is more
// than 3% faster).  Trial
// sources count once, like any other (BC is an exact integer sum).  This is
// the measure-then-split idea of the paper's variable partitioning (Sec.
// V-D) applied to the launch configuration.
constexpr int kTuneBlocks = 4;
constexpr int kTuneConfigs = 5;
constexpr long long kTuneMinSources = 2LL * kTuneConfigs * kTuneBlocks * kLanes;
constexpr double kTuneMargin = 0.03;

bool tune_wanted(gbbc_graph* g, const std::vector<int32_t>& gid, long long k) {
    if (g->tuned || !g->auto_width || !g->auto_heavy || g->k_dist || (g->opt.flags & (GBBC_TRACE | GBBC_DEVICE_LOOP)))
        return false;
    if (g->goff.size() != 2 || k < kTuneMinSources) return false;
    if (!(g->opt.schedule == GBBC_SCHEDULE_AUTO || g->opt.schedule == GBBC_SCHEDULE_GRID)) return false;
    BatchDesc b;
    b.gi = 0;
    b.lo = 0;
    b.hi = g->n;
    (void)gid;
    return g->opt.schedule == GBBC_SCHEDULE_GRID || grid_graph(g, b);
}

gbbc_status autotune(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<long long>& order,
                     std::vector<char>& taken, cudaStream_t st) {
    struct Cfg {
        int width, heavy;
        bool device;
    };
    const Cfg cfgs[kTuneConfigs] = {{64, 1024, false}, {64, 512, false}, {64, 2048, false}, {32, 1024, false},
                                    {64, 1024, true}};
    const long long k = (long long)order.size();
    const int nblk = kTuneConfigs * kTuneBlocks;
    std::vector<std::vector<int32_t>> src(kTuneConfigs);
    for (int j = 0; j < nblk; ++j) {
        long long start = (long long)(((double)j + 0.5) * (double)k / nblk) - kLanes / 2;
        start = std::max(0LL, std::min(start, k - kLanes));
        for (long long p = start; p < start + kLanes; ++p)
            if (!taken[p]) {
                taken[p] = 1;
                src[j % kTuneConfigs].push_back(gsrc[order[p]]);
            }
    }
    // one-time set-up outside the timed trials
    CKS(alloc_slot(g));
    const int W = grid_workers(g, 64);
    CKS(ensure_workers(g, W - 1));
    CKS(persist_prepare(g, std::min(W, kMaxPSlots)));
    double best_rate = -1.0;
    int best = 0;
    for (int c = 0; c < kTuneConfigs; ++c) {
        g->opt.batch_width = cfgs[c].width;
        g->opt.heavy_degree = cfgs[c].heavy;
        g->tuned_device = cfgs[c].device;
        std::vector<BatchDesc> bs;
        for (size_t i = 0; i < src[c].size();) {
            BatchDesc b;
            b.gi = 0;
            b.lo = 0;
            b.hi = g->n;
            b.first = 0;
            b.nsrc = 0;
            while (i < src[c].size() && b.nsrc < cfgs[c].width) b.src[b.nsrc++] = src[c][i++];
            bs.push_back(b);
        }
        CK(g, cudaStreamSynchronize(st));
        const double t0 = now_s();
        CKS(run_grid_batches(g, bs.data(), bs.size(), st));
        CK(g, cudaStreamSynchronize(st));
        const double rate = (double)src[c].size() / std::max(now_s() - t0, 1e-9);
        // the default (configuration 0) is kept unless another beats it by
        // more than kTuneMargin: trials on different sources are noisy
        const double bar = c == 0 ? 0.0 : (best == 0 ? best_rate * (1.0 + kTuneMargin) : best_rate);
        if (c == 0 || rate > bar) {
            best_rate = rate;
            best = c;
        }
    }
    g->opt.batch_width = cfgs[best].width;
    g->opt.heavy_degree = cfgs[best].heavy;
    g->tuned_device = cfgs[best].device;
    g->tuned = true;
    g->stats.batch_width = cfgs[best].width;
    g->stats.tuned_heavy_degree = cfgs[best].heavy;
    g->stats.tuned_device_loop = cfgs[best].device ? 1 : 0;
    return GBBC_OK;
}

// The bitset schedules (grid, block): sources packed 64 (or 32) per word.
gbbc_status compute_batched(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<int32_t>& gid,
                            cudaStream_t st, bool mixed) {
    long long k = (long long)gsrc.size();
    if (g->opt.batch_width == 1) {  // plain: one source at a time, list order
        if (g->opt.schedule == GBBC_SCHEDULE_BLOCK && !g->k_dist && !(g->opt.flags & GBBC_TRACE))
            return run_plain_blocks(g, gsrc, st);
        CKS(alloc_plain(g));
        for (long long i = 0; i < k; ++i)
            CKS(run_plain(g, gsrc[i], (int32_t)g->goff[gid[i]], (int32_t)g->goff[gid[i] + 1], i, st));
        return GBBC_OK;
    }
    // group by graph (stable), then pack up to 64 consecutive sources; with a
    // grouping network loaded (and no per-source state kept), each graph's
    // sources are ordered by the network's score so that sources whose BFS
    // levels line up share a word
    std::vector<long long> order(k);
    for (long long i = 0; i < k; ++i) order[i] = i;
    if (g->d_grouping && !g->k_dist) {
        std::vector<float> score;
        CKS(grouping_scores(g, gsrc, gid, score, st));
        std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) {
            return gid[a] != gid[b] ? gid[a] < gid[b] : score[a] < score[b];
        });
    } else {
        std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return gid[a] < gid[b]; });
    }
    if (tune_wanted(g, gid, k)) {  // trial runs on spread blocks of the list, then the rest
        std::vector<char> taken((size_t)k, 0);
        CKS(autotune(g, gsrc, order, taken, st));
        std::vector<long long> rest;
        rest.reserve((size_t)k);
        for (long long i = 0; i < k; ++i)
            if (!taken[i]) rest.push_back(order[i]);
        order.swap(rest);
        k = (long long)order.size();
    }
    std::vector<BatchDesc> batches;
    const int width = g->opt.batch_width == 32 ? 32 : kLanes;
    long long i = 0;
    while (i < k) {
        BatchDesc b;
        int32_t gi = gid[order[i]];
        b.gi = gi;
        b.lo = (int32_t)g->goff[gi];
        b.hi = (int32_t)g->goff[gi + 1];
        b.first = order[i];
        b.nsrc = 0;
        bool contiguous = true;
        while (i < k && b.nsrc < width && gid[order[i]] == gi) {
            if (order[i] != b.first + b.nsrc) contiguous = false;
            b.src[b.nsrc++] = gsrc[order[i]];
            ++i;
        }
        // KEEP_STATE writes rows by the batch lane's position in the list
        if (g->k_dist && !contiguous)
            return fail(g, GBBC_ERR_INVALID, "GBBC_KEEP_STATE needs the sources of each graph to be contiguous");
        batches.push_back(b);
    }
    CKS(dispatch(g, batches, st));
    if (mixed) g->stats.schedule = GBBC_SCHEDULE_AUTO;  // pair and bitset schedules in one call
    return GBBC_OK;
}

// ---- weighted graphs ----------------------------------------------------------

double wslot_bytes(long long nslot, int L, int B) {
    const long long levcap = 2 * nslot + 4096;
    return (double)nslot * L * (4 + 8 + 8 + 4 + 1) + (double)B * nslot * L * 4 + (double)(nslot * L + L) * 4 +
           (double)levcap * 4 + (double)(levcap + 1) * 8;
}

gbbc_status alloc_wslots(gbbc_graph* g, long long nslot, int L, int B, int want) {
    WSlots& S = g->wsl;
    if (S.count >= want && S.nslot >= nslot && S.B == B && S.L == L) return GBBC_OK;
    for (void* p : {(void*)S.dist, (void*)S.sp, (void*)S.blist, (void*)S.qv, (void*)S.levD, (void*)S.levOff,
                    (void*)S.sN, (void*)S.sX, (void*)S.wf})
        dfree(g, p);
    S = WSlots();
    const long long qcap = nslot * L + L;
    const long long levcap = 2 * nslot + 4096;
    const long long bcap = nslot * L;  // a pair is listed at most once per bucket between its visits
    const double per_slot = wslot_bytes(nslot, L, B);
    double budget = 0.5 * (double)avail_bytes(g->device);
    if (g->opt.mem_limit_bytes > 0) budget = std::min(budget, (double)g->opt.mem_limit_bytes - (double)g->bytes);
    int count = (int)std::min<double>((double)want, std::floor(budget / per_slot));
    if (count < 1) return fail(g, GBBC_ERR_OOM, "no room for one weighted-path slot (%.0f bytes)", per_slot);
    const size_t c = (size_t)count, ns = (size_t)nslot;
    S.nslot = nslot;
    S.qcap = qcap;
    S.levcap = levcap;
    S.bcap = bcap;
    S.count = count;
    S.B = B;
    S.L = L;
    CKS(dalloc_t(g, &S.dist, c * ns * L));
    CKS(dalloc_t(g, &S.sp, c * ns * L));
    CKS(dalloc_t(g, &S.blist, c * (size_t)B * (size_t)bcap));
    CKS(dalloc_t(g, &S.qv, c * (size_t)qcap));
    CKS(dalloc_t(g, &S.levD, c * (size_t)levcap));
    CKS(dalloc_t(g, &S.levOff, c * (size_t)(levcap + 1)));
    CKS(dalloc_t(g, &S.sN, c * ns * L));
    CKS(dalloc_t(g, &S.sX, c * ns * L));
    CKS(dalloc_t(g, &S.wf, c * ns * L));
    return GBBC_OK;
}

// Pair-granular kernel (bc_weighted.cu), for weighted graphs and for
// unweighted ones under GBBC_SCHEDULE_PAIR (all weights 1): sources in list
// order (by graph), L per batch, one CTA per batch, every batch in one
// launch.  L = ceil(k / (SMs x resident blocks per SM)), at most 64, so that
// every resident block gets a batch (one block per SM left it latency-bound;
// two gave 1.5-1.6x).  Work items are (vertex, lane) pairs, so narrower
// batches lose nothing.
gbbc_status compute_weighted(gbbc_graph* g, const std::vector<int32_t>& gsrc, const std::vector<int32_t>& gid,
                             cudaStream_t st) {
    if (g->opt.batch_width == 1)
        return fail(g, GBBC_ERR_INVALID, "the pair-granular path has no one-source form (batch_width 1)");
    const int W = g->d_w ? g->max_w : 1;
    const long long k = (long long)gsrc.size();
    if (k == 0) return GBBC_OK;
    std::vector<long long> order(k);
    for (long long i = 0; i < k; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return gid[a] < gid[b]; });
    long long nslot = 1;
    for (long long i = 0; i < k; ++i)
        nslot = std::max<long long>(nslot, g->goff[gid[i] + 1] - g->goff[gid[i]]);
    // a slot's memory grows with L, so when fewer slots than SMs fit, wider
    // batches do not raise the number of pairs in flight: L depends on k and
    // on the resident blocks only (every resident block gets a batch)
    if (g->w_bps == 0) g->w_bps = weighted_blocks_per_sm();
    const long long blocks = (long long)g->nsm * g->w_bps;
    const int L = (int)std::max<long long>(1, std::min<long long>(kLanes, (k + blocks - 1) / blocks));
    if ((double)nslot * L >= 2147483647.0)
        return fail(g, GBBC_ERR_INVALID, "weighted path: n x lanes must stay below 2^31");
    std::vector<WBatch> hb;
    std::vector<int32_t> hsrc;
    for (long long i = 0; i < k;) {
        const int32_t gi = gid[order[i]];
        WBatch b;
        b.lo = (int32_t)g->goff[gi];
        b.hi = (int32_t)g->goff[gi + 1];
        b.first = order[i];
        b.src_off = (long long)hsrc.size();
        b.nsrc = 0;
        b.gi = gi;
        b.wide = g->wide_graph[gi];
        b.pad = 0;
        while (i < k && b.nsrc < L && gid[order[i]] == gi) {
            if (g->k_dist && order[i] != b.first + b.nsrc)
                return fail(g, GBBC_ERR_INVALID, "GBBC_KEEP_STATE needs the sources of each graph to be contiguous");
            hsrc.push_back(gsrc[order[i]]);
            ++b.nsrc;
            ++i;
        }
        hb.push_back(b);
    }
    const int nb = (int)hb.size();
    CKS(alloc_wslots(g, nslot, L, W + 1, (int)std::min<long long>(nb, blocks)));
    const size_t ngraphs = g->wide_graph.size();
    if (!g->d_gwide) CKS(dalloc_t(g, &g->d_gwide, ngraphs));
    CK(g, cudaMemsetAsync(g->d_gwide, 0, ngraphs * sizeof(int), st));
    if (g->d_wb_cap < nb) {
        dfree(g, g->d_wb);
        CKS(dalloc_t(g, &g->d_wb, (size_t)nb));
        g->d_wb_cap = nb;
    }
    if (g->d_bsrc_cap < (long long)hsrc.size()) {
        dfree(g, g->d_bsrc);
        CKS(dalloc_t(g, &g->d_bsrc, hsrc.size()));
        g->d_bsrc_cap = (long long)hsrc.size();
    }
    if (!g->d_next) CKS(dalloc_t(g, &g->d_next, 1));
    if (!g->d_bstats) CKS(dalloc_t(g, &g->d_bstats, 4));
    CK(g, cudaMemcpyAsync(g->d_wb, hb.data(), hb.size() * sizeof(WBatch), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemcpyAsync(g->d_bsrc, hsrc.data(), hsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemsetAsync(g->d_next, 0, sizeof(unsigned), st));
    CK(g, cudaMemsetAsync(g->d_bstats, 0, 4 * sizeof(unsigned long long), st));
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    CK(g, launch_weighted_batches(c, g->d_w, g->wsl, g->d_wb, nb, g->d_bsrc, g->d_next, g->d_bc, W, g->k_dist,
                                  reinterpret_cast<u64*>(g->k_sigma), g->k_ovf, g->n, g->d_gwide, g->d_bstats, st));
    g->stats.kernel_launches++;
    unsigned long long hst[4];
    std::vector<int> gw(ngraphs);
    CK(g, cudaMemcpyAsync(hst, g->d_bstats, sizeof(hst), cudaMemcpyDeviceToHost, st));
    CK(g, cudaMemcpyAsync(gw.data(), g->d_gwide, ngraphs * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    const unsigned err = (unsigned)(hst[3] & 0xffffffffull);
    if (err) return fail(g, GBBC_ERR_CAPACITY, "pair-granular path: capacity exceeded (flags %u)", err);
    if ((int)hst[0] != nb) return fail(g, GBBC_ERR_CUDA, "pair-granular path ran %llu of %d batches", hst[0], nb);
    g->stats.batches += nb;
    g->stats.sources += k;
    g->stats.levels_fwd += (long long)hst[1];
    g->stats.levels_push += (long long)hst[1];
    for (const WBatch& b : hb) g->stats.wide_batches += b.wide;
    g->stats.wide_batches += (long long)hst[2];
    for (size_t i = 0; i < ngraphs; ++i)
        if (gw[i]) g->wide_graph[i] = 1;  // later batches of this graph start wide
    g->stats.schedule = GBBC_SCHEDULE_PAIR;
    return GBBC_OK;
}

// ---- block-per-batch schedule ----------------------------------------------

gbbc_status alloc_block(gbbc_graph* g, long long nslot, int want) {
    BlockSlots& S = g->blk;
    if (S.count >= want && S.nslot >= nslot) return GBBC_OK;
    // release the old slots
    for (void* p : {(void*)S.vis, (void*)S.nx, (void*)S.ovf, (void*)S.F, (void*)S.sigma, (void*)S.psi, (void*)S.sN,
                    (void*)S.sX, (void*)S.psi_e, (void*)S.qv, (void*)S.qm, (void*)S.lev, (void*)S.ctr,
                    (void*)S.slot_batch, S.lsp})
        dfree(g, p);
    S = BlockSlots();
    const long long qcap = nslot * kLanes + kLanes;
    const double per_slot = (double)nslot * (3 * 8 + 2 * sizeof(MaskTag) + kLanes * (8 + 8 + 8 + 4 + 4) + 8) +
                            (double)qcap * 12 + sizeof(Counters);
    double budget = 0.5 * (double)avail_bytes(g->device);
    if (g->opt.mem_limit_bytes > 0) budget = std::min(budget, (double)g->opt.mem_limit_bytes - (double)g->bytes);
    int count = (int)std::min<double>((double)want, std::floor(budget / per_slot));
    if (count < 1) return fail(g, GBBC_ERR_OOM, "no room for one block-schedule slot (%.0f bytes)", per_slot);
    const size_t ns = (size_t)nslot, c = (size_t)count;
    S.nslot = nslot;
    S.qcap = qcap;
    S.count = count;
    CKS(dalloc_t(g, &S.vis, c * ns));
    CKS(dalloc_t(g, &S.nx, c * ns));
    CKS(dalloc_t(g, &S.ovf, c * ns));
    CKS(dalloc_t(g, &S.F, c * 2 * ns));
    CKS(dalloc_t(g, &S.sigma, c * ns * kLanes));
    CKS(dalloc_t(g, &S.psi, c * ns * kLanes));
    CKS(dalloc_t(g, &S.sN, c * ns * kLanes));
    CKS(dalloc_t(g, &S.sX, c * ns * kLanes));
    CKS(dalloc_t(g, &S.psi_e, c * ns * kLanes));
    CKS(dalloc_t(g, &S.qv, c * (size_t)qcap));
    CKS(dalloc_t(g, &S.qm, c * (size_t)qcap));
    CKS(dalloc_t(g, &S.lev, c * (ns + 2)));
    CKS(dalloc_t(g, &S.ctr, c));
    CKS(dalloc_t(g, &S.slot_batch, c));
    CKS(dalloc(g, &S.lsp, c * (ns + 2)));
    return GBBC_OK;
}

gbbc_status ensure_graph_arrays(gbbc_graph* g) {
    if (!g->d_graph_max_deg) {
        CKS(dalloc_t(g, &g->d_graph_max_deg, g->graph_max_deg.size()));
        CK(g, cudaMemcpy(g->d_graph_max_deg, g->graph_max_deg.data(), g->graph_max_deg.size() * sizeof(long long),
                         cudaMemcpyHostToDevice));
    }
    if (!g->d_goff) {
        CKS(dalloc_t(g, &g->d_goff, g->goff.size()));
        CK(g, cudaMemcpy(g->d_goff, g->goff.data(), g->goff.size() * sizeof(long long), cudaMemcpyHostToDevice));
    }
    return GBBC_OK;
}

// Features of k sources (whole-handle ids) into device x[k][6].
gbbc_status source_features(gbbc_graph* g, const std::vector<int32_t>& src, const std::vector<int32_t>& gid,
                            float* d_x, cudaStream_t st) {
    long long k = (long long)src.size();
    if (k == 0) return GBBC_OK;
    CKS(ensure_graph_arrays(g));
    int32_t *d_src = nullptr, *d_gid = nullptr;
    CKS(dalloc_t(g, &d_src, (size_t)k));
    gbbc_status r = dalloc_t(g, &d_gid, (size_t)k);
    if (r == GBBC_OK) {
        Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
        if (cudaMemcpyAsync(d_src, src.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_gid, gid.data(), k * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            launch_source_features(c, d_src, d_gid, k, g->d_goff, g->d_graph_max_deg, d_x, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            r = fail(g, GBBC_ERR_CUDA, "source features failed");
        g->stats.kernel_launches++;
    }
    dfree(g, d_src);
    dfree(g, d_gid);
    return r;
}

// Predicted grouping score of each source (learned network, FP16 weights).
gbbc_status grouping_scores(gbbc_graph* g, const std::vector<int32_t>& src, const std::vector<int32_t>& gid,
                            std::vector<float>& score, cudaStream_t st) {
    long long k = (long long)src.size();
    score.assign((size_t)k, 0.f);
    if (k == 0) return GBBC_OK;
    float *d_x = nullptr, *d_s = nullptr;
    CKS(dalloc_t(g, &d_x, (size_t)k * 6));
    gbbc_status r = dalloc_t(g, &d_s, (size_t)k);
    if (r == GBBC_OK) r = source_features(g, src, gid, d_x, st);
    if (r == GBBC_OK) {
        if (launch_group_score(g->d_grouping, d_x, k, d_s, st) != cudaSuccess ||
            cudaMemcpyAsync(score.data(), d_s, k * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            r = fail(g, GBBC_ERR_CUDA, "grouping scores failed");
        g->stats.kernel_launches++;
    }
    dfree(g, d_x);
    dfree(g, d_s);
    return r;
}

int ilog2(int x) {
    int r = 0;
    while (x > 1) x >>= 1, ++r;
    return r;
}

// Cluster size of the block schedule for nb batches (see run_block_mode).
int block_csize(gbbc_graph* g, int nb) {
    if (g->max_clusters[0] == 0)
        for (int i = 0; i < 4; ++i) g->max_clusters[i] = std::max(1, block_max_clusters(1 << i));
    int csize = 1;
    while (csize < 8 && (long long)nb * csize * 2 <= g->nsm) csize *= 2;
    return csize;
}

gbbc_status run_block_mode(gbbc_graph* g, const BatchDesc* bs, int nb, cudaStream_t st) {
    if (nb <= 0) return GBBC_OK;
    long long nslot = 1;
    std::vector<BlockBatch> hb((size_t)nb);
    std::vector<int32_t> hsrc;
    for (int i = 0; i < nb; ++i) {
        nslot = std::max<long long>(nslot, (long long)bs[i].hi - bs[i].lo);
        hb[i].gi = bs[i].gi;
        hb[i].lo = bs[i].lo;
        hb[i].hi = bs[i].hi;
        hb[i].nsrc = bs[i].nsrc;
        hb[i].src_off = (long long)hsrc.size();
        hb[i].wide = g->wide_graph[bs[i].gi];
        hb[i].pad = 0;
        hsrc.insert(hsrc.end(), bs[i].src, bs[i].src + bs[i].nsrc);
    }
    // Longest batches first (the work list hands them out in this order), so
    // that the last batches to start are short ones and no cluster runs alone
    // at the end.  Estimated cost: edges and vertices of the batch's graph
    // times a level count (about sqrt(n) on sparse, road-like graphs, log2(n)
    // otherwise), tripled in the wide sigma format.  BC does not depend on
    // the order.
    {
        std::vector<double> cost((size_t)nb);
        for (int i = 0; i < nb; ++i) {
            const double nr = (double)hb[i].hi - hb[i].lo;
            const double er = (double)(g->h_row_ptr[hb[i].hi] - g->h_row_ptr[hb[i].lo]);
            const double levels = er <= 6.0 * nr ? std::sqrt(nr) : std::log2(nr + 2.0);
            cost[i] = (er + nr) * levels * (hb[i].wide ? 3.0 : 1.0) * (double)hb[i].nsrc;
        }
        std::vector<int> ord((size_t)nb);
        for (int i = 0; i < nb; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::vector<BlockBatch> sorted((size_t)nb);
        for (int i = 0; i < nb; ++i) sorted[i] = hb[ord[i]];
        hb.swap(sorted);
    }
    // clusters: few batches get several SMs each (up to 8 CTAs, the portable
    // cluster size), many batches one SM each.  A batch's time falls about in
    // proportion to its cluster's CTAs (measured on the 1024^2 grid: 8 CTAs
    // 1.1 s, 4 CTAs 2.3 s), so the larger cluster wins even when fewer of its
    // clusters are resident (they are placed within GPCs: 15 of 8 CTAs fit)
    // and a batch waits for a second round.  Slots beyond the resident
    // clusters would only hold memory.
    int csize = block_csize(g, nb);
    const int resident = g->max_clusters[ilog2(csize)];
    CKS(alloc_block(g, nslot, std::max(1, std::min(nb, std::min(resident, g->nsm / csize)))));
    g->blk.csize = csize;
    if (g->d_bb_cap < nb) {
        dfree(g, g->d_bb);
        CKS(dalloc_t(g, &g->d_bb, (size_t)nb));
        g->d_bb_cap = nb;
    }
    if (g->d_bsrc_cap < (long long)hsrc.size()) {
        dfree(g, g->d_bsrc);
        CKS(dalloc_t(g, &g->d_bsrc, hsrc.size()));
        g->d_bsrc_cap = (long long)hsrc.size();
    }
    if (!g->d_next) CKS(dalloc_t(g, &g->d_next, 1));
    if (!g->d_bstats) CKS(dalloc_t(g, &g->d_bstats, 4));
    const size_t ngraphs = g->wide_graph.size();
    if (!g->d_gwide) CKS(dalloc_t(g, &g->d_gwide, ngraphs));
    CKS(ensure_graph_arrays(g));
    CK(g, cudaMemcpyAsync(g->d_bb, hb.data(), hb.size() * sizeof(BlockBatch), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemcpyAsync(g->d_bsrc, hsrc.data(), hsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemsetAsync(g->d_next, 0, sizeof(unsigned), st));
    CK(g, cudaMemsetAsync(g->d_bstats, 0, 4 * sizeof(unsigned long long), st));
    // batches are taken from a work list, so a slot may get none; its counters
    // (read below) must then be zero rather than whatever the memory held
    CK(g, cudaMemsetAsync(g->blk.ctr, 0, (size_t)g->blk.count * sizeof(Counters), st));
    CK(g, cudaMemsetAsync(g->d_gwide, 0, ngraphs * sizeof(int), st));
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    CK(g, launch_block_batches(c, g->blk, g->d_bb, nb, g->d_bsrc, g->d_next, g->d_bc, effective_policy(g),
                               g->d_policy, g->d_graph_max_deg, g->d_bstats, g->d_gwide, st));
    g->stats.kernel_launches++;
    unsigned long long hst[4];
    CK(g, cudaMemcpyAsync(hst, g->d_bstats, sizeof(hst), cudaMemcpyDeviceToHost, st));
    std::vector<Counters> hc((size_t)g->blk.count);
    CK(g, cudaMemcpyAsync(hc.data(), g->blk.ctr, hc.size() * sizeof(Counters), cudaMemcpyDeviceToHost, st));
    std::vector<int> gw(ngraphs);
    CK(g, cudaMemcpyAsync(gw.data(), g->d_gwide, ngraphs * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    for (const Counters& x : hc)
        if (x.err) return fail(g, GBBC_ERR_CAPACITY, "block schedule: queue capacity exceeded (flags %u)", x.err);
    if ((int)hst[0] != nb) return fail(g, GBBC_ERR_CUDA, "block schedule ran %llu of %d batches", hst[0], nb);
    g->stats.batches += nb;
    for (int i = 0; i < nb; ++i) g->stats.sources += bs[i].nsrc;
    g->stats.levels_fwd += (long long)hst[1];
    g->stats.levels_pull += (long long)hst[2];
    g->stats.levels_push += (long long)(hst[1] - hst[2]);
    for (int i = 0; i < nb; ++i) g->stats.wide_batches += hb[i].wide;
    g->stats.wide_batches += (long long)hst[3];
    for (size_t i = 0; i < ngraphs; ++i)
        if (gw[i]) g->wide_graph[i] = 1;  // later batches of this graph start wide
    g->stats.block_slots = g->blk.count;
    return GBBC_OK;
}

// dst[i] += src[i] for n u128 fixed-point values (a worker's BC into the handle's)
__global__ void k_add_fixed(u64* dst, const u64* src, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        u128 a = {dst[2 * i], dst[2 * i + 1]}, b = {src[2 * i], src[2 * i + 1]};
        a = add128(a, b);
        dst[2 * i] = a.lo;
        dst[2 * i + 1] = a.hi;
    }
}

void launch_add_fixed(u64* dst, const u64* src, long long n, cudaStream_t st) {
    if (n <= 0) return;
    k_add_fixed<<<1216, 256, 0, st>>>(dst, src, n);
}

void stats_add(gbbc_stats& a, gbbc_stats& b) {
    a.sources += b.sources;
    a.batches += b.batches;
    a.levels_fwd += b.levels_fwd;
    a.levels_push += b.levels_push;
    a.levels_pull += b.levels_pull;
    a.wide_batches += b.wide_batches;
    a.kernel_launches += b.kernel_launches;
    std::memset(&b, 0, sizeof(b));
}

// Concurrent batches of the grid schedule: up to opt.streams (default 8)
// batches at once, worker 0 on the caller's stream and slot, the others on
// their own streams, slots and fixed-point BC accumulators, each driven by a
// host thread taking the next batch from a shared counter.  A single batch's
// levels leave much of the GPU idle (small frontiers, host read-back per
// level); overlapping batches fills it (R-MAT 18, 4096 sources: 1.36x with 2,
// 1.56x with 4, 1.63x with 6, 1.66x with 8).  The accumulators are added into the handle's BC at the end:
// integer sums, so BC does not depend on which worker ran which batch.
int grid_workers(gbbc_graph* g, size_t nb) {
    if ((g->opt.flags & GBBC_TRACE) || g->k_dist || nb < 2) return 1;
    int want = g->opt.streams == 0 ? 8 : g->opt.streams;
    want = (int)std::min<size_t>((size_t)want, nb);
    if (want <= 1) return 1;
    const double n = (double)std::max<int32_t>(g->n, 1);
    // per extra worker: the slot (as alloc_slot_into) and its BC accumulator
    const double per = n * (3 * 8 + 2 * sizeof(MaskTag) + kLanes * 16 + 8 + 8) + (n * kLanes + kLanes) * 12 + 16 * n;
    double budget = 0.5 * (double)avail_bytes(g->device);
    if (g->opt.mem_limit_bytes > 0) budget = std::min(budget, (double)g->opt.mem_limit_bytes - (double)g->bytes);
    const int have = (int)g->workers.size();
    const int fit = have + (int)std::max(0.0, std::floor(budget / per));
    return std::max(1, std::min(want, 1 + fit));
}

gbbc_status ensure_workers(gbbc_graph* g, int count) {
    const size_t n1 = (size_t)std::max<int32_t>(g->n, 1);
    while ((int)g->workers.size() < count) {
        g->workers.emplace_back();
        gbbc_graph::Worker& w = g->workers.back();
        std::memset(&w.stats, 0, sizeof(w.stats));
        CK(g, cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking));
        CK(g, cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming));
        CKS(alloc_slot_into(g, w.slot));
        CKS(dalloc_t(g, &w.bc, 2 * n1));
        CK(g, cudaMemset(w.bc, 0, 2 * n1 * sizeof(u64)));
    }
    if (!g->ev_start) CK(g, cudaEventCreateWithFlags(&g->ev_start, cudaEventDisableTiming));
    return GBBC_OK;
}

gbbc_status run_persistent(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st,
                           std::vector<BatchDesc>& wide_out);
gbbc_status run_grid_host(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st);

// The grid schedule: the host-driven level loop, or the persistent kernel for
// narrow batches when GBBC_DEVICE_LOOP is set or the autotuner chose it
// (never with tracing or kept state, which need the host loop); batches in
// the wide format always run the host loop.
gbbc_status run_grid_batches(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st) {
    if (nb == 0) return GBBC_OK;
    const bool device = ((g->opt.flags & GBBC_DEVICE_LOOP) || g->tuned_device) &&
                        !(g->opt.flags & GBBC_TRACE) && !g->k_dist;
    if (!device) return run_grid_host(g, bs, nb, st);
    std::vector<BatchDesc> narrow, wide;
    for (size_t i = 0; i < nb; ++i) (g->wide_graph[bs[i].gi] ? wide : narrow).push_back(bs[i]);
    CKS(run_persistent(g, narrow.data(), narrow.size(), st, wide));
    return run_grid_host(g, wide.data(), wide.size(), st);
}

// The grid schedule driven from the host: per-step kernels and a counter
// read-back per level, up to opt.streams batches at once on host threads.
gbbc_status run_grid_host(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st) {
    if (nb == 0) return GBBC_OK;
    CKS(alloc_slot(g));
    const int C = grid_workers(g, nb);
    if (C <= 1) {
        for (size_t i = 0; i < nb; ++i) CKS(run_batch(g, bs[i], st));
        return GBBC_OK;
    }
    CKS(ensure_workers(g, C - 1));
    CK(g, cudaEventRecord(g->ev_start, st));
    for (int w = 0; w < C - 1; ++w) CK(g, cudaStreamWaitEvent(g->workers[w].st, g->ev_start, 0));
    std::atomic<size_t> next{0};
    std::atomic<int> status{GBBC_OK};
    auto work = [&](Slot* slot, u64* bc, gbbc_stats* stats, cudaStream_t ws) {
        for (;;) {
            if (status.load() != GBBC_OK) break;
            const size_t i = next.fetch_add(1);
            if (i >= nb) break;
            const gbbc_status r = run_batch(g, bs[i], ws, *slot, bc, *stats);
            if (r != GBBC_OK) {
                int expect = GBBC_OK;
                status.compare_exchange_strong(expect, (int)r);
                break;
            }
        }
    };
    std::vector<std::thread> th;
    for (int w = 0; w < C - 1; ++w) {
        gbbc_graph::Worker& wk = g->workers[w];
        th.emplace_back(work, &wk.slot, wk.bc, &wk.stats, wk.st);
    }
    work(&g->slot, g->d_bc, &g->stats, st);
    for (std::thread& t : th) t.join();
    const size_t n1 = (size_t)std::max<int32_t>(g->n, 1);
    for (int w = 0; w < C - 1; ++w) {
        gbbc_graph::Worker& wk = g->workers[w];
        CK(g, cudaEventRecord(wk.ev, wk.st));
        CK(g, cudaStreamWaitEvent(st, wk.ev, 0));
        launch_add_fixed(g->d_bc, wk.bc, (long long)n1, st);
        CK(g, cudaMemsetAsync(wk.bc, 0, 2 * n1 * sizeof(u64), st));
        stats_add(g->stats, wk.stats);
        g->stats.kernel_launches++;
    }
    CK(g, cudaGetLastError());
    return (gbbc_status)status.load();
}

// The persistent grid schedule (bc_persist.cu): every narrow batch of the
// call in one cooperative launch, W batches in flight on W slots (the handle's
// slot and the workers' slots), the level loop on the device.  Batches whose
// counts reach 2^64 come back in a list and are rerun wide by the host loop.
// One-time set-up of the persistent kernel for W slots: the slots, the
// device copies of their descriptors and control words, level boundaries,
// events and the cooperative grid size.
gbbc_status persist_prepare(gbbc_graph* g, int W) {
    CKS(alloc_slot(g));
    CKS(ensure_workers(g, W - 1));
    if (g->p_blocks == 0) {
        const int per_sm = persist_blocks_per_sm();
        if (per_sm < 1) return fail(g, GBBC_ERR_CUDA, "persistent kernel: occupancy query failed");
        g->p_blocks = per_sm * g->nsm;
    }
    const size_t n2 = (size_t)std::max<int32_t>(g->n, 1) + 2;
    if (!g->p_slots) {
        CKS(dalloc_t(g, &g->p_slots, kMaxPSlots));
        CKS(dalloc_t(g, &g->p_ctl, kMaxPSlots));
        CKS(dalloc_t(g, &g->p_glob, 1));
    }
    if (g->p_lev_rows < W) {
        dfree(g, g->p_lev);
        g->p_lev = nullptr;
        CKS(dalloc_t(g, &g->p_lev, (size_t)W * n2));
        g->p_lev_rows = W;
    }
    if (!g->p_ev[0]) {
        CK(g, cudaEventCreate(&g->p_ev[0]));
        CK(g, cudaEventCreate(&g->p_ev[1]));
    }
    return GBBC_OK;
}

gbbc_status run_persistent(gbbc_graph* g, const BatchDesc* bs, size_t nb, cudaStream_t st,
                           std::vector<BatchDesc>& wide_out) {
    if (nb == 0) return GBBC_OK;
    const int W = std::max(1, std::min(grid_workers(g, nb), kMaxPSlots));
    CKS(persist_prepare(g, W));
    const size_t n2 = (size_t)std::max<int32_t>(g->n, 1) + 2;
    if (g->p_wide_cap < (long long)nb) {
        dfree(g, g->p_wide);
        g->p_wide = nullptr;
        CKS(dalloc_t(g, &g->p_wide, nb));
        g->p_wide_cap = (long long)nb;
    }
    std::vector<Slot> hs((size_t)W);
    hs[0] = g->slot;
    for (int w = 1; w < W; ++w) hs[w] = g->workers[w - 1].slot;
    if (g->p_dirty) {  // an earlier launch stopped in the middle of a step
        for (const Slot& x : hs) {
            CK(g, cudaMemsetAsync(x.hacc, 0, (size_t)x.hcap * kLanes * 2 * sizeof(u64), st));
            CK(g, cudaMemsetAsync(x.hcarry, 0, (size_t)x.hcap * sizeof(u64), st));
        }
        g->p_dirty = false;
    }
    std::vector<BlockBatch> hb(nb);
    std::vector<int32_t> hsrc;
    for (size_t i = 0; i < nb; ++i) {
        hb[i].gi = bs[i].gi;
        hb[i].lo = bs[i].lo;
        hb[i].hi = bs[i].hi;
        hb[i].nsrc = bs[i].nsrc;
        hb[i].src_off = (long long)hsrc.size();
        hb[i].wide = 0;
        hb[i].pad = 0;
        hsrc.insert(hsrc.end(), bs[i].src, bs[i].src + bs[i].nsrc);
    }
    if (g->d_bb_cap < (long long)nb) {
        dfree(g, g->d_bb);
        CKS(dalloc_t(g, &g->d_bb, nb));
        g->d_bb_cap = (long long)nb;
    }
    if (g->d_bsrc_cap < (long long)hsrc.size()) {
        dfree(g, g->d_bsrc);
        CKS(dalloc_t(g, &g->d_bsrc, hsrc.size()));
        g->d_bsrc_cap = (long long)hsrc.size();
    }
    CKS(ensure_graph_arrays(g));
    for (const Slot& x : hs) CK(g, cudaMemsetAsync(x.ctr, 0, sizeof(Counters), st));
    CK(g, cudaMemcpyAsync(g->p_slots, hs.data(), W * sizeof(Slot), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemsetAsync(g->p_ctl, 0, W * sizeof(PCtl), st));
    CK(g, cudaMemsetAsync(g->p_glob, 0, sizeof(PGlobal), st));
    CK(g, cudaMemcpyAsync(g->d_bb, hb.data(), nb * sizeof(BlockBatch), cudaMemcpyHostToDevice, st));
    CK(g, cudaMemcpyAsync(g->d_bsrc, hsrc.data(), hsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const long long spins = g->opt.timeout_spins > 0 ? (long long)g->opt.timeout_spins : GBBC_DEFAULT_SPINS;
    Csr c{g->n, g->nnz, g->d_row_ptr, g->d_col};
    CK(g, cudaEventRecord(g->p_ev[0], st));
    CK(g, launch_persist(c, g->p_slots, W, g->p_ctl, g->p_lev, (long long)n2, g->d_bb, (int)nb, g->d_bsrc, g->d_bc,
                         effective_policy(g), g->d_policy, g->d_graph_max_deg, g->opt.heavy_degree, spins, g->p_glob,
                         g->p_wide, g->p_blocks, st));
    CK(g, cudaEventRecord(g->p_ev[1], st));
    g->stats.kernel_launches++;
    PGlobal hg;
    CK(g, cudaMemcpyAsync(&hg, g->p_glob, sizeof(PGlobal), cudaMemcpyDeviceToHost, st));
    CK(g, cudaStreamSynchronize(st));
    {
        float ms = 0.f;
        CK(g, cudaEventElapsedTime(&ms, g->p_ev[0], g->p_ev[1]));
        g->stats.persist_launches++;
        g->stats.persist_ms += ms;
        g->stats.persist_slots = W;
        g->stats.persist_blocks = g->p_blocks;
    }
    if (hg.err & 1u) {
        g->p_dirty = true;
        return fail(g, GBBC_ERR_TIMEOUT,
                    "persistent grid schedule: a grid barrier wait passed timeout_spins=%lld polls; the handle's BC "
                    "is undefined until bc_reset", spins);
    }
    if (hg.err & 2u) {
        g->p_dirty = true;
        return fail(g, GBBC_ERR_CAPACITY,
                    "persistent grid schedule: capacity exceeded (flags %u, step kind %u, direction %u, level %u)",
                    hg.err_info & 15u, (hg.err_info >> 4) & 7u, (hg.err_info >> 7) & 1u, (hg.err_info >> 8) & 0xffffu);
    }
    std::vector<int32_t> wl(hg.wide);
    if (hg.wide)
        CK(g, cudaMemcpy(wl.data(), g->p_wide, hg.wide * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<char> rerun(nb, 0);
    for (int32_t b : wl)
        if (b >= 0 && (size_t)b < nb) rerun[b] = 1;
    g->stats.batches += (long long)hg.batches;
    g->stats.levels_fwd += (long long)hg.levels_fwd;
    g->stats.levels_pull += (long long)hg.levels_pull;
    g->stats.levels_push += (long long)(hg.levels_fwd - hg.levels_pull);
    for (size_t i = 0; i < nb; ++i) {
        if (rerun[i]) {
            std::lock_guard<std::recursive_mutex> lk(g->mtx);
            g->wide_graph[bs[i].gi] = 1;  // later batches of this graph start wide
            wide_out.push_back(bs[i]);
        } else {
            g->stats.sources += bs[i].nsrc;
        }
    }
    return GBBC_OK;
}

double now_s() {
    return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count() * 1e-9;
}

// Graphs above this many vertices with an average degree above
// kBlockMaxAvgDegree run in the grid schedule: one cluster per batch cannot
// hide the latency of their wide levels.  Sparse large graphs (road-like,
// thousands of levels) run block: their cost is per level, not per edge.
#ifndef GBBC_BLOCK_MAX_VERTICES
#define GBBC_BLOCK_MAX_VERTICES 65536
#endif
constexpr long long kBlockMaxVertices = GBBC_BLOCK_MAX_VERTICES;
constexpr double kBlockMaxAvgDegree = 6.0;

bool grid_graph(const gbbc_graph* g, const BatchDesc& b) {
    long long n = (long long)b.hi - b.lo;
    if (n <= kBlockMaxVertices) return false;
    double nnz = (double)g->h_row_ptr[b.hi] - (double)g->h_row_ptr[b.lo];
    return nnz > kBlockMaxAvgDegree * (double)n;
}

// Grid or block for each batch: fixed by the options, forced to grid when
// per-level state is kept or traced.  Under GBBC_SCHEDULE_AUTO, batches of
// large dense graphs (grid_graph) run grid; the others run block unless a
// timed trial (batches spread over the call's list, whose results are kept)
// shows grid faster; the choice is kept per handle.
gbbc_status dispatch(gbbc_graph* g, const std::vector<BatchDesc>& bs, cudaStream_t st) {
    int sched = g->opt.schedule;
    if (g->k_dist || (g->opt.flags & GBBC_TRACE)) sched = GBBC_SCHEDULE_GRID;
    std::vector<BatchDesc> small, large;
    if (sched == GBBC_SCHEDULE_AUTO) {
        for (const BatchDesc& b : bs) (grid_graph(g, b) ? large : small).push_back(b);
    } else {
        (sched == GBBC_SCHEDULE_BLOCK ? small : large) = bs;
    }
    int small_sched = sched == GBBC_SCHEDULE_AUTO ? g->tuned_schedule : sched;
    if (!small.empty() && small_sched == 0) {
        if (small.size() >= (size_t)std::max(2, g->nsm / 4)) {
            // enough batches to give every SM a cluster of its own: the grid
            // schedule, one batch at a time with a read-back per level, cannot
            // win, and a trial of it on a long batch would cost seconds
            g->tuned_schedule = GBBC_SCHEDULE_BLOCK;
            small_sched = GBBC_SCHEDULE_BLOCK;
        } else if (small.size() >= 2) {
            // Timed trial on batches spread evenly over the list (the list may
            // be sorted by cost, e.g. by the grouping network): one in the grid
            // schedule (three from 32 batches on), one wave of up to nsm in the
            // block schedule.
            // Throughput is compared in source-edge units, since the batches
            // of a multi-graph handle differ in size.  The trial's results are
            // kept; the other batches follow in list order.
            const size_t m = small.size();
            std::vector<char> used(m, 0);
            std::vector<BatchDesc> tg, tb, rest;
            auto work = [&](const BatchDesc& b) {
                return (double)b.nsrc * (1.0 + (double)(g->h_row_ptr[b.hi] - g->h_row_ptr[b.lo]));
            };
            const size_t ngrid = m >= 32 ? 3 : 1;
            for (size_t j = 0; j < ngrid; ++j) {
                size_t i = (size_t)(((double)j + 0.5) * (double)m / (double)ngrid);
                if (i < m && !used[i]) used[i] = 1, tg.push_back(small[i]);
            }
            const size_t nblk = std::min<size_t>(m - tg.size(), (size_t)g->nsm);
            for (size_t j = 0; j < nblk; ++j) {
                size_t i = (size_t)(((double)j + 0.5) * (double)m / (double)nblk);
                while (i < m && used[i]) ++i;
                if (i >= m) {
                    i = 0;
                    while (i < m && used[i]) ++i;
                }
                if (i < m) used[i] = 1, tb.push_back(small[i]);
            }
            for (size_t i = 0; i < m; ++i)
                if (!used[i]) rest.push_back(small[i]);
            CKS(alloc_slot(g));
            CK(g, cudaStreamSynchronize(st));
            double w_grid = 0, w_block = 0;
            double t0 = now_s();
            for (const BatchDesc& b : tg) {
                CKS(run_batch(g, b, st));
                w_grid += work(b);
            }
            CK(g, cudaStreamSynchronize(st));
            double t_grid = now_s() - t0;
            for (const BatchDesc& b : tb) w_block += work(b);
            t0 = now_s();
            if (!tb.empty()) CKS(run_block_mode(g, tb.data(), (int)tb.size(), st));
            double t_block = now_s() - t0;
            g->tuned_schedule = tb.empty() || w_block / t_block > w_grid / t_grid ? GBBC_SCHEDULE_BLOCK
                                                                                  : GBBC_SCHEDULE_GRID;
            small_sched = g->tuned_schedule;
            small.swap(rest);
        } else {
            small_sched = GBBC_SCHEDULE_BLOCK;
        }
    }
    if (small_sched == GBBC_SCHEDULE_BLOCK) {
        // A few batches beyond a whole number of resident-cluster rounds would
        // each run a last round alone on one cluster.  On large graphs the
        // grid schedule runs such a batch on the whole GPU in about half that
        // time (1024^2 grid: 0.37 s against 0.75 s), so they go there.
        const int nb = (int)small.size();
        if (nb > 0) {
            const int csize = block_csize(g, nb);
            const int R = std::max(1, std::min(g->max_clusters[ilog2(csize)], g->nsm / csize));
            const int rounds = (nb + R - 1) / R;
            const int left = nb - (rounds - 1) * R;
            long long nmin = LLONG_MAX;
            for (const BatchDesc& b : small) nmin = std::min<long long>(nmin, (long long)b.hi - b.lo);
            if (rounds >= 2 && left <= R / 4 && nmin > kBlockMaxVertices) {
                CKS(run_grid_batches(g, small.data() + (nb - left), (size_t)left, st));
                small.resize((size_t)(nb - left));
            }
        }
        if (!small.empty()) CKS(run_block_mode(g, small.data(), (int)small.size(), st));
    } else {
        CKS(run_grid_batches(g, small.data(), small.size(), st));
    }
    CKS(run_grid_batches(g, large.data(), large.size(), st));
    g->stats.schedule = large.empty() ? small_sched : (small.empty() ? GBBC_SCHEDULE_GRID : GBBC_SCHEDULE_AUTO);
    return GBBC_OK;
}

gbbc_status finish_create(gbbc_graph* g, cudaStream_t st) {
    bc_clear_trace(g);
    size_t count = g->goff.size() - 1;
    g->graph_max_deg.assign(count, 0);
    g->wide_graph.assign(count, 0);
    for (size_t i = 0; i < count; ++i)
        for (long long v = g->goff[i]; v < g->goff[i + 1]; ++v)
            g->graph_max_deg[i] = std::max<long long>(g->graph_max_deg[i], g->h_row_ptr[v + 1] - g->h_row_ptr[v]);
    size_t n1 = (size_t)std::max<int32_t>(g->n, 1);
    CKS(dalloc_t(g, &g->d_bc, 2 * n1));
    CKS(dalloc_t(g, &g->d_bc_out, n1));
    CK(g, cudaMemsetAsync(g->d_bc, 0, 2 * n1 * sizeof(u64), st));
    g->stats.batch_width = g->opt.batch_width == 0 ? 64 : g->opt.batch_width;
    g->stats.schedule = g->opt.schedule;
    g->stats.policy = g->opt.policy;
    CK(g, cudaStreamSynchronize(st));
    return GBBC_OK;
}

}  // namespace

extern "C" {

void bc_options_init(gbbc_options* opt) {
    if (opt) *opt = default_options();
}

gbbc_status bc_graph_create(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                            const gbbc_options* opt, void* stream, gbbc_graph** out) {
    if (!out) return GBBC_ERR_INVALID;
    *out = nullptr;
    if (n < 0 || nnz < 0 || nnz >= 0x7fffffffLL || !row_ptr || (nnz > 0 && !col)) return GBBC_ERR_INVALID;
    gbbc_graph* g = new gbbc_graph();
    std::memset(&g->stats, 0, sizeof(g->stats));
    cudaStream_t st = (cudaStream_t)stream;
    gbbc_status r = read_options(g, opt);
    if (r == GBBC_OK) r = init_device(g);
    if (r == GBBC_OK) {
        g->n = n;
        g->nnz = nnz;
        g->goff = {0, (long long)n};
        r = to_host(g, g->h_row_ptr, row_ptr, (size_t)n + 1, st);
    }
    if (r == GBBC_OK) r = check_row_ptr(g);
    if (r == GBBC_OK) r = dalloc_t(g, &g->d_row_ptr, (size_t)n + 1);
    if (r == GBBC_OK) r = dalloc_t(g, &g->d_col, (size_t)std::max<int64_t>(nnz, 1));
    if (r == GBBC_OK) r = to_device(g, g->d_row_ptr, g->h_row_ptr.data(), ((size_t)n + 1) * sizeof(int32_t), st);
    if (r == GBBC_OK) r = to_device(g, g->d_col, col, (size_t)nnz * sizeof(int32_t), st);
    if (r == GBBC_OK) r = check_graph(g, st);
    if (r == GBBC_OK) r = finish_create(g, st);
    if (r != GBBC_OK) {
        release_failed(g, r);
        return r;
    }
    *out = g;
    return GBBC_OK;
}

gbbc_status bc_graph_create_weighted(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                                     const int32_t* weight, const gbbc_options* opt, void* stream,
                                     gbbc_graph** out) {
    if (!out) return GBBC_ERR_INVALID;
    *out = nullptr;
    if (nnz > 0 && !weight) return GBBC_ERR_INVALID;
    gbbc_status r = bc_graph_create(n, nnz, row_ptr, col, opt, stream, out);
    if (r != GBBC_OK) return r;
    gbbc_graph* g = *out;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> w;
    r = to_host(g, w, weight, (size_t)nnz, st);
    int32_t maxw = 1;
    if (r == GBBC_OK) {
        for (long long p = 0; p < nnz; ++p) {
            if (w[p] < 1 || w[p] > kMaxWeight) {
                r = fail(g, GBBC_ERR_INVALID, "weight %d at entry %lld outside [1, %d]", w[p], p, kMaxWeight);
                break;
            }
            maxw = std::max(maxw, w[p]);
        }
    }
    if (r == GBBC_OK && (long long)maxw * std::max<long long>(n - 1, 0) > 0x7fffffffLL - kMaxWeight)
        r = fail(g, GBBC_ERR_INVALID, "max weight %d times n - 1 may exceed the int32 distance range", maxw);
    if (r == GBBC_OK && g->opt.validate) {  // symmetric weights: w(u, v) == w(v, u)
        std::vector<int32_t> hc((size_t)nnz);
        if (nnz > 0 && cudaMemcpy(hc.data(), g->d_col, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
                           cudaSuccess)
            r = fail(g, GBBC_ERR_CUDA, "copy of col failed");
        for (int32_t u = 0; u < n && r == GBBC_OK; ++u)
            for (int32_t p = g->h_row_ptr[u]; p < g->h_row_ptr[u + 1]; ++p) {
                const int32_t v = hc[p];
                const int32_t* b = hc.data() + g->h_row_ptr[v];
                const int32_t* e = hc.data() + g->h_row_ptr[v + 1];
                const int32_t* q = std::lower_bound(b, e, u);  // rows are sorted (checked by validation)
                if (q == e || *q != u || w[q - hc.data()] != w[p]) {
                    r = fail(g, GBBC_ERR_INVALID, "weight of edge (%d, %d) differs from (%d, %d)", u, v, v, u);
                    break;
                }
            }
    }
    if (r == GBBC_OK) r = dalloc_t(g, &g->d_w, (size_t)std::max<int64_t>(nnz, 1));
    if (r == GBBC_OK) r = to_device(g, g->d_w, w.data(), (size_t)nnz * sizeof(int32_t), st);
    if (r == GBBC_OK && cudaStreamSynchronize(st) != cudaSuccess) r = fail(g, GBBC_ERR_CUDA, "sync failed");
    if (r != GBBC_OK) {
        release_failed(g, r);
        *out = nullptr;
        return r;
    }
    g->max_w = maxw;
    return GBBC_OK;
}

gbbc_status bc_graph_create_multi(int32_t count, const int32_t* n, const int64_t* nnz, const int32_t* const* row_ptr,
                                  const int32_t* const* col, const gbbc_options* opt, void* stream,
                                  gbbc_graph** out) {
    if (!out) return GBBC_ERR_INVALID;
    *out = nullptr;
    if (count < 0 || (count > 0 && (!n || !nnz || !row_ptr || !col))) return GBBC_ERR_INVALID;
    long long N = 0, M = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (n[i] < 0 || nnz[i] < 0 || !row_ptr[i] || (nnz[i] > 0 && !col[i])) return GBBC_ERR_INVALID;
        N += n[i];
        M += nnz[i];
    }
    if (N >= 0x7fffffffLL || M >= 0x7fffffffLL) return GBBC_ERR_INVALID;
    gbbc_graph* g = new gbbc_graph();
    std::memset(&g->stats, 0, sizeof(g->stats));
    cudaStream_t st = (cudaStream_t)stream;
    gbbc_status r = read_options(g, opt);
    if (r == GBBC_OK) r = init_device(g);
    if (r == GBBC_OK) {
        g->n = (int32_t)N;
        g->nnz = M;
        g->goff.assign(1, 0);
        g->h_row_ptr.assign(1, 0);
        r = dalloc_t(g, &g->d_row_ptr, (size_t)N + 1);
    }
    if (r == GBBC_OK) r = dalloc_t(g, &g->d_col, (size_t)std::max<long long>(M, 1));
    int32_t* tmp = nullptr;
    long long maxm = 1;
    for (int32_t i = 0; i < count; ++i) maxm = std::max<long long>(maxm, nnz[i]);
    if (r == GBBC_OK) r = dalloc_t(g, &tmp, (size_t)maxm);
    long long voff = 0, eoff = 0;
    std::vector<int32_t> rp;
    for (int32_t i = 0; i < count && r == GBBC_OK; ++i) {
        r = to_host(g, rp, row_ptr[i], (size_t)n[i] + 1, st);
        if (r != GBBC_OK) break;
        if (rp[0] != 0 || (long long)rp[n[i]] != nnz[i]) {
            r = fail(g, GBBC_ERR_INVALID, "graph %d: row_ptr[0] must be 0 and row_ptr[n] = nnz", i);
            break;
        }
        for (int32_t v = 0; v < n[i]; ++v)
            if (rp[v + 1] < rp[v]) r = fail(g, GBBC_ERR_INVALID, "graph %d: row_ptr decreases at %d", i, v);
        if (r != GBBC_OK) break;
        for (int32_t v = 1; v <= n[i]; ++v) g->h_row_ptr.push_back((int32_t)(rp[v] + eoff));
        if (nnz[i] > 0) {
            r = to_device(g, tmp, col[i], (size_t)nnz[i] * sizeof(int32_t), st);
            if (r != GBBC_OK) break;
            launch_offset_copy(tmp, g->d_col + eoff, nnz[i], (int32_t)voff, st);
            g->stats.kernel_launches++;
        }
        voff += n[i];
        eoff += nnz[i];
        g->goff.push_back(voff);
    }
    if (r == GBBC_OK && cudaStreamSynchronize(st) != cudaSuccess) r = fail(g, GBBC_ERR_CUDA, "union copy failed");
    if (tmp) dfree(g, tmp);
    if (r == GBBC_OK) r = to_device(g, g->d_row_ptr, g->h_row_ptr.data(), ((size_t)N + 1) * sizeof(int32_t), st);
    if (r == GBBC_OK) r = check_graph(g, st);
    if (r == GBBC_OK) r = finish_create(g, st);
    if (r != GBBC_OK) {
        release_failed(g, r);
        return r;
    }
    *out = g;
    return GBBC_OK;
}

gbbc_status bc_compute(gbbc_graph* g, const int32_t* sources, int64_t k, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (k < 0 || (k > 0 && !sources)) return fail(g, GBBC_ERR_INVALID, "bad source list");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> src;
    CKS(to_host(g, src, sources, (size_t)k, st));
    std::vector<int32_t> gid((size_t)k);
    for (long long i = 0; i < k; ++i) {
        if (src[i] < 0 || src[i] >= g->n)
            return fail(g, GBBC_ERR_INVALID, "source %lld = %d outside [0, %d)", i, src[i], g->n);
        // graph of the source (multi-graph handles): last offset <= src
        gid[i] = (int32_t)(std::upper_bound(g->goff.begin(), g->goff.end(), (long long)src[i]) - g->goff.begin()) - 1;
    }
    return compute_impl(g, src, gid, st);
}

gbbc_status bc_compute_multi(gbbc_graph* g, const int32_t* graph_id, const int32_t* local_src, int64_t k,
                             void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (k < 0 || (k > 0 && (!graph_id || !local_src))) return fail(g, GBBC_ERR_INVALID, "bad source list");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> gid, loc;
    CKS(to_host(g, gid, graph_id, (size_t)k, st));
    CKS(to_host(g, loc, local_src, (size_t)k, st));
    int32_t count = (int32_t)g->goff.size() - 1;
    std::vector<int32_t> src((size_t)k);
    for (long long i = 0; i < k; ++i) {
        if (gid[i] < 0 || gid[i] >= count) return fail(g, GBBC_ERR_INVALID, "graph_id[%lld] = %d", i, gid[i]);
        long long nv = g->goff[gid[i] + 1] - g->goff[gid[i]];
        if (loc[i] < 0 || loc[i] >= nv)
            return fail(g, GBBC_ERR_INVALID, "local source %lld = %d outside graph %d", i, loc[i], gid[i]);
        src[i] = (int32_t)(g->goff[gid[i]] + loc[i]);
    }
    return compute_impl(g, src, gid, st);
}

gbbc_status bc_read(gbbc_graph* g, double* bc_out, int32_t graph_id, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (!bc_out) return fail(g, GBBC_ERR_INVALID, "bc_out is NULL");
    int32_t count = (int32_t)g->goff.size() - 1;
    if (graph_id < -1 || graph_id >= count) return fail(g, GBBC_ERR_INVALID, "graph_id %d", graph_id);
    long long lo = graph_id < 0 ? 0 : g->goff[graph_id];
    long long hi = graph_id < 0 ? g->n : g->goff[graph_id + 1];
    cudaStream_t st = (cudaStream_t)stream;
    if (hi > lo) {
        bool dev = is_device_ptr(bc_out);
        double* dst = dev ? bc_out : g->d_bc_out;
        launch_bc_to_double(g->d_bc + 2 * lo, dst, hi - lo, false, st);
        g->stats.kernel_launches++;
        CK(g, cudaGetLastError());
        if (!dev)
            CK(g, cudaMemcpyAsync(bc_out, dst, (size_t)(hi - lo) * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(g, cudaStreamSynchronize(st));
    return GBBC_OK;
}

gbbc_status bc_read_fixed(gbbc_graph* g, uint64_t* out, int32_t graph_id, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (!out) return fail(g, GBBC_ERR_INVALID, "out is NULL");
    int32_t count = (int32_t)g->goff.size() - 1;
    if (graph_id < -1 || graph_id >= count) return fail(g, GBBC_ERR_INVALID, "graph_id %d", graph_id);
    long long lo = graph_id < 0 ? 0 : g->goff[graph_id];
    long long hi = graph_id < 0 ? g->n : g->goff[graph_id + 1];
    cudaStream_t st = (cudaStream_t)stream;
    if (hi > lo)
        CK(g, cudaMemcpyAsync(out, g->d_bc + 2 * lo, (size_t)(hi - lo) * 2 * sizeof(u64), cudaMemcpyDefault, st));
    CK(g, cudaStreamSynchronize(st));
    return GBBC_OK;
}

gbbc_status bc_add_fixed(gbbc_graph* g, const uint64_t* partial, int32_t graph_id, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (!partial) return fail(g, GBBC_ERR_INVALID, "partial is NULL");
    int32_t count = (int32_t)g->goff.size() - 1;
    if (graph_id < -1 || graph_id >= count) return fail(g, GBBC_ERR_INVALID, "graph_id %d", graph_id);
    long long lo = graph_id < 0 ? 0 : g->goff[graph_id];
    long long hi = graph_id < 0 ? g->n : g->goff[graph_id + 1];
    cudaStream_t st = (cudaStream_t)stream;
    if (hi > lo) {
        const size_t bytes = (size_t)(hi - lo) * 2 * sizeof(u64);
        const u64* src = reinterpret_cast<const u64*>(partial);
        u64* stage = nullptr;
        if (!is_device_ptr(partial)) {  // host partial: stage it on the device
            CKS(dalloc(g, (void**)&stage, bytes));
            cudaError_t e = cudaMemcpyAsync(stage, partial, bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) {
                dfree(g, stage);
                return fail(g, GBBC_ERR_CUDA, "staging copy failed: %s", cudaGetErrorString(e));
            }
            src = stage;
        }
        launch_add_fixed(g->d_bc + 2 * lo, src, hi - lo, st);
        g->stats.kernel_launches++;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (stage) dfree(g, stage);
        if (e != cudaSuccess) return fail(g, GBBC_ERR_CUDA, "bc_add_fixed: %s", cudaGetErrorString(e));
    }
    g->last_stream = st;
    return GBBC_OK;
}

gbbc_status bc_read_source_state(gbbc_graph* g, int64_t source_index, int32_t* dist, uint64_t* sigma,
                                 uint8_t* overflow) {
    if (!g) return GBBC_ERR_INVALID;
    if (!g->k_dist) return fail(g, GBBC_ERR_STATE, "no kept state (set GBBC_KEEP_STATE and call bc_compute)");
    if (source_index < 0 || source_index >= g->k_count)
        return fail(g, GBBC_ERR_INVALID, "source_index %lld outside [0, %lld)", (long long)source_index, g->k_count);
    size_t at = (size_t)source_index * (size_t)g->n;
    CK(g, cudaStreamSynchronize(g->last_stream));
    if (dist) CK(g, cudaMemcpy(dist, g->k_dist + at, (size_t)g->n * sizeof(int32_t), cudaMemcpyDefault));
    if (sigma) CK(g, cudaMemcpy(sigma, g->k_sigma + at, (size_t)g->n * sizeof(uint64_t), cudaMemcpyDefault));
    if (overflow) CK(g, cudaMemcpy(overflow, g->k_ovf + at, (size_t)g->n, cudaMemcpyDefault));
    return GBBC_OK;
}

gbbc_status bc_reset(gbbc_graph* g) {
    if (!g) return GBBC_ERR_INVALID;
    CK(g, cudaStreamSynchronize(g->last_stream));
    CK(g, cudaMemset(g->d_bc, 0, 2 * (size_t)std::max<int32_t>(g->n, 1) * sizeof(u64)));
    CKS(alloc_keep(g, 0, nullptr));
    return GBBC_OK;
}

gbbc_status bc_sync(gbbc_graph* g) {
    if (!g) return GBBC_ERR_INVALID;
    CK(g, cudaStreamSynchronize(g->last_stream));
    CK(g, cudaGetLastError());
    return GBBC_OK;
}

void bc_graph_destroy(gbbc_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    const bool pooled = g->ast && device_pool(g->device);
    for (auto& a : g->allocs) {
        if (pooled) cudaFreeAsync(a.first, g->ast);
        else cudaFree(a.first);
    }
    g->allocs.clear();
    if (g->ast) {
        cudaStreamSynchronize(g->ast);
        cudaStreamDestroy(g->ast);
    }
    if (g->slot.hctr) cudaFreeHost(g->slot.hctr);
    for (auto& w : g->workers) {
        if (w.slot.hctr) cudaFreeHost(w.slot.hctr);
        if (w.st) cudaStreamDestroy(w.st);
        if (w.ev) cudaEventDestroy(w.ev);
    }
    if (g->ev_start) cudaEventDestroy(g->ev_start);
    for (cudaEvent_t e : g->p_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    delete g;
}

const char* bc_status_string(gbbc_status s) {
    switch (s) {
        case GBBC_OK: return "GBBC_OK";
        case GBBC_ERR_INVALID: return "GBBC_ERR_INVALID";
        case GBBC_ERR_OOM: return "GBBC_ERR_OOM";
        case GBBC_ERR_CUDA: return "GBBC_ERR_CUDA";
        case GBBC_ERR_TIMEOUT: return "GBBC_ERR_TIMEOUT";
        case GBBC_ERR_CAPACITY: return "GBBC_ERR_CAPACITY";
        case GBBC_ERR_STATE: return "GBBC_ERR_STATE";
    }
    return "GBBC_UNKNOWN_STATUS";
}

gbbc_status bc_last_error_detail(const gbbc_graph* g, char* buf, size_t len) {
    if (!buf || len == 0) return GBBC_ERR_INVALID;
    std::snprintf(buf, len, "%s", g ? g->err.c_str() : tl_create_err.c_str());
    return GBBC_OK;
}

gbbc_status bc_policy_load(gbbc_graph* g, const float* params, size_t bytes) {
    if (!g) return GBBC_ERR_INVALID;
    const size_t want = (size_t)bc_mlp_param_count(2) * sizeof(float);
    if (!params) {  // unload
        if (g->d_policy) dfree(g, g->d_policy);
        g->d_policy = nullptr;
        return GBBC_OK;
    }
    if (bytes != want) return fail(g, GBBC_ERR_INVALID, "policy weights: %zu bytes, expected %zu", bytes, want);
    float* tmp = nullptr;
    CKS(dalloc(g, (void**)&tmp, want));
    gbbc_status r = to_device(g, tmp, params, want, g->last_stream);
    if (r == GBBC_OK && !g->d_policy) r = dalloc(g, &g->d_policy, (want / sizeof(float)) * 2);
    if (r == GBBC_OK && policy_to_half(tmp, g->d_policy, g->last_stream) != cudaSuccess)
        r = fail(g, GBBC_ERR_CUDA, "policy conversion failed");
    if (r == GBBC_OK && cudaStreamSynchronize(g->last_stream) != cudaSuccess) r = fail(g, GBBC_ERR_CUDA, "sync");
    dfree(g, tmp);
    return r;
}

gbbc_status bc_release_memory(int32_t device) {
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GBBC_ERR_CUDA;
    }
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return GBBC_OK;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
        cudaGetLastError();
        return GBBC_ERR_CUDA;
    }
    return GBBC_OK;
}

gbbc_status bc_grouping_load(gbbc_graph* g, const float* params, size_t bytes) {
    if (!g) return GBBC_ERR_INVALID;
    const int np = (int)bc_mlp_param_count(1);
    const size_t want = (size_t)np * sizeof(float);
    if (!params) {
        if (g->d_grouping) dfree(g, g->d_grouping);
        g->d_grouping = nullptr;
        return GBBC_OK;
    }
    if (bytes != want) return fail(g, GBBC_ERR_INVALID, "grouping weights: %zu bytes, expected %zu", bytes, want);
    float* tmp = nullptr;
    CKS(dalloc(g, (void**)&tmp, want));
    gbbc_status r = to_device(g, tmp, params, want, g->last_stream);
    if (r == GBBC_OK && !g->d_grouping) r = dalloc(g, &g->d_grouping, (size_t)np * 2);
    if (r == GBBC_OK && mlp_to_half(tmp, g->d_grouping, np, g->last_stream) != cudaSuccess)
        r = fail(g, GBBC_ERR_CUDA, "grouping conversion failed");
    if (r == GBBC_OK && cudaStreamSynchronize(g->last_stream) != cudaSuccess) r = fail(g, GBBC_ERR_CUDA, "sync");
    dfree(g, tmp);
    return r;
}

namespace {
gbbc_status grouping_sources(gbbc_graph* g, const int32_t* sources, int64_t k, const void* out,
                             std::vector<int32_t>& src, std::vector<int32_t>& gid, cudaStream_t st) {
    if (!g) return GBBC_ERR_INVALID;
    if (k < 0 || (k > 0 && (!sources || !out))) return fail(g, GBBC_ERR_INVALID, "bad arguments");
    CKS(to_host(g, src, sources, (size_t)k, st));
    gid.assign((size_t)k, 0);
    for (long long i = 0; i < k; ++i) {
        if (src[i] < 0 || src[i] >= g->n) return fail(g, GBBC_ERR_INVALID, "source %lld outside [0, n)", i);
        gid[i] = (int32_t)(std::upper_bound(g->goff.begin(), g->goff.end(), (long long)src[i]) - g->goff.begin()) - 1;
    }
    return GBBC_OK;
}
}  // namespace

gbbc_status bc_grouping_scores(gbbc_graph* g, const int32_t* sources, int64_t k, float* out, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (!g->d_grouping) return fail(g, GBBC_ERR_STATE, "no grouping weights loaded");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> src, gid;
    CKS(grouping_sources(g, sources, k, out, src, gid, st));
    if (k == 0) return GBBC_OK;
    std::vector<float> score;
    CKS(grouping_scores(g, src, gid, score, st));
    CK(g, cudaMemcpy(out, score.data(), (size_t)k * sizeof(float), cudaMemcpyDefault));
    return GBBC_OK;
}

gbbc_status bc_source_features(gbbc_graph* g, const int32_t* sources, int64_t k, float* out, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> src, gid;
    CKS(grouping_sources(g, sources, k, out, src, gid, st));
    if (k == 0) return GBBC_OK;
    float* d_x = nullptr;
    CKS(dalloc_t(g, &d_x, (size_t)k * 6));
    gbbc_status r = source_features(g, src, gid, d_x, st);
    if (r == GBBC_OK && cudaMemcpy(out, d_x, (size_t)k * 6 * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        r = fail(g, GBBC_ERR_CUDA, "copy failed");
    dfree(g, d_x);
    return r;
}

gbbc_status bc_get_trace(const gbbc_graph* g, gbbc_level_trace* out, int64_t max, int64_t* count) {
    if (!g || (max > 0 && !out)) return GBBC_ERR_INVALID;
    long long n = (long long)g->trace.size();
    if (count) *count = n;
    for (long long i = 0; i < n && i < max; ++i) out[i] = g->trace[i];
    return GBBC_OK;
}

gbbc_status bc_clear_trace(gbbc_graph* g) {
    if (!g) return GBBC_ERR_INVALID;
    g->trace.clear();
    for (int k = 0; k < PK_COUNT; ++k) {
        std::memset(&g->prof[k], 0, sizeof(gbbc_kernel_profile));
        std::snprintf(g->prof[k].name, sizeof(g->prof[k].name), "%s", kProfNames[k]);
    }
    return GBBC_OK;
}

gbbc_status bc_get_profile(const gbbc_graph* g, gbbc_kernel_profile* out, int32_t max, int32_t* count) {
    if (!g || (max > 0 && !out)) return GBBC_ERR_INVALID;
    if (count) *count = PK_COUNT;
    for (int k = 0; k < PK_COUNT && k < max; ++k) out[k] = g->prof[k];
    return GBBC_OK;
}

gbbc_status bc_partition(gbbc_graph* g, const int32_t* part, int32_t P, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (g->goff.size() != 2 || g->d_w)
        return fail(g, GBBC_ERR_INVALID, "bc_partition: single-graph, unweighted handles only");
    if (P < 1 || P > std::max<int32_t>(g->n, 1) || P > kMaxParts)
        return fail(g, GBBC_ERR_INVALID, "bc_partition: P = %d (1 to %d, at most n)", P, kMaxParts);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = g->n;
    std::vector<int32_t> hp;
    if (part) {
        CKS(to_host(g, hp, part, (size_t)n, st));
        for (int32_t v = 0; v < n; ++v)
            if (hp[v] < 0 || hp[v] >= P) return fail(g, GBBC_ERR_INVALID, "part[%d] = %d outside [0, %d)", v, hp[v], P);
    } else {  // P contiguous ranges of vertex ids
        hp.resize((size_t)n);
        for (int32_t v = 0; v < n; ++v) hp[v] = (int32_t)(((long long)v * P) / std::max<int32_t>(n, 1));
    }
    std::vector<int32_t> col((size_t)g->nnz);
    if (g->nnz > 0)
        CK(g, cudaMemcpy(col.data(), g->d_col, (size_t)g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    // intra-part and border-edge CSRs, border nodes by part then id
    const std::vector<int32_t>& rp = g->h_row_ptr;
    std::vector<int32_t> in_rp((size_t)n + 1, 0), cut_rp((size_t)n + 1, 0), in_col, cut_col;
    in_col.reserve((size_t)g->nnz);
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) (hp[col[p]] == hp[v] ? in_col : cut_col).push_back(col[p]);
        in_rp[v + 1] = (int32_t)in_col.size();
        cut_rp[v + 1] = (int32_t)cut_col.size();
    }
    std::vector<std::vector<int32_t>> byp((size_t)P);
    for (int32_t v = 0; v < n; ++v)
        if (cut_rp[v + 1] > cut_rp[v]) byp[hp[v]].push_back(v);
    std::vector<int32_t> border, bpart, bidx((size_t)n, -1);
    std::vector<long long> boff((size_t)P + 1, 0), moff((size_t)P + 1, 0);
    for (int32_t q = 0; q < P; ++q) {
        for (int32_t v : byp[q]) {
            bidx[v] = (int32_t)border.size();
            border.push_back(v);
            bpart.push_back(q);
        }
        const long long B = (long long)byp[q].size();
        boff[q + 1] = boff[q] + B;
        moff[q + 1] = moff[q] + B * B;
    }
    const long long nbt = (long long)border.size(), entries = moff[P];
    const double need = (double)entries * (4 + 21) + (double)nbt * kLanes * (2 * 4 + 3 * 21);
    if (entries >= 0x7fffffffLL || need > 0.5 * (double)avail_bytes(g->device))
        return fail(g, GBBC_ERR_OOM, "bc_partition: %lld border nodes need %.3g bytes of border matrices", nbt, need);
    free_partition(g);
    gbbc_graph::Part& q = g->pt;
    const size_t n1 = (size_t)std::max<int32_t>(n, 1);
    const size_t e1 = (size_t)std::max<long long>(entries, 1), c1 = (size_t)std::max<long long>(nbt, 1) * kLanes;
    CKS(dalloc_t(g, &q.part, n1));
    CKS(dalloc_t(g, &q.in_rp, n1 + 1));
    CKS(dalloc_t(g, &q.in_col, std::max<size_t>(in_col.size(), 1)));
    CKS(dalloc_t(g, &q.cut_rp, n1 + 1));
    CKS(dalloc_t(g, &q.cut_col, std::max<size_t>(cut_col.size(), 1)));
    CKS(dalloc_t(g, &q.border, std::max<size_t>(border.size(), 1)));
    CKS(dalloc_t(g, &q.bidx, n1));
    CKS(dalloc_t(g, &q.bpart, std::max<size_t>(bpart.size(), 1)));
    CKS(dalloc_t(g, &q.boff, boff.size()));
    CKS(dalloc_t(g, &q.moff, moff.size()));
    CKS(dalloc_t(g, &q.BM, e1));
    CKS(alloc_wide_arr(g, q.SM, e1));
    CKS(dalloc_t(g, &q.D, c1));
    CKS(dalloc_t(g, &q.D1, c1));
    CKS(alloc_wide_arr(g, q.S1, c1));
    CKS(alloc_wide_arr(g, q.A, c1));
    CKS(alloc_wide_arr(g, q.Sig, c1));
    CKS(dalloc_t(g, &q.changed, 1));
    CKS(dalloc_t(g, &q.lane_b, kLanes));
    CKS(dalloc_t(g, &q.dist, n1 * kLanes));
    CKS(dalloc_t(g, &q.need, (size_t)P * (n1 + 1)));
    CKS(dalloc_t(g, &q.done, (size_t)P));
    CKS(dalloc_t(g, &q.ctl, (size_t)(2 + 2 * P)));
    CKS(dalloc_t(g, &q.off, n1 + 2));
    q.in_nnz = (long long)in_col.size();
    q.cut_nnz = (long long)cut_col.size();
    q.nbt = nbt;
    q.h_boff = boff;
    q.h_moff = moff;
    CKS(to_device(g, q.part, hp.data(), (size_t)n * sizeof(int32_t), st));
    CKS(to_device(g, q.in_rp, in_rp.data(), in_rp.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.in_col, in_col.data(), in_col.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.cut_rp, cut_rp.data(), cut_rp.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.cut_col, cut_col.data(), cut_col.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.border, border.data(), border.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.bidx, bidx.data(), (size_t)n * sizeof(int32_t), st));
    CKS(to_device(g, q.bpart, bpart.data(), bpart.size() * sizeof(int32_t), st));
    CKS(to_device(g, q.boff, boff.data(), boff.size() * sizeof(long long), st));
    CKS(to_device(g, q.moff, moff.data(), moff.size() * sizeof(long long), st));
    launch_fill_i32(q.BM, (long long)e1, -1, st);
    CKS(clear_wide_arr(g, q.SM, e1, st));
    // border matrices (Sec. IV-B) and sigma matrices (Sec. V-A): a BFS inside
    // its part from every border node, 64 border nodes per batch
    CKS(alloc_slot(g));
    Csr cin{n, q.in_nnz, q.in_rp, q.in_col};
    bool wide = g->wide_graph[0] != 0;
    for (long long b0 = 0; b0 < nbt; b0 += kLanes) {
        BatchDesc bd;
        bd.gi = 0;
        bd.lo = 0;
        bd.hi = n;
        bd.first = 0;
        bd.nsrc = (int)std::min<long long>(kLanes, nbt - b0);
        int32_t lane_b[kLanes];
        for (int j = 0; j < kLanes; ++j) lane_b[j] = j < bd.nsrc ? (int32_t)(b0 + j) : -1;
        for (int j = 0; j < bd.nsrc; ++j) bd.src[j] = border[(size_t)(b0 + j)];
        CK(g, cudaMemcpyAsync(q.lane_b, lane_b, sizeof(lane_b), cudaMemcpyHostToDevice, st));
        std::vector<long long> off;
        CKS(part_forward(g, cin, bd, st, wide, off, nullptr));
        for (size_t l = 0; l + 1 < off.size(); ++l)
            launch_part_extract(g->slot, off[l], off[l + 1], (int)l, wide, 0, q.bidx, q.bpart, q.boff, q.moff,
                                q.lane_b, q.BM, q.SM.mod, q.SM.N, q.SM.X, q.SM.big, g->nsm, st);
        CK(g, cudaGetLastError());
        CK(g, cudaStreamSynchronize(st));  // lane_b is reused by the next batch
    }
    q.P = P;
    g->last_stream = st;
    return GBBC_OK;
}

gbbc_status bc_partition_info(const gbbc_graph* g, gbbc_partition_info* out) {
    if (!g || !out) return GBBC_ERR_INVALID;
    std::memset(out, 0, sizeof(*out));
    out->parts = g->pt.P;
    out->border_nodes = g->pt.nbt;
    out->border_edges = g->pt.cut_nnz;
    out->intra_entries = g->pt.in_nnz;
    out->matrix_entries = g->pt.P ? g->pt.h_moff.back() : 0;
    out->refinement_sweeps = g->pt.sweeps;
    out->backward_waits = g->pt.waits;
    return GBBC_OK;
}

gbbc_status bc_read_border_matrix(gbbc_graph* g, int32_t p, int64_t* nodes, int32_t* border, int32_t* bm,
                                  uint64_t* sigma_m, uint8_t* overflow) {
    if (!g) return GBBC_ERR_INVALID;
    const gbbc_graph::Part& q = g->pt;
    if (!q.P) return fail(g, GBBC_ERR_STATE, "no partition (bc_partition)");
    if (p < 0 || p >= q.P) return fail(g, GBBC_ERR_INVALID, "part %d outside [0, %d)", p, q.P);
    const long long b0 = q.h_boff[p], B = q.h_boff[p + 1] - b0, m0 = q.h_moff[p];
    if (nodes) *nodes = B;
    CK(g, cudaStreamSynchronize(g->last_stream));
    if (B == 0) return GBBC_OK;
    if (border) CK(g, cudaMemcpy(border, q.border + b0, (size_t)B * sizeof(int32_t), cudaMemcpyDefault));
    if (bm) CK(g, cudaMemcpy(bm, q.BM + m0, (size_t)(B * B) * sizeof(int32_t), cudaMemcpyDefault));
    if (sigma_m) CK(g, cudaMemcpy(sigma_m, q.SM.mod + m0, (size_t)(B * B) * sizeof(uint64_t), cudaMemcpyDefault));
    if (overflow) CK(g, cudaMemcpy(overflow, q.SM.big + m0, (size_t)(B * B), cudaMemcpyDefault));
    return GBBC_OK;
}

gbbc_status bc_compute_partitioned(gbbc_graph* g, const int32_t* sources, int64_t k, void* stream) {
    if (!g) return GBBC_ERR_INVALID;
    if (!g->pt.P) return fail(g, GBBC_ERR_STATE, "no partition (call bc_partition first)");
    if (k < 0 || (k > 0 && !sources)) return fail(g, GBBC_ERR_INVALID, "bad source list");
    if (g->opt.batch_width == 1) return fail(g, GBBC_ERR_INVALID, "the partitioned method has no one-source form");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> src;
    CKS(to_host(g, src, sources, (size_t)k, st));
    for (long long i = 0; i < k; ++i)
        if (src[i] < 0 || src[i] >= g->n)
            return fail(g, GBBC_ERR_INVALID, "source %lld = %d outside [0, %d)", i, src[i], g->n);
    CKS(alloc_keep(g, k, st));
    CKS(alloc_slot(g));
    g->last_stream = st;
    g->pt.sweeps = 0;
    g->pt.waits = 0;
    const int width = g->opt.batch_width == 32 ? 32 : kLanes;
    for (long long i = 0; i < k; i += width) {
        BatchDesc b;
        b.gi = 0;
        b.lo = 0;
        b.hi = g->n;
        b.first = i;
        b.nsrc = (int)std::min<long long>(width, k - i);
        for (int j = 0; j < b.nsrc; ++j) b.src[j] = src[(size_t)(i + j)];
        CKS(part_batch(g, b, st));
    }
    CK(g, cudaStreamSynchronize(st));
    return GBBC_OK;
}

gbbc_status bc_get_stats(const gbbc_graph* g, gbbc_stats* out) {
    if (!g || !out) return GBBC_ERR_INVALID;
    *out = g->stats;
    out->device_bytes = (int64_t)g->bytes;
    return GBBC_OK;
}

}  // extern "C"
