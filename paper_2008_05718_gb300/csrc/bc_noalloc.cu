// bc_compute_noalloc: exact Brandes BC for one small graph without any device
// (or host heap) allocation, for callers that may not allocate memory
// themselves -- for example code running inside a memory pool that owns the
// whole device, a plug-in host whose allocator must not be bypassed, or a
// real-time loop where cudaMalloc's implicit synchronisation is not allowed.
//
// All per-batch working state lives in one file-scope device array,
// g_noalloc_scratch, sized for kNoallocMaxVertices vertices.  It is part of
// the library image: every GPU that loads libgbbc.so holds it until the
// process exits.  Every call shares it, so two calls whose work overlapped on
// the GPU would race and give wrong results.  The library rules that out
// within one process: calls on one device hold a per-device host lock for
// their whole duration, and each call returns only after its work on the
// stream has finished.  The array keeps the previous call's contents:
// everything a batch needs at zero is cleared at the start of that batch.
// The host-side level boundaries of a batch live in a static per-device
// array too (not on the caller's stack, which may be small), used under the
// same lock.
//
// Host code cannot use the array's name as a device address (in host code
// the symbol is a host-side stand-in), so the device address is looked up
// with cudaGetSymbolAddress once per device, the first time a call runs on
// that device with it current.
//
// Each call first checks the caller's CSR on the device (row bounds, column
// range, sorted rows without duplicates or self-loops, symmetry) with the
// library's validation kernel, writing its flags into a word of the scratch,
// so that no later kernel reads or writes outside the caller's arrays or the
// scratch.
//
// The kernels are the same ones bc_compute launches (64 sources per batch);
// this path always expands top-down, keeps this call's BC in the scratch's
// 128-bit fixed-point vector and adds it into the caller's BC vector.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bc_internal.cuh"

using namespace gbbc;

namespace {

constexpr long long kNoallocMaxVertices = 16384;  // also in include/gbbc.h
constexpr long long kNoallocQcap = kNoallocMaxVertices * kLanes + kLanes;

constexpr long long align256(long long x) { return (x + 255) / 256 * 256; }

// Byte offsets of the regions inside the scratch array.
constexpr long long kOffVis = 0;
constexpr long long kOffNx = kOffVis + align256(8 * kNoallocMaxVertices);
constexpr long long kOffOvf = kOffNx + align256(8 * kNoallocMaxVertices);
constexpr long long kOffF = kOffOvf + align256(8 * kNoallocMaxVertices);
constexpr long long kOffSigma = kOffF + align256(2 * (long long)sizeof(MaskTag) * kNoallocMaxVertices);
constexpr long long kOffPsi = kOffSigma + align256(8 * kLanes * kNoallocMaxVertices);
constexpr long long kOffBc = kOffPsi + align256(8 * kLanes * kNoallocMaxVertices);
constexpr long long kOffQv = kOffBc + align256(16 * kNoallocMaxVertices);
constexpr long long kOffQm = kOffQv + align256(4 * kNoallocQcap);
constexpr long long kOffHeavy = kOffQm + align256(8 * kNoallocQcap);
constexpr long long kOffMedium = kOffHeavy + align256(4 * kNoallocMaxVertices);
constexpr long long kNoallocTcap = kNoallocMaxVertices * kNoallocMaxVertices / kChunk + kNoallocMaxVertices;
constexpr long long kOffHentry = kOffMedium + align256(4 * kNoallocMaxVertices);
constexpr long long kOffHacc = kOffHentry + align256(4 * kNoallocMaxVertices);
constexpr long long kOffHcarry = kOffHacc + align256(16 * kLanes * kNoallocMaxVertices);
constexpr long long kOffTasks = kOffHcarry + align256(8 * kNoallocMaxVertices);
constexpr long long kOffCtr = kOffTasks + align256(8 * kNoallocTcap);
constexpr long long kOffSrc = kOffCtr + align256((long long)sizeof(Counters));
constexpr long long kOffFlags = kOffSrc + align256(4 * kLanes);  // validation flags
constexpr long long kScratchBytes = kOffFlags + align256(4);
static_assert(kScratchBytes < (64ll << 20), "no-allocation scratch above 64 MiB");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};
// Per device: the lock that serialises calls, and the level boundaries of
// the batch in flight (static storage: untouched pages cost no memory).
std::mutex g_call_mutex[kMaxDevices];
long long g_level_off[kMaxDevices][kNoallocMaxVertices + 2];

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

bool device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

#define NA_CK(call)                               \
    do {                                          \
        if ((call) != cudaSuccess) return GBBC_ERR_CUDA; \
    } while (0)

extern "C" gbbc_status bc_compute_noalloc(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                                          const int32_t* sources, int64_t k, double* bc_out, void* stream) {
    if (n < 0 || nnz < 0 || nnz >= 0x7fffffffLL || k < 0) return GBBC_ERR_INVALID;
    if (n > kNoallocMaxVertices) return GBBC_ERR_CAPACITY;
    if (k == 0 || n == 0) return GBBC_OK;
    if (!row_ptr || !col || !sources || !bc_out) return GBBC_ERR_INVALID;
    if (!device_pointer(row_ptr) || !device_pointer(col) || !device_pointer(bc_out) || device_pointer(sources))
        return GBBC_ERR_INVALID;
    for (int64_t i = 0; i < k; ++i)
        if (sources[i] < 0 || sources[i] >= n) return GBBC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    NA_CK(scratch_address(&base));
    int dev = 0, nsm = 152;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GBBC_ERR_CUDA;
    NA_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    std::lock_guard<std::mutex> call_lock(g_call_mutex[dev]);
    long long* off = g_level_off[dev];  // level boundaries of a batch

    Slot s;
    s.n = n;
    s.vis = (u64*)(base + kOffVis);
    s.nx = (u64*)(base + kOffNx);
    s.ovf = (u64*)(base + kOffOvf);
    s.F = (MaskTag*)(base + kOffF);
    s.sigma = (u64*)(base + kOffSigma);
    s.psi = (u64*)(base + kOffPsi);
    u64* bc_fixed = (u64*)(base + kOffBc);  // this call's BC, 128-bit fixed point
    s.qv = (int32_t*)(base + kOffQv);
    s.qm = (u64*)(base + kOffQm);
    s.heavy = (int32_t*)(base + kOffHeavy);
    s.medium = (int32_t*)(base + kOffMedium);
    s.hentry = (int32_t*)(base + kOffHentry);
    s.hacc = (u64*)(base + kOffHacc);
    s.hcarry = (u64*)(base + kOffHcarry);
    s.tasks = (int2*)(base + kOffTasks);
    s.hcap = kNoallocMaxVertices;     // a row is heavy at most once per step
    s.tcap = kNoallocTcap;            // nnz <= n^2 entries in chunks, plus one partial chunk per row
    s.ctr = (Counters*)(base + kOffCtr);
    s.d_src = (int32_t*)(base + kOffSrc);
    s.qcap = (long long)n * kLanes + kLanes;
    // F is indexed [parity][n] with the stride of this graph's n
    Csr c{n, (long long)nnz, row_ptr, col};
    const int heavy_deg = 1024;
    const size_t disc_off = offsetof(Counters, heavy), disc_bytes = offsetof(Counters, err) - disc_off;
    const size_t gath_off = offsetof(Counters, lane_sum), gath_bytes = offsetof(Counters, medium) - gath_off;

    // The caller's CSR: row_ptr[0] = 0 and row_ptr[n] = nnz, then the device
    // check of every row (flags in the scratch; any flag rejects the graph).
    int32_t ends[2] = {-1, -1};
    NA_CK(cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(&ends[1], row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (ends[0] != 0 || (long long)ends[1] != (long long)nnz) return GBBC_ERR_INVALID;
    int32_t* d_flags = (int32_t*)(base + kOffFlags);
    NA_CK(cudaMemsetAsync(d_flags, 0, sizeof(int32_t), st));
    launch_validate(c, d_flags, st);
    NA_CK(cudaGetLastError());
    int32_t flags = 0;
    NA_CK(cudaMemcpyAsync(&flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (flags) return GBBC_ERR_INVALID;

    NA_CK(cudaMemsetAsync(bc_fixed, 0, 2 * (size_t)n * sizeof(u64), st));
    // heavy-row accumulators must start at zero (they are left at zero by
    // every completed step, but the array may hold an aborted call's state)
    NA_CK(cudaMemsetAsync(s.hacc, 0, (size_t)n * kLanes * 2 * sizeof(u64), st));
    NA_CK(cudaMemsetAsync(s.hcarry, 0, (size_t)n * sizeof(u64), st));
    for (int64_t b0 = 0; b0 < k; b0 += kLanes) {
        const int nsrc = (int)((k - b0) < kLanes ? (k - b0) : kLanes);
        const int32_t* bsrc = sources + b0;
        // clear what a batch needs at zero (the array keeps the last contents)
        NA_CK(cudaMemsetAsync(s.vis, 0, (size_t)n * sizeof(u64), st));
        NA_CK(cudaMemsetAsync(s.nx, 0, (size_t)n * sizeof(u64), st));
        NA_CK(cudaMemsetAsync(s.ovf, 0, (size_t)n * sizeof(u64), st));
        NA_CK(cudaMemsetAsync(s.F, 0xff, 2 * (size_t)n * sizeof(MaskTag), st));
        NA_CK(cudaMemcpyAsync(s.d_src, bsrc, nsrc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        long long nq0 = 0;
        for (int j = 0; j < nsrc; ++j) {
            bool first = true;
            for (int i = 0; i < j; ++i)
                if (bsrc[i] == bsrc[j]) { first = false; break; }
            nq0 += first;
        }
        Counters hc;
        std::memset(&hc, 0, sizeof(hc));
        hc.qtail = (unsigned long long)nq0;
        NA_CK(cudaMemcpyAsync(s.ctr, &hc, sizeof(Counters), cudaMemcpyHostToDevice, st));
        NA_CK(cudaStreamSynchronize(st));  // hc is on the stack
        launch_seed(s, nsrc, st);
        NA_CK(cudaGetLastError());
        off[0] = 0;
        off[1] = nq0;
        int level = 0;
        for (;;) {
            const long long q_lo = off[level], q_hi = off[level + 1];
            NA_CK(cudaMemsetAsync((char*)s.ctr + disc_off, 0, disc_bytes, st));
            launch_push(c, s, q_lo, q_hi, level, heavy_deg, nsm, st);
            NA_CK(cudaGetLastError());
            NA_CK(cudaMemcpyAsync(&hc, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            NA_CK(cudaStreamSynchronize(st));
            if (hc.err) return GBBC_ERR_CAPACITY;
            const long long new_hi = (long long)hc.qtail;
            if (new_hi == q_hi) break;
            if (level + 2 > kNoallocMaxVertices + 1) return GBBC_ERR_CAPACITY;
            off[level + 2] = new_hi;
            NA_CK(cudaMemsetAsync((char*)s.ctr + gath_off, 0, gath_bytes, st));
            launch_fwd_gather(c, s, q_hi, level, heavy_deg, nsm, st, false);
            NA_CK(cudaGetLastError());
            ++level;
        }
        const int nlev = level + 1;
        NA_CK(cudaMemcpyAsync(&hc, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (hc.err || hc.carry) return GBBC_ERR_CAPACITY;
        for (int l = nlev - 1; l >= 1; --l) {
            NA_CK(cudaMemsetAsync(&s.ctr->heavy, 0, 2 * sizeof(unsigned long long), st));  // heavy, tasks
            launch_bwd(c, s, bc_fixed, off[l], off[l + 1], l, heavy_deg, nsm, st, false);
        }
        NA_CK(cudaGetLastError());
    }
    launch_bc_to_double(bc_fixed, bc_out, n, true, st);
    NA_CK(cudaGetLastError());
    NA_CK(cudaStreamSynchronize(st));
    return GBBC_OK;
}
