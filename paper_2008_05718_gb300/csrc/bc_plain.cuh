// The plain path with one source per thread block (batch width 1 on the
// block schedule): per-block state and launch.
#pragma once
#include "bc_internal.cuh"

namespace gbbc {

// Rows of n per block (dist -1 and sigma 0 between sources) and the block's
// level boundaries in its queue.
constexpr int kPlainBlock = 512;
struct PlainBlocks {
    int32_t n = 0;
    int count = 0;             // thread blocks (sources in flight)
    int32_t* dist = nullptr;   // [count][n]
    u64* sigma = nullptr;      // [count][n]
    u64* psi = nullptr;        // [count][n]
    int32_t* queue = nullptr;  // [count][n]
    int32_t* lev = nullptr;    // [count][n + 2]
    Counters* ctr = nullptr;   // [count]
};

int plain_blocks_per_sm();
// Every source of src[k] on the blocks of B (stats[0] += sources, stats[1] +=
// forward levels, low word of stats[2] |= 1 when a count reached 2^64).
cudaError_t launch_plain_blocks(const Csr& g, const PlainBlocks& B, const int32_t* src, long long k,
                                unsigned long long* next, u64* bc, unsigned long long* stats, cudaStream_t st);

}  // namespace gbbc
