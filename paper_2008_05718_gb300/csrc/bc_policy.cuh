// Direction policy of the forward phase and the small MLP behind it.
//
// Features of a forward step at level l (all from device counters):
//   x0 frontier popcount    log2(1 + (vertex, lane) pairs at level l) / log2(1 + 64 n)
//   x1 frontier edge sum    log2(1 + sum of degrees of level-l vertices) / log2(1 + nnz)
//   x2 unvisited count      log2(1 + unvisited (vertex, active lane) pairs) / log2(1 + 64 n)
//   x3 level index          log2(1 + l) / 8
//   x4 degree mean          log2(1 + nnz / n) / 16
//   x5 degree max           log2(1 + max degree) / 24
// Network: 6 -> 32 (ReLU) -> 32 (ReLU) -> K outputs; K = 2 logits (push,
// pull) for the direction head.  Inference keeps the weights in FP16 and
// accumulates in FP32.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "bc_internal.cuh"

namespace gbbc {

constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 32;
constexpr int kMlpMaxOut = 2;

// Parameter offsets (FP32 master copy and FP16 inference copy share them).
constexpr int kW1 = 0;                                  // [32][6]
constexpr int kB1 = kW1 + kMlpHidden * kMlpIn;          // [32]
constexpr int kW2 = kB1 + kMlpHidden;                   // [32][32]
constexpr int kB2 = kW2 + kMlpHidden * kMlpHidden;      // [32]
constexpr int kW3 = kB2 + kMlpHidden;                   // [K][32]
__host__ __device__ constexpr int mlp_b3(int k_out) { return kW3 + k_out * kMlpHidden; }
__host__ __device__ constexpr int mlp_params(int k_out) { return mlp_b3(k_out) + k_out; }

// One warp evaluates the network for one feature vector: thread t owns
// hidden unit t of both layers.  Weights in FP16, sums in FP32; the summation
// order is fixed, so the result is deterministic.  Returns output o on every
// thread.
__device__ __forceinline__ void mlp_warp_eval(const __half* w, int k_out, const float* x, float* out) {
    const int t = threadIdx.x & 31;
    float h1 = __half2float(w[kB1 + t]);
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) h1 += __half2float(w[kW1 + t * kMlpIn + i]) * x[i];
    h1 = fmaxf(h1, 0.f);
    float h2 = __half2float(w[kB2 + t]);
#pragma unroll
    for (int k = 0; k < kMlpHidden; ++k) h2 += __half2float(w[kW2 + t * kMlpHidden + k]) * __shfl_sync(0xffffffffu, h1, k);
    h2 = fmaxf(h2, 0.f);
    for (int o = 0; o < k_out; ++o) {
        float v = __half2float(w[kW3 + o * kMlpHidden + t]) * h2;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        out[o] = v + __half2float(w[mlp_b3(k_out) + o]);
    }
}

__device__ __forceinline__ float log2p1(float x) { return log2f(1.f + (x > 0.f ? x : 0.f)); }

__device__ __forceinline__ void policy_features(float pairs, float edges, float unvisited, int level, float n,
                                                float nnz, float max_deg, float* x) {
    x[0] = log2p1(pairs) / fmaxf(log2p1(64.f * n), 1.f);
    x[1] = log2p1(edges) / fmaxf(log2p1(nnz), 1.f);
    x[2] = log2p1(unvisited) / fmaxf(log2p1(64.f * n), 1.f);
    x[3] = log2p1((float)level) / 8.f;
    x[4] = log2p1(nnz / (n > 0.f ? n : 1.f)) / 16.f;
    x[5] = log2p1(max_deg) / 24.f;
}

// Decision for the step at `level`, by one warp (all 32 threads call it):
// entries [q_lo, c->qtail), degree sum c->edge_sum, (vertex, lane) pairs
// c->lane_sum, active lanes c->lanes.  Writes c->dir, the features and the
// running state (visited pairs, explored edges, threshold hysteresis).
__device__ __forceinline__ void decide_step(Counters* c, long long q_lo, int level, int policy, const __half* w,
                                            float n_range, float nnz_range, float max_deg) {
    const int t = threadIdx.x & 31;
    unsigned long long nv = c->qtail - (unsigned long long)q_lo;
    unsigned long long ne = c->edge_sum;
    unsigned long long pairs = c->lane_sum;
    unsigned long long visited = c->visited + pairs;
    float active = (float)__popcll(c->lanes);
    float x[kMlpIn];
    policy_features((float)pairs, (float)ne, active * n_range - (float)visited, level, n_range, nnz_range, max_deg,
                    x);
    int dir = 0;
    float out[2] = {0.f, 0.f};
    if (policy == GBBC_POLICY_LEARNED && w) {
        mlp_warp_eval(w, 2, x, out);
        dir = out[1] > out[0] ? 1 : 0;
    } else if (policy == GBBC_POLICY_PUSH) {
        dir = 0;
    } else if (policy == GBBC_POLICY_PULL) {
        dir = level >= 1 ? 1 : 0;
    } else {
        // threshold rule (Beamer, Asanovic, Patterson, SC'12): go bottom-up
        // once the frontier's edges exceed the unexplored edges / alpha; come
        // back once the frontier holds fewer than n / beta vertices
        const float alpha = 14.f, beta = 24.f;
        float m_u = fmaxf(nnz_range - (float)c->explored, 1.f);
        int st = c->pull_state;
        if (!st) {
            if ((float)ne > m_u / alpha) st = 1;
        } else if ((float)nv < n_range / beta) {
            st = 0;
        }
        dir = st;
    }
    __syncwarp();
    if (t == 0) {
        if (!(policy == GBBC_POLICY_LEARNED && w) && policy != GBBC_POLICY_PUSH && policy != GBBC_POLICY_PULL)
            c->pull_state = dir;
        c->dir = dir;
        c->visited = visited;
        c->explored += ne;
        for (int i = 0; i < kMlpIn; ++i) c->feat[i] = x[i];
        c->logit[0] = out[0];
        c->logit[1] = out[1];
    }
    __syncwarp();
}

}  // namespace gbbc
