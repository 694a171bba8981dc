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

}  // namespace gbbc
