// Direction decisions in the level loop and the MLP that can make them.
//
// k_decide runs once per forward level (one warp) between the gather of the
// level's vertices and the host's read-back: it computes the policy
// features from the device counters and the direction of the next step,
// either by the threshold rule of Beamer, Asanovic and Patterson (SC'12) or
// by the learned network (FP16 weights, FP32 sums).  The rule and the
// network only steer the schedule: both directions compute the same level.
//
// Training (bc_mlp_*): full-batch gradient descent with Adam on traces of
// per-level features and measured push/pull times.  All kernels are FP32;
// every reduction over samples runs in sample order inside one thread, so
// gradients and losses are deterministic.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "bc_internal.cuh"
#include "bc_policy.cuh"

namespace gbbc {

// ---------------------------------------------------------------------------
// Decision for the step at `level` (see decide_step in bc_policy.cuh).
__global__ void k_decide(Slot s, long long q_lo, int level, int policy, const __half* w, float n_range,
                         float nnz_range, float max_deg) {
    decide_step(s.ctr, q_lo, level, policy, w, n_range, nnz_range, max_deg);
}

void launch_decide(const Slot& s, long long q_lo, int level, int policy, const void* weights_fp16, long long n_range,
                   long long nnz_range, long long max_deg, cudaStream_t st) {
    k_decide<<<1, 32, 0, st>>>(s, q_lo, level, policy, (const __half*)weights_fp16, (float)n_range,
                               (float)nnz_range, (float)max_deg);
}

// ---------------------------------------------------------------------------
// Training kernels (FP32).
__global__ void k_mlp_fwd(const float* p, int k, const float* x, long long n, float* h1, float* h2, float* out) {
    for (long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; sidx < n;
         sidx += (long long)gridDim.x * blockDim.x) {
        const float* xs = x + sidx * kMlpIn;
        float a1[kMlpHidden];
        for (int j = 0; j < kMlpHidden; ++j) {
            float v = p[kB1 + j];
            for (int i = 0; i < kMlpIn; ++i) v += p[kW1 + j * kMlpIn + i] * xs[i];
            a1[j] = fmaxf(v, 0.f);
            h1[sidx * kMlpHidden + j] = a1[j];
        }
        float a2[kMlpHidden];
        for (int j = 0; j < kMlpHidden; ++j) {
            float v = p[kB2 + j];
            for (int i = 0; i < kMlpHidden; ++i) v += p[kW2 + j * kMlpHidden + i] * a1[i];
            a2[j] = fmaxf(v, 0.f);
            h2[sidx * kMlpHidden + j] = a2[j];
        }
        for (int o = 0; o < k; ++o) {
            float v = p[mlp_b3(k) + o];
            for (int j = 0; j < kMlpHidden; ++j) v += p[kW3 + o * kMlpHidden + j] * a2[j];
            out[sidx * k + o] = v;
        }
    }
}

// loss kinds: 0 = weighted softmax cross-entropy over k classes (target is
// the class index), 1 = weighted squared error (k = 1).  Weights are
// normalised by their sum.
__global__ void k_mlp_bwd(const float* p, int k, const float* target, const float* wgt, long long n,
                          const float* wsum, int loss, const float* h1, const float* h2, const float* out,
                          float* dout, float* dh2, float* dh1, float* sloss) {
    const float W = *wsum > 0.f ? *wsum : 1.f;
    for (long long sidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; sidx < n;
         sidx += (long long)gridDim.x * blockDim.x) {
        float ws = (wgt ? wgt[sidx] : 1.f) / W;
        float d[kMlpMaxOut];
        const float* o = out + sidx * k;
        if (loss == 0) {
            float mx = o[0];
            for (int c = 1; c < k; ++c) mx = fmaxf(mx, o[c]);
            float z = 0.f;
            for (int c = 0; c < k; ++c) z += expf(o[c] - mx);
            int tc = (int)target[sidx];
            float lse = mx + logf(z);
            sloss[sidx] = ws * (lse - o[tc]);
            for (int c = 0; c < k; ++c) d[c] = ws * (expf(o[c] - lse) - (c == tc ? 1.f : 0.f));
        } else {
            float r = o[0] - target[sidx];
            sloss[sidx] = ws * r * r;
            d[0] = 2.f * ws * r;
        }
        for (int c = 0; c < k; ++c) dout[sidx * k + c] = d[c];
        float g2[kMlpHidden];
        for (int j = 0; j < kMlpHidden; ++j) {
            float v = 0.f;
            for (int c = 0; c < k; ++c) v += p[kW3 + c * kMlpHidden + j] * d[c];
            g2[j] = h2[sidx * kMlpHidden + j] > 0.f ? v : 0.f;
            dh2[sidx * kMlpHidden + j] = g2[j];
        }
        for (int i = 0; i < kMlpHidden; ++i) {
            float v = 0.f;
            for (int j = 0; j < kMlpHidden; ++j) v += p[kW2 + j * kMlpHidden + i] * g2[j];
            dh1[sidx * kMlpHidden + i] = h1[sidx * kMlpHidden + i] > 0.f ? v : 0.f;
        }
    }
}

// One thread per parameter; sums over samples in index order.
__global__ void k_mlp_grad(int k, const float* x, long long n, const float* h1, const float* h2, const float* dout,
                           const float* dh2, const float* dh1, float* grad) {
    const int np = mlp_params(k);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
        float acc = 0.f;
        if (q < kB1) {
            int j = (q - kW1) / kMlpIn, i = (q - kW1) % kMlpIn;
            for (long long s = 0; s < n; ++s) acc += dh1[s * kMlpHidden + j] * x[s * kMlpIn + i];
        } else if (q < kW2) {
            int j = q - kB1;
            for (long long s = 0; s < n; ++s) acc += dh1[s * kMlpHidden + j];
        } else if (q < kB2) {
            int j = (q - kW2) / kMlpHidden, i = (q - kW2) % kMlpHidden;
            for (long long s = 0; s < n; ++s) acc += dh2[s * kMlpHidden + j] * h1[s * kMlpHidden + i];
        } else if (q < kW3) {
            int j = q - kB2;
            for (long long s = 0; s < n; ++s) acc += dh2[s * kMlpHidden + j];
        } else if (q < mlp_b3(k)) {
            int o = (q - kW3) / kMlpHidden, j = (q - kW3) % kMlpHidden;
            for (long long s = 0; s < n; ++s) acc += dout[s * k + o] * h2[s * kMlpHidden + j];
        } else {
            int o = q - mlp_b3(k);
            for (long long s = 0; s < n; ++s) acc += dout[s * k + o];
        }
        grad[q] = acc;
    }
}

// Sum of v[0..n) by one block (fixed tree order).
__global__ void k_sum(const float* v, long long n, float* out) {
    __shared__ float part[256];
    float a = 0.f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) a += v ? v[i] : 1.f;
    part[threadIdx.x] = a;
    __syncthreads();
    for (int h = blockDim.x / 2; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long count, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float mi = b1 * m[i] + (1.f - b1) * g[i];
        float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_to_half(const float* p, __half* h, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        h[i] = __float2half_rn(p[i]);
}

// Inference path of the level loop on a batch of feature vectors (a warp each).
__global__ void k_policy_eval(const __half* w, const float* x, long long n, float* logits, int32_t* choice) {
    const int lane = threadIdx.x & 31;
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long sidx = wid; sidx < n; sidx += nw) {
        float xv[kMlpIn];
        for (int i = 0; i < kMlpIn; ++i) xv[i] = x[sidx * kMlpIn + i];
        float out[2];
        mlp_warp_eval(w, 2, xv, out);
        if (lane == 0) {
            if (logits) {
                logits[2 * sidx] = out[0];
                logits[2 * sidx + 1] = out[1];
            }
            if (choice) choice[sidx] = out[1] > out[0] ? 1 : 0;
        }
    }
}

}  // namespace gbbc

using namespace gbbc;

namespace {

struct MlpScratch {
    float *h1 = nullptr, *h2 = nullptr, *out = nullptr, *dout = nullptr, *dh2 = nullptr, *dh1 = nullptr,
          *sloss = nullptr, *wsum = nullptr;
    bool ok = false;
    cudaError_t alloc(long long n, int k) {
        cudaError_t e;
        size_t hn = (size_t)n * kMlpHidden * sizeof(float), on = (size_t)n * k * sizeof(float);
        if ((e = cudaMalloc(&h1, hn)) || (e = cudaMalloc(&h2, hn)) || (e = cudaMalloc(&dh1, hn)) ||
            (e = cudaMalloc(&dh2, hn)) || (e = cudaMalloc(&out, on)) || (e = cudaMalloc(&dout, on)) ||
            (e = cudaMalloc(&sloss, (size_t)n * sizeof(float))) || (e = cudaMalloc(&wsum, sizeof(float))))
            return e;
        ok = true;
        return cudaSuccess;
    }
    ~MlpScratch() {
        for (float* p : {h1, h2, out, dout, dh2, dh1, sloss, wsum})
            if (p) cudaFree(p);
    }
};

bool valid_k(int k) { return k >= 1 && k <= kMlpMaxOut; }

gbbc_status mlp_loss_grad(const float* params, int k, const float* x, const float* target, const float* weight,
                          long long n, int loss, float* grad, float* loss_out, cudaStream_t st, MlpScratch& sc) {
    int blocks = (int)((n + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    k_mlp_fwd<<<blocks, 256, 0, st>>>(params, k, x, n, sc.h1, sc.h2, sc.out);
    k_sum<<<1, 256, 0, st>>>(weight, n, sc.wsum);
    k_mlp_bwd<<<blocks, 256, 0, st>>>(params, k, target, weight, n, sc.wsum, loss, sc.h1, sc.h2, sc.out, sc.dout,
                                      sc.dh2, sc.dh1, sc.sloss);
    k_mlp_grad<<<(mlp_params(k) + 127) / 128, 128, 0, st>>>(k, x, n, sc.h1, sc.h2, sc.dout, sc.dh2, sc.dh1, grad);
    if (loss_out) k_sum<<<1, 256, 0, st>>>(sc.sloss, n, loss_out);
    return cudaGetLastError() == cudaSuccess ? GBBC_OK : GBBC_ERR_CUDA;
}

}  // namespace

extern "C" {

int64_t bc_mlp_param_count(int32_t k_out) { return valid_k(k_out) ? mlp_params(k_out) : -1; }

gbbc_status bc_mlp_forward(const float* params, int32_t k_out, const float* x, int64_t n, float* out, void* stream) {
    if (!valid_k(k_out) || n < 0 || !params || !x || !out) return GBBC_ERR_INVALID;
    if (n == 0) return GBBC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    float *h1 = nullptr, *h2 = nullptr;
    if (cudaMalloc(&h1, (size_t)n * kMlpHidden * sizeof(float)) != cudaSuccess) return GBBC_ERR_OOM;
    if (cudaMalloc(&h2, (size_t)n * kMlpHidden * sizeof(float)) != cudaSuccess) {
        cudaFree(h1);
        return GBBC_ERR_OOM;
    }
    int blocks = (int)((n + 255) / 256);
    k_mlp_fwd<<<blocks > 1024 ? 1024 : blocks, 256, 0, st>>>(params, k_out, x, n, h1, h2, out);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(h1);
    cudaFree(h2);
    return e == cudaSuccess ? GBBC_OK : GBBC_ERR_CUDA;
}

gbbc_status bc_mlp_loss_grad(const float* params, int32_t k_out, const float* x, const float* target,
                             const float* weight, int64_t n, int32_t loss, float* grad, float* loss_out,
                             void* stream) {
    if (!valid_k(k_out) || n <= 0 || !params || !x || !target || !grad || (loss != 0 && loss != 1) ||
        (loss == 1 && k_out != 1))
        return GBBC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    MlpScratch sc;
    if (sc.alloc(n, k_out) != cudaSuccess) return GBBC_ERR_OOM;
    gbbc_status r = mlp_loss_grad(params, k_out, x, target, weight, n, loss, grad, loss_out, st, sc);
    if (cudaStreamSynchronize(st) != cudaSuccess) return GBBC_ERR_CUDA;
    return r;
}

gbbc_status bc_mlp_adam_step(float* params, const float* grad, float* m, float* v, int64_t count, float lr,
                             float beta1, float beta2, float eps, int32_t t, void* stream) {
    if (!params || !grad || !m || !v || count <= 0 || t < 1) return GBBC_ERR_INVALID;
    float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<(int)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, beta1, beta2,
                                                                        eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? GBBC_OK : GBBC_ERR_CUDA;
}

gbbc_status bc_mlp_train(float* params, int32_t k_out, const float* x, const float* target, const float* weight,
                         int64_t n, int32_t loss, int32_t epochs, float lr, float* loss_hist, void* stream) {
    if (!valid_k(k_out) || n <= 0 || epochs < 0 || !params || !x || !target) return GBBC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    MlpScratch sc;
    if (sc.alloc(n, k_out) != cudaSuccess) return GBBC_ERR_OOM;
    const int np = mlp_params(k_out);
    float *g = nullptr, *m = nullptr, *v = nullptr;
    if (cudaMalloc(&g, np * sizeof(float)) || cudaMalloc(&m, np * sizeof(float)) ||
        cudaMalloc(&v, np * sizeof(float))) {
        cudaFree(g);
        cudaFree(m);
        cudaFree(v);
        return GBBC_ERR_OOM;
    }
    cudaMemsetAsync(m, 0, np * sizeof(float), st);
    cudaMemsetAsync(v, 0, np * sizeof(float), st);
    gbbc_status r = GBBC_OK;
    for (int ep = 0; ep < epochs && r == GBBC_OK; ++ep) {
        r = mlp_loss_grad(params, k_out, x, target, weight, n, loss, g, loss_hist ? loss_hist + ep : nullptr, st, sc);
        if (r == GBBC_OK) r = bc_mlp_adam_step(params, g, m, v, np, lr, 0.9f, 0.999f, 1e-8f, ep + 1, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) r = GBBC_ERR_CUDA;
    cudaFree(g);
    cudaFree(m);
    cudaFree(v);
    return r;
}

gbbc_status bc_policy_eval(const float* params, const float* x, int64_t n, float* logits, int32_t* choice,
                           void* stream) {
    if (!params || !x || n < 0) return GBBC_ERR_INVALID;
    if (n == 0) return GBBC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    __half* w = nullptr;
    const int np = mlp_params(2);
    if (cudaMalloc(&w, np * sizeof(__half)) != cudaSuccess) return GBBC_ERR_OOM;
    k_to_half<<<(np + 255) / 256, 256, 0, st>>>(params, w, np);
    long long blocks = (n * 32 + 255) / 256;
    k_policy_eval<<<(int)(blocks > 4096 ? 4096 : blocks), 256, 0, st>>>(w, x, n, logits, choice);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(w);
    return e == cudaSuccess ? GBBC_OK : GBBC_ERR_CUDA;
}

}  // extern "C"

namespace gbbc {

// ---------------------------------------------------------------------------
// Source-grouping features (a warp per source): log-scaled degree of s, sum
// and maximum of its neighbours' degrees, and the size, mean degree and
// maximum degree of s's graph.
__global__ void k_source_features(Csr g, const int32_t* src, const int32_t* gid, long long k, const long long* goff,
                                  const long long* gmaxdeg, float* x) {
    const int lane = threadIdx.x & 31;
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wid; i < k; i += nw) {
        int32_t s = src[i];
        int gi = gid[i];
        int32_t beg = g.row_ptr[s], end = g.row_ptr[s + 1];
        unsigned long long sum = 0;
        int mx = 0;
        for (int32_t p = beg + lane; p < end; p += 32) {
            int32_t u = g.col[p];
            int d = g.row_ptr[u + 1] - g.row_ptr[u];
            sum += (unsigned long long)d;
            mx = d > mx ? d : mx;
        }
        for (int o = 16; o >= 1; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            int om = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = om > mx ? om : mx;
        }
        if (lane == 0) {
            float n = (float)(goff[gi + 1] - goff[gi]);
            float nnz = (float)(g.row_ptr[goff[gi + 1]] - g.row_ptr[goff[gi]]);
            float* xi = x + i * kMlpIn;
            xi[0] = log2p1((float)(end - beg)) / 24.f;
            xi[1] = log2p1((float)sum) / 32.f;
            xi[2] = log2p1((float)mx) / 24.f;
            xi[3] = log2p1(n) / 32.f;
            xi[4] = log2p1(nnz / (n > 0.f ? n : 1.f)) / 16.f;
            xi[5] = log2p1((float)gmaxdeg[gi]) / 24.f;
        }
    }
}

// Grouping score (the network's single output) of each feature vector.
__global__ void k_group_score(const __half* w, const float* x, long long k, float* score) {
    const int lane = threadIdx.x & 31;
    long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = wid; i < k; i += nw) {
        float xv[kMlpIn];
        for (int j = 0; j < kMlpIn; ++j) xv[j] = x[i * kMlpIn + j];
        float out[1];
        mlp_warp_eval(w, 1, xv, out);
        if (lane == 0) score[i] = out[0];
    }
}

cudaError_t launch_source_features(const Csr& g, const int32_t* src, const int32_t* gid, long long k,
                                   const long long* goff, const long long* gmaxdeg, float* x, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    long long blocks = (k * 32 + 255) / 256;
    k_source_features<<<(int)(blocks > 4096 ? 4096 : blocks), 256, 0, st>>>(g, src, gid, k, goff, gmaxdeg, x);
    return cudaGetLastError();
}

cudaError_t launch_group_score(const void* w_half, const float* x, long long k, float* score, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    long long blocks = (k * 32 + 255) / 256;
    k_group_score<<<(int)(blocks > 4096 ? 4096 : blocks), 256, 0, st>>>((const __half*)w_half, x, k, score);
    return cudaGetLastError();
}

cudaError_t mlp_to_half(const float* params_dev, void* half_dev, int count, cudaStream_t st) {
    k_to_half<<<(count + 255) / 256, 256, 0, st>>>(params_dev, (__half*)half_dev, count);
    return cudaGetLastError();
}

// FP16 copy of a direction network for a handle (bc_policy_load).
cudaError_t policy_to_half(const float* params_dev, void* half_dev, cudaStream_t st) {
    k_to_half<<<(mlp_params(2) + 255) / 256, 256, 0, st>>>(params_dev, (__half*)half_dev, mlp_params(2));
    return cudaGetLastError();
}
}  // namespace gbbc
