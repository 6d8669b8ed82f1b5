// rtlfs_sched.cu -- the learned and heuristic schedulers: per-fault features, the load
// predictor (a 5-64-64-1 MLP with BF16 weights and FP32 accumulation on the CUDA cores),
// its training kernels, and the device-side ordering of the work queue.
//
// The paper balances load with a runtime monitor: a node whose share of the run time
// exceeds a threshold is split over the fault dimension (Sec. IV-C-2). Here the same
// decision -- which work is heavy and what runs first -- is taken before the faulty
// kernels start, from a prediction of each fault's propagation load (node evaluations
// summed over cycles, which the simulator records). The prediction only orders and
// assigns work; results never depend on it.
#include "rtlfs_internal.h"
#include "rtlfs_sched.h"

#include <cuda_bf16.h>

namespace rtlfs {

// ---- features ------------------------------------------------------------------------
// One warp per fault: static features come from per-net tables built at load time, the
// toggle rate of the site bit from the good trace (lanes read 32 consecutive cycles).
__global__ void features_kernel(const DevDesign *__restrict__ designs, DevFaults f,
                                const float *__restrict__ const *net_static, float *X,
                                float *heur, uint32_t t_limit) {
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (warp >= f.F) return;
    const uint32_t fid = warp;
    const uint32_t di = f.design[fid];
    const DevDesign &D = designs[di];
    const uint32_t site = f.site[fid], bit = f.bit[fid];
    const uint64_t *col = D.gcol + (size_t)site * D.T;
    const uint32_t T = min(D.T, t_limit);   // cycles the toggle rate is measured over
    uint32_t toggles = 0;
    uint32_t prev_last = 0;   // bit at the last cycle of the previous 32-cycle block
    for (uint32_t t0 = 0; t0 < T; t0 += 32) {
        const uint32_t t = t0 + lane;
        const uint32_t b = t < T ? (uint32_t)((__ldg(col + t) >> bit) & 1ull) : 0u;
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, b);
        const uint32_t valid = (T - t0) >= 32 ? 0xFFFFFFFFu : ((1u << (T - t0)) - 1u);
        // toggles inside the block, plus across the block boundary
        const uint32_t shifted = (bits << 1) | (t0 ? prev_last : (bits & 1u));
        toggles += __popc((bits ^ shifted) & valid);
        const uint32_t last = 31 - __clz(valid);
        prev_last = (bits >> last) & 1u;
    }
    if (lane == 0) {
        const float *ns = net_static[di];   // [n_net][4]: cone, level, regdepth, width
        const float cone = ns[4 * (size_t)site + 0];
        const float tog = T > 1 ? (float)toggles / (float)(T - 1) : 0.f;
        float *x = X + (size_t)fid * MLP_IN;
        x[0] = cone;
        x[1] = ns[4 * (size_t)site + 1];
        x[2] = ns[4 * (size_t)site + 2];
        x[3] = ns[4 * (size_t)site + 3];
        x[4] = tog;
        // heuristic score: static cone size x toggle rate (both as fractions of their range)
        heur[fid] = cone * tog;
    }
}

// ---- MLP -------------------------------------------------------------------------------
// Parameter layout (MLP_PARAMS values): W1[5][64], b1[64], W2[64][64], b2[64], w3[64], b3.
// W1[i][j] connects input i to hidden unit j; W2[i][j] hidden-1 unit i to hidden-2 unit j.
__device__ __forceinline__ void load_params(const __nv_bfloat16 *__restrict__ wb, float *sw) {
    for (uint32_t i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) sw[i] = __bfloat162float(wb[i]);
}

// One thread per sample; weights (as FP32 copies of the BF16 values) in shared memory.
__global__ void mlp_forward_kernel(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ X,
                                   uint32_t n, float *y) {
    __shared__ float sw[MLP_PARAMS];
    load_params(wb, sw);
    __syncthreads();
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float *W1 = sw, *b1 = sw + MLP_OFF_B1, *W2 = sw + MLP_OFF_W2, *b2 = sw + MLP_OFF_B2;
    const float *w3 = sw + MLP_OFF_W3;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[(size_t)s * MLP_IN + i];
    float h1[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        float a = b1[j];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(x[i], W1[i * MLP_H + j], a);
        h1[j] = a > 0.f ? a : 0.f;
    }
    float out = sw[MLP_OFF_B3];
    for (int j = 0; j < MLP_H; ++j) {
        float a = b2[j];
#pragma unroll
        for (int i = 0; i < MLP_H; ++i) a = fmaf(h1[i], W2[i * MLP_H + j], a);
        a = a > 0.f ? a : 0.f;
        out = fmaf(a, w3[j], out);
    }
    y[s] = out;
}

// Forward + backward of the mean squared error over n samples for one tile of MLP_TILE
// samples per CTA; the tile's parameter gradients are added into grad (FP32 atomics) and
// its squared errors into loss_sum.
__global__ void __launch_bounds__(256)
mlp_grad_kernel(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ X,
                const float *__restrict__ tgt, uint32_t n, float *grad, float *loss_sum) {
    extern __shared__ float gsh[];
    float *sw = gsh;                                   // [MLP_PARAMS]
    float *h1 = sw + MLP_PARAMS;                       // [TILE][H]  post-activation
    float *h2 = h1 + MLP_TILE * MLP_H;                 // [TILE][H]  post-activation
    float *d2 = h2 + MLP_TILE * MLP_H;                 // [TILE][H]  dL/d(pre-activation 2)
    float *d1 = d2 + MLP_TILE * MLP_H;                 // [TILE][H]  dL/d(pre-activation 1)
    float *xs = d1 + MLP_TILE * MLP_H;                 // [TILE][IN]
    float *dy = xs + MLP_TILE * MLP_IN;                // [TILE]
    load_params(wb, sw);
    const float *W1 = sw, *b1 = sw + MLP_OFF_B1, *W2 = sw + MLP_OFF_W2, *b2 = sw + MLP_OFF_B2;
    const float *w3 = sw + MLP_OFF_W3;
    const uint32_t s0 = blockIdx.x * MLP_TILE, tid = threadIdx.x, B = blockDim.x;
    for (uint32_t k = tid; k < MLP_TILE * MLP_IN; k += B) {
        const uint32_t s = s0 + k / MLP_IN;
        xs[k] = s < n ? X[(size_t)s0 * MLP_IN + k] : 0.f;
    }
    __syncthreads();
    // layer 1
    for (uint32_t k = tid; k < MLP_TILE * MLP_H; k += B) {
        const uint32_t s = k / MLP_H, j = k % MLP_H;
        float a = b1[j];
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(xs[s * MLP_IN + i], W1[i * MLP_H + j], a);
        h1[k] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    // layer 2
    for (uint32_t k = tid; k < MLP_TILE * MLP_H; k += B) {
        const uint32_t s = k / MLP_H, j = k % MLP_H;
        float a = b2[j];
        for (int i = 0; i < MLP_H; ++i) a = fmaf(h1[s * MLP_H + i], W2[i * MLP_H + j], a);
        h2[k] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    // output, error and dL/dy = 2 (y - t) / n
    if (tid < MLP_TILE) {
        const uint32_t s = s0 + tid;
        float e = 0.f;
        if (s < n) {
            float out = sw[MLP_OFF_B3];
            for (int j = 0; j < MLP_H; ++j) out = fmaf(h2[tid * MLP_H + j], w3[j], out);
            e = out - tgt[s];
            atomicAdd(loss_sum, e * e);
        }
        dy[tid] = 2.f * e / (float)n;
    }
    __syncthreads();
    for (uint32_t k = tid; k < MLP_TILE * MLP_H; k += B) {
        const uint32_t s = k / MLP_H, j = k % MLP_H;
        d2[k] = h2[k] > 0.f ? w3[j] * dy[s] : 0.f;
    }
    __syncthreads();
    for (uint32_t k = tid; k < MLP_TILE * MLP_H; k += B) {
        const uint32_t s = k / MLP_H, i = k % MLP_H;
        float a = 0.f;
        for (int j = 0; j < MLP_H; ++j) a = fmaf(W2[i * MLP_H + j], d2[s * MLP_H + j], a);
        d1[k] = h1[k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients of this tile
    for (uint32_t k = tid; k < MLP_H * MLP_H; k += B) {          // W2
        const uint32_t i = k / MLP_H, j = k % MLP_H;
        float a = 0.f;
        for (uint32_t s = 0; s < MLP_TILE; ++s) a = fmaf(h1[s * MLP_H + i], d2[s * MLP_H + j], a);
        atomicAdd(grad + MLP_OFF_W2 + k, a);
    }
    for (uint32_t k = tid; k < MLP_IN * MLP_H; k += B) {         // W1
        const uint32_t i = k / MLP_H, j = k % MLP_H;
        float a = 0.f;
        for (uint32_t s = 0; s < MLP_TILE; ++s) a = fmaf(xs[s * MLP_IN + i], d1[s * MLP_H + j], a);
        atomicAdd(grad + k, a);
    }
    for (uint32_t j = tid; j < MLP_H; j += B) {                  // b1, b2, w3
        float g1 = 0.f, g2 = 0.f, g3 = 0.f;
        for (uint32_t s = 0; s < MLP_TILE; ++s) {
            g1 += d1[s * MLP_H + j];
            g2 += d2[s * MLP_H + j];
            g3 = fmaf(h2[s * MLP_H + j], dy[s], g3);
        }
        atomicAdd(grad + MLP_OFF_B1 + j, g1);
        atomicAdd(grad + MLP_OFF_B2 + j, g2);
        atomicAdd(grad + MLP_OFF_W3 + j, g3);
    }
    if (tid == 0) {
        float g = 0.f;
        for (uint32_t s = 0; s < MLP_TILE; ++s) g += dy[s];
        atomicAdd(grad + MLP_OFF_B3, g);
    }
}

// Adam step on the FP32 master parameters; the BF16 copy (round to nearest even) is what
// the forward pass uses. Clears the gradient for the next step.
__global__ void mlp_adam_kernel(float *master, __nv_bfloat16 *wb, float *grad, float *m, float *v,
                                float lr, float beta1, float beta2, float eps, float bc1, float bc2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_PARAMS) return;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    master[i] = p;
    wb[i] = __float2bfloat16_rn(p);
    grad[i] = 0.f;
}

// ---- queue order -----------------------------------------------------------------------
// Counting sort of the faults by score, descending, into SORT_BUCKETS buckets over [lo, hi].
// With k > 0 score classes (a power of two up to 64) the buckets are k classes of
// SORT_BUCKETS / k sub-buckets each: fault i of n goes to its class's sub-bucket
// i * (SORT_BUCKETS / k) / n, so inside a class the queue keeps the fault-list order (by
// site), at the granularity of a sub-bucket. Every bucket index is below SORT_BUCKETS.
__device__ __forceinline__ uint32_t bucket_of(float s, float lo, float hi, uint32_t i, uint32_t n,
                                              uint32_t k) {
    float u = hi > lo ? (s - lo) / (hi - lo) : 0.f;
    u = fminf(fmaxf(u, 0.f), 1.f);
    if (k == 0) {
        const uint32_t b = (uint32_t)(u * (float)(SORT_BUCKETS - 1) + 0.5f);
        return (SORT_BUCKETS - 1) - b;    // descending score = ascending bucket
    }
    const uint32_t per = SORT_BUCKETS / k;
    const uint32_t c = min((uint32_t)(u * (float)k), k - 1u);
    const uint32_t sb = min((uint32_t)(((uint64_t)i * per) / max(n, 1u)), per - 1u);
    return (k - 1u - c) * per + sb;
}

__device__ __forceinline__ int map_key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : (int)(0x80000000u - (uint32_t)i);
}

__global__ void minmax_init_kernel(float *mm) {
    reinterpret_cast<int *>(mm)[0] = map_key(3.0e38f);
    reinterpret_cast<int *>(mm)[1] = map_key(-3.0e38f);
}

__device__ __forceinline__ float unmap_key(int k) {
    return k >= 0 ? __int_as_float(k) : __int_as_float((int)(0x80000000u - (uint32_t)k));
}

__global__ void minmax_kernel(const float *score, uint32_t n, float *mm) {
    float lo = 3.0e38f, hi = -3.0e38f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        lo = fminf(lo, score[i]);
        hi = fmaxf(hi, score[i]);
    }
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if ((threadIdx.x & 31u) == 0) {
        // order-preserving float -> int mapping so that integer atomics compare floats
        atomicMin(reinterpret_cast<int *>(mm) + 0, map_key(lo));
        atomicMax(reinterpret_cast<int *>(mm) + 1, map_key(hi));
    }
}

__global__ void histogram_kernel(const float *score, uint32_t n, const float *mm, uint32_t *hist,
                                 uint32_t k) {
    __shared__ uint32_t h[SORT_BUCKETS];
    for (uint32_t b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const float lo = unmap_key(reinterpret_cast<const int *>(mm)[0]);
    const float hi = unmap_key(reinterpret_cast<const int *>(mm)[1]);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[bucket_of(score[i], lo, hi, i, n, k)], 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < SORT_BUCKETS; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Single CTA: exclusive scan of the histogram into bucket cursors.
__global__ void scan_kernel(uint32_t *hist) {
    __shared__ uint32_t part[1024];
    const uint32_t tid = threadIdx.x;
    constexpr uint32_t PER = SORT_BUCKETS / 1024;
    uint32_t loc[PER], sum = 0;
    for (uint32_t k = 0; k < PER; ++k) { loc[k] = hist[tid * PER + k]; sum += loc[k]; }
    part[tid] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
        const uint32_t v = tid >= off ? part[tid - off] : 0u;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint32_t run = part[tid] - sum;
    for (uint32_t k = 0; k < PER; ++k) { hist[tid * PER + k] = run; run += loc[k]; }
}

// Scatter fault ids into their buckets (order inside a bucket is unspecified), then the
// first n_heavy go to the heavy kernel's initial list and the rest form the light queue.
__global__ void scatter_kernel(const float *score, uint32_t n, const float *mm, uint32_t *cursor,
                               uint32_t *order, uint32_t k) {
    const float lo = unmap_key(reinterpret_cast<const int *>(mm)[0]);
    const float hi = unmap_key(reinterpret_cast<const int *>(mm)[1]);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t p = atomicAdd(&cursor[bucket_of(score[i], lo, hi, i, n, k)], 1u);
        order[p] = i;
    }
}

__global__ void heavy_items_kernel(const uint32_t *order, uint32_t n_heavy, HeavyItem *items) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_heavy) return;
    HeavyItem h{};
    h.fault = order[i];
    items[i] = h;
}

// ---- launchers ------------------------------------------------------------------------

cudaError_t launch_features(const DevDesign *d_designs, DevFaults f, const float *const *net_static,
                            float *X, float *heur, cudaStream_t s, uint32_t t_limit) {
    if (!f.F) return cudaSuccess;
    const uint32_t threads = 256, warps_per = threads / 32;
    features_kernel<<<(f.F + warps_per - 1) / warps_per, threads, 0, s>>>(d_designs, f, net_static, X, heur,
                                                                          t_limit);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void *wb, const float *X, uint32_t n, float *y, cudaStream_t s) {
    if (!n) return cudaSuccess;
    mlp_forward_kernel<<<(n + 127) / 128, 128, 0, s>>>((const __nv_bfloat16 *)wb, X, n, y);
    return cudaGetLastError();
}

size_t mlp_grad_smem() {
    return (MLP_PARAMS + 4 * MLP_TILE * MLP_H + MLP_TILE * MLP_IN + MLP_TILE) * sizeof(float);
}

cudaError_t launch_mlp_grad(const void *wb, const float *X, const float *t, uint32_t n, float *grad,
                            float *loss_sum, cudaStream_t s) {
    if (!n) return cudaSuccess;
    const size_t smem = mlp_grad_smem();
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp_grad_kernel<<<(n + MLP_TILE - 1) / MLP_TILE, 256, smem, s>>>((const __nv_bfloat16 *)wb, X, t, n,
                                                                     grad, loss_sum);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *master, void *wb, float *grad, float *m, float *v, float lr,
                            float beta1, float beta2, float eps, int step, cudaStream_t s) {
    const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
    mlp_adam_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, s>>>(master, (__nv_bfloat16 *)wb, grad, m, v, lr,
                                                            beta1, beta2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_order(const float *score, uint32_t n, float *mm, uint32_t *hist, uint32_t *order,
                         uint32_t n_heavy, HeavyItem *items, cudaStream_t s, uint32_t classes) {
    if (!n) return cudaSuccess;
    if (classes > 64 || (classes & (classes - 1))) return cudaErrorInvalidValue;
    minmax_init_kernel<<<1, 1, 0, s>>>(mm);
    cudaError_t e = cudaMemsetAsync(hist, 0, SORT_BUCKETS * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint32_t g = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    minmax_kernel<<<g, 256, 0, s>>>(score, n, mm);
    histogram_kernel<<<g, 256, 0, s>>>(score, n, mm, hist, classes);
    scan_kernel<<<1, 1024, 0, s>>>(hist);
    scatter_kernel<<<g, 256, 0, s>>>(score, n, mm, hist, order, classes);
    if (n_heavy) heavy_items_kernel<<<(n_heavy + 255) / 256, 256, 0, s>>>(order, n_heavy, items);
    return cudaGetLastError();
}

}  // namespace rtlfs
