// Learned slab sizing: a small MLP that predicts how many edges each vertex
// will gain, so that a rebuilt graph can give it enough buckets up front.
// The paper fixes bucket counts a priori from the load factor and the
// current degree (Sec. "Motivation"); this is a project addition on top of
// that rule, which stays its fallback and its yardstick.  It may change the
// memory layout (bucket counts) but never a result.
//
// Network: 8 inputs -> 64 ReLU -> 64 ReLU -> 1.  Master weights are fp32;
// every forward and backward pass uses them rounded to bf16 (round to
// nearest even) and accumulates in fp32.  Loss = mean squared error.
// Gradients are with respect to the bf16-rounded weights (the rounding is
// treated as the identity), and Adam updates the fp32 masters.
//
// Kernels: one block of 128 threads takes a tile of 128 samples at a time
// (grid-stride over tiles); weights and the tile's activations live in
// shared memory (activation rows padded to 65 floats so that a column walk
// is free of bank conflicts); each block accumulates its weight gradients in
// shared memory across its tiles and adds them to the global gradient with
// one atomicAdd per weight at the end.
#include "mk_host.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

using namespace mk;

namespace {

constexpr int kIn = 8, kHid = 64;
constexpr int kW1 = 0, kB1 = kW1 + kIn * kHid, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kHid, kNParams = kB3 + 1; // 4801
constexpr int kTile = 128, kPad = kHid + 1;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct Smem {
    float w1[kIn * kHid], b1[kHid], w2[kHid * kHid], b2[kHid], w3[kHid], b3;
    float x[kTile * kIn];
    float h1[kTile * kPad];
    float h2[kTile * kPad];
    float dy[kTile];
};

__device__ void load_weights(Smem &s, const float *P)
{
    for (int i = threadIdx.x; i < kIn * kHid; i += blockDim.x)
        s.w1[i] = bf16r(P[kW1 + i]);
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x)
        s.w2[i] = bf16r(P[kW2 + i]);
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        s.b1[i] = bf16r(P[kB1 + i]);
        s.b2[i] = bf16r(P[kB2 + i]);
        s.w3[i] = bf16r(P[kW3 + i]);
    }
    if (threadIdx.x == 0)
        s.b3 = bf16r(P[kB3]);
}

// Forward pass of sample t (row t of the tile); returns y.
__device__ float forward_row(Smem &s, int t)
{
    float *h1 = s.h1 + t * kPad, *h2 = s.h2 + t * kPad;
    const float *x = s.x + t * kIn;
    for (int j = 0; j < kHid; ++j) {
        float a = s.b1[j];
#pragma unroll
        for (int i = 0; i < kIn; ++i)
            a = fmaf(x[i], s.w1[i * kHid + j], a);
        h1[j] = fmaxf(a, 0.f);
    }
    float y = s.b3;
    for (int j = 0; j < kHid; ++j) {
        float a = s.b2[j];
        for (int k = 0; k < kHid; ++k)
            a = fmaf(h1[k], s.w2[k * kHid + j], a);
        a = fmaxf(a, 0.f);
        h2[j] = a;
        y = fmaf(a, s.w3[j], y);
    }
    return y;
}

__global__ void __launch_bounds__(kTile) k_mlp_forward(const float *P, const float *X, uint64_t n, float *Y)
{
    extern __shared__ float smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    load_weights(s, P);
    __syncthreads();
    for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < n; base += (uint64_t)gridDim.x * kTile) {
        const uint64_t i = base + threadIdx.x;
        for (int f = 0; f < kIn; ++f)
            s.x[threadIdx.x * kIn + f] = i < n ? X[i * kIn + f] : 0.f;
        if (i < n)
            Y[i] = forward_row(s, threadIdx.x);
    }
}

// Gradient of mean((y - T)^2) over n samples, accumulated into G (kNParams
// floats, zeroed by the caller); the sum of squared errors into *sse.
__global__ void __launch_bounds__(kTile) k_mlp_backward(const float *P, const float *X, const float *T, uint64_t n,
                                                        float inv_n, float *G, double *sse)
{
    extern __shared__ float smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ float g_w2[kHid * kHid];
    __shared__ float g_small[kIn * kHid + 3 * kHid + 1]; // w1, b1, b2, w3, b3
    float *gw1 = g_small, *gb1 = g_small + kIn * kHid, *gb2 = gb1 + kHid, *gw3 = gb2 + kHid, *gb3 = gw3 + kHid;
    load_weights(s, P);
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x)
        g_w2[i] = 0.f;
    for (int i = threadIdx.x; i < kIn * kHid + 3 * kHid + 1; i += blockDim.x)
        g_small[i] = 0.f;
    double my_sse = 0.0;
    __syncthreads();
    const int t = threadIdx.x;
    for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < n; base += (uint64_t)gridDim.x * kTile) {
        const uint64_t i = base + t;
        const bool valid = i < n;
        for (int f = 0; f < kIn; ++f)
            s.x[t * kIn + f] = valid ? X[i * kIn + f] : 0.f;
        const float y = forward_row(s, t);
        const float e = valid ? y - T[i] : 0.f;
        my_sse += (double)e * e;
        const float dy = 2.f * e * inv_n;
        s.dy[t] = dy;
        // dz2 (overwrites h2 after using its sign); w3 / b3 gradients need h2
        float *h2 = s.h2 + t * kPad;
        __syncthreads();
        // gw3[j] = sum_t h2[t][j] dy[t]; gb3 = sum dy  (thread j < 64 reduces column j)
        if (t < kHid) {
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a = fmaf(s.h2[r * kPad + t], s.dy[r], a);
            gw3[t] += a;
        } else if (t == kHid) {
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a += s.dy[r];
            *gb3 += a;
        }
        __syncthreads();
        for (int j = 0; j < kHid; ++j)
            h2[j] = h2[j] > 0.f ? dy * s.w3[j] : 0.f;
        __syncthreads();
        // gw2[k][j] = sum_t h1[t][k] dz2[t][j]: thread t owns 32 of the 4096
        for (int o = t; o < kHid * kHid; o += kTile) {
            const int k = o / kHid, j = o % kHid;
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a = fmaf(s.h1[r * kPad + k], s.h2[r * kPad + j], a);
            g_w2[o] += a;
        }
        if (t < kHid) {
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a += s.h2[r * kPad + t];
            gb2[t] += a;
        }
        __syncthreads();
        // dz1[t][k] = (sum_j dz2[t][j] w2[k][j]) * (h1[t][k] > 0), over h1
        float *h1 = s.h1 + t * kPad;
        for (int k = 0; k < kHid; ++k) {
            float a = 0.f;
            for (int j = 0; j < kHid; ++j)
                a = fmaf(h2[j], s.w2[k * kHid + j], a);
            h1[k] = h1[k] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // gw1[i][k] = sum_t x[t][i] dz1[t][k]; gb1[k] = sum_t dz1[t][k]
        for (int o = t; o < kIn * kHid; o += kTile) {
            const int f = o / kHid, k = o % kHid;
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a = fmaf(s.x[r * kIn + f], s.h1[r * kPad + k], a);
            gw1[o] += a;
        }
        if (t < kHid) {
            float a = 0.f;
            for (int r = 0; r < kTile; ++r)
                a += s.h1[r * kPad + t];
            gb1[t] += a;
        }
        __syncthreads();
    }
    for (int o = threadIdx.x; o < kHid * kHid; o += blockDim.x)
        atomicAdd(&G[kW2 + o], g_w2[o]);
    for (int o = threadIdx.x; o < kIn * kHid; o += blockDim.x)
        atomicAdd(&G[kW1 + o], gw1[o]);
    for (int o = threadIdx.x; o < kHid; o += blockDim.x) {
        atomicAdd(&G[kB1 + o], gb1[o]);
        atomicAdd(&G[kB2 + o], gb2[o]);
        atomicAdd(&G[kW3 + o], gw3[o]);
    }
    if (threadIdx.x == 0)
        atomicAdd(&G[kB3], *gb3);
    // block sum of squared errors
    for (int o = 16; o; o >>= 1)
        my_sse += __shfl_xor_sync(kFull, my_sse, o);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(sse, my_sse);
}

// Adam (Kingma and Ba, ICLR 2015) on the fp32 master weights.
__global__ void k_adam(float *P, const float *G, float *M, float *Vv, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * Vv[i] + (1.f - b2) * g * g;
    M[i] = m;
    Vv[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// Degree trace: out/in degree += sign for every edge flagged 1.
__global__ void k_degree_update(const uint32_t *src, const uint32_t *dst, const uint8_t *flags, uint64_t n, int sign,
                                uint32_t V, uint32_t *out_deg, uint32_t *in_deg)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n || (flags && !flags[i]))
        return;
    const uint32_t s = src[i], d = dst[i];
    if (s >= V || d >= V)
        return;
    if (out_deg)
        atomicAdd(&out_deg[s], (uint32_t)sign);
    if (in_deg)
        atomicAdd(&in_deg[d], (uint32_t)sign);
}

__device__ __forceinline__ float lg1p(float x) { return log1pf(fmaxf(x, 0.f)); }

// Features of each vertex from its out-degree snapshots (hist[k * V + v] =
// out-degree k batches ago, k = 0..4), in-degree and bucket count.
__global__ void k_features(const uint32_t *hist, const uint32_t *in_deg, const uint32_t *buckets, uint32_t V, float *X)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const float d0 = (float)hist[v];
    float *x = X + (uint64_t)v * kIn;
    x[0] = lg1p(d0);
    for (int k = 1; k <= 4; ++k)
        x[k] = lg1p(d0 - (float)hist[(uint64_t)k * V + v]);
    const float din = (float)in_deg[v];
    x[5] = lg1p(din);
    x[6] = lg1p(din) - lg1p(d0);
    x[7] = d0 / (15.f * (float)(buckets[v] ? buckets[v] : 1));
}

// Bucket counts from the predicted growth: y = log1p(edges gained per
// batch); future degree = degree + horizon * expm1(y); buckets =
// max(1, ceil(future degree / (load_factor * 15))).
__global__ void k_learned_buckets(const float *Y, const uint32_t *deg, uint32_t V, float horizon, float lf,
                                  uint32_t max_buckets, uint32_t *buckets)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const float growth = fmaxf(expm1f(fmaxf(Y[v], 0.f)), 0.f);
    const double fut = (double)deg[v] + (double)horizon * growth;
    double b = ceil(fut / (double)(lf * 15.f));
    if (b < 1)
        b = 1;
    if (b > max_buckets)
        b = max_buckets;
    buckets[v] = (uint32_t)b;
}

// Training target of each vertex: log1p of the out-edges it gained per batch
// between two snapshots h batches apart.
__global__ void k_growth_targets(const uint32_t *deg_then, const uint32_t *deg_later, uint32_t V, float h, float *T)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const float gain = (float)deg_later[v] - (float)deg_then[v];
    T[v] = log1pf(fmaxf(gain, 0.f) / h);
}

size_t smem_bytes() { return sizeof(Smem); }

int mlp_grid(uint64_t n)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
        cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
    }
    const uint64_t tiles = (n + kTile - 1) / kTile;
    const uint64_t g = std::min<uint64_t>(tiles, (uint64_t)sms * 2);
    return (int)std::max<uint64_t>(g, 1);
}

// splitmix64, for the initial weights
uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

} // namespace

struct mk_mlp {
    float *P = nullptr, *G = nullptr, *M = nullptr, *Vv = nullptr;
    double *sse = nullptr;
    uint64_t steps = 0;
};

extern "C" {

mk_status mk_mlp_create(uint64_t seed, mk_mlp **out)
{
    if (!out)
        return MK_ERR_INVALID_ARG;
    mk_mlp *m = new mk_mlp;
    const size_t bytes = kNParams * sizeof(float);
    if (cudaMalloc(&m->P, bytes) != cudaSuccess || cudaMalloc(&m->G, bytes) != cudaSuccess ||
        cudaMalloc(&m->M, bytes) != cudaSuccess || cudaMalloc(&m->Vv, bytes) != cudaSuccess ||
        cudaMalloc(&m->sse, sizeof(double)) != cudaSuccess) {
        mk_mlp_destroy(m);
        return MK_ERR_NO_MEMORY;
    }
    // He-uniform initial weights, zero biases
    std::vector<float> h(kNParams, 0.f);
    auto uni = [&](uint64_t i) { return (double)(mix64(seed * 0x9E3779B97F4A7C15ULL + i + 1) >> 11) / 9007199254740992.0; };
    for (int i = 0; i < kIn * kHid; ++i)
        h[kW1 + i] = (float)((2 * uni(i) - 1) * std::sqrt(6.0 / kIn));
    for (int i = 0; i < kHid * kHid; ++i)
        h[kW2 + i] = (float)((2 * uni(10000 + i) - 1) * std::sqrt(6.0 / kHid));
    for (int i = 0; i < kHid; ++i)
        h[kW3 + i] = (float)((2 * uni(20000 + i) - 1) * std::sqrt(6.0 / kHid));
    if (cudaMemcpy(m->P, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->M, 0, bytes) != cudaSuccess || cudaMemset(m->Vv, 0, bytes) != cudaSuccess) {
        mk_mlp_destroy(m);
        return MK_ERR_CUDA;
    }
    *out = m;
    return MK_OK;
}

mk_status mk_mlp_destroy(mk_mlp *m)
{
    if (!m)
        return MK_ERR_INVALID_ARG;
    cudaFree(m->P);
    cudaFree(m->G);
    cudaFree(m->M);
    cudaFree(m->Vv);
    cudaFree(m->sse);
    delete m;
    return MK_OK;
}

int mk_mlp_num_params(void) { return kNParams; }

mk_status mk_mlp_get_params(mk_mlp *m, float *h_out)
{
    if (!m || !h_out)
        return MK_ERR_INVALID_ARG;
    MK_CUDA(cudaMemcpy(h_out, m->P, kNParams * sizeof(float), cudaMemcpyDeviceToHost));
    return MK_OK;
}

mk_status mk_mlp_set_params(mk_mlp *m, const float *h_in)
{
    if (!m || !h_in)
        return MK_ERR_INVALID_ARG;
    MK_CUDA(cudaMemcpy(m->P, h_in, kNParams * sizeof(float), cudaMemcpyHostToDevice));
    MK_CUDA(cudaMemset(m->M, 0, kNParams * sizeof(float)));
    MK_CUDA(cudaMemset(m->Vv, 0, kNParams * sizeof(float)));
    m->steps = 0;
    return MK_OK;
}

mk_status mk_mlp_forward(mk_mlp *m, const float *d_x, uint64_t n, float *d_y, void *stream)
{
    if (!m || (n && (!d_x || !d_y)))
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_forward<<<mlp_grid(n), kTile, smem_bytes(), s>>>(m->P, d_x, n, d_y);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_mlp_gradient(mk_mlp *m, const float *d_x, const float *d_t, uint64_t n, float *d_grad, double *d_sse,
                          void *stream)
{
    if (!m || !n || !d_x || !d_t || !d_grad)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MK_CUDA(cudaMemsetAsync(d_grad, 0, kNParams * sizeof(float), s));
    double *sse = d_sse ? d_sse : m->sse;
    MK_CUDA(cudaMemsetAsync(sse, 0, sizeof(double), s));
    k_mlp_backward<<<mlp_grid(n), kTile, smem_bytes(), s>>>(m->P, d_x, d_t, n, 1.f / (float)n, d_grad, sse);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_mlp_adam_step(mk_mlp *m, const float *d_x, const float *d_t, uint64_t n, float lr, double *d_sse,
                           void *stream)
{
    if (!m || !n || !d_x || !d_t || !(lr > 0.f))
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MK_TRY(mk_mlp_gradient(m, d_x, d_t, n, m->G, d_sse, stream));
    m->steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->steps), c2 = 1.f - std::pow(b2, (float)m->steps);
    k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(m->P, m->G, m->M, m->Vv, kNParams, lr, b1, b2, 1e-8f, c1, c2);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_degree_update(uint32_t V, const uint32_t *d_src, const uint32_t *d_dst, const uint8_t *d_flags,
                           uint64_t n, int sign, uint32_t *d_out_deg, uint32_t *d_in_deg, void *stream)
{
    if (!V || (n && (!d_src || !d_dst)) || (sign != 1 && sign != -1))
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    k_degree_update<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(d_src, d_dst, d_flags, n, sign, V, d_out_deg,
                                                                        d_in_deg);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_sizing_features(uint32_t V, const uint32_t *d_out_hist, const uint32_t *d_in_deg,
                             const uint32_t *d_buckets, float *d_x, void *stream)
{
    if (!V || !d_out_hist || !d_in_deg || !d_buckets || !d_x)
        return MK_ERR_INVALID_ARG;
    k_features<<<grid_for(V, 256), 256, 0, (cudaStream_t)stream>>>(d_out_hist, d_in_deg, d_buckets, V, d_x);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_sizing_targets(uint32_t V, const uint32_t *d_deg_then, const uint32_t *d_deg_later, float horizon,
                            float *d_t, void *stream)
{
    if (!V || !d_deg_then || !d_deg_later || !d_t || !(horizon > 0.f))
        return MK_ERR_INVALID_ARG;
    k_growth_targets<<<grid_for(V, 256), 256, 0, (cudaStream_t)stream>>>(d_deg_then, d_deg_later, V, horizon, d_t);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_sizing_buckets(mk_mlp *m, const float *d_x, const uint32_t *d_out_deg, uint32_t V, float horizon,
                            float load_factor, uint32_t max_buckets, float *d_y, uint32_t *d_buckets, void *stream)
{
    if (!m || !V || !d_x || !d_out_deg || !d_y || !d_buckets || !(load_factor > 0.f) || load_factor > 1.f ||
        horizon < 0.f || max_buckets == 0)
        return MK_ERR_INVALID_ARG;
    MK_TRY(mk_mlp_forward(m, d_x, V, d_y, stream));
    k_learned_buckets<<<grid_for(V, 256), 256, 0, (cudaStream_t)stream>>>(d_y, d_out_deg, V, horizon, load_factor,
                                                                          max_buckets, d_buckets);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

} // extern "C"
