// MLP cost model kernels: a network of three hidden ReLU layers of width 64 and one
// linear output, predicting log(run time) of a contraction variant from problem and
// descriptor features.  Forward (inference), loss + gradient (mean squared error),
// a deterministic cross-block gradient reduction, and the Adam update, all FP32.
//
// Parameter vector (float), in this order:
//   W1[64][din], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4[1]
// A CTA of 64 threads keeps the whole network in shared memory; thread h owns hidden
// unit h of every layer.
#include <cuda_runtime.h>

#include "lc_internal.h"

namespace lc {

static constexpr int kH = 64;       // hidden width
static constexpr int kMaxDin = 32;  // input features (keeps the network under 48 KB of shared memory)
static constexpr int kHp = kH + 1;  // padded row (column reads of W without bank conflicts)

__host__ __device__ inline long long mlp_nparams(int din) { return (long long)kH * din + kH + 2LL * (kH * kH + kH) + kH + 1; }

struct MlpSmem {
    float W1[kH][kMaxDin + 1];
    float W2[kH][kHp];
    float W3[kH][kHp];
    float b1[kH], b2[kH], b3[kH], w4[kH];
    float b4;
    float x[kMaxDin];
    float a1[kH], a2[kH], a3[kH];
    float g2[kH], g3[kH];
    float red[2];
};

__device__ void mlp_load(MlpSmem &S, const float *__restrict__ p, int din)
{
    const int h = threadIdx.x;
    const float *W1 = p, *b1 = W1 + kH * din, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH;
    const float *b3 = W3 + kH * kH, *w4 = b3 + kH, *b4 = w4 + kH;
    for (int k = 0; k < din; ++k)
        S.W1[h][k] = W1[h * din + k];
    for (int k = 0; k < kH; ++k) {
        S.W2[h][k] = W2[h * kH + k];
        S.W3[h][k] = W3[h * kH + k];
    }
    S.b1[h] = b1[h];
    S.b2[h] = b2[h];
    S.b3[h] = b3[h];
    S.w4[h] = w4[h];
    if (h == 0)
        S.b4 = b4[0];
}

// Forward pass of one sample already in S.x; returns y on every thread, keeps z > 0 flags.
__device__ float mlp_forward_one(MlpSmem &S, int din, bool &p1, bool &p2, bool &p3)
{
    const int h = threadIdx.x;
    float z = S.b1[h];
    for (int k = 0; k < din; ++k)
        z = fmaf(S.W1[h][k], S.x[k], z);
    p1 = z > 0.f;
    S.a1[h] = p1 ? z : 0.f;
    __syncthreads();
    z = S.b2[h];
#pragma unroll 8
    for (int k = 0; k < kH; ++k)
        z = fmaf(S.W2[h][k], S.a1[k], z);
    p2 = z > 0.f;
    S.a2[h] = p2 ? z : 0.f;
    __syncthreads();
    z = S.b3[h];
#pragma unroll 8
    for (int k = 0; k < kH; ++k)
        z = fmaf(S.W3[h][k], S.a2[k], z);
    p3 = z > 0.f;
    S.a3[h] = p3 ? z : 0.f;
    // output: sum_h w4[h] a3[h] + b4 (two warps)
    float v = S.w4[h] * S.a3[h];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((h & 31) == 0)
        S.red[h >> 5] = v;
    __syncthreads();
    const float y = S.red[0] + S.red[1] + S.b4;
    __syncthreads();
    return y;
}

__global__ void __launch_bounds__(kH) mlp_forward_kernel(const float *__restrict__ p, const float *__restrict__ X,
                                                         float *__restrict__ y, int n, int din)
{
    __shared__ MlpSmem S;
    mlp_load(S, p, din);
    __syncthreads();
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        if (threadIdx.x < din)
            S.x[threadIdx.x] = X[(size_t)s * din + threadIdx.x];
        __syncthreads();
        bool p1, p2, p3;
        const float out = mlp_forward_one(S, din, p1, p2, p3);
        if (threadIdx.x == 0)
            y[s] = out;
    }
}

// Per-block partial loss and gradient of L = (1/B) sum_s (y_s - t_s)^2 over the samples
// s = blockIdx.x, blockIdx.x + gridDim.x, ... < n; written to part[blockIdx.x][0..np],
// entry np holding the partial loss.
__global__ void __launch_bounds__(kH) mlp_grad_kernel(const float *__restrict__ p, const float *__restrict__ X,
                                                      const float *__restrict__ t, int n, int din, float inv_b,
                                                      float *__restrict__ part)
{
    __shared__ MlpSmem S;
    const int h = threadIdx.x;
    mlp_load(S, p, din);
    __syncthreads();
    // thread h accumulates the rows h of dW1, dW2, dW3 and the entries h of the vectors
    float dW1[kMaxDin];
    float dW2[kH], dW3[kH];
    float db1 = 0.f, db2 = 0.f, db3 = 0.f, dw4 = 0.f, db4 = 0.f, loss = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxDin; ++k)
        dW1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        dW2[k] = 0.f;
        dW3[k] = 0.f;
    }
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        if (h < din)
            S.x[h] = X[(size_t)s * din + h];
        __syncthreads();
        bool p1, p2, p3;
        const float yv = mlp_forward_one(S, din, p1, p2, p3);
        const float r = yv - t[s];
        loss += r * r;
        const float dy = 2.f * r * inv_b;
        db4 += dy;
        dw4 += dy * S.a3[h];
        const float g3 = p3 ? dy * S.w4[h] : 0.f;  // dL/dz3[h]
        S.g3[h] = g3;
        db3 += g3;
#pragma unroll
        for (int k = 0; k < kH; ++k)
            dW3[k] = fmaf(g3, S.a2[k], dW3[k]);
        __syncthreads();
        float s2 = 0.f;  // dL/da2[h] = sum_o W3[o][h] g3[o]
#pragma unroll 8
        for (int o = 0; o < kH; ++o)
            s2 = fmaf(S.W3[o][h], S.g3[o], s2);
        const float g2 = p2 ? s2 : 0.f;
        S.g2[h] = g2;
        db2 += g2;
#pragma unroll
        for (int k = 0; k < kH; ++k)
            dW2[k] = fmaf(g2, S.a1[k], dW2[k]);
        __syncthreads();
        float s1 = 0.f;
#pragma unroll 8
        for (int o = 0; o < kH; ++o)
            s1 = fmaf(S.W2[o][h], S.g2[o], s1);
        const float g1 = p1 ? s1 : 0.f;
        db1 += g1;
#pragma unroll
        for (int k = 0; k < kMaxDin; ++k)
            if (k < din)
                dW1[k] = fmaf(g1, S.x[k], dW1[k]);
        __syncthreads();
    }
    const long long np = mlp_nparams(din);
    float *g = part + (size_t)blockIdx.x * (np + 1);
    float *gW1 = g, *gb1 = gW1 + kH * din, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gW3 = gb2 + kH;
    float *gb3 = gW3 + kH * kH, *gw4 = gb3 + kH, *gb4 = gw4 + kH;
#pragma unroll
    for (int k = 0; k < kMaxDin; ++k)
        if (k < din)
            gW1[h * din + k] = dW1[k];
#pragma unroll
    for (int k = 0; k < kH; ++k) {
        gW2[h * kH + k] = dW2[k];
        gW3[h * kH + k] = dW3[k];
    }
    gb1[h] = db1;
    gb2[h] = db2;
    gb3[h] = db3;
    gw4[h] = dw4;
    if (h == 0) {
        gb4[0] = db4;
        g[np] = loss * inv_b;
    }
}

// grad[q] = sum over blocks of part[b][q] (fixed order), q in [0, np]; entry np = loss.
__global__ void mlp_reduce_kernel(const float *__restrict__ part, int nblocks, long long np1, float *__restrict__ out)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < np1; q += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b)
            s += part[(size_t)b * np1 + q];
        out[q] = s;
    }
}

__global__ void mlp_adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                                float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                                float c2)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

static constexpr int kGradBlocks = 64;

}  // namespace lc

using namespace lc;

extern "C" {

lc_status lc_mlp_param_count(int32_t din, int64_t *count)
{
    if (din < 1 || din > kMaxDin || !count)
        return LC_ERR_INVALID_ARGUMENT;
    *count = mlp_nparams(din);
    return LC_OK;
}

lc_status lc_mlp_forward(const float *params, const float *X, int64_t n, int32_t din, float *y, void *stream)
{
    if (!params || (n > 0 && (!X || !y)) || n < 0 || din < 1 || din > kMaxDin)
        return LC_ERR_INVALID_ARGUMENT;
    if (n == 0)
        return LC_OK;
    const int grid = (int)std::min<long long>(n, 1024);
    mlp_forward_kernel<<<grid, kH, 0, (cudaStream_t)stream>>>(params, X, y, (int)n, din);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

lc_status lc_mlp_workspace_size(int32_t din, size_t *bytes)
{
    if (din < 1 || din > kMaxDin || !bytes)
        return LC_ERR_INVALID_ARGUMENT;
    *bytes = sizeof(float) * (size_t)kGradBlocks * (mlp_nparams(din) + 1);
    return LC_OK;
}

lc_status lc_mlp_loss_grad(const float *params, const float *X, const float *t, int64_t n, int32_t din,
                           float *grad_loss, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!params || !X || !t || !grad_loss || !workspace || n <= 0 || din < 1 || din > kMaxDin)
        return LC_ERR_INVALID_ARGUMENT;
    size_t need = 0;
    lc_mlp_workspace_size(din, &need);
    if (workspace_bytes < need)
        return LC_ERR_BUFFER_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<long long>(n, kGradBlocks);
    float *part = static_cast<float *>(workspace);
    mlp_grad_kernel<<<blocks, kH, 0, s>>>(params, X, t, (int)n, din, 1.f / (float)n, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    const long long np1 = mlp_nparams(din) + 1;
    mlp_reduce_kernel<<<(int)((np1 + 255) / 256), 256, 0, s>>>(part, blocks, np1, grad_loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

lc_status lc_mlp_adam_step(float *params, const float *grad, float *m, float *v, int64_t n, int32_t step, float lr,
                           float beta1, float beta2, float eps, void *stream)
{
    if (!params || !grad || !m || !v || n <= 0 || step < 1)
        return LC_ERR_INVALID_ARGUMENT;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    mlp_adam_kernel<<<(int)std::min<long long>((n + 255) / 256, 1024), 256, 0, (cudaStream_t)stream>>>(
        params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

}  // extern "C"
