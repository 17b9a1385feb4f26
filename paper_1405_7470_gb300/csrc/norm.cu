// FP64 error norm on the GPU: sums[0] = sum (out - ref)^2, sums[1] = sum ref^2.
// Two launches with a fixed grid, so the summation order (and the result) is the
// same on every call: per-block partial sums, then one block adds them in order.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "lc_internal.h"
#include "tma.cuh"

namespace lc {

// Self-test of the bounded-wait error path: wait on an mbarrier phase that nothing
// completes; after limit_ns the wait gives up and the kernel records the timeout in
// the device error word, as every pipeline wait in the library does.
__global__ void selftest_wait_kernel(unsigned long long limit_ns, unsigned int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_ns(&bar, 0, limit_ns);
    if (!__syncthreads_and(ok) && threadIdx.x == 0)
        atomicOr(err, 1u);
}

static constexpr int kNormBlocks = 2048;
static constexpr int kNormThreads = 256;

__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? sh[2 * l] : 0.0;
        b = l < nw ? sh[2 * l + 1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kNormThreads) norm_partial_kernel(const T *__restrict__ out,
                                                                    const double *__restrict__ ref,
                                                                    long long n, double *partial)
{
    __shared__ double sh[2 * (kNormThreads / 32)];
    double s0 = 0.0, s1 = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // four grid-strided elements per step: eight independent loads in flight per thread
    for (; k + 3 * stride < n; k += 4 * stride) {
        double r[4], o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            r[q] = __ldcs(ref + k + q * stride);
            o[q] = (double)__ldcs(out + k + q * stride);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double d = o[q] - r[q];
            s0 = fma(d, d, s0);
            s1 = fma(r[q], r[q], s1);
        }
    }
    for (; k < n; k += stride) {
        const double r = ref[k];
        const double d = (double)out[k] - r;
        s0 = fma(d, d, s0);
        s1 = fma(r, r, s1);
    }
    block_sum2(s0, s1, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
    }
}

__global__ void __launch_bounds__(kNormThreads) norm_final_kernel(const double *__restrict__ partial,
                                                                  int nblocks, double *sums)
{
    __shared__ double sh[2 * (kNormThreads / 32)];
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        s0 += partial[2 * k];
        s1 += partial[2 * k + 1];
    }
    block_sum2(s0, s1, sh);
    if (threadIdx.x == 0) {
        sums[0] = s0;
        sums[1] = s1;
    }
}

size_t norm_workspace_bytes() { return sizeof(double) * 2 * kNormBlocks; }

lc_status norm_launch(const void *out, int dtype, const double *ref, long long n, double *sums,
                      double *partial, cudaStream_t s)
{
    if (dtype == LC_DTYPE_F32)
        norm_partial_kernel<float><<<kNormBlocks, kNormThreads, 0, s>>>(static_cast<const float *>(out), ref,
                                                                        n, partial);
    else
        norm_partial_kernel<double><<<kNormBlocks, kNormThreads, 0, s>>>(static_cast<const double *>(out),
                                                                         ref, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    norm_final_kernel<<<1, kNormThreads, 0, s>>>(partial, kNormBlocks, sums);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

// ---------------------------------------------------------------- no-allocation variant
//
// Some callers cannot hand the library a workspace: code that runs where cudaMalloc is
// off limits (it synchronises the whole device, so latency-bound serving loops and
// real-time callers forbid it), or plugins whose host framework owns every allocation
// and offers none to its extensions.  For them the same two-kernel reduction can take
// its partial sums from a fixed array that the library places in device memory.
//
// The array holds one (sum of squared differences, sum of squares) pair per block of
// the first kernel.  The grid is fixed by n alone: one block per kNoallocPerBlock
// elements, at most kNoallocMaxBlocks blocks, which grid-stride through the rest, so
// small inputs still spread over every SM.  One call handles at most kNoallocMaxElems
// elements (2^28), the documented limit of this entry point.  Every GPU that
// loads the library keeps these 64 KiB until the process exits.  All calls share the
// array: calls whose kernels overlap on the GPU (different streams, or threads) race on
// it and must be serialised by the caller.  Each call overwrites every slot it reads, so
// nothing needs clearing between calls.
static constexpr long long kNoallocPerBlock = 4LL * kNormThreads;
static constexpr int kNoallocMaxBlocks = 4096;
static constexpr long long kNoallocMaxElems = 1LL << 28;
static __device__ __align__(256) double g_norm_scratch[2 * kNoallocMaxBlocks];

static std::mutex g_scratch_mu;
static std::map<int, double *> g_scratch_addr;  // device -> address of g_norm_scratch

// The device address of g_norm_scratch on the current device.  Host code must not pass
// the symbol itself to a kernel: on the host it names a stand-in, not device memory.
static lc_status norm_scratch(double **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) {
        *ptr = it->second;
        return LC_OK;
    }
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_norm_scratch);
    if (e != cudaSuccess)
        return cuda_fail(e);
    g_scratch_addr[dev] = p;
    *ptr = p;
    return LC_OK;
}

}  // namespace lc

extern "C" {

lc_status lc_error_norm_noalloc(const void *out, int32_t out_dtype, const double *ref, int64_t n, double *sums,
                                void *stream)
{
    if (!out || !ref || !sums || n < 1)
        return LC_ERR_INVALID_ARGUMENT;
    if (out_dtype != LC_DTYPE_F32 && out_dtype != LC_DTYPE_F64)
        return LC_ERR_INVALID_ARGUMENT;
    if (n > lc::kNoallocMaxElems)
        return LC_ERR_BUFFER_TOO_SMALL;  // beyond the entry point's documented size limit
    if (((uintptr_t)ref & 7u) || ((uintptr_t)sums & 7u) || ((uintptr_t)out & (out_dtype == LC_DTYPE_F64 ? 7u : 3u)))
        return LC_ERR_MISALIGNED;
    double *scratch = nullptr;
    lc_status st = lc::norm_scratch(&scratch);
    if (st != LC_OK)
        return st;
    const int blocks =
        (int)std::min<long long>(lc::kNoallocMaxBlocks, (n + lc::kNoallocPerBlock - 1) / lc::kNoallocPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    if (out_dtype == LC_DTYPE_F32)
        lc::norm_partial_kernel<float><<<blocks, lc::kNormThreads, 0, s>>>(static_cast<const float *>(out), ref, n,
                                                                             scratch);
    else
        lc::norm_partial_kernel<double><<<blocks, lc::kNormThreads, 0, s>>>(static_cast<const double *>(out), ref,
                                                                              n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return lc::cuda_fail(e);
    lc::norm_final_kernel<<<1, lc::kNormThreads, 0, s>>>(scratch, blocks, sums);
    e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : lc::cuda_fail(e);
}

lc_status lc_selftest_wait_timeout(int64_t limit_ns, void *stream)
{
    if (limit_ns < 1 || limit_ns > 1000000000LL)
        return LC_ERR_INVALID_ARGUMENT;
    unsigned int *err = lc::error_word();
    if (!err)
        return LC_ERR_NO_DEVICE;
    lc::selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((unsigned long long)limit_ns, err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : lc::cuda_fail(e);
}

lc_status lc_error_norm_workspace_size(int64_t n, size_t *bytes)
{
    if (n < 0 || !bytes)
        return LC_ERR_INVALID_ARGUMENT;
    *bytes = lc::norm_workspace_bytes();
    return LC_OK;
}

lc_status lc_error_norm(const void *out, int32_t out_dtype, const double *ref, int64_t n, double *sums,
                        void *workspace, size_t workspace_bytes, void *stream)
{
    if (!out || !ref || !sums || !workspace || n < 0)
        return LC_ERR_INVALID_ARGUMENT;
    if (out_dtype != LC_DTYPE_F32 && out_dtype != LC_DTYPE_F64)
        return LC_ERR_INVALID_ARGUMENT;
    if (workspace_bytes < lc::norm_workspace_bytes())
        return LC_ERR_BUFFER_TOO_SMALL;
    if (((uintptr_t)workspace & 15u) || ((uintptr_t)ref & 7u) || ((uintptr_t)sums & 7u) ||
        ((uintptr_t)out & (out_dtype == LC_DTYPE_F64 ? 7u : 3u)))
        return LC_ERR_MISALIGNED;
    return lc::norm_launch(out, out_dtype, ref, n, sums, static_cast<double *>(workspace),
                           (cudaStream_t)stream);
}

}  // extern "C"
