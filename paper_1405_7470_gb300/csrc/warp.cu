// Small-N kernel: one warp holds 32 / N elements at a time, lane (s, n) owning
// node n of element slot s.  Each lane keeps its rows D[f][n][:] in registers;
// u[e][j] reaches lane (s, n) by a warp shuffle from lane (s, j), so the j
// reduction (the sum instruction of Section 2.1) runs lane-locally with no
// shared memory.  Element-major loads and stores are contiguous across the warp.
#include <cuda_runtime.h>

#include "lc_internal.h"

namespace lc {

template <typename T, int NMAX, int FMAX, bool NODE>
__global__ void __launch_bounds__(512) warp_contract_kernel(WarpArgs a)
{
    const int N = a.N, F = a.F, P = a.per_warp;
    const long long E = a.E;
    const T *__restrict__ D = static_cast<const T *>(a.D);
    const T *__restrict__ u = static_cast<const T *>(a.u);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int lane = threadIdx.x & 31;
    const int s = lane / N, n = lane - (lane / N) * N;
    const bool active = s < P;
    T dr[FMAX][NMAX];
#pragma unroll
    for (int f = 0; f < FMAX; ++f)
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
            dr[f][j] = (active && f < F && j < N) ? D[((size_t)f * N + n) * N + j] : T(0);

    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < a.ngroups;
         g += warps) {
        const long long e = g * P + s;
        const bool valid = active && e < E;
        T x = T(0);
        if (valid)
            x = NODE ? __ldg(u + (size_t)n * E + e) : __ldg(u + e * N + n);
        T acc[FMAX];
#pragma unroll
        for (int f = 0; f < FMAX; ++f)
            acc[f] = T(0);
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
            if (j < N) {
                const T xj = __shfl_sync(0xffffffffu, x, (s * N + j) & 31);
#pragma unroll
                for (int f = 0; f < FMAX; ++f)
                    acc[f] = fma(dr[f][j], xj, acc[f]);
            }
        }
        if (valid) {
#pragma unroll
            for (int f = 0; f < FMAX; ++f)
                if (f < F) {
                    if (NODE)
                        out[((size_t)f * N + n) * E + e] = acc[f];
                    else
                        out[((size_t)f * E + e) * N + n] = acc[f];
                }
        }
    }
}

template <typename T, bool NODE>
static void *warp_pick(int N)
{
    if (N <= 8)
        return reinterpret_cast<void *>(&warp_contract_kernel<T, 8, 4, NODE>);
    if (N <= 16)
        return reinterpret_cast<void *>(&warp_contract_kernel<T, 16, 4, NODE>);
    // FP64 above 16 nodes: one operator's row in registers (the planner admits F = 1 only)
    if constexpr (sizeof(T) == 8)
        return reinterpret_cast<void *>(&warp_contract_kernel<T, 32, 1, NODE>);
    else
        return reinterpret_cast<void *>(&warp_contract_kernel<T, 32, 4, NODE>);
}

lc_status warp_launch(const WarpArgs &a, int layout, int fp64, int grid, int threads, cudaStream_t s)
{
    const bool node = layout == LC_LAYOUT_NODE_MAJOR;
    void *fn = fp64 ? (node ? warp_pick<double, true>(a.N) : warp_pick<double, false>(a.N))
                    : (node ? warp_pick<float, true>(a.N) : warp_pick<float, false>(a.N));
    WarpArgs args = a;
    void *params[] = {&args};
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, 0, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

}  // namespace lc
