// K-split SIMT kernel (FP32) for the element-local contraction
//     out[f,e,i] = sum_j D[f,i,j] * u[e,j]                (dG FEM volume, Table 1)
// read as the product of the u tile [BM x N] and D^T [N x F*N] (column c = f*N + i).
//
// Transformations (Section 2.4) and how they map here:
//   split_iname(e, BM)       one tile of BM elements per CTA step (persistent, grid-stride);
//                            rows past E are zeros and are not stored.
//   split_iname(j, BK)       the reduction in chunks of BK; the D^T slice of each chunk is
//                            fetched asynchronously (cp.async, 4-byte elements, zero-filled
//                            past N or past the last column) into a two-slot ring one chunk
//                            ahead, so D^T never has to fit in shared memory at once.
//   add_prefetch(u)          the u tile, transposed to [j][e], stays resident for every
//                            column block of the tile; with two buffers the next tile's
//                            u is fetched while this one is used.
//   ilp on e and on i        8 x 8 register block per thread: elements {4ty..4ty+3,
//                            BM/2+4ty..}, columns {4tx..4tx+3, 64+4tx..} of a 128-column
//                            block; the operand reads are 16-byte vector loads.
//   unr on j                 the chunk loop is fully unrolled.
// Column blocks of 128 cover F*N columns; the u tile is read once per tile for all of them.
#include <cuda_runtime.h>

#include "lc_internal.h"
#include "tma.cuh"

namespace lc {

static constexpr int kKsBN = 128;  // output columns per block

// 4-byte asynchronous copy global -> shared; `bytes` 0 writes a zero (nothing is read).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(bytes)
                 : "memory");
}

// 16-byte asynchronous copy; the first `bytes` (0..16) come from src, the rest are zeros.
__device__ __forceinline__ void cp_async16(float *dst, const float *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int LAYOUT, int BM, int BK>
struct KsShape {
    static constexpr int TH = BM / 8 * 16;  // threads: (BM / 8) x 16
    static constexpr int LDA = BM + 4;      // u tile row (one j): BM elements, padded
    static constexpr int LDB = kKsBN + 4;   // D^T chunk row (one j): 128 columns, padded
    static constexpr int TPC = TH / kKsBN;  // threads per column of a D^T chunk (1 or 2)
    static constexpr int KPT = BK / TPC;    // chunk rows each of them copies
};

// Copy the u tile of elements e0 .. e0+BM-1 into ut[j][e] (j < Kp; zeros past N or E).
template <int LAYOUT, int BM, int BK>
__device__ __forceinline__ void ks_load_u(const KsArgs &a, float *ut, long long e0, int tid)
{
    using S = KsShape<LAYOUT, BM, BK>;
    const int N = a.N, Kp = a.Kp;
    const long long E = a.E;
    if (LAYOUT == LC_LAYOUT_NODE_MAJOR) {
        // rows j of u[N][E] are contiguous in e: 16-byte pieces when E % 4 == 0
        if (a.vec_u) {
            constexpr int Q = BM / 4;
            for (int idx = tid; idx < Kp * Q; idx += S::TH) {
                const int j = idx / Q, e = (idx - j * Q) * 4;
                const long long left = E - (e0 + e);
                const uint32_t bytes = (j < N && left > 0) ? (uint32_t)(left >= 4 ? 16 : left * 4) : 0u;
                cp_async16(ut + j * S::LDA + e, bytes ? a.u + (size_t)j * E + e0 + e : a.u, bytes);
            }
        } else {
            for (int idx = tid; idx < Kp * BM; idx += S::TH) {
                const int j = idx / BM, e = idx - j * BM;
                const bool ok = j < N && e0 + e < E;
                cp_async4(ut + j * S::LDA + e, ok ? a.u + (size_t)j * E + e0 + e : a.u, ok ? 4u : 0u);
            }
        }
    } else {
        // rows e of u[E][N] are contiguous in j: j fastest across threads (coalesced reads),
        // written transposed; the walk idx = e * Kp + j advances by TH without divisions
        const int de = S::TH / Kp, dj = S::TH - de * Kp;
        int e = tid / Kp, j = tid - e * Kp;
        while (e < BM) {
            const bool ok = j < N && e0 + e < E;
            cp_async4(ut + j * S::LDA + e, ok ? a.u + (e0 + e) * N + j : a.u, ok ? 4u : 0u);
            e += de;
            j += dj;
            if (j >= Kp) {
                j -= Kp;
                ++e;
            }
        }
    }
}

// Copy rows kc*BK .. kc*BK+BK-1 of the D^T column block starting at column c0 into bs[k][c].
// Each thread copies KPT rows of one column: `drow` is that column's D row (null past C).
template <int LAYOUT, int BM, int BK>
__device__ __forceinline__ void ks_load_b(const KsArgs &a, float *bs, const float *drow, int kc, int tid)
{
    using S = KsShape<LAYOUT, BM, BK>;
    const int cl = tid / S::TPC, k0 = (tid - cl * S::TPC) * S::KPT;
#pragma unroll
    for (int q = 0; q < S::KPT; ++q) {
        const int j = kc * BK + k0 + q;
        const bool ok = drow != nullptr && j < a.N;
        cp_async4(bs + (k0 + q) * S::LDB + cl, ok ? drow + j : a.D, ok ? 4u : 0u);
    }
}

// The D row feeding column cl of block cb (null past the last column): column c = f*N + i
// reads D[f][i][:].
__device__ __forceinline__ const float *ks_drow(const KsArgs &a, int cb, int cl)
{
    const int c = cb * kKsBN + cl;
    if (c >= a.C)
        return nullptr;
    const int f = c / a.N, i = c - f * a.N;
    return a.D + ((size_t)f * a.N + i) * a.N;
}

// Resident CTAs the register budget is sized for (128 registers a thread at 2 x 256 or
// 3 x 128 threads).
#ifndef KS_MIN_CTAS_128
#define KS_MIN_CTAS_128 2
#endif
#ifndef KS_MIN_CTAS_64
#define KS_MIN_CTAS_64 3
#endif

template <int LAYOUT, int BM, int BK>
__global__ void __launch_bounds__(BM / 8 * 16, BM == 128 ? KS_MIN_CTAS_128 : KS_MIN_CTAS_64)
    ks_contract_kernel(const __grid_constant__ KsArgs a)
{
    using S = KsShape<LAYOUT, BM, BK>;
    constexpr bool NODE = LAYOUT == LC_LAYOUT_NODE_MAJOR;
    extern __shared__ __align__(16) float ks_smem[];
    const int N = a.N, Kp = a.Kp, nkc = a.nkc, nb = a.nblocks;
    const long long E = a.E;
    float *ubuf = ks_smem;                                    // [ubufs][Kp][LDA]
    float *bbuf = ks_smem + (size_t)a.ubufs * Kp * S::LDA;    // [2][BK][LDB]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int cl = tid / S::TPC;  // the D^T column this thread copies
    const long long t0 = blockIdx.x, dt = gridDim.x;
    if (t0 >= a.ntiles)
        return;

    float acc[8][8];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y)
            acc[x][y] = 0.f;

    // prologue: the first tile's u and the first chunk
    const float *drow = ks_drow(a, 0, cl);
    ks_load_u<LAYOUT, BM, BK>(a, ubuf, t0 * BM, tid);
    ks_load_b<LAYOUT, BM, BK>(a, bbuf, drow, 0, tid);
    cp_async_commit();
    int sl = 0;  // ring slot of the current chunk
    int ti = 0;
    for (long long t = t0; t < a.ntiles; t += dt, ++ti) {
        const long long e0 = t * BM;
        const int ub = a.ubufs == 2 ? (ti & 1) : 0;
        const float *ut = ubuf + (size_t)ub * Kp * S::LDA;
        const bool has_next_tile = t + dt < a.ntiles;
        for (int cb = 0; cb < nb; ++cb) {
            for (int kc = 0; kc < nkc; ++kc) {
                cp_async_wait_all();  // this thread's copies of the current chunk (and tile) landed
                __syncthreads();      // everyone's landed; everyone is done with the other slot
                if (a.ubufs == 1 && ti > 0 && cb == 0 && kc == 0) {
                    // one u buffer: the previous tile's reads are over only now
                    ks_load_u<LAYOUT, BM, BK>(a, ubuf, e0, tid);
                    cp_async_commit();
                    cp_async_wait_all();
                    __syncthreads();
                }
                // the next chunk: (cb, kc + 1), (cb + 1, 0) or the next tile's (0, 0)
                int nkc_ = kc + 1, ncb = cb;
                if (nkc_ == nkc) {
                    nkc_ = 0;
                    ncb = cb + 1;
                }
                const bool next_in_tile = ncb < nb;
                if (next_in_tile || has_next_tile) {
                    if (ncb == nb)
                        ncb = 0;
                    if (nkc_ == 0)
                        drow = ks_drow(a, ncb, cl);
                    ks_load_b<LAYOUT, BM, BK>(a, bbuf + (size_t)(sl ^ 1) * BK * S::LDB, drow, nkc_, tid);
                }
                if (a.ubufs == 2 && cb == 0 && kc == 0 && has_next_tile)
                    ks_load_u<LAYOUT, BM, BK>(a, ubuf + (size_t)(ub ^ 1) * Kp * S::LDA, (t + dt) * BM, tid);
                cp_async_commit();

                const float *A = ut + (size_t)kc * BK * S::LDA;
                const float *B = bbuf + (size_t)sl * BK * S::LDB;
#pragma unroll
                for (int k = 0; k < BK; ++k) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(A + k * S::LDA + 4 * ty);
                    const float4 a1 = *reinterpret_cast<const float4 *>(A + k * S::LDA + BM / 2 + 4 * ty);
                    const float4 b0 = *reinterpret_cast<const float4 *>(B + k * S::LDB + 4 * tx);
                    const float4 b1 = *reinterpret_cast<const float4 *>(B + k * S::LDB + 64 + 4 * tx);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int x = 0; x < 8; ++x)
#pragma unroll
                        for (int y = 0; y < 8; ++y)
                            acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
                }
                sl ^= 1;
            }
            // the 8 x 8 block of column block cb: rows 4ty + (0..3) and BM/2 + 4ty + (0..3),
            // columns 4tx + (0..3) and 64 + 4tx + (0..3)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c4 = cb * kKsBN + 64 * h + 4 * tx;  // first of 4 consecutive columns
                if (c4 >= a.C)
                    continue;
                if (NODE) {
                    // out[f][i][e]: per column, 4 consecutive elements
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        const int c = c4 + y;
                        if (c >= a.C)
                            break;
                        const int f = c / N, i = c - f * N;
                        float *col = a.out + ((size_t)f * N + i) * E;
#pragma unroll
                        for (int g = 0; g < 2; ++g) {
                            const long long eb = e0 + g * (BM / 2) + 4 * ty;
                            const float v0 = acc[4 * g][4 * h + y], v1 = acc[4 * g + 1][4 * h + y];
                            const float v2 = acc[4 * g + 2][4 * h + y], v3 = acc[4 * g + 3][4 * h + y];
                            if (a.vec_out && eb + 3 < E) {
                                *reinterpret_cast<float4 *>(col + eb) = make_float4(v0, v1, v2, v3);
                            } else {
                                const float vv[4] = {v0, v1, v2, v3};
#pragma unroll
                                for (int z = 0; z < 4; ++z)
                                    if (eb + z < E)
                                        col[eb + z] = vv[z];
                            }
                        }
                    }
                } else {
                    // out[f][e][i]: per element, 4 consecutive columns (one operator's when
                    // N % 4 == 0: then one 16-byte store)
                    const int f4 = c4 / N, i4 = c4 - f4 * N;
#pragma unroll
                    for (int x = 0; x < 8; ++x) {
                        const long long e = e0 + (x < 4 ? 4 * ty + x : BM / 2 + 4 * ty + x - 4);
                        if (e >= E)
                            continue;
                        if (a.vec_out) {
                            *reinterpret_cast<float4 *>(a.out + ((size_t)f4 * E + e) * N + i4) =
                                make_float4(acc[x][4 * h], acc[x][4 * h + 1], acc[x][4 * h + 2], acc[x][4 * h + 3]);
                        } else {
                            int f = f4, i = i4;
#pragma unroll
                            for (int y = 0; y < 4; ++y) {
                                if (c4 + y < a.C)
                                    a.out[((size_t)f * E + e) * N + i] = acc[x][4 * h + y];
                                if (++i == N) {
                                    i = 0;
                                    ++f;
                                }
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y)
                    acc[x][y] = 0.f;
        }
    }
    cp_async_wait_all();  // no copy outlives the CTA
}

size_t ks_smem_bytes(int Kp, int bm, int bk, int ubufs)
{
    return sizeof(float) * ((size_t)ubufs * Kp * (bm + 4) + 2 * (size_t)bk * (kKsBN + 4));
}

template <int LAYOUT>
static void *ks_fn(int bm, int bk)
{
    if (bm == 128)
        return bk == 16 ? reinterpret_cast<void *>(&ks_contract_kernel<LAYOUT, 128, 16>)
                        : reinterpret_cast<void *>(&ks_contract_kernel<LAYOUT, 128, 8>);
    return bk == 16 ? reinterpret_cast<void *>(&ks_contract_kernel<LAYOUT, 64, 16>)
                    : reinterpret_cast<void *>(&ks_contract_kernel<LAYOUT, 64, 8>);
}

lc_status ks_launch(const KsArgs &a, int layout, int bm, int bk, int grid, cudaStream_t s, bool set_attr)
{
    if (!(bm == 64 || bm == 128) || !(bk == 8 || bk == 16))
        return LC_ERR_INVALID_VARIANT;
    void *fn = layout == LC_LAYOUT_NODE_MAJOR ? ks_fn<LC_LAYOUT_NODE_MAJOR>(bm, bk) : ks_fn<LC_LAYOUT_ELEM_MAJOR>(bm, bk);
    const size_t smem = ks_smem_bytes(a.Kp, bm, bk, a.ubufs);
    cudaError_t e = cudaSuccess;
    if (set_attr) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return cuda_fail(e);
    }
    if (grid <= 0)
        return LC_OK;  // attribute set only (a capture launches later)
    KsArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(bm / 8 * 16), params, smem, s);
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

}  // namespace lc
