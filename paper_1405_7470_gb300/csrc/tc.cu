// Tensor-core (tcgen05 / TMEM) kernel for the element-local contraction
//     out[f,e,i] = sum_j D[f,i,j] * u[e,j]                (dG FEM volume, Table 1)
// as a GEMM per tile of 128 elements: A = u tile [128 x K] (K = nodes j, padded to a
// multiple of 16), B = D^T columns [CB x K] (c = f*N + i for the G operators of this
// CTA's column block), accumulator [128 x CB] FP32 in tensor memory.
//
// Precision paths (FP32 accumulation in both):
//   BF16    operands rounded to bfloat16 (nearest-even), one product.
//   BF16X3  x = hi + mid + lo (three bfloat16 terms, exact for binary32); the six
//           products hh, hm, mh, hl, lh, mm are accumulated, small ones first; the
//           dropped products (ml, lm, ll) are below 2^-24 relative.
//
// Structure (one CTA of 128 threads per SM; thread r owns tile row / TMEM lane r):
//   setup    warp 0 allocates 2 accumulators in TMEM; all threads split D into the
//            B-operand terms in shared memory (K-major, hardware swizzle layout).
//   loop     the bulk-copy engine fetches the next u tile (fp32) into a stage buffer;
//            threads convert the tile into the A-operand terms; thread 0 issues the
//            MMAs for tile k into accumulator k % 2 and commits them to an mbarrier;
//            meanwhile all threads drain accumulator (k-1) % 2 (tcgen05.ld) and store
//            it: element-major through shared memory and one bulk store per operator,
//            node-major straight from registers (coalesced along e).
// Every mbarrier wait is bounded in time; on a timeout the kernel sets the device
// error word, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lc_internal.h"
#include "tma.cuh"

namespace lc {

// ------------------------------------------------------------------ tcgen05 helpers

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, M = 128, N and K = 16 per the instruction descriptor.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on an mbarrier once all previously issued MMAs of this thread have completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q)
        v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor, K-major, swizzle atom of W bytes per row (32, 64, 128):
// start address, leading offset 16 B (unused for swizzled K-major), stride between
// 8-row groups = 8*W, descriptor version 1, layout type per swizzle width.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int W)
{
    const uint64_t layout = W == 128 ? 2ull : (W == 64 ? 4ull : 6ull);
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)((8u * W) >> 4) << 32) | (1ull << 46) |
           (layout << 61);
}

// Instruction descriptor: kind::f16, A = B = bf16, K-major both, D = f32, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of the 16-byte chunk (row, chunk16) inside a K-block of rows of W bytes with
// the hardware swizzle (16-byte chunk index XORed with address bits 7.. of the row).
__device__ __forceinline__ uint32_t swz_off(int row, int chunk16, int W)
{
    const int mask = W / 16 - 1;
    return (uint32_t)(row * W + ((chunk16 ^ ((row * W >> 7) & mask)) << 4));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Split 8 floats into NT bfloat16 terms (hi, mid, lo), each packed as 16 bytes.
template <int NT>
__device__ __forceinline__ void split8(const float *x, uint4 *t)
{
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * q]), h1 = __float2bfloat16_rn(x[2 * q + 1]);
        w[0][q] = pack2(h0, h1);
        if (NT == 3) {
            const float r0 = x[2 * q] - __bfloat162float(h0), r1 = x[2 * q + 1] - __bfloat162float(h1);
            __nv_bfloat16 m0 = __float2bfloat16_rn(r0), m1 = __float2bfloat16_rn(r1);
            const float s0 = r0 - __bfloat162float(m0), s1 = r1 - __bfloat162float(m1);
            w[1][q] = pack2(m0, m1);
            w[2][q] = pack2(__float2bfloat16_rn(s0), __float2bfloat16_rn(s1));
        }
    }
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
        t[tt] = make_uint4(w[tt][0], w[tt][1], w[tt][2], w[tt][3]);
}

// ------------------------------------------------------------------ kernel

template <int LAYOUT, int NT>
__global__ void __launch_bounds__(128, 1) tc_contract_kernel(const __grid_constant__ TcArgs a)
{
    constexpr bool NODE = LAYOUT == LC_LAYOUT_NODE_MAJOR;
    constexpr int TE = 128;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte aligned base for the swizzled operand tiles
    const uint32_t raw = smem_addr(smem_dyn);
    unsigned char *smem = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sbase = smem_addr(smem);

    const int N = a.N, G = a.G, CB = a.CB, CBp = a.CBp, Kp = a.Kp, KB = a.KB, nkb = a.nkb;
    const int W = 2 * KB;  // bytes per row of a K-block
    const long long E = a.E;
    const int S = a.stages;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int blk = blockIdx.x % a.nblocks;  // this CTA's column block
    const int f0 = blk * G;
    const int Gb = min(G, a.F - f0);         // operators in this block
    const int CBb = Gb * N;                  // valid columns

    const uint32_t offB = 0;
    const uint32_t termB = (uint32_t)nkb * CBp * W;  // bytes per B term
    const uint32_t offA = offB + NT * termB;
    const uint32_t termA = (uint32_t)nkb * TE * W;
    float *stage = reinterpret_cast<float *>(smem + a.off_stage);  // S x [TE*N] fp32
    float *ost = reinterpret_cast<float *>(smem + a.off_out);      // [G][TE][N] (element-major)
    uint64_t *bar_u = reinterpret_cast<uint64_t *>(smem + a.off_bar);
    uint64_t *bar_mma = bar_u + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar_u + 4);

    if (warp == 0)
        tmem_alloc(tmem_holder, 2u * a.tmem_cols);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bar_u[s], 1);
            mbar_init(&bar_mma[s], 1);
        }
        fence_mbar_init();
    }

    // B terms: row n = f_local*N + i of this block, column k = j; zero padding.
    {
        const int c8n = Kp / 8;
        for (int idx = tid; idx < CBp * c8n; idx += blockDim.x) {
            const int n = idx / c8n, c8 = idx - n * c8n;
            float x[8];
            const int fl = n / N, i = n - fl * N;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = c8 * 8 + q;
                x[q] = (n < CBb && j < N) ? a.D[((size_t)(f0 + fl) * N + i) * N + j] : 0.f;
            }
            uint4 t[3];
            split8<NT>(x, t);
            const int kb = (c8 * 8) / KB, ch = ((c8 * 8) % KB) / 8;
            const uint32_t off = offB + (uint32_t)kb * CBp * W + swz_off(n, ch, W);
#pragma unroll
            for (int tt = 0; tt < NT; ++tt)
                *reinterpret_cast<uint4 *>(smem + off + tt * termB) = t[tt];
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    const long long my_first = blockIdx.x / a.nblocks;
    const long long my_step = gridDim.x / a.nblocks;

    // Fetch u tile t into stage slot s (thread 0). Tiles the bulk engine cannot fetch
    // (unaligned tails) are read from global memory during the conversion.
    auto tile_bulk_bytes = [&](long long t) -> uint32_t {
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);
        if (!a.bulk_u)
            return 0;
        const uint32_t bytes = (uint32_t)TEv * N * 4u;
        return (bytes & 15u) ? 0u : bytes;
    };
    auto issue_u = [&](long long t, int s) {
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);
        const uint32_t bytes = tile_bulk_bytes(t);
        mbar_arrive_expect_tx(&bar_u[s], bytes);
        if (!bytes)
            return;
        float *dst = stage + (size_t)s * TE * N;
        if (NODE) {
            for (int j = 0; j < N; ++j)
                bulk_g2s(dst + (size_t)j * TE, a.u + (size_t)j * E + e0, (uint32_t)TEv * 4u, &bar_u[s]);
        } else {
            bulk_g2s(dst, a.u + e0 * N, bytes, &bar_u[s]);
        }
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            const long long t = my_first + s * my_step;
            if (t < a.ntiles)
                issue_u(t, s);
        }
    }

    const uint32_t idesc = instr_desc(CBp);
    const int ksteps = Kp / 16;
    bool failed = false;

    // Drain accumulator `acc` of tile `t` to global memory.
    auto epilogue = [&](long long t, int acc) {
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);
        const int r = tid;  // tile row == TMEM lane
        const uint32_t tbase = tmem_base + (uint32_t)acc * a.tmem_cols + ((uint32_t)(warp * 32) << 16);
        if (!NODE) {
            if (tid == 0)
                bulk_wait_read0();  // previous bulk stores have read ost
            __syncthreads();
        }
        int fl = 0, i = 0;
        for (int c0 = 0; c0 < CBp; c0 += 32) {
            float v[32];
            tmem_ld32(tbase + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int c = c0 + q;
                if (c < CBb) {
                    if (NODE) {
                        if (r < TEv)
                            a.out[((size_t)(f0 + fl) * N + i) * E + e0 + r] = v[q];
                    } else {
                        ost[((size_t)fl * TE + r) * N + i] = v[q];
                    }
                    if (++i == N) {
                        i = 0;
                        ++fl;
                    }
                }
            }
        }
        tc_fence_before();
        if (!NODE) {
            fence_async_smem();
            __syncthreads();
            const int total = TEv * N;
            const bool bulk = a.bulk_store && ((total * 4) & 15) == 0;
            if (bulk) {
                if (tid == 0) {
                    for (int g = 0; g < Gb; ++g)
                        bulk_s2g(a.out + ((size_t)(f0 + g) * E + e0) * N, ost + (size_t)g * TE * N,
                                 (uint32_t)total * 4u);
                    bulk_commit();
                }
            } else {
                for (int g = 0; g < Gb; ++g) {
                    const float *src = ost + (size_t)g * TE * N;
                    float *dst = a.out + ((size_t)(f0 + g) * E + e0) * N;
                    for (int q = tid; q < total; q += blockDim.x)
                        dst[q] = src[q];
                }
            }
        }
    };

    long long prev_tile = -1;
    int k = 0;
    for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
        const int acc = k & 1;
        const int s = S == 2 ? (k & 1) : 0;
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);

        // u tile landed, and the MMAs of the previous tile (readers of the A terms) are done
        bool ok = mbar_wait(&bar_u[s], (uint32_t)((k / S) & 1));
        if (k >= 1)
            ok = ok && mbar_wait(&bar_mma[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1));
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        tc_fence_after();

        // convert row r of the u tile into the A terms
        {
            const int r = tid;
            const bool from_stage = tile_bulk_bytes(t) != 0;
            const float *st = stage + (size_t)s * TE * N;
            const int c8n = Kp / 8;
            for (int c8 = 0; c8 < c8n; ++c8) {
                float x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = c8 * 8 + q;
                    float val = 0.f;
                    if (j < N && r < TEv) {
                        if (from_stage)
                            val = NODE ? st[j * TE + r] : st[r * N + j];
                        else
                            val = NODE ? a.u[(size_t)j * E + e0 + r] : a.u[(e0 + r) * N + j];
                    }
                    x[q] = val;
                }
                uint4 tt4[3];
                split8<NT>(x, tt4);
                const int kb = (c8 * 8) / KB, ch = ((c8 * 8) % KB) / 8;
                const uint32_t off = offA + (uint32_t)kb * TE * W + swz_off(r, ch, W);
#pragma unroll
                for (int tt = 0; tt < NT; ++tt)
                    *reinterpret_cast<uint4 *>(smem + off + tt * termA) = tt4[tt];
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        if (tid == 0) {
            // stage slot s is consumed: fetch the tile S steps ahead
            const long long tn = t + (long long)S * my_step;
            if (tn < a.ntiles)
                issue_u(tn, s);
            // MMAs: pairs (D term, u term), small products first
            // (D term, u term): lh, hl, mm, mh, hm, hh
            const uint32_t dtm = tmem_base + (uint32_t)acc * a.tmem_cols;
            constexpr int npairs = NT == 3 ? 6 : 1;
#pragma unroll
            for (int p = 0; p < npairs; ++p) {
                const int bt = NT == 3 ? (p == 0 ? 2 : (p == 2 || p == 3) ? 1 : 0) : 0;
                const int at = NT == 3 ? (p == 1 ? 2 : (p == 2 || p == 4) ? 1 : 0) : 0;
                for (int kk = 0; kk < ksteps; ++kk) {
                    const int kb = (kk * 16) / KB, kin = ((kk * 16) % KB) * 2;  // byte offset in the row
                    const uint64_t ad = smem_desc(sbase + offA + at * termA + kb * TE * W + kin, W);
                    const uint64_t bd = smem_desc(sbase + offB + bt * termB + kb * CBp * W + kin, W);
                    tc_mma(dtm, ad, bd, idesc, (p > 0 || kk > 0) ? 1u : 0u);
                }
            }
            tc_commit(&bar_mma[acc]);
        }

        if (prev_tile >= 0)
            epilogue(prev_tile, acc ^ 1);
        prev_tile = t;
    }

    if (!failed && prev_tile >= 0) {
        const bool ok = mbar_wait(&bar_mma[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1));
        if (__syncthreads_and(ok)) {
            tc_fence_after();
            epilogue(prev_tile, (k - 1) & 1);
        } else {
            failed = true;
        }
    }
    if (failed && tid == 0)
        atomicOr(a.err, 1u);
    if (!NODE && tid == 0)
        bulk_wait0();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tmem_base, 2u * a.tmem_cols);
}

lc_status tc_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s)
{
    void *fn;
    const bool node = layout == LC_LAYOUT_NODE_MAJOR;
    if (nterms == 3)
        fn = node ? reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3>)
                  : reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3>);
    else
        fn = node ? reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1>)
                  : reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem_bytes);
    if (e != cudaSuccess)
        return cuda_fail(e);
    TcArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(128), params, a.smem_bytes, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

}  // namespace lc
