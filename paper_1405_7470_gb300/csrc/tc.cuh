// Tensor-core (tcgen05 / TMEM) kernel for the element-local contraction
//     out[f,e,i] = sum_j D[f,i,j] * u[e,j]                (dG FEM volume, Table 1)
// as a GEMM per tile of 128 elements: A = u tile [128 x K] (K = nodes j, padded to a
// multiple of 16), B = D^T columns [CB x K] (c = f*Np + i for the G operators of this
// CTA's column block, each padded to Np columns), accumulator [128 x CB] FP32 in tensor
// memory.  Operands live in K-blocks of 16, 32 or 64 bf16 per row (32/64/128-byte swizzle).
//
// Precision paths (FP32 accumulation in both):
//   BF16    operands rounded to bfloat16 (nearest-even), one product.
//   BF16X3  x = hi + mid + lo (three bfloat16 terms, exact for binary32); the six
//           products hh, hm, mh, hl, lh, mm are accumulated with the large hh sum kept
//           apart from (or after) the others; the dropped products (ml, lm, ll) are
//           below 2^-24 relative.
//
// Structure: a persistent, warp-specialised CTA per SM, roles linked by full/empty
// mbarrier pairs (no CTA-wide barrier inside the tile loop):
//   producer warp  the bulk-copy engine fetches u tiles (fp32) into a ring of
//                  `stages` shared-memory buffers;
//   MMA warp       one lane issues the tcgen05.mma chain of tile k into TMEM
//                  accumulator k % 2 (two accumulators), K-block by K-block,
//                  committing each block of the A buffer back as it is done, then the
//                  accumulator to the epilogue;
//   4*Hc converters convert the fp32 tile into the bf16 A-operand terms (K-major,
//                  hardware swizzle layout; Hc threads share a tile row's K chunks),
//                  K-block by K-block;
//   4*He epilogue  drain the accumulator of a finished tile (tcgen05.ld; the He warps
//                  of a TMEM lane quarter split its columns) and store it: element-
//                  major through shared-memory slots and bulk stores (every operator
//                  of the tile per slot, or one operator per slot in store groups of
//                  lane quarters), node-major straight from registers (coalesced
//                  along e);
//   store warp     issues the bulk stores of the whole-tile slots and hands each slot
//                  back once the copies have read it (idle in the other layouts).
// Setup: the MMA warp allocates the accumulators; all threads split D into the
// B-operand terms, resident for the CTA's lifetime.
// Every mbarrier wait is bounded in time; on a timeout the kernel sets the device
// error word, frees its tensor memory and returns.
#pragma once

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

// 16 consecutive accumulator columns of this thread's TMEM lane (complete after tmem_wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

// 8 consecutive accumulator columns of this thread's TMEM lane (complete after tmem_wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Store 4 consecutive 32-bit columns of this thread's TMEM lane (complete after tmem_wait_st).
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint4 &v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem desc]^T: A (M = 128 rows, one per TMEM lane; K = 16 bf16 packed
// two per 32-bit column, 8 columns) read from tensor memory.
__device__ __forceinline__ void tc_mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
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

// Round two floats to a packed bfloat16 pair (nearest-even): lo half = a, hi half = b.
__device__ __forceinline__ uint32_t cvt_bf16x2(float a, float b)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// Split 8 floats into NT bfloat16 terms (hi, mid, lo), each packed as 16 bytes:
// hi = rn(x), mid = rn(x - hi), lo = rn(x - hi - mid); both differences are exact.
template <int NT>
__device__ __forceinline__ void split8(const float *x, uint4 *t)
{
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float x0 = x[2 * q], x1 = x[2 * q + 1];
        const uint32_t h = cvt_bf16x2(x0, x1);
        w[0][q] = h;
        if (NT == 3) {
            const float r0 = x0 - __uint_as_float(h << 16), r1 = x1 - __uint_as_float(h & 0xffff0000u);
            const uint32_t m = cvt_bf16x2(r0, r1);
            const float s0 = r0 - __uint_as_float(m << 16), s1 = r1 - __uint_as_float(m & 0xffff0000u);
            w[1][q] = m;
            w[2][q] = cvt_bf16x2(s0, s1);
        }
    }
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
        t[tt] = make_uint4(w[tt][0], w[tt][1], w[tt][2], w[tt][3]);
}

// ------------------------------------------------------------------ kernel

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Named barrier `id` (immediate) over `nthreads` threads that also returns the OR of `v`
// over them.
#define LC_BAR_OR(ID)                                                                              \
    __device__ __forceinline__ bool bar_or_##ID(int nthreads, bool v)                              \
    {                                                                                              \
        uint32_t r;                                                                                \
        asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, " #ID          \
                     ", %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"                                            \
                     : "=r"(r)                                                                     \
                     : "r"((uint32_t)v), "r"(nthreads)                                             \
                     : "memory");                                                                  \
        return r != 0;                                                                             \
    }
LC_BAR_OR(1)
LC_BAR_OR(2)
LC_BAR_OR(3)
LC_BAR_OR(4)
LC_BAR_OR(5)
#undef LC_BAR_OR

__device__ __forceinline__ bool bar_or(int id, int nthreads, bool v)
{
    switch (id) {
    case 1: return bar_or_1(nthreads, v);
    case 2: return bar_or_2(nthreads, v);
    case 3: return bar_or_3(nthreads, v);
    case 4: return bar_or_4(nthreads, v);
    default: return bar_or_5(nthreads, v);
    }
}

// K-blocks per A buffer with their own full/empty barrier pair
static constexpr int kTcMaxKB = 16;

// Accumulator chunks (CW columns each) an epilogue warp loads before one wait: 32 registers
// of loaded values, half of them per region when the BF16X3 terms are stacked.
template <int NT, int CW>
struct EpiBatch {
    static constexpr int value = (NT == 3 ? 16 : 32) / CW;
};

template <int CW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t *r)
{
    if (CW == 16)
        tmem_ld16(taddr, r);
    else
        tmem_ld8(taddr, r);
}

// FG = 0: the contraction, one output per operator.  FG = F (2 or 3): the volume derivative
// with per-element geometric factors, out[d,e,i] = sum_f r[e,d,f] * (sum_j D[f,i,j] u[e,j]),
// every operator in the CTA's one column block; the epilogue mixes the F partial sums of a
// node with its element's F x F factors before the store.
//
// The body is shared by the plain launch (column block and tile share from the CTA index)
// and the grouped launch (each CTA one (group, column block) unit of a table): `blk` is the
// CTA's column block, its tiles are my_first, my_first + my_step, ... below a.ntiles.
template <int LAYOUT, int NT, int CW, int FG, bool ATM>
__device__ __forceinline__ void tc_body(const TcArgs &a, const int blk, const long long my_first,
                                        const long long my_step)
{
    constexpr bool NODE = LAYOUT == LC_LAYOUT_NODE_MAJOR;
    constexpr int TE = 128;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte aligned base for the swizzled operand tiles
    const uint32_t raw = smem_addr(smem_dyn);
    unsigned char *smem = smem_dyn + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sbase = smem_addr(smem);

    const int N = a.N, G = a.G, CBp = a.CBp, KB = a.KB, nkb = a.nkb;
    // The A terms in tensor memory are compiled into the BF16 instances and into separate
    // three-term instances (ATM): in the three-term instances for shared-memory A, the
    // warp-uniform conversion loops the tensor-memory stores need measured slower, and with
    // three terms the A reads from tensor memory are slower beside the epilogue's loads, so
    // those plans take them only where the shared-memory plan does not fit (large N).
    constexpr bool kATmem = ATM;
    const int Np = a.Np;  // accumulator columns per operator (N rounded up to 16)
    // K columns the MMAs read: N rounded up to the 16 of one instruction.  A K-block
    // wider than that keeps its last columns unread, so nothing writes them.
    const int Kn = a.Kt;
    // K columns that hold nodes (N rounded up to a chunk of 8, at most Kn): the conversion
    // writes these; the chunks beyond, up to Kn, stay zero from the set-up (A in shared memory)
    const int Kz8 = (kATmem && a.a_tmem) ? Kn : min(Kn, (N + 7) & ~7);
    const int W = 2 * KB;  // bytes per row of a K-block
    const long long E = a.E;
    const int S = a.stages, NA = a.abufs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int He = a.threads_per_row, Hc = a.conv_threads_per_row;  // threads per tile row per role
    const int NW = 4 * He, NC = 4 * Hc;  // epilogue warps 0..NW-1, conversion warps NW..NW+NC-1
    const int row = 32 * (warp & 3) + lane;  // tile row (== TMEM lane for epilogue warps)
    const int part = (warp < NW ? warp : warp - NW) >> 2;  // which share of the row's K chunks / columns
    const int f0 = blk * G;
    const int Gb = min(G, a.F - f0);  // operators in this block

    // B: per K-block, the NT terms of D^T stacked along rows (term t, column n -> row t*CBp + n)
    const uint32_t bkb = (uint32_t)NT * CBp * W;  // bytes per K-block of B
    const uint32_t offA = (uint32_t)nkb * bkb;
    const uint32_t termA = (uint32_t)nkb * TE * W;  // bytes per A term
    const uint32_t bufA = NT * termA;               // bytes per A buffer
    float *stage = reinterpret_cast<float *>(smem + a.off_stage);  // S x [TE*N] fp32
    float *ost0 = reinterpret_cast<float *>(smem + a.off_out);     // obufs x [4][32][N] slots (element-major)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + a.off_bar);
    uint64_t *u_full = bar, *u_empty = bar + 3, *acc_full = bar + 6, *acc_empty = bar + 8;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 10);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bar + 11);
    // A buffers are handed over per K-block: a_full/a_empty[ab * kTcMaxKB + kb]
    uint64_t *a_full = bar + 16, *a_empty = bar + 16 + 2 * kTcMaxKB;
    // element-major whole-tile staging slots handed between the epilogue and the store warp
    uint64_t *slot_full = bar + 16 + 4 * kTcMaxKB, *slot_empty = slot_full + 4;

    const int prod_warp = NW + NC, mma_warp = NW + NC + 1, store_warp = NW + NC + 2;
    if (warp == mma_warp)
        tmem_alloc(tmem_holder, (uint32_t)a.tmem_alloc);
    if (tid == 0) {
        for (int q = 0; q < 3; ++q) {
            mbar_init(&u_full[q], 1);
            mbar_init(&u_empty[q], NC);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], NW);
        }
        for (int q = 0; q < 2 * kTcMaxKB; ++q) {
            mbar_init(&a_full[q], NC);
            mbar_init(&a_empty[q], 1);
        }
        for (int q = 0; q < 4; ++q) {
            mbar_init(&slot_full[q], NW);
            mbar_init(&slot_empty[q], 1);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }

    // B terms: column n = f_local*Np + i of this block (i < N), K index = j; zero padding.
    {
        const int c8n = Kn / 8;
        for (int idx = tid; idx < CBp * c8n; idx += blockDim.x) {
            const int n = idx / c8n, c8 = idx - n * c8n;
            float x[8];
            const int fl = n / Np, i = n - fl * Np;
            const bool valid = fl < Gb && i < N;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = c8 * 8 + q;
                x[q] = (valid && j < N) ? a.D[((size_t)(f0 + fl) * N + i) * N + j] : 0.f;
            }
            uint4 t[3];
            split8<NT>(x, t);
            const int kb = (c8 * 8) / KB, ch = ((c8 * 8) % KB) / 8;
#pragma unroll
            for (int tt = 0; tt < NT; ++tt)
                *reinterpret_cast<uint4 *>(smem + (uint32_t)kb * bkb + swz_off(tt * CBp + n, ch, W)) = t[tt];
        }
        // A chunks past the last node (all zeros in every tile) are written once here; the
        // conversion warps skip them
        if (!(kATmem && a.a_tmem)) {
            const int zc = Kn / 8 - Kz8 / 8;  // zero chunks per row
            for (int idx = tid; idx < NA * NT * TE * zc; idx += blockDim.x) {
                int rest = idx;
                const int c8 = Kz8 / 8 + rest % zc;
                rest /= zc;
                const int rw = rest % TE;
                rest /= TE;
                const int tt = rest % NT, ab = rest / NT;
                const int kb = (c8 * 8) / KB, ch = ((c8 * 8) % KB) / 8;
                *reinterpret_cast<uint4 *>(smem + offA + (uint32_t)ab * bufA + (uint32_t)tt * termA +
                                           (uint32_t)kb * TE * W + swz_off(rw, ch, W)) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    // bulk-copy bytes of u tile t (0: not fetchable by the bulk engine, read from global)
    auto tile_bulk_bytes = [&](long long t) -> uint32_t {
        const int TEv = (int)min((long long)TE, E - t * TE);
        if (!a.bulk_u)
            return 0;
        const uint32_t bytes = (uint32_t)TEv * N * 4u;
        return (bytes & 15u) ? 0u : bytes;
    };
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.err, 1u);
    };

    if (warp == prod_warp) {
        // ---------------- producer: u tiles into the stage ring
        int k = 0;
        for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
            const int s = k % S;
            const uint32_t n = (uint32_t)(k / S);
            if (!mbar_wait(&u_empty[s], (n & 1u) ^ 1u)) {
                if (lane == 0)
                    fail();
                break;
            }
            const long long e0 = t * TE;
            const int TEv = (int)min((long long)TE, E - e0);
            const uint32_t bytes = tile_bulk_bytes(t);
            if (lane == 0)
                mbar_arrive_expect_tx(&u_full[s], bytes);
            __syncwarp();
            if (bytes) {
                float *dst = stage + (size_t)s * TE * N;
                if (NODE) {
                    for (int j = lane; j < N; j += 32)
                        bulk_g2s(dst + (size_t)j * TE, a.u + (size_t)j * E + e0, (uint32_t)TEv * 4u, &u_full[s]);
                } else if (lane == 0) {
                    bulk_g2s(dst, a.u + e0 * N, bytes, &u_full[s]);
                }
            }
            if (*abort_flag)
                break;
        }
    } else if (warp == mma_warp) {
        // ---------------- MMA issuer
        // BF16 and stacked BF16X3: K-blocks outermost; the MMAs of block kb (every product)
        // are followed by a commit that hands that block of the A buffer back to the
        // conversion warps, which refill it for a later tile while the remaining blocks are
        // multiplied.  Unstacked BF16X3: products outermost, small ones first over all of K
        // (the large hh sum is accumulated last); a block is handed back after its last
        // product.
        const uint32_t idesc = instr_desc(CBp), idesc2 = instr_desc(2 * CBp);
        // the K steps of block kb of one product: A term `at` times the B rows from `brow`,
        // into accumulator columns dcol.. (a descriptor advances by byte offset / 16)
        // A in tensor memory: term `at` of buffer ab starts at column ab * a_cols + at * Kn / 2,
        // 8 columns per K step
        const uint32_t a_tm0 = tmem_base + 2u * (uint32_t)a.tmem_cols;
        uint32_t a_tmb = a_tm0;  // the current tile's A buffer
        auto mma_block = [&](uint32_t dtm, uint64_t a0, uint64_t b0, int kb, int at, int brow, uint32_t id,
                             uint32_t dcol, uint32_t accumulate) {
            const int steps = min(KB, Kn - kb * KB) / 16;  // all-zero K steps skipped
            const uint64_t ad = a0 + ((uint32_t)(at * termA + kb * TE * W) >> 4);
            const uint64_t bd = b0 + ((uint32_t)(brow * W + kb * bkb) >> 4);
            const uint32_t at_tm = a_tmb + (uint32_t)(at * (Kn / 2) + kb * KB / 2);
            for (int ki = 0; ki < steps; ++ki) {
                if (kATmem && a.a_tmem)
                    tc_mma_ta(dtm + dcol, at_tm + 8u * ki, bd + 2 * ki, id, accumulate);
                else
                    tc_mma(dtm + dcol, ad + 2 * ki, bd + 2 * ki, id, accumulate);  // +32 bytes per K step
                accumulate = 1;
            }
        };
        const bool k_outer = NT == 1 || a.stack;
        int k = 0;
        for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
            const int b = k & 1, ab = k % NA;
            const uint32_t n = (uint32_t)(k >> 1), na = (uint32_t)(k / NA);
            bool ok = mbar_wait(&acc_empty[b], (n & 1u) ^ 1u);
            const uint32_t dtm = tmem_base + (uint32_t)b * a.tmem_cols;
            a_tmb = a_tm0 + (uint32_t)(ab * a.a_cols);
            const uint64_t a0 = smem_desc(sbase + offA + (uint32_t)ab * bufA, W);
            const uint64_t b0 = smem_desc(sbase, W);
            const int npass = k_outer ? 1 : 6;
            for (int p = 0; p < npass && ok; ++p) {
                for (int kb = 0; kb < nkb; ++kb) {
                    if (p == 0) {
                        ok = mbar_wait(&a_full[ab * kTcMaxKB + kb], na & 1u);
                        if (!ok)
                            break;
                        tc_fence_after();
                    }
                    if (lane == 0) {
                        const uint32_t acc = kb > 0;  // block 0 of a region's first product overwrites
                        if (NT == 1) {
                            mma_block(dtm, a0, b0, kb, 0, 0, idesc, 0, acc);
                        } else if (a.stack) {
                            // regions R0 = columns [0, CBp) and R1 = [CBp, 2 CBp), summed by the
                            // epilogue: u_hi x [D_hi; D_mid] puts hh in R0 and hm in R1; the
                            // smaller products lh, hl, mm, mh all go to R1, so the large R0 sum
                            // takes one rounding per K step, as a plain FP32 dot product would
                            mma_block(dtm, a0, b0, kb, 0, 0, idesc2, 0, acc);
                            mma_block(dtm, a0, b0, kb, 2, 0, idesc, (uint32_t)CBp, 1);
                            mma_block(dtm, a0, b0, kb, 0, 2 * CBp, idesc, (uint32_t)CBp, 1);
                            mma_block(dtm, a0, b0, kb, 1, CBp, idesc, (uint32_t)CBp, 1);
                            mma_block(dtm, a0, b0, kb, 1, 0, idesc, (uint32_t)CBp, 1);
                        } else {
                            // (D term, u term) of pass p: lh, hl, mm, mh, hm, hh
                            const int bt = p == 0 ? 2 : (p == 2 || p == 3) ? 1 : 0;
                            const int at = p == 1 ? 2 : (p == 2 || p == 4) ? 1 : 0;
                            mma_block(dtm, a0, b0, kb, at, bt * CBp, idesc, 0, p == 0 ? acc : 1u);
                        }
                        if (p == npass - 1)
                            tc_commit(&a_empty[ab * kTcMaxKB + kb]);
                    }
                    __syncwarp();
                }
            }
            if (!ok) {
                if (lane == 0)
                    fail();
                break;
            }
            if (lane == 0)
                tc_commit(&acc_full[b]);
            __syncwarp();
            if (*abort_flag)
                break;
        }
    } else if (warp == store_warp) {
        // ---------------- store warp: element-major whole-tile slots -> out.  Once every
        // epilogue warp has staged tile k into slot k % R, one lane issues the bulk stores of
        // the block's operators, waits until they have read the slot and hands it back, so
        // the epilogue warps never wait on the bulk-copy engine themselves.
        if (!NODE && a.store_quarters == 4) {
            const int R = a.obufs;
            int k = 0;
            bool ok = true;
            for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
                const int s = k % R;
                if (!mbar_wait(&slot_full[s], (uint32_t)(k / R) & 1u)) {
                    ok = false;
                    break;
                }
                const long long e0 = t * TE;
                const int total = (int)min((long long)TE, E - e0) * N;
                const float *ost = ost0 + (size_t)s * G * TE * N;
                if (a.bulk_store && ((total * 4) & 15) == 0) {
                    if (lane == 0) {
                        for (int g = 0; g < Gb; ++g)
                            bulk_s2g(a.out + ((size_t)(f0 + g) * E + e0) * N, ost + (size_t)g * TE * N,
                                     (uint32_t)total * 4u);
                        bulk_commit();
                        bulk_wait_read0();
                    }
                } else {
                    // unaligned tail: plain copy
                    for (int g = 0; g < Gb; ++g) {
                        const float *src = ost + (size_t)g * TE * N;
                        float *dst = a.out + ((size_t)(f0 + g) * E + e0) * N;
                        for (int idx = lane; idx < total; idx += 32)
                            dst[idx] = src[idx];
                    }
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&slot_empty[s]);
                if (*abort_flag)
                    break;
            }
            if (lane == 0)
                bulk_wait0();
            if (!ok && lane == 0)
                fail();
        }
    } else if (warp >= NW) {
        // ---------------- conversion warps: fp32 u tile -> bf16 A-operand terms, K-block by K-block
        // A thread converts K chunks c8 (8 values of j) of its tile row: within K-block kb the
        // chunks c8_lo + part, c8_lo + part + Hc, ...  The A terms go to shared memory (hardware
        // swizzle) or to tensor memory (tcgen05.st into this warp's lane quarter, warp-uniform
        // loops; rows past the tile and nodes past N are zeros).
        // Early release (descriptor prefetch_smem = 2): when K is one block and a thread has at
        // most kMaxEarly chunks, it loads them, splits them into their terms in registers and
        // hands the u stage back to the producer at once, so the next tile's bulk copy overlaps
        // this tile's conversion and MMAs, and only the stores of the terms wait for the A
        // buffer (threads with more chunks take the plain path).
        // chunks a thread may hold: three (BF16, one term each) or two (three terms each)
        constexpr int kMaxEarly = NT == 1 ? 3 : 2;
        int k = 0;
        bool ok = true;
        const int nch8 = Kz8 / 8;
        const int my_chunks = (nkb == 1 && a.early_release) ? (nch8 - part + Hc - 1) / Hc : kMaxEarly + 1;
        const uint32_t lane_q = (uint32_t)(32 * (warp & 3)) << 16;
        for (long long t = my_first; t < a.ntiles && ok; t += my_step, ++k) {
            const int s = k % S, ab = k % NA;
            const uint32_t ns = (uint32_t)(k / S), na = (uint32_t)(k / NA);
            if (!mbar_wait(&u_full[s], ns & 1u)) {
                ok = false;
                break;
            }
            const long long e0 = t * TE;
            const int TEv = (int)min((long long)TE, E - e0);
            const bool from_stage = tile_bulk_bytes(t) != 0;
            const float *st = stage + (size_t)s * TE * N;
            unsigned char *Ab = smem + offA + (size_t)ab * bufA;
            const bool rowv = row < TEv;
            constexpr int JS = NODE ? TE : 1;
            const float *src_s = NODE ? st + row : st + row * N;
            const float *src_g = NODE ? a.u + e0 + row : a.u + (e0 + row) * N;
            const long long jsg = NODE ? E : 1;
            const uint32_t abase = tmem_base + 2u * (uint32_t)a.tmem_cols + (uint32_t)(ab * a.a_cols) + lane_q;
            // the 8 values of chunk c8 of this thread's row (zeros past the row or past N)
            auto load_chunk = [&](int c8, float *x) {
                if (from_stage && c8 * 8 + 8 <= N) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        x[q] = rowv ? src_s[(c8 * 8 + q) * JS] : 0.f;
                } else if (from_stage) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        x[q] = (rowv && c8 * 8 + q < N) ? src_s[(c8 * 8 + q) * JS] : 0.f;
                } else {
                    // unaligned tail tile, read from global memory
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        x[q] = (rowv && c8 * 8 + q < N) ? src_g[(long long)(c8 * 8 + q) * jsg] : 0.f;
                }
            };
            // chunk c8 -> the A terms
            // the NT terms of chunk c8 -> the A buffer
            auto put_terms = [&](int c8, const uint4 *tt4) {
                if (kATmem && a.a_tmem) {
#pragma unroll
                    for (int tt = 0; tt < NT; ++tt)
                        tmem_st4(abase + (uint32_t)(tt * (Kn / 2) + c8 * 4), tt4[tt]);
                } else {
                    const int kb = (c8 * 8) / KB, ch = ((c8 * 8) % KB) / 8;
                    const uint32_t off = (uint32_t)kb * TE * W + swz_off(row, ch, W);
#pragma unroll
                    for (int tt = 0; tt < NT; ++tt)
                        *reinterpret_cast<uint4 *>(Ab + off + tt * termA) = tt4[tt];
                }
            };
            auto put = [&](int c8, const float *x) {
                uint4 tt4[3];
                split8<NT>(x, tt4);
                put_terms(c8, tt4);
            };
            // block kb written: make it visible to the tensor core and hand it to the MMA warp
            auto block_done = [&](int kb) {
                if (kATmem && a.a_tmem) {
                    tmem_wait_st();
                    tc_fence_before();
                } else {
                    fence_async_smem();
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&a_full[ab * kTcMaxKB + kb]);
            };
            bool released = false;
            if (from_stage && my_chunks <= kMaxEarly) {
                // the chunks are split into their terms before the A buffer is free, so that
                // only the stores of the terms wait for the MMAs of the previous tile
                uint4 tv[kMaxEarly][3];
#pragma unroll
                for (int m = 0; m < kMaxEarly; ++m) {
                    const int c8 = part + Hc * m;
                    float x[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        x[q] = (m < my_chunks && rowv && c8 * 8 + q < N) ? src_s[(c8 * 8 + q) * JS] : 0.f;
                    split8<NT>(x, tv[m]);
                }
                // the loads are complete before the stage is handed back (no load may be
                // deferred past the arrive to the point where the values are used)
                __threadfence_block();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&u_empty[s]);  // the stage is free for the next bulk copy
                released = true;
                if (!mbar_wait(&a_empty[ab * kTcMaxKB], (na & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int m = 0; m < kMaxEarly; ++m)
                    if (m < my_chunks)
                        put_terms(part + Hc * m, tv[m]);
                block_done(0);
            } else {
                const int full8 = rowv ? N / 8 : 0;  // chunks with all 8 values inside the row
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&a_empty[ab * kTcMaxKB + kb], (na & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int c8_lo = kb * KB / 8, c8_hi = min(Kz8, (kb + 1) * KB) / 8;
                    if (kATmem && a.a_tmem) {
                        // tcgen05.st is warp-collective: every lane runs the same chunks (the
                        // trip count depends on the warp's share only), rows past the tile are
                        // zeros by predicated loads
                        for (int c8 = c8_lo + part; c8 < c8_hi; c8 += Hc) {
                            float x[8];
                            load_chunk(c8, x);
                            put(c8, x);
                        }
                    } else if (from_stage) {
                        // staged tile: compile-time stride along j; two whole chunks in flight, then
                        // the chunks cut by N or past the tile (zeros) one by one
                        const int f_hi = min(full8, c8_hi);
                        int c8 = c8_lo + part;
                        for (; c8 + Hc < f_hi; c8 += 2 * Hc) {
                            float x[8], y[8];
                            const float *p0 = src_s + c8 * 8 * JS, *p1 = src_s + (c8 + Hc) * 8 * JS;
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                x[q] = p0[q * JS];
                                y[q] = p1[q * JS];
                            }
                            put(c8, x);
                            put(c8 + Hc, y);
                        }
                        for (; c8 < c8_hi; c8 += Hc) {
                            float x[8];
                            const float *p0 = src_s + c8 * 8 * JS;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                x[q] = (rowv && c8 * 8 + q < N) ? p0[q * JS] : 0.f;
                            put(c8, x);
                        }
                    } else {
                        for (int c8 = c8_lo + part; c8 < c8_hi; c8 += Hc) {
                            float x[8];
                            load_chunk(c8, x);
                            put(c8, x);
                        }
                    }
                    block_done(kb);
                }
            }
            if (!ok)
                break;
            if (!released) {
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&u_empty[s]);  // every block of this tile has been read from the stage
            }
            if (*abort_flag)
                break;
        }
        if (!ok && lane == 0)
            fail();
    } else {
        // ---------------- epilogue warps: TMEM accumulators -> out
        // Warp w reads TMEM lane quarter q = w % 4 (tile rows 32q..32q+31); the He warps of a
        // quarter split the CW-column chunks of the accumulator (with stacked BF16X3 terms a
        // chunk is the sum of regions R0 and R1).
        //   node-major        stores straight from registers, coalesced along e;
        //   element-major     staged in shared memory, then bulk stores of contiguous rows:
        //     store_quarters = 4   all epilogue warps stage every operator of the tile into
        //                          one of R slots, then one thread issues G stores;
        //     store_quarters < 4   a store group of SQ quarters stages one operator at a time
        //                          into its own ring of R slots and stores 32 SQ rows of it,
        //                          with no CTA-wide barrier.
        const int q = warp & 3;
        const int R = a.obufs;
        const int SQ = NODE ? 4 : a.store_quarters;
        const int NWT = NW * 32;
        const bool stack = NT == 3 && a.stack;
        // Load, sum and store the chunks of columns [c_begin, c_end) of this warp's lane
        // quarter; element-major values go to stage + ((operator - f_stage) * TE + row) * N.
        // operators packed without padding (Np = N, N not a multiple of the chunk): a chunk of
        // columns c = f N + i may run into the next operator
        const bool packed = Np == N && N % CW != 0;
        auto drain = [&](int c_begin, int c_end, const uint32_t tbase, float *stage, int f_stage, long long e0,
                         int TEv) {
            constexpr int EB = EpiBatch<NT, CW>::value;
            for (int c0 = c_begin + part * CW; c0 < c_end; c0 += EB * CW * He) {
                uint32_t r[EB][CW], r2[EB][CW];
#pragma unroll
                for (int k4 = 0; k4 < EB; ++k4)
                    if (c0 + k4 * CW * He < c_end) {
                        tmem_ld<CW>(tbase + (uint32_t)(c0 + k4 * CW * He), r[k4]);
                        if (stack)
                            tmem_ld<CW>(tbase + (uint32_t)(CBp + c0 + k4 * CW * He), r2[k4]);
                    }
                tmem_wait();
#pragma unroll
                for (int k4 = 0; k4 < EB; ++k4) {
                    const int cc = c0 + k4 * CW * He;
                    if (cc >= c_end)
                        continue;
                    const int fl = cc / Np, i0 = cc - fl * Np;
                    const int nv = min(CW, N - i0);  // valid columns of this chunk (>= 1)
                    if (stack) {
#pragma unroll
                        for (int qq = 0; qq < CW; ++qq)
                            r[k4][qq] = __float_as_uint(__uint_as_float(r[k4][qq]) + __uint_as_float(r2[k4][qq]));
                    }
                    if (packed) {
                        if (NODE) {
                            if (row < TEv) {
                                float *o = a.out + ((size_t)f0 * N + cc) * E + e0 + row;  // (f0 + f) N + i = f0 N + c
#pragma unroll
                                for (int qq = 0; qq < CW; ++qq) {
                                    if (cc + qq < c_end)
                                        *o = __uint_as_float(r[k4][qq]);
                                    o += E;
                                }
                            }
                        } else {
                            // (f, row, i) at (f TE + row) N + i: past the operator's last node the
                            // next operator's row starts (TE - 1) N further on
                            float *o = stage + ((fl - f_stage) * TE + row) * N + i0;
                            const int jump = (TE - 1) * N, rest = N - i0;
                            if (rest >= CW && cc + CW <= c_end) {
#pragma unroll
                                for (int qq = 0; qq < CW; ++qq)  // the chunk inside one operator
                                    o[qq] = __uint_as_float(r[k4][qq]);
                            } else {
#pragma unroll
                                for (int qq = 0; qq < CW; ++qq)
                                    if (cc + qq < c_end)
                                        o[qq + (qq >= rest ? jump : 0)] = __uint_as_float(r[k4][qq]);
                            }
                        }
                        continue;
                    }
                    if (NODE) {
                        if (row < TEv) {
                            float *o = a.out + ((size_t)(f0 + fl) * N + i0) * E + e0 + row;
#pragma unroll
                            for (int qq = 0; qq < CW; ++qq) {
                                if (qq < nv)
                                    *o = __uint_as_float(r[k4][qq]);
                                o += E;
                            }
                        }
                    } else {
                        float *o = stage + ((fl - f_stage) * TE + row) * N + i0;
                        if ((N & 3) == 0) {
                            // 16-byte aligned rows: vector stores (nv is a multiple of 4)
#pragma unroll
                            for (int h = 0; h < CW / 4; ++h)
                                if (4 * h < nv)
                                    *reinterpret_cast<uint4 *>(o + 4 * h) =
                                        make_uint4(r[k4][4 * h], r[k4][4 * h + 1], r[k4][4 * h + 2], r[k4][4 * h + 3]);
                        } else if (nv == CW) {
#pragma unroll
                            for (int qq = 0; qq < CW; ++qq)
                                o[qq] = __uint_as_float(r[k4][qq]);
                        } else {
#pragma unroll
                            for (int qq = 0; qq < CW; ++qq)
                                if (qq < nv)
                                    o[qq] = __uint_as_float(r[k4][qq]);
                        }
                    }
                }
            }
        };
        // Geometric factors of this thread's element (row) for the current tile: rr[d][f].
        constexpr int FGm = FG > 0 ? FG : 1;
        float rr[FGm][FGm];
        auto load_r = [&](long long e0, int TEv) {
#pragma unroll
            for (int d = 0; d < FGm; ++d)
#pragma unroll
                for (int f = 0; f < FGm; ++f) {
                    const long long e = e0 + row;
                    rr[d][f] = row >= TEv ? 0.f
                                          : (NODE ? a.r[((long long)d * FGm + f) * E + e]
                                                  : a.r[(e * FGm + d) * FGm + f]);
                }
        };
        // Volume derivative epilogue: per chunk of CW nodes, the F partial sums (both regions
        // added when the terms are stacked), then out[d] = sum_f rr[d][f] * partial[f] in FP32,
        // f ascending; element-major into the staging slot [d][TE][N], node-major to global.
        auto drain_geo = [&](const uint32_t tbase, float *stage, long long e0, int TEv) {
            for (int c0 = part * CW; c0 < N; c0 += CW * He) {
                float acc[FGm][CW];
#pragma unroll
                for (int f = 0; f < FGm; ++f) {
                    uint32_t r0[CW], r1[CW];
                    tmem_ld<CW>(tbase + (uint32_t)(f * Np + c0), r0);
                    if (stack)
                        tmem_ld<CW>(tbase + (uint32_t)(CBp + f * Np + c0), r1);
                    tmem_wait();
#pragma unroll
                    for (int qq = 0; qq < CW; ++qq)
                        acc[f][qq] = stack ? __uint_as_float(r0[qq]) + __uint_as_float(r1[qq]) : __uint_as_float(r0[qq]);
                }
                const int nv = min(CW, N - c0);
#pragma unroll
                for (int d = 0; d < FGm; ++d) {
                    float o[CW];
#pragma unroll
                    for (int qq = 0; qq < CW; ++qq) {
                        float v = rr[d][0] * acc[0][qq];
#pragma unroll
                        for (int f = 1; f < FGm; ++f)
                            v = fmaf(rr[d][f], acc[f][qq], v);
                        o[qq] = v;
                    }
                    if (NODE) {
                        if (row < TEv) {
                            float *op = a.out + ((size_t)d * N + c0) * E + e0 + row;
#pragma unroll
                            for (int qq = 0; qq < CW; ++qq) {
                                if (qq < nv)
                                    *op = o[qq];
                                op += E;
                            }
                        }
                    } else {
                        float *op = stage + ((size_t)d * TE + row) * N + c0;
#pragma unroll
                        for (int qq = 0; qq < CW; ++qq)
                            if (qq < nv)
                                op[qq] = o[qq];
                    }
                }
            }
        };
        auto release_acc = [&](int b) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&acc_empty[b]);
        };
        int k = 0;
        bool ok = true;
        if (SQ == 4) {
            // ---- node-major, or element-major with whole-tile slots
            for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
                const int b = k & 1;
                const long long e0 = t * TE;
                const int TEv = (int)min((long long)TE, E - e0);
                const bool got = mbar_wait(&acc_full[b], (uint32_t)((k >> 1) & 1));
                float *ost = ost0 + (size_t)(k % R) * G * TE * N;
                // every warp goes its own way (no named barrier; every wait is bounded)
                if (!got || *abort_flag) {
                    ok = got;
                    break;
                }
                // element-major: the store warp has finished reading this slot
                if (!NODE && !mbar_wait(&slot_empty[k % R], ((uint32_t)(k / R) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem_base + (uint32_t)b * a.tmem_cols + ((uint32_t)(q * 32) << 16);
                if (FG > 0) {
                    load_r(e0, TEv);
                    drain_geo(tbase, ost, e0, TEv);
                } else {
                    drain(0, Gb * Np, tbase, ost, 0, e0, TEv);
                }
                release_acc(b);
                if (!NODE) {
                    // this warp's staged values, ordered before the store warp's bulk copies
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(&slot_full[k % R]);
                }
            }
        } else {
            // ---- element-major, one operator per slot, store groups of SQ quarters
            const int gq = q / SQ, qin = q % SQ;  // store group, quarter within it
            const int gthreads = 32 * He * SQ;
            const bool leader = part == 0 && lane == 0 && qin == 0;  // issues and waits on the group's stores
            // named barrier 2 + gq (immediate operands)
            auto group_sync = [&]() {
                switch (gq) {
                case 0: asm volatile("bar.sync 2, %0;" ::"r"(gthreads) : "memory"); break;
                case 1: asm volatile("bar.sync 3, %0;" ::"r"(gthreads) : "memory"); break;
                case 2: asm volatile("bar.sync 4, %0;" ::"r"(gthreads) : "memory"); break;
                default: asm volatile("bar.sync 5, %0;" ::"r"(gthreads) : "memory"); break;
                }
            };
            const int r0 = 32 * SQ * gq;  // first tile row of this store group
            int ns = 0;                   // slots used by this store group
            for (long long t = my_first; t < a.ntiles; t += my_step, ++k) {
                const int b = k & 1;
                const long long e0 = t * TE;
                const int TEv = (int)min((long long)TE, E - e0);
                const int rows_g = max(0, min(32 * SQ, TEv - r0));  // valid rows of this store group
                const bool got = mbar_wait(&acc_full[b], (uint32_t)((k >> 1) & 1));
                const uint32_t tbase = tmem_base + (uint32_t)b * a.tmem_cols + ((uint32_t)(q * 32) << 16);
                bool stop = false;
                for (int g = 0; g < Gb; ++g) {
                    float *slot = ost0 + (size_t)(ns % R) * TE * N;  // [TE][N], this group's rows r0..
                    ++ns;
                    if (leader)
                        bulk_wait_read(R - 1);  // the store that last read this slot is done reading
                    if (g > 0) {
                        group_sync();
                    } else {
                        // the warps of a store group leave together (they meet at named barriers)
                        if (bar_or(2 + gq, gthreads, !got || *abort_flag)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                    }
                    drain(g * Np, (g + 1) * Np, tbase, slot, g, e0, TEv);
                    if (g == Gb - 1)
                        release_acc(b);
                    fence_async_smem();
                    group_sync();
                    const uint32_t bytes = (uint32_t)rows_g * N * 4u;
                    float *dst = a.out + ((size_t)(f0 + g) * E + e0 + r0) * N;
                    const float *src = slot + (size_t)r0 * N;
                    if (a.bulk_store && (bytes & 15u) == 0) {
                        if (leader && bytes) {
                            bulk_s2g(dst, src, bytes);
                            bulk_commit();
                        }
                    } else {
                        // unaligned tail: plain copy; the next barrier on this slot orders reuse
                        for (int idx = (qin * He + part) * 32 + lane; idx < rows_g * N; idx += gthreads)
                            dst[idx] = src[idx];
                    }
                }
                if (stop) {
                    ok = got;
                    break;
                }
            }
            if (leader)
                bulk_wait0();
        }
        if (!ok && lane == 0)
            fail();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == mma_warp)
        tmem_dealloc(tmem_base, (uint32_t)a.tmem_alloc);
}

template <int LAYOUT, int NT, int CW, int FG, bool ATM = (NT == 1)>
__global__ void __launch_bounds__(864, 1) tc_contract_kernel(const __grid_constant__ TcArgs a)
{
    tc_body<LAYOUT, NT, CW, FG, ATM>(a, (int)(blockIdx.x % a.nblocks), blockIdx.x / a.nblocks,
                                     gridDim.x / a.nblocks);
}

// Grouped launch: CTA b runs unit P.map[b] = {group, column block, first tile, tile step} of
// the group's own plan P.g[group] (one unit per CTA, no group switching inside a CTA).
template <int LAYOUT, int NT, bool ATM = (NT == 1)>
__global__ void __launch_bounds__(864, 1) tc_grouped_kernel(const __grid_constant__ TcGroupedParams P)
{
    const int4 m = P.map[blockIdx.x];
    tc_body<LAYOUT, NT, 8, 0, ATM>(P.g[m.x], m.y, m.z, m.w);
}

// Set the shared-memory size of one kernel instance and launch it.
static inline lc_status tc_launch_fn(void *fn, const TcArgs &a, int grid, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem_bytes);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (grid <= 0)
        return LC_OK;  // attribute set only (a capture launches later)
    TcArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(tc_threads(a)), params,
                         a.smem_bytes, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

}  // namespace lc
