// Surface part of the dG operator (the dG FEM surface workload of Table 1):
//
//     out[e,i] (+)= sum_{f,p} L[i,f,p] * s[e,f] * ( u[e, fmask[f,p]] - u_flat[vmapP[e,f,p]] )
//
// the jumps between each face node's interior trace and the exterior trace gathered through
// the face-node map vmapP, scaled per face and lifted to the volume nodes.  FP32 throughout
// (the contraction has K = Nf * Nfp and about 5 flops per byte moved: the FMA pipes are not
// the limit, so the tensor cores would buy nothing here).
//
// One CTA walks element tiles of TE elements (persistent, grid-stride):
//   stage    (add_prefetch, descriptor prefetch_smem = 1) the bulk-copy engine fetches, one
//            or two tiles ahead of the compute (descriptor stages: staging buffers), the
//            tile's vmapP rows, its face scales and a u window: the rows of the tile and of
//            `halo` elements on either side, one
//            contiguous run.  Exterior traces inside the window (on a structured mesh, all
//            of them) are read from shared memory, the others from global memory;
//            (prefetch_smem = 0: every operand is read from global memory)
//   gather   the tile's fluxes flux[m][t] = s[e, m / Nfp] * (u[e, fmask[m]] - u[vmapP[e, m]]),
//            m-fastest, several items per thread in flight, written transposed into shared
//            memory (padded rows per m);
//   lift     each thread accumulates a RE x 4 register block (elements x nodes) over m with
//            L^T (resident in shared memory for the CTA's lifetime), m ascending;
//   store    out rows, adding to the previous values when accumulating.
#include <cuda_runtime.h>

#include <algorithm>

#include "lc_internal.h"
#include "tma.cuh"

namespace lc {

// elements per tile: 64 or 128 (descriptor tile_e), a template parameter of the kernel
static constexpr int kLiftRE = 4;      // elements per thread
static constexpr int kLiftRC = 4;      // nodes per thread
static constexpr int kLiftPad = 4;     // padding of a flux row: 16-byte rows (one vector load of a thread's
                                       // four elements), transposed writes at most 4-way bank conflicts
static constexpr int kLiftG = 4;       // gathered items per thread in flight

__host__ __device__ inline size_t lift_r4(size_t n) { return (n + 3) & ~(size_t)3; }

// Shared memory: L^T [M][NP], the flux tile [M][TP], {node, face} per face node, two
// mbarriers, then (staged) nbuf buffers of {u window, vmapP tile, scale tile}, 16-byte
// aligned.
struct LiftSmem {
    size_t flux, fmf, bars, buf, buf_bytes, win, vm, sc, total;
};
__host__ __device__ inline LiftSmem lift_smem(int N, int M, int Nf, int halo, int nbuf, int TE)
{
    LiftSmem L;
    const size_t NP = (size_t)(N + kLiftRC - 1) / kLiftRC * kLiftRC, TP = TE + kLiftPad;
    L.flux = sizeof(float) * (size_t)M * NP;
    L.fmf = L.flux + sizeof(float) * (size_t)M * TP;
    L.bars = L.fmf + sizeof(int2) * (size_t)M;
    L.buf = (L.bars + 2 * sizeof(uint64_t) + 15) & ~(size_t)15;
    L.win = 0;
    L.vm = halo < 0 ? 0 : sizeof(float) * lift_r4((size_t)(TE + 2 * halo) * N);
    L.sc = L.vm + sizeof(int) * lift_r4((size_t)TE * M);
    L.buf_bytes = halo < 0 ? 0 : L.sc + sizeof(float) * lift_r4((size_t)TE * Nf);
    L.total = L.buf + (size_t)nbuf * L.buf_bytes;
    return L;
}

template <bool STAGED, int TE>
__global__ void __launch_bounds__(512) lift_kernel(LiftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(kLiftRE == 4 && kLiftRC == 4, "the inner loop reads four elements and four nodes");
    const int N = a.N, M = a.M, Nfp = a.Nfp, Nf = a.Nf;
    const int CG = (N + kLiftRC - 1) / kLiftRC;  // column groups
    const int NP = CG * kLiftRC;                 // padded node count
    const int TP = TE + kLiftPad;                // flux row stride
    const int H = STAGED ? a.halo : 0;
    const int NB = STAGED ? a.nbuf : 1;  // staging buffers (1 or 2)
    const LiftSmem lay = lift_smem(N, M, Nf, STAGED ? H : -1, NB, TE);
    float *LT = reinterpret_cast<float *>(smem_raw);  // [M][NP]
    float *flux = reinterpret_cast<float *>(smem_raw + lay.flux);  // [M][TP]
    int2 *fmf = reinterpret_cast<int2 *>(smem_raw + lay.fmf);      // [M] {node, face}
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + lay.bars);
    const long long E = a.E;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < M * NP; idx += nthr) {
        const int m = idx / NP, i = idx - m * NP;
        LT[idx] = i < N ? a.L[(size_t)i * M + m] : 0.f;
    }
    for (int m = tid; m < M; m += nthr) {
        const int j = a.fmask[m];
        const bool bad = j < 0 || j >= N;
        fmf[m] = make_int2(bad ? 0 : j, m / Nfp);  // out of range: recorded, node 0 read instead
        if (bad)
            atomicOr(a.err, 2u);
    }
    const long long ntiles = (E + TE - 1) / TE;
    // bulk parts (16-byte multiples) of tile t's three runs; the rest is read by plain loads
    auto runs = [&](long long t, long long &lo, int &wn, int &vn, int &sn) {
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);
        lo = max(0LL, e0 - H);
        const long long hi = min(E, e0 + TE + H);
        wn = (int)((hi - lo) * N);
        vn = TEv * M;
        sn = TEv * Nf;
    };
    auto issue = [&](long long t, int b) {
        long long lo;
        int wn, vn, sn;
        runs(t, lo, wn, vn, sn);
        unsigned char *buf = smem_raw + lay.buf + (size_t)b * lay.buf_bytes;
        const uint32_t wb = (uint32_t)(wn * 4) & ~15u, vb = (uint32_t)(vn * 4) & ~15u, sb = (uint32_t)(sn * 4) & ~15u;
        mbar_arrive_expect_tx(&bars[b], wb + vb + sb);
        const long long e0 = t * TE;
        if (wb)
            bulk_g2s(buf + lay.win, a.u + lo * N, wb, &bars[b]);
        if (vb)
            bulk_g2s(buf + lay.vm, a.vmapP + e0 * M, vb, &bars[b]);
        if (sb)
            bulk_g2s(buf + lay.sc, a.s + e0 * Nf, sb, &bars[b]);
    };
    if (STAGED && tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (STAGED && tid == 0) {
        for (int b = 0; b < NB; ++b)
            if (blockIdx.x + (long long)b * gridDim.x < ntiles)
                issue(blockIdx.x + (long long)b * gridDim.x, b);
    }
    const int EN = (int)(E * N);  // E * N < 2^31 (checked by the host): flat u indices are ints
    // the gather walks idx = te * M + m = tid, tid + nthr, ...: one step adds dte to te and
    // dm (< M) to m, with a carry
    const int dte = nthr / M, dm = nthr - dte * M;
    const int te_first = tid / M, m_first = tid - te_first * M;
    // register block of this thread: elements eg*RE.., nodes cg*RC..
    const int cg = tid % CG, eg = tid / CG;
    const bool active = eg < TE / kLiftRE;
    int k = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const long long e0 = t * TE;
        const int TEv = (int)min((long long)TE, E - e0);
        const int b = NB == 2 ? (k & 1) : 0;
        const uint32_t ph = (uint32_t)((NB == 2 ? k >> 1 : k) & 1);
        long long lo = 0;
        int wn = 0, vn = 0, sn = 0;
        const float *win = nullptr, *scb = nullptr;
        const int *vm = nullptr;
        if (STAGED) {
            runs(t, lo, wn, vn, sn);
            unsigned char *buf = smem_raw + lay.buf + (size_t)b * lay.buf_bytes;
            const bool ok = mbar_wait(&bars[b], ph);
            if (!__syncthreads_and(ok)) {
                if (tid == 0)
                    atomicOr(a.err, 1u);
                break;
            }
            float *w = reinterpret_cast<float *>(buf + lay.win);
            int *v = reinterpret_cast<int *>(buf + lay.vm);
            float *c = reinterpret_cast<float *>(buf + lay.sc);
            // the parts past the last 16-byte multiple of each run
            for (int q = ((wn * 4) & ~15) / 4 + tid; q < wn; q += nthr)
                w[q] = a.u[lo * N + q];
            for (int q = ((vn * 4) & ~15) / 4 + tid; q < vn; q += nthr)
                v[q] = a.vmapP[e0 * M + q];
            for (int q = ((sn * 4) & ~15) / 4 + tid; q < sn; q += nthr)
                c[q] = a.s[e0 * Nf + q];
            __syncthreads();
            win = w;
            vm = v;
            scb = c;
        }
        const int wb = (int)(lo * N);                 // flat u index of the window's first value
        const int ib = (int)(e0 - lo) * N;            // window index of the tile's first row
        // gather the tile's fluxes, kLiftG items per thread in flight: all index loads first,
        // then all trace loads, then the fluxes
        int te_c = te_first, m_c = m_first;
        while (te_c < TE) {
            int te[kLiftG], m[kLiftG], q[kLiftG];
            float ui[kLiftG], ux[kLiftG], sc[kLiftG];
#pragma unroll
            for (int g = 0; g < kLiftG; ++g) {
                te[g] = te_c;
                m[g] = m_c;
                te_c += dte;
                m_c += dm;
                if (m_c >= M) {
                    m_c -= M;
                    ++te_c;
                }
                const bool live = te[g] < TEv;
                q[g] = live ? (STAGED ? vm[te[g] * M + m[g]] : a.vmapP[(e0 + te[g]) * M + m[g]]) : 0;
            }
#pragma unroll
            for (int g = 0; g < kLiftG; ++g) {
                const bool live = te[g] < TEv;
                const bool in = live && (unsigned)q[g] < (unsigned)EN;
                const int2 nf = fmf[live ? m[g] : 0];
                if (STAGED) {
                    const int qw = q[g] - wb;  // position in the window
                    ux[g] = in ? ((unsigned)qw < (unsigned)wn ? win[qw] : a.u[q[g]]) : 0.f;
                    ui[g] = live ? win[ib + te[g] * N + nf.x] : 0.f;  // the tile lies in the window
                    sc[g] = live ? scb[te[g] * Nf + nf.y] : 0.f;
                } else {
                    ux[g] = in ? a.u[q[g]] : 0.f;
                    ui[g] = live ? a.u[(e0 + te[g]) * N + nf.x] : 0.f;
                    sc[g] = live ? a.s[(e0 + te[g]) * Nf + nf.y] : 0.f;
                }
            }
#pragma unroll
            for (int g = 0; g < kLiftG; ++g) {
                if (te[g] >= TE)
                    break;
                float v = 0.f;
                if (te[g] < TEv) {
                    if ((unsigned)q[g] < (unsigned)EN) {
                        v = __fmul_rn(sc[g], __fsub_rn(ui[g], ux[g]));
                    } else {
                        v = __int_as_float(0x7fc00000);  // out-of-range index: NaN, recorded
                        atomicOr(a.err, 2u);
                    }
                }
                flux[(size_t)m[g] * TP + te[g]] = v;
            }
        }
        fence_async_smem();
        __syncthreads();
        if (STAGED && tid == 0) {
            // buffer b is consumed: fetch the tile NB steps ahead into it
            const long long nt = t + (long long)NB * gridDim.x;
            if (nt < ntiles)
                issue(nt, b);
        }
        if (active) {
            float acc[kLiftRE][kLiftRC];
#pragma unroll
            for (int x = 0; x < kLiftRE; ++x)
#pragma unroll
                for (int y = 0; y < kLiftRC; ++y)
                    acc[x][y] = 0.f;
            const float *fp = flux + eg * kLiftRE;
            const float *lp = LT + cg * kLiftRC;
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const float4 l4 = *reinterpret_cast<const float4 *>(lp);
                const float4 f4 = *reinterpret_cast<const float4 *>(fp);
                const float fv[4] = {f4.x, f4.y, f4.z, f4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int x = 0; x < kLiftRE; ++x)
#pragma unroll
                    for (int y = 0; y < kLiftRC; ++y)
                        acc[x][y] = fmaf(fv[x], lv[y], acc[x][y]);
                fp += TP;
                lp += NP;
            }
#pragma unroll
            for (int x = 0; x < kLiftRE; ++x) {
                const int te = eg * kLiftRE + x;
                if (te >= TEv)
                    continue;
                float *o = a.out + (e0 + te) * N;
#pragma unroll
                for (int y = 0; y < kLiftRC; ++y) {
                    const int i = cg * kLiftRC + y;
                    if (i < N)
                        o[i] = a.accumulate ? __fadd_rn(o[i], acc[x][y]) : acc[x][y];
                }
            }
        }
        __syncthreads();  // the flux tile is rewritten next
    }
}

size_t lift_smem_bytes(int N, int M, int Nf, int halo, int nbuf, int te)
{
    return lift_smem(N, M, Nf, halo, nbuf, te).total;
}

int lift_threads(int N, int te)
{
    const int CG = (N + kLiftRC - 1) / kLiftRC;
    const int t = CG * (te / kLiftRE);
    return (t + 31) / 32 * 32;
}

lc_status lift_launch(const LiftArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = lift_smem_bytes(a.N, a.M, a.Nf, a.halo, a.nbuf, a.te);
    void *fn = a.te == 128 ? (a.halo >= 0 ? reinterpret_cast<void *>(&lift_kernel<true, 128>)
                                          : reinterpret_cast<void *>(&lift_kernel<false, 128>))
                           : (a.halo >= 0 ? reinterpret_cast<void *>(&lift_kernel<true, 64>)
                                          : reinterpret_cast<void *>(&lift_kernel<false, 64>));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    // a persistent grid no larger than the CTAs that are resident at once (shared memory may
    // allow fewer per SM than asked for; the rest would wait for a second wave)
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, lift_threads(a.N, a.te), smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    const int sms = sm_count();
    if (per_sm > 0 && sms > 0)
        grid = std::min(grid, per_sm * sms);
    LiftArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(lift_threads(a.N, a.te)), params, smem, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

}  // namespace lc

using namespace lc;

extern "C" {

lc_status lc_lift(const lc_kernel *kh, const lc_variant *v, const float *L, const int32_t *fmask,
                  const int32_t *vmapP, const float *s, const float *u, float *out, int64_t E, int32_t N,
                  int32_t Nf, int32_t Nfp, int32_t accumulate, void *stream)
{
    if (!kh || !v || v->struct_size != sizeof(lc_variant))
        return LC_ERR_INVALID_ARGUMENT;
    if (kh->k.kind != KIND_LIFT)
        return LC_ERR_UNSUPPORTED;
    if (E < 0 || N < 1 || N > 128 || Nf < 1 || Nfp < 1 || Nf * Nfp > 256 || E * (long long)N >= (1LL << 31) ||
        (accumulate != 0 && accumulate != 1))
        return LC_ERR_INVALID_ARGUMENT;
    if (!L || !fmask || (E > 0 && (!vmapP || !s || !u || !out)))
        return LC_ERR_INVALID_ARGUMENT;
    // FP32 SIMT engine; prefetch_smem (the u window), ctas_per_sm and max_ctas size the
    // persistent grid; nothing else is used
    if (v->engine != LC_ENGINE_SIMT || v->precision != LC_PREC_FP32 || v->layout != LC_LAYOUT_ELEM_MAJOR ||
        v->ctas_per_sm < 0 || v->ctas_per_sm > 8 || v->max_ctas < 0 || v->prefetch_smem < 0 ||
        v->prefetch_smem > 1 || v->stages < 1 || v->stages > 2 || (v->tile_e != 64 && v->tile_e != 128))
        return LC_ERR_INVALID_VARIANT;
    const int nbuf = v->stages;  // staging buffers
    const int te = v->tile_e;    // elements per tile
    for (const void *p : {(const void *)L, (const void *)fmask, (const void *)vmapP, (const void *)s,
                          (const void *)u, (const void *)out})
        if ((uintptr_t)p & 3u)
            return LC_ERR_MISALIGNED;
    {
        // out must not overlap an input
        const uintptr_t o0 = (uintptr_t)out, o1 = o0 + (size_t)E * N * 4;
        const uintptr_t in[5][2] = {{(uintptr_t)u, (uintptr_t)u + (size_t)E * N * 4},
                                    {(uintptr_t)L, (uintptr_t)L + (size_t)N * Nf * Nfp * 4},
                                    {(uintptr_t)s, (uintptr_t)s + (size_t)E * Nf * 4},
                                    {(uintptr_t)vmapP, (uintptr_t)vmapP + (size_t)E * Nf * Nfp * 4},
                                    {(uintptr_t)fmask, (uintptr_t)fmask + (size_t)Nf * Nfp * 4}};
        for (auto &x : in)
            if (E > 0 && o0 < x[1] && x[0] < o1)
                return LC_ERR_INVALID_ARGUMENT;
    }
    int major = 0, minor = 0;
    if (current_cc(&major, &minor) != 0 || major != 10 || minor != 3)
        return LC_ERR_NO_DEVICE;
    // the window's halo: 64 elements (the largest face-neighbour offset of a structured
    // strip of width 64), halved while the CTA's shared memory would keep ctas_per_sm (at
    // least 2) CTAs from sharing an SM; none without prefetch_smem
    // The staged path needs 16-byte aligned u, vmapP and s (bulk copies); others read every
    // operand from global memory.
    int halo = -1;
    if (v->prefetch_smem && ((((uintptr_t)u | (uintptr_t)vmapP | (uintptr_t)s) & 15u) == 0)) {
        // (a multiple of 4: the window's first row then starts on a 16-byte boundary)
        halo = 64;
        const int want = std::max(2, v->ctas_per_sm ? v->ctas_per_sm : 4);
        const size_t fit = smem_optin_limit() / want - 1024;  // (1 KB reserved per CTA)
        while (halo > 0 && lift_smem_bytes(N, Nf * Nfp, Nf, halo, nbuf, te) > fit)
            halo = halo > 4 ? halo / 2 : 0;
        if (lift_smem_bytes(N, Nf * Nfp, Nf, halo, nbuf, te) > smem_optin_limit())
            halo = -1;
    }
    if (lift_smem_bytes(N, Nf * Nfp, Nf, halo, nbuf, te) > smem_optin_limit())
        return LC_ERR_INVALID_VARIANT;
    if (E == 0)
        return LC_OK;
    const int sms = sm_count();
    if (sms <= 0)
        return LC_ERR_NO_DEVICE;
    LiftArgs a;
    a.L = L;
    a.fmask = fmask;
    a.vmapP = vmapP;
    a.s = s;
    a.u = u;
    a.out = out;
    a.E = E;
    a.N = N;
    a.Nf = Nf;
    a.Nfp = Nfp;
    a.M = Nf * Nfp;
    a.accumulate = accumulate;
    a.halo = halo;
    a.nbuf = nbuf;
    a.te = te;
    a.err = error_word();
    const long long ntiles = (E + te - 1) / te;
    long long grid = std::min<long long>(ntiles, (long long)(v->ctas_per_sm ? v->ctas_per_sm : 4) * sms);
    if (v->max_ctas > 0)
        grid = std::min<long long>(grid, v->max_ctas);
    return lift_launch(a, (int)std::max<long long>(grid, 1), (cudaStream_t)stream);
}

}  // extern "C"
