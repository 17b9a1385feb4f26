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
//   gather   the tile's fluxes flux[m][t] = s[e, m / Nfp] * (u[e, fmask[m]] - u[vmapP[e, m]]),
//            m-fastest so the vmapP rows are read contiguously, written transposed into
//            shared memory (rows of odd stride per m: no bank conflicts);
//   lift     each thread accumulates a RE x 4 register block (elements x nodes) over m with
//            L^T (resident in shared memory for the CTA's lifetime), m ascending;
//   store    out rows, adding to the previous values when accumulating.
#include <cuda_runtime.h>

#include <algorithm>

#include "lc_internal.h"

namespace lc {

static constexpr int kLiftTE = 64;     // elements per tile
static constexpr int kLiftRE = 4;      // elements per thread
static constexpr int kLiftRC = 4;      // nodes per thread
static constexpr int kLiftPad = 1;     // padding of a flux row: odd stride, conflict-free transposed writes

__global__ void __launch_bounds__(512) lift_kernel(LiftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(kLiftRE == 4 && kLiftRC == 4, "the inner loop reads four elements and four nodes");
    const int N = a.N, M = a.M, Nfp = a.Nfp, Nf = a.Nf;
    const int CG = (N + kLiftRC - 1) / kLiftRC;  // column groups
    const int NP = CG * kLiftRC;                 // padded node count
    const int TP = kLiftTE + kLiftPad;           // flux row stride
    float *LT = reinterpret_cast<float *>(smem_raw);  // [M][NP]
    float *flux = LT + (size_t)M * NP;                // [M][TP]
    int *fm = reinterpret_cast<int *>(flux + (size_t)M * TP);  // [M]
    const long long E = a.E;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < M * NP; idx += nthr) {
        const int m = idx / NP, i = idx - m * NP;
        LT[idx] = i < N ? a.L[(size_t)i * M + m] : 0.f;
    }
    for (int m = tid; m < M; m += nthr) {
        const int j = a.fmask[m];
        const bool bad = j < 0 || j >= N;
        fm[m] = bad ? 0 : j;  // out of range: recorded, node 0 read instead
        if (bad)
            atomicOr(a.err, 2u);
    }
    __syncthreads();
    // register block of this thread: elements eg*RE.., nodes cg*RC..
    const int cg = tid % CG, eg = tid / CG;
    const bool active = eg < kLiftTE / kLiftRE;
    const long long ntiles = (E + kLiftTE - 1) / kLiftTE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long e0 = t * kLiftTE;
        const int TEv = (int)min((long long)kLiftTE, E - e0);
        // gather the tile's fluxes (m fastest: contiguous vmapP rows)
        for (int idx = tid; idx < kLiftTE * M; idx += nthr) {
            const int te = idx / M, m = idx - te * M;
            float v = 0.f;
            if (te < TEv) {
                const long long e = e0 + te;
                const int q = a.vmapP[e * M + m];
                if (q >= 0 && (long long)q < E * N) {
                    const float jump = __fsub_rn(a.u[e * N + fm[m]], a.u[q]);
                    v = __fmul_rn(a.s[e * Nf + m / Nfp], jump);
                } else {
                    v = __int_as_float(0x7fc00000);  // out-of-range index: NaN, recorded
                    atomicOr(a.err, 2u);
                }
            }
            flux[(size_t)m * TP + te] = v;
        }
        __syncthreads();
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
                const float fv[4] = {fp[0], fp[1], fp[2], fp[3]}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
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

size_t lift_smem_bytes(int N, int M)
{
    const int NP = (N + kLiftRC - 1) / kLiftRC * kLiftRC;
    return sizeof(float) * ((size_t)M * NP + (size_t)M * (kLiftTE + kLiftPad)) + sizeof(int) * (size_t)M;
}

int lift_threads(int N)
{
    const int CG = (N + kLiftRC - 1) / kLiftRC;
    const int t = CG * (kLiftTE / kLiftRE);
    return (t + 31) / 32 * 32;
}

lc_status lift_launch(const LiftArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = lift_smem_bytes(a.N, a.M);
    cudaError_t e = cudaFuncSetAttribute(lift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    lift_kernel<<<grid, lift_threads(a.N), smem, s>>>(a);
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
    // FP32 SIMT engine; ctas_per_sm and max_ctas size the persistent grid; nothing else is used
    if (v->engine != LC_ENGINE_SIMT || v->precision != LC_PREC_FP32 || v->layout != LC_LAYOUT_ELEM_MAJOR ||
        v->ctas_per_sm < 0 || v->ctas_per_sm > 8 || v->max_ctas < 0)
        return LC_ERR_INVALID_VARIANT;
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
    if (lift_smem_bytes(N, Nf * Nfp) > smem_optin_limit())
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
    a.err = error_word();
    const long long ntiles = (E + 63) / 64;
    long long grid = std::min<long long>(ntiles, (long long)(v->ctas_per_sm ? v->ctas_per_sm : 4) * sms);
    if (v->max_ctas > 0)
        grid = std::min<long long>(grid, v->max_ctas);
    return lift_launch(a, (int)std::max<long long>(grid, 1), (cudaStream_t)stream);
}

}  // extern "C"
