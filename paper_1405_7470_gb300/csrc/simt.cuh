// SIMT (FP32 / FP64 FMA) kernels for the element-local contraction
//     out[f,e,i] = sum_j D[f,i,j] * u[e,j]                (dG FEM volume, Table 1)
//
// The descriptor's transformations (Section 2.4) map onto this template:
//   split_iname(e, TE)       one tile of TE elements per CTA step, e = e_in + TE*e_out
//                            (Eq. 1); the last tile is guarded unless tail_free.
//   ilp on e_in / on i       register block of RE elements x RC output columns per
//                            thread (columns c = f*N + i, all F operators fused).
//   unr on j                 UNR-fold unrolled reduction loop.
//   vec                      16-byte vector loads and stores along the contiguous axis.
//   add_prefetch(u)          PREFETCH: the u tile is staged in shared memory,
//                            transposed to [j][e]; otherwise loaded from global
//                            memory inside the j loop.
//   precompute(D)            D^T staged once per CTA in shared memory, columns
//                            permuted so each thread's RC columns are contiguous.
//   layout tags              element-major u[E][N], out[F][E][N]: outputs are staged
//                            in shared memory and written as contiguous [TE][N] runs;
//                            node-major u[N][E], out[F][N][E]: coalesced vector stores
//                            straight from registers.
#pragma once

#include <cuda_runtime.h>

#include "lc_internal.h"

namespace lc {

template <typename T>
struct VecT;
template <>
struct VecT<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct VecT<double> {
    using type = double2;
    static constexpr int n = 2;
};

template <typename T, int RE, int RC, int UNR, int LAYOUT, bool PREFETCH>
__global__ void __launch_bounds__(512) simt_contract_kernel(SimtArgs a)
{
    constexpr int VEC = VecT<T>::n;
    using V = typename VecT<T>::type;
    constexpr int QE = RE / VEC;  // element vectors per thread
    constexpr int QC = RC / VEC;  // column vectors per thread
    static_assert(RE % VEC == 0 && RC % VEC == 0, "register block must be whole vectors");
    constexpr bool NODE = LAYOUT == LC_LAYOUT_NODE_MAJOR;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.N, F = a.F, C = a.C, TE = a.TE, EG = a.EG, CG = a.CG, CW = a.CW;
    const long long E = a.E;
    const T *__restrict__ D = static_cast<const T *>(a.D);
    const T *__restrict__ u = static_cast<const T *>(a.u);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    // Lane order: element groups fastest for node-major (coalesced stores along e),
    // column groups fastest for element-major (conflict-free staging along i).
    const int eg = NODE ? tid % EG : tid / CG;
    const int cg = NODE ? tid / EG : tid % CG;
    const int TEp = NODE ? TE : TE + VEC;  // padded row of the transposed u tile

    T *Ds = reinterpret_cast<T *>(smem_raw);                 // [N][CW]
    T *uT = Ds + (size_t)N * CW;                             // [N][TEp]   (PREFETCH)
    T *ost = uT + (PREFETCH ? (size_t)N * TEp : 0);          // [F][TE][N] (element-major)

    // precompute(D): Ds[j][cg*RC + m] = D[f][i][j] with c = ch*CW + cg + m*CG = f*N + i.
    auto load_D = [&](int ch) {
        for (int idx = tid; idx < N * CW; idx += nthr) {
            int j = idx / CW, p = idx - j * CW;
            int g = p / RC, m = p - g * RC;
            int c = ch * CW + g + m * CG;
            T val = T(0);
            if (c < C) {
                int f = c / N, i = c - f * N;
                val = D[((size_t)f * N + i) * N + j];
            }
            Ds[idx] = val;
        }
    };
    if (a.nchunks == 1) {
        load_D(0);
    }

    for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const long long e0 = tile * (long long)TE;
        const bool full = a.tail_free || (e0 + TE <= E);
        const int TEv = full ? TE : (int)(E - e0);
        __syncthreads();  // previous tile finished with uT / ost

        if (PREFETCH) {
            if (NODE) {
                // rows u[j][e0 : e0+TE] -> uT[j][0:TE]
                const int QT = TE / VEC;
                const bool vec_ok = full && (E % VEC == 0);
                for (int idx = tid; idx < N * QT; idx += nthr) {
                    int j = idx / QT, q = idx - j * QT;
                    const T *src = u + (size_t)j * E + e0 + q * VEC;
                    V val;
                    if (vec_ok) {
                        val = *reinterpret_cast<const V *>(src);
                    } else {
                        T *pv = reinterpret_cast<T *>(&val);
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            pv[v] = (q * VEC + v < TEv) ? src[v] : T(0);
                    }
                    *reinterpret_cast<V *>(uT + (size_t)j * TEp + q * VEC) = val;
                }
            } else {
                // contiguous block u[e0 : e0+TEv][0:N] -> uT[j][e], zero-filled tail
                const T *src = u + e0 * N;
                const int total = TEv * N;
                int e = tid / N, j = tid - (tid / N) * N;
                const int de = nthr / N, dj = nthr - (nthr / N) * N;
                for (int k = tid; k < total; k += nthr) {
                    uT[(size_t)j * TEp + e] = src[k];
                    e += de;
                    j += dj;
                    if (j >= N) {
                        j -= N;
                        ++e;
                    }
                }
                if (!full) {
                    for (int idx = tid; idx < N * (TE - TEv); idx += nthr) {
                        int j2 = idx / (TE - TEv), e2 = TEv + idx % (TE - TEv);
                        uT[(size_t)j2 * TEp + e2] = T(0);
                    }
                }
            }
        }
        __syncthreads();

        for (int ch = 0; ch < a.nchunks; ++ch) {
            if (a.nchunks > 1) {
                __syncthreads();
                load_D(ch);
                __syncthreads();
            }
            T acc[RE][RC];
#pragma unroll
            for (int x = 0; x < RE; ++x)
#pragma unroll
                for (int y = 0; y < RC; ++y)
                    acc[x][y] = T(0);

#pragma unroll UNR
            for (int j = 0; j < N; ++j) {
                T av[RE], bv[RC];
                if (PREFETCH) {
#pragma unroll
                    for (int q = 0; q < QE; ++q)
                        *reinterpret_cast<V *>(&av[q * VEC]) =
                            *reinterpret_cast<const V *>(uT + (size_t)j * TEp + (eg + q * EG) * VEC);
                } else if (NODE) {
#pragma unroll
                    for (int q = 0; q < QE; ++q) {
                        const long long eb = e0 + (long long)(eg + q * EG) * VEC;
                        const T *src = u + (size_t)j * E + eb;
                        if (full && (E % VEC == 0)) {
                            *reinterpret_cast<V *>(&av[q * VEC]) = __ldg(reinterpret_cast<const V *>(src));
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                av[q * VEC + v] = (eb + v < E) ? __ldg(src + v) : T(0);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < QE; ++q)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const long long e = e0 + (long long)(eg + q * EG) * VEC + v;
                            av[q * VEC + v] = (full || e < E) ? __ldg(u + e * N + j) : T(0);
                        }
                }
#pragma unroll
                for (int r = 0; r < QC; ++r)
                    *reinterpret_cast<V *>(&bv[r * VEC]) =
                        *reinterpret_cast<const V *>(Ds + (size_t)j * CW + cg * RC + r * VEC);
#pragma unroll
                for (int x = 0; x < RE; ++x)
#pragma unroll
                    for (int y = 0; y < RC; ++y)
                        acc[x][y] = fma(av[x], bv[y], acc[x][y]);
            }

            // Stores.
#pragma unroll
            for (int y = 0; y < RC; ++y) {
                const int c = ch * CW + cg + y * CG;
                if (c >= C)
                    continue;
                const int f = c / N, i = c - f * N;
                if (NODE) {
                    T *orow = out + ((size_t)f * N + i) * E;
#pragma unroll
                    for (int q = 0; q < QE; ++q) {
                        const long long eb = e0 + (long long)(eg + q * EG) * VEC;
                        if (full && (E % VEC == 0)) {
                            V val;
                            T *pv = reinterpret_cast<T *>(&val);
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                pv[v] = acc[q * VEC + v][y];
                            *reinterpret_cast<V *>(orow + eb) = val;
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                if (eb + v < E)
                                    orow[eb + v] = acc[q * VEC + v][y];
                        }
                    }
                } else {
                    T *o = ost + (size_t)f * TE * N + i;
#pragma unroll
                    for (int q = 0; q < QE; ++q)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            o[(size_t)((eg + q * EG) * VEC + v) * N] = acc[q * VEC + v][y];
                }
            }
        }

        if (!NODE) {
            // out[f][e0 : e0+TEv][0:N] is one contiguous run per operator.
            __syncthreads();
            const int total = TEv * N;
            for (int f = 0; f < F; ++f) {
                const T *src = ost + (size_t)f * TE * N;
                T *dst = out + ((size_t)f * E + e0) * N;
                const bool vec_ok = ((((size_t)f * E + e0) * N) % VEC) == 0;
                int done = 0;
                if (vec_ok) {
                    const int nv = total / VEC;
                    for (int k = tid; k < nv; k += nthr)
                        reinterpret_cast<V *>(dst)[k] = reinterpret_cast<const V *>(src)[k];
                    done = nv * VEC;
                }
                for (int k = done + tid; k < total; k += nthr)
                    dst[k] = src[k];
            }
        }
    }
}

// Host-side dispatch over the compiled instances of one element type and layout.
template <typename T, int LAYOUT, int RE, int RC, int UNR, bool PF>
static void *simt_kernel_ptr()
{
    return reinterpret_cast<void *>(&simt_contract_kernel<T, RE, RC, UNR, LAYOUT, PF>);
}

template <typename T, int LAYOUT, int RE, int RC, int UNR>
static void *simt_pick_pf(int pf)
{
    return pf ? simt_kernel_ptr<T, LAYOUT, RE, RC, UNR, true>()
              : simt_kernel_ptr<T, LAYOUT, RE, RC, UNR, false>();
}

template <typename T, int LAYOUT, int RE, int RC>
static void *simt_pick_unr(int unr, int pf)
{
    switch (unr) {
    case 1: return simt_pick_pf<T, LAYOUT, RE, RC, 1>(pf);
    case 2: return simt_pick_pf<T, LAYOUT, RE, RC, 2>(pf);
    case 4: return simt_pick_pf<T, LAYOUT, RE, RC, 4>(pf);
    case 8: return simt_pick_pf<T, LAYOUT, RE, RC, 8>(pf);
    default: return nullptr;
    }
}

template <typename T, int LAYOUT>
static lc_status simt_launch_impl(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                                  cudaStream_t s)
{
    constexpr int V = VecT<T>::n;
    void *fn = nullptr;
    if (g.RE == V && g.RC == V) fn = simt_pick_unr<T, LAYOUT, V, V>(unroll, prefetch);
    else if (g.RE == V && g.RC == 2 * V) fn = simt_pick_unr<T, LAYOUT, V, 2 * V>(unroll, prefetch);
    else if (g.RE == 2 * V && g.RC == V) fn = simt_pick_unr<T, LAYOUT, 2 * V, V>(unroll, prefetch);
    else if (g.RE == 2 * V && g.RC == 2 * V) fn = simt_pick_unr<T, LAYOUT, 2 * V, 2 * V>(unroll, prefetch);
    if (!fn)
        return LC_ERR_INVALID_VARIANT;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    SimtArgs args = a;
    void *params[] = {&args};
    e = cudaLaunchKernel(fn, dim3(g.grid), dim3(g.threads), params, g.smem, s);
    if (e != cudaSuccess)
        return cuda_fail(e);
    return LC_OK;
}

}  // namespace lc
