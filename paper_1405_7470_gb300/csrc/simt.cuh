// SIMT (FP32 / FP64 FMA) kernels for the element-local contraction
//     out[f,e,i] = sum_j D[f,i,j] * u[e,j]                (dG FEM volume, Table 1)
//
// The descriptor's transformations (Section 2.4) map onto this template:
//   split_iname(e, TE)       one tile of TE elements per CTA step, e = e_in + TE*e_out
//                            (Eq. 1); the last tile is guarded unless tail_free.
//   ilp on e_in / on i       register block of RE consecutive elements x RC output
//                            columns per thread (columns c = f*N + i, all F operators
//                            fused). A warp is a WE x WC grid of lanes (WE*WC = 32) so
//                            that shared-memory operand loads are broadcasts; operand
//                            addresses advance by one pointer increment per j.
//   unr on j                 UNR-fold unrolled reduction loop.
//   vec                      16-byte vector loads and stores along the contiguous axis.
//   add_prefetch(u)          PREFETCH: u tiles are fetched by the bulk-copy engine
//                            (cp.async.bulk, mbarrier completion) into a ring of
//                            `stages` shared-memory buffers, ahead of the compute;
//                            otherwise u is read from global memory inside the j loop.
//   precompute(D)            D^T staged once per CTA in shared memory, columns
//                            permuted so each thread's RC columns are contiguous.
//   layout tags              element-major u[E][N], out[F][E][N]: the u tile is
//                            transposed to [j][e] in shared memory and each operator's
//                            output tile [TE][N] is written by one bulk store;
//                            node-major u[N][E], out[F][N][E]: the fetched tile is
//                            already [j][e] and outputs leave registers as coalesced
//                            16-byte stores.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "lc_internal.h"
#include "tma.cuh"

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

// Threads per CTA allowed for a register block (the 8 x 8 FP32 block needs > 128 registers).
__host__ __device__ constexpr int simt_max_threads(int re, int rc) { return re * rc >= 64 ? 256 : 512; }

// One CTA's share of a contraction: column block `ch` (operators ch*G .. ch*G + G - 1,
// their D^T resident in shared memory for the whole call) of the tiles t_first,
// t_first + t_step, ... below t_end.  Used by the plain kernel (grid-stride over all
// tiles) and by the grouped kernel (contiguous tile ranges of several problems).
template <typename T, int RE, int RC, int UNR, int LAYOUT, bool PREFETCH>
__device__ __forceinline__ void simt_tiles(const SimtArgs &a, int ch, long long t_first, long long t_step,
                                           long long t_end, unsigned char *smem_raw)
{
    constexpr int VEC = VecT<T>::n;
    using V = typename VecT<T>::type;
    constexpr int QE = RE / VEC;  // element vectors per thread
    constexpr int QC = RC / VEC;  // column vectors per thread
    static_assert(RE % VEC == 0 && RC % VEC == 0, "register block must be whole vectors");
    constexpr bool NODE = LAYOUT == LC_LAYOUT_NODE_MAJOR;
    constexpr int ES = (int)sizeof(T);

    const int N = a.N, F = a.F, TE = a.TE, EG = a.EG, CG = a.CG, CW = a.CW;
    // Column block `ch`: G whole operators (isplit == 0), or rows [i_lo, i_lo + width) of
    // one operator (isplit = width > 0, when one operator's D^T does not fit).
    const bool whole = a.isplit == 0;
    const int nsub = whole ? 1 : (N + a.isplit - 1) / a.isplit;
    const int f0 = whole ? ch * a.G : ch / nsub;                 // first operator of the block
    const int Gb = whole ? min(a.G, F - f0) : 1;                 // operators in the block
    const int i_lo = whole ? 0 : (ch % nsub) * a.isplit;
    const int Cb = whole ? Gb * N : min(a.isplit, N - i_lo);     // columns of the block
    const int orow = whole ? N : Cb;                             // staged output row length
    const long long E = a.E;
    const int S = a.stages;
    const T *__restrict__ D = static_cast<const T *>(a.D);
    const T *__restrict__ u = static_cast<const T *>(a.u);
    T *__restrict__ out = static_cast<T *>(a.out);
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int WC = a.WC, WE = 32 / WC;
    const int nwe = EG / WE;
    const int eg = (warp % nwe) * WE + lane % WE;
    const int cg = (warp / nwe) * WC + lane / WE;
    // warps beyond the EG x CG thread grid (a grouped CTA sized for a larger group) only
    // take part in the cooperative loads, copies and barriers
    const bool active = warp < (EG * CG) / 32;
    const int TEp = TE + VEC;  // padded row of the transposed element-major tile

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);  // two mbarriers
    T *Ds = reinterpret_cast<T *>(smem_raw + 16);              // [N][CW]
    T *p = Ds + (size_t)N * CW;
    T *uT = nullptr, *stage = nullptr, *ost = nullptr;
    if (PREFETCH) {
        if (NODE) {
            stage = p;  // S x [N][TE]
            p += (size_t)S * N * TE;
        } else {
            uT = p;  // [N][TEp]
            p += (size_t)N * TEp;
            stage = p;  // S x [TE*N]
            p += (size_t)S * TE * N;
        }
    }
    if (!NODE)
        ost = p;  // [Gb][TE][N]

    // precompute(D): Ds[j][cg*RC + m] = D[f][i][j] for block column c = cg + m*CG < Cb.
    auto load_D = [&]() {
        for (int idx = tid; idx < N * CW; idx += nthr) {
            int j = idx / CW, q = idx - j * CW;
            int g = q / RC, m = q - g * RC;
            int c = g + m * CG;
            T val = T(0);
            if (c < Cb) {
                int fl = whole ? c / N : 0, i = whole ? c - fl * N : i_lo + c;
                val = D[((size_t)(f0 + fl) * N + i) * N + j];
            }
            Ds[idx] = val;
        }
    };

    const bool bulk = PREFETCH && a.bulk;
    if (bulk && tid == 0) {
        for (int s = 0; s < S; ++s)
            mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    load_D();
    __syncthreads();

    // Warp 0 fetches tile `t` into ring slot `buf`.
    auto issue = [&](long long t, int buf) {
        const long long e0 = t * (long long)TE;
        const int TEv = (int)min((long long)TE, E - e0);
        if (NODE) {
            const uint32_t bytes = (uint32_t)TEv * ES;  // a multiple of 16 when bulk is set
            if (lane == 0)
                mbar_arrive_expect_tx(&bars[buf], bytes * (uint32_t)N);
            __syncwarp();
            T *dst = stage + (size_t)buf * N * TE;
            for (int j = lane; j < N; j += 32)
                bulk_g2s(dst + (size_t)j * TE, u + (size_t)j * E + e0, bytes, &bars[buf]);
        } else if (lane == 0) {
            const uint32_t bytes = ((uint32_t)TEv * N * ES) & ~15u;
            mbar_arrive_expect_tx(&bars[buf], bytes);
            if (bytes)
                bulk_g2s(stage + (size_t)buf * TE * N, u + e0 * N, bytes, &bars[buf]);
        }
    };
    if (bulk && warp == 0) {
        for (int s = 0; s < S; ++s) {
            const long long t = t_first + (long long)s * t_step;
            if (t < t_end)
                issue(t, s);
        }
    }

    // Output offsets of this thread's RC columns c = cg + y*CG of the block (-1: padding).
    using Off = typename std::conditional<NODE, long long, int>::type;
    Off coff[RC];
#pragma unroll
    for (int y = 0; y < RC; ++y) {
        const int c = cg + y * CG;
        const int fl = whole ? c / N : 0, il = whole ? c - fl * N : c;  // il: index in the staged row
        coff[y] = c >= Cb ? Off(-1)
                          : (NODE ? Off(((long long)(f0 + fl) * N + i_lo + il) * E) : Off(fl * TE * orow + il));
    }

    int k = 0;
    for (long long tile = t_first; tile < t_end; tile += t_step, ++k) {
        const long long e0 = tile * (long long)TE;
        const bool full = a.tail_free || (e0 + TE <= E);
        const int TEv = full ? TE : (int)(E - e0);
        const int buf = bulk ? k % S : 0;
        const T *ut = nullptr;  // [N][ldu] tile the compute reads
        int ldu = 0;

        if (PREFETCH) {
            if (bulk) {
                const bool ok = mbar_wait(&bars[buf], (uint32_t)((k / S) & 1));
                if (!__syncthreads_and(ok)) {
                    if (tid == 0)
                        atomicOr(a.err, 1u);
                    break;
                }
            } else {
                // no bulk path (node-major with E % VEC != 0): cooperative synchronous loads
                __syncthreads();
                if (NODE) {
                    for (int idx = tid; idx < N * TE; idx += nthr) {
                        int j = idx / TE, e = idx - j * TE;
                        stage[idx] = e < TEv ? u[(size_t)j * E + e0 + e] : T(0);
                    }
                }
            }
            if (NODE) {
                ut = stage + (size_t)buf * N * TE;
                ldu = TE;
            } else {
                // transpose the [TE][N] tile into uT[j][e]; lanes walk e so the writes are
                // conflict-free; the part the bulk copy did not cover comes from global memory
                const T *st = stage + (size_t)buf * TE * N;
                const int total = TEv * N;
                const int kb = bulk ? (int)((((uint32_t)total * ES) & ~15u) / ES) : 0;
                int j = tid / TE, e = tid - (tid / TE) * TE;
                const int dj = nthr / TE, de = nthr - (nthr / TE) * TE;
                if (kb == N * TE) {
                    for (int idx = tid; idx < N * TE; idx += nthr) {
                        uT[j * TEp + e] = st[e * N + j];
                        e += de;
                        j += dj;
                        if (e >= TE) {
                            e -= TE;
                            ++j;
                        }
                    }
                } else {
                    for (int idx = tid; idx < N * TE; idx += nthr) {
                        const int kk = e * N + j;
                        uT[j * TEp + e] = kk < kb ? st[kk] : (kk < total ? u[e0 * N + kk] : T(0));
                        e += de;
                        j += dj;
                        if (e >= TE) {
                            e -= TE;
                            ++j;
                        }
                    }
                }
                ut = uT;
                ldu = TEp;
            }
            if (!NODE) {
                if (tid == 0)
                    bulk_wait_read0();  // previous tile's output stores have read ost
                fence_async_smem();
            }
            __syncthreads();
            if (!NODE && bulk && warp == 0) {
                // stage[buf] is consumed: fetch the tile S steps ahead into it
                const long long nt = tile + (long long)S * t_step;
                if (nt < t_end)
                    issue(nt, buf);
            }
        } else if (!NODE) {
            if (tid == 0)
                bulk_wait_read0();
            __syncthreads();
        }

        if (active) {
            T acc[RE][RC];
#pragma unroll
            for (int x = 0; x < RE; ++x)
#pragma unroll
                for (int y = 0; y < RC; ++y)
                    acc[x][y] = T(0);

            const T *dp = Ds + cg * RC;
            const T *up = PREFETCH ? ut + eg * RE : nullptr;
            const long long eb0 = e0 + (long long)eg * RE;  // this thread's first element
#pragma unroll UNR
            for (int j = 0; j < N; ++j) {
                T av[RE], bv[RC];
                if (PREFETCH) {
#pragma unroll
                    for (int q = 0; q < QE; ++q)
                        *reinterpret_cast<V *>(&av[q * VEC]) = *reinterpret_cast<const V *>(up + q * VEC);
                    up += ldu;
                } else if (NODE) {
                    const T *src = u + (size_t)j * E + eb0;
#pragma unroll
                    for (int q = 0; q < QE; ++q) {
                        if (full && (E % VEC == 0)) {
                            *reinterpret_cast<V *>(&av[q * VEC]) = __ldg(reinterpret_cast<const V *>(src + q * VEC));
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                av[q * VEC + v] = (eb0 + q * VEC + v < E) ? __ldg(src + q * VEC + v) : T(0);
                        }
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < RE; ++x) {
                        const long long e = eb0 + x;
                        av[x] = (full || e < E) ? __ldg(u + e * N + j) : T(0);
                    }
                }
#pragma unroll
                for (int r = 0; r < QC; ++r)
                    *reinterpret_cast<V *>(&bv[r * VEC]) = *reinterpret_cast<const V *>(dp + r * VEC);
                dp += CW;
#pragma unroll
                for (int x = 0; x < RE; ++x)
#pragma unroll
                    for (int y = 0; y < RC; ++y)
                        acc[x][y] = fma(av[x], bv[y], acc[x][y]);
            }

            if (NODE) {
                const bool vec_ok = full && (E % VEC == 0);
#pragma unroll
                for (int y = 0; y < RC; ++y) {
                    if (coff[y] < 0)
                        continue;
                    T *orow = out + coff[y] + eb0;
#pragma unroll
                    for (int q = 0; q < QE; ++q) {
                        if (vec_ok) {
                            V val;
                            T *pv = reinterpret_cast<T *>(&val);
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                pv[v] = acc[q * VEC + v][y];
                            *reinterpret_cast<V *>(orow + q * VEC) = val;
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                if (eb0 + q * VEC + v < E)
                                    orow[q * VEC + v] = acc[q * VEC + v][y];
                        }
                    }
                }
            } else {
                T *o = ost + eg * RE * orow;
#pragma unroll
                for (int x = 0; x < RE; ++x) {
#pragma unroll
                    for (int y = 0; y < RC; ++y)
                        if (coff[y] >= 0)
                            o[coff[y]] = acc[x][y];
                    o += orow;
                }
            }
        }

        if (NODE) {
            if (bulk) {
                __syncthreads();  // every warp is done reading stage[buf]
                if (warp == 0) {
                    const long long nt = tile + (long long)S * t_step;
                    if (nt < t_end)
                        issue(nt, buf);
                }
            }
        } else {
            // out[f][e0 : e0+TEv][0:N] is one contiguous run per operator
            fence_async_smem();
            __syncthreads();
            const int total = TEv * N;
            if (!whole) {
                // rows [i_lo, i_lo + Cb) of each element: one short segment per element
                for (int q = tid; q < TEv * Cb; q += nthr) {
                    const int e = q / Cb, c = q - e * Cb;
                    out[((size_t)f0 * E + e0 + e) * N + i_lo + c] = ost[q];
                }
            } else if (a.bulk_store && ((total * ES) & 15) == 0) {
                if (tid == 0) {
                    for (int g = 0; g < Gb; ++g)
                        bulk_s2g(out + ((size_t)(f0 + g) * E + e0) * N, ost + (size_t)g * TE * N,
                                 (uint32_t)total * ES);
                    bulk_commit();
                }
            } else {
                for (int g = 0; g < Gb; ++g) {
                    const int f = f0 + g;
                    const T *src = ost + (size_t)g * TE * N;
                    T *dst = out + ((size_t)f * E + e0) * N;
                    int done = 0;
                    if (((((size_t)f * E + e0) * N) % VEC) == 0) {
                        const int nv = total / VEC;
                        for (int q = tid; q < nv; q += nthr)
                            reinterpret_cast<V *>(dst)[q] = reinterpret_cast<const V *>(src)[q];
                        done = nv * VEC;
                    }
                    for (int q = done + tid; q < total; q += nthr)
                        dst[q] = src[q];
                }
            }
        }
    }
    if (!NODE && tid == 0)
        bulk_wait0();
    // leave the mbarriers and shared memory reusable by the next tile range
    __syncthreads();
    if (bulk && tid == 0)
        for (int s = 0; s < S; ++s)
            mbar_inval(&bars[s]);
    __syncthreads();
}

template <typename T, int RE, int RC, int UNR, int LAYOUT, bool PREFETCH>
__global__ void __launch_bounds__(simt_max_threads(RE, RC)) simt_contract_kernel(SimtArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nb = a.nchunks;
    simt_tiles<T, RE, RC, UNR, LAYOUT, PREFETCH>(a, blockIdx.x % nb, blockIdx.x / nb, gridDim.x / nb, a.ntiles,
                                                 smem_raw);
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
