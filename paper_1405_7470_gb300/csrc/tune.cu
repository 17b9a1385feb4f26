// Autotuner: enumerate the valid descriptors for a problem and time each on the GPU
// with CUDA events (warm-up launch, then the median of `reps` timed launches).  The
// same candidate list is what the MLP cost model ranks.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lc_internal.h"

namespace lc {

static std::vector<lc_variant> candidates(int N, int F, int layout, int precision)
{
    std::vector<lc_variant> out;
    lc_variant b;
    memset(&b, 0, sizeof b);
    b.struct_size = sizeof(lc_variant);
    b.layout = layout;
    b.precision = precision;
    if (precision == LC_PREC_FP32 || precision == LC_PREC_FP64) {
        const int V = precision == LC_PREC_FP64 ? 2 : 4;
        const int blocks[3][2] = {{V, 2 * V}, {2 * V, V}, {2 * V, 2 * V}};
        const int pfst[2][2] = {{0, 1}, {1, 2}};
        for (auto &rb : blocks)
            for (int tm : {8, 16})
                for (int unr : {1, 4})
                    for (auto &ps : pfst) {
                        lc_variant v = b;
                        v.engine = LC_ENGINE_SIMT;
                        v.elems_per_thread = rb[0];
                        v.split_i = rb[1];
                        v.tile_e = rb[0] * tm;
                        v.unroll = unr;
                        v.prefetch_smem = ps[0];
                        v.stages = ps[1];
                        v.ctas_per_sm = 2;
                        out.push_back(v);
                    }
        if (precision == LC_PREC_FP32) {
            // K-split: tile 64 or 128 elements, j chunks of 8 or 16, one or two u buffers
            for (int bm : {64, 128})
                for (int bk : {8, 16})
                    for (int st : {1, 2}) {
                        lc_variant v = b;
                        v.engine = LC_ENGINE_KSPLIT;
                        v.tile_e = bm;
                        v.elems_per_thread = 8;
                        v.split_i = 8;
                        v.unroll = bk;
                        v.prefetch_smem = 1;
                        v.stages = st;
                        out.push_back(v);
                    }
        }
        if (N <= 32 && (precision != LC_PREC_FP64 || N <= 16 || F == 1)) {
            for (int warps : {4, 8}) {
                lc_variant v = b;
                v.engine = LC_ENGINE_WARP;
                v.tile_e = (32 / N) * warps;
                v.elems_per_thread = 1;
                v.split_i = 1;
                v.unroll = 1;
                v.stages = 1;
                v.ctas_per_sm = 4;
                out.push_back(v);
            }
        }
    } else {
        const bool node = layout == LC_LAYOUT_NODE_MAJOR;
        // stage ring depth 1, 2, 3, and one stage released early (prefetch_smem = 2)
        for (int st : {1, 2, 3, 0}) {
            for (int tpr : {2, 3, 4})
                for (int g : {0, 1})
                    for (int kbw : {1, 64})
                        for (int rows : {32, 128}) {
                            if (node && rows != 32)
                                continue;  // node-major stores from registers
                            lc_variant v = b;
                            v.engine = LC_ENGINE_TCGEN05;
                            v.tile_e = 128;
                            v.elems_per_thread = kbw;
                            v.split_i = g;
                            v.unroll = tpr;
                            v.prefetch_smem = st == 0 ? 2 : 1;
                            v.stages = st == 0 ? 1 : st;
                            v.store_rows = node ? 0 : rows;
                            out.push_back(v);
                        }
        }
    }
    return out;
}

}  // namespace lc

using namespace lc;

extern "C" {

lc_status lc_enumerate_variants(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout,
                                int32_t precision, lc_variant *out, int32_t cap, int32_t *count)
{
    if (!k || !count || cap < 0 || (cap > 0 && !out))
        return LC_ERR_INVALID_ARGUMENT;
    std::vector<lc_variant> cand = candidates(N, F, layout, precision);
    if (precision == LC_PREC_BF16 || precision == LC_PREC_BF16X3) {
        // when no tensor-core plan fits (large N), the FP32 SIMT variants serve the request:
        // their error is below both reduced-precision bounds
        bool any = false;
        for (const lc_variant &v : cand)
            any = any || lc_variant_validate(k, E, N, F, &v) == LC_OK;
        if (!any)
            cand = candidates(N, F, layout, LC_PREC_FP32);
    }
    int n = 0;
    for (const lc_variant &v : cand) {
        if (lc_variant_validate(k, E, N, F, &v) != LC_OK)
            continue;
        // leave out plans that shrink to one warp per CTA (the column block split until
        // the tile's operators fit shared memory): one warp then holds a whole SM
        lc_plan p;
        memset(&p, 0, sizeof p);
        p.struct_size = sizeof(lc_plan);
        if (lc_variant_plan(k, E, N, F, &v, &p) != LC_OK || p.threads < 64)
            continue;
        // keep one copy of descriptors that resolve to the same launch (e.g. G = F)
        bool dup = false;
        for (int q = 0; q < std::min(n, cap); ++q)
            if (memcmp(&out[q], &v, sizeof v) == 0)
                dup = true;
        if (dup)
            continue;
        if (n < cap)
            out[n] = v;
        ++n;
    }
    *count = n;
    return n > cap ? LC_ERR_BUFFER_TOO_SMALL : LC_OK;
}

lc_status lc_autotune(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t precision,
                      const void *D, const void *u, void *out, int32_t reps, lc_variant *variants, float *ms,
                      int32_t cap, int32_t *count, void *stream)
{
    if (!k || !variants || !ms || !count || reps < 1 || cap <= 0)
        return LC_ERR_INVALID_ARGUMENT;
    int n = 0;
    lc_status st = lc_enumerate_variants(k, E, N, F, layout, precision, variants, cap, &n);
    if (st != LC_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess)
        ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess)
        return cuda_fail(ce);
    std::vector<float> times;
    for (int c = 0; c < n; ++c) {
        st = lc_contract(k, &variants[c], D, u, out, E, N, F, stream);  // warm-up
        if (st != LC_OK)
            break;
        times.clear();
        for (int r = 0; r < reps && st == LC_OK; ++r) {
            cudaEventRecord(e0, s);
            st = lc_contract(k, &variants[c], D, u, out, E, N, F, stream);
            cudaEventRecord(e1, s);
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                st = cuda_fail(ce);
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            times.push_back(t);
        }
        if (st != LC_OK)
            break;
        std::sort(times.begin(), times.end());
        ms[c] = times[times.size() / 2];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LC_OK)
        return st;
    // best first
    std::vector<int> idx(n);
    for (int q = 0; q < n; ++q)
        idx[q] = q;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return ms[x] < ms[y]; });
    std::vector<lc_variant> vv(n);
    std::vector<float> tt(n);
    for (int q = 0; q < n; ++q) {
        vv[q] = variants[idx[q]];
        tt[q] = ms[idx[q]];
    }
    for (int q = 0; q < n; ++q) {
        variants[q] = vv[q];
        ms[q] = tt[q];
    }
    *count = n;
    return LC_OK;
}

}  // extern "C"
