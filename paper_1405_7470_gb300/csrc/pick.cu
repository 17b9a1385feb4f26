// Learned variant pick behind the C ABI: the cost model's input features of a
// (problem, descriptor) pair, and the pick itself (enumerate the candidates, build their
// features, run the network, or each network of an ensemble, with lc_mlp_forward on the
// device, take the argmin of the (mean) prediction).
//
// The paper leaves the choice of transformations to the controlling program, which can
// react to the target and the workload (Section 1); here that program is a small network
// trained on the autotuner's own timings.  Every feature is O(1) so one network serves
// problems of any size.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lc_internal.h"

namespace lc {

static constexpr int kPickCap = 256;  // candidates the workspace is sized for

static double log2_pos(double x) { return std::log2(std::max(x, 1.0)); }

// The feature vector; the order and scaling are part of the trained network's contract.
static lc_status features(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t path,
                          const lc_variant *v, float *x)
{
    lc_plan p;
    memset(&p, 0, sizeof p);
    p.struct_size = sizeof(lc_plan);
    lc_status st = lc_variant_plan(k, E, N, F, v, &p);
    if (st != LC_OK)
        return st;
    const int eng = v->engine;
    const double units = (double)p.tiles * p.column_blocks / std::max(p.grid, 1);  // tiles per CTA
    const double f[LC_FEATURES] = {
        log2_pos((double)E) / 23.0,
        N / 165.0,
        (N % 16) / 16.0,
        F / 4.0,
        (double)(path == LC_PREC_FP32),
        (double)(path == LC_PREC_BF16),
        (double)(path == LC_PREC_BF16X3),
        (double)(layout == LC_LAYOUT_ELEM_MAJOR),
        (double)(layout == LC_LAYOUT_NODE_MAJOR),
        log2_pos((double)E * N * F) / 32.0,
        (double)p.stacked,
        (double)(std::log2((double)N) / 8.0),
        (double)(eng == LC_ENGINE_SIMT),  // (the K-split engine: zero in all three)
        (double)(eng == LC_ENGINE_TCGEN05),
        (double)(eng == LC_ENGINE_WARP),
        log2_pos((double)v->tile_e) / 10.0,
        eng == LC_ENGINE_TCGEN05 ? v->elems_per_thread / 64.0 : v->elems_per_thread / 8.0,
        v->split_i / 8.0,
        log2_pos((double)v->unroll) / 3.0,
        (double)v->prefetch_smem,
        v->stages / 3.0,
        v->ctas_per_sm / 4.0,
        (double)(v->precision == LC_PREC_FP32),
        (double)(v->precision == LC_PREC_BF16 || v->precision == LC_PREC_BF16X3),
        v->store_rows / 128.0,
        log2_pos((double)p.grid) / 10.0,
        (double)(std::log2(1.0 + units) / 16.0),
        p.column_blocks / 8.0,
        p.smem_bytes / 232448.0,
        p.threads / 1024.0,
        (double)(std::log2(1.0 + (double)p.mma_per_tile * units) / 20.0),
        p.a_buffers / 2.0 + p.out_slots / 8.0,
    };
    for (int q = 0; q < LC_FEATURES; ++q)
        x[q] = (float)f[q];
    return LC_OK;
}

static size_t pick_bytes() { return sizeof(float) * (size_t)kPickCap * (LC_FEATURES + 1); }

}  // namespace lc

extern "C" {

lc_status lc_variant_features(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t precision,
                              const lc_variant *v, float *x)
{
    if (!k || !v || !x)
        return LC_ERR_INVALID_ARGUMENT;
    if (layout != LC_LAYOUT_ELEM_MAJOR && layout != LC_LAYOUT_NODE_MAJOR)
        return LC_ERR_INVALID_ARGUMENT;
    if (precision < LC_PREC_FP64 || precision > LC_PREC_BF16X3)
        return LC_ERR_INVALID_ARGUMENT;
    return lc::features(k, E, N, F, layout, precision, v, x);
}

lc_status lc_pick_workspace_size(size_t *bytes)
{
    if (!bytes)
        return LC_ERR_INVALID_ARGUMENT;
    *bytes = lc::pick_bytes();
    return LC_OK;
}

lc_status lc_pick_variant_ensemble(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout,
                                   int32_t precision, const float *params_dev, int32_t n_models, void *workspace_dev,
                                   size_t workspace_bytes, lc_variant *picked, float *predicted, void *stream)
{
    if (!k || !params_dev || !workspace_dev || !picked || n_models < 1 || n_models > 64)
        return LC_ERR_INVALID_ARGUMENT;
    if (workspace_bytes < lc::pick_bytes())
        return LC_ERR_BUFFER_TOO_SMALL;
    if (((uintptr_t)workspace_dev & 15u) || ((uintptr_t)params_dev & 3u))
        return LC_ERR_MISALIGNED;
    int64_t P = 0;
    lc_status st = lc_mlp_param_count(LC_FEATURES, &P);
    if (st != LC_OK)
        return st;
    std::vector<lc_variant> cand(lc::kPickCap);
    int n = 0;
    st = lc_enumerate_variants(k, E, N, F, layout, precision, cand.data(), lc::kPickCap, &n);
    if (st != LC_OK)
        return st;
    if (n == 0)
        return LC_ERR_UNSUPPORTED;
    std::vector<float> X((size_t)n * LC_FEATURES), y(n), sum(n, 0.f);
    for (int c = 0; c < n; ++c) {
        st = lc::features(k, E, N, F, layout, precision, &cand[c], &X[(size_t)c * LC_FEATURES]);
        if (st != LC_OK)
            return st;
    }
    float *Xd = static_cast<float *>(workspace_dev);
    float *yd = Xd + (size_t)lc::kPickCap * LC_FEATURES;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(Xd, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return lc::cuda_fail(e);
    // the models' predicted log times, averaged in model order
    for (int q = 0; q < n_models; ++q) {
        st = lc_mlp_forward(params_dev + (size_t)q * P, Xd, n, LC_FEATURES, yd, stream);
        if (st != LC_OK)
            return st;
        e = cudaMemcpyAsync(y.data(), yd, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return lc::cuda_fail(e);
        for (int c = 0; c < n; ++c)
            sum[c] += y[c];
    }
    int best = 0;
    for (int c = 1; c < n; ++c)
        if (sum[c] < sum[best])
            best = c;
    *picked = cand[best];
    if (predicted)
        *predicted = sum[best] / (float)n_models;
    return LC_OK;
}

lc_status lc_pick_variant(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t precision,
                          const float *params_dev, void *workspace_dev, size_t workspace_bytes, lc_variant *picked,
                          float *predicted, void *stream)
{
    return lc_pick_variant_ensemble(k, E, N, F, layout, precision, params_dev, 1, workspace_dev, workspace_bytes,
                                    picked, predicted, stream);
}

}  // extern "C"
