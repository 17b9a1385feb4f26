// Grouped tensor-core launch: one persistent launch over the groups that have a tensor-core
// plan, each CTA running one (group, column block) unit of its group's own plan (the group's
// B terms staged once, its tiles strided over the unit's CTAs).  The kernel body is the plain
// contraction's (tc.cuh); the epilogue works in 8-column chunks for every group.
#include "tc.cuh"

namespace lc {

lc_status tc_grouped_launch(const TcGroupedParams &P, int layout, int nterms, int grid, int threads, size_t smem,
                            cudaStream_t s, void **fn_out)
{
    // three terms: the instance with tensor-memory A stores when any group's plan uses them
    bool atm = false;
    for (int g = 0; g < P.ngroups; ++g)
        atm = atm || P.g[g].a_tmem;
    static void *const fns[2][3] = {{reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_ELEM_MAJOR, 1>),
                                     reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_ELEM_MAJOR, 3>),
                                     reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_ELEM_MAJOR, 3, true>)},
                                    {reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_NODE_MAJOR, 1>),
                                     reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_NODE_MAJOR, 3>),
                                     reinterpret_cast<void *>(&tc_grouped_kernel<LC_LAYOUT_NODE_MAJOR, 3, true>)}};
    void *fn = fns[layout == LC_LAYOUT_NODE_MAJOR][nterms == 3 ? (atm ? 2 : 1) : 0];
    if (fn_out)
        *fn_out = fn;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (grid <= 0)
        return LC_OK;  // attribute set only (a capture launches later)
    TcGroupedParams p = P;
    void *params[] = {&p};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, smem, s);
    return e == cudaSuccess ? LC_OK : cuda_fail(e);
}

}  // namespace lc
