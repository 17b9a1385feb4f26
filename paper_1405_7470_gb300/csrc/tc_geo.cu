// Tensor-core volume derivative with per-element geometric factors (the dG FEM volume
// workload of Table 1 with the chain rule applied in the kernel's epilogue):
//     out[d,e,i] = sum_f r[e,d,f] * sum_j D[f,i,j] * u[e,j],   d, f < F
// The kernel template is in tc.cuh (instances with FG = F); the contraction part is the
// same pipeline as the plain kernel, the F partial sums of a node never leave the SM.
#include "tc.cuh"

namespace lc {

lc_status tc_geo_launch_node(const TcArgs &a, int nterms, int grid, cudaStream_t s);

lc_status tc_geo_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s)
{
    if (a.F < 2 || a.F > 3 || a.chunk != 8)
        return LC_ERR_INVALID_VARIANT;
    if (layout == LC_LAYOUT_NODE_MAJOR)
        return tc_geo_launch_node(a, nterms, grid, s);  // node-major instances (tc_geo_node.cu)
    // element-major instance per (terms, operators); 8-column epilogue chunks
    static void *const fns[2][2] = {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 8, 2>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 8, 3>)},
                                    {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 8, 2>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 8, 3>)}};
    return tc_launch_fn(fns[nterms == 3][a.F == 3], a, grid, s);
}

}  // namespace lc
