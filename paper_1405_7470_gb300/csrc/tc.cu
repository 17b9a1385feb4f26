// Tensor-core contraction: the element-major kernel instances of the plain contraction (one
// output per operator) and the launcher.  The kernel template is in tc.cuh; the node-major
// instances are in tc_node.cu (separate translation units compile in parallel).
#include "tc.cuh"

namespace lc {

lc_status tc_launch_node(const TcArgs &a, int nterms, int grid, cudaStream_t s);
lc_status tc_launch_tmem3(const TcArgs &a, int layout, int grid, cudaStream_t s);

lc_status tc_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s)
{
    if (nterms == 3 && a.a_tmem)
        return tc_launch_tmem3(a, layout, grid, s);  // three terms, A in tensor memory (tc_tmem3.cu)
    if (layout == LC_LAYOUT_NODE_MAJOR)
        return tc_launch_node(a, nterms, grid, s);  // the node-major instances (tc_node.cu)
    // element-major instance per (terms, epilogue chunk width)
    static void *const fns[2][2] = {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 8, 0>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 16, 0>)},
                                    {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 8, 0>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 16, 0>)}};
    return tc_launch_fn(fns[nterms == 3][a.chunk == 16], a, grid, s);
}

}  // namespace lc
