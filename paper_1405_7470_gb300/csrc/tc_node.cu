// Tensor-core contraction: the node-major kernel instances (the template is in tc.cuh).
#include "tc.cuh"

namespace lc {

lc_status tc_launch_node(const TcArgs &a, int nterms, int grid, cudaStream_t s)
{
    static void *const fns[2][2] = {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 8, 0>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 16, 0>)},
                                    {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 8, 0>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 16, 0>)}};
    return tc_launch_fn(fns[nterms == 3][a.chunk == 16], a, grid, s);
}

}  // namespace lc
