// Volume derivative with per-element geometric factors: the node-major kernel instances
// (the template is in tc.cuh, the element-major instances and the launcher in tc_geo.cu).
#include "tc.cuh"

namespace lc {

lc_status tc_geo_launch_node(const TcArgs &a, int nterms, int grid, cudaStream_t s)
{
    static void *const fns[2][2] = {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 8, 2>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 8, 3>)},
                                    {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 8, 2>),
                                     reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 8, 3>)}};
    return tc_launch_fn(fns[nterms == 3][a.F == 3], a, grid, s);
}

}  // namespace lc
