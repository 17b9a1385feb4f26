// Tensor-core contraction: the kernel instances of the plain contraction (one output per
// operator) and their launcher.  The kernel template is in tc.cuh.
#include "tc.cuh"

namespace lc {

lc_status tc_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s)
{
    // kernel instance per (layout, terms, epilogue chunk width)
    static void *const fns[2][2][2] = {
        {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 8, 0>),
          reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 1, 16, 0>)},
         {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 8, 0>),
          reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 16, 0>)}},
        {{reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 8, 0>),
          reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 1, 16, 0>)},
         {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 8, 0>),
          reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 16, 0>)}}};
    return tc_launch_fn(fns[layout == LC_LAYOUT_NODE_MAJOR][nterms == 3][a.chunk == 16], a, grid, s);
}

}  // namespace lc
