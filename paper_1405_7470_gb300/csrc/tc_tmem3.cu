// Tensor-core contraction, three-term split (BF16X3) with the A terms in tensor memory: the
// plans for large N whose shared-memory plan does not fit (both layouts, both epilogue chunk
// widths).  The kernel template is in tc.cuh.
#include "tc.cuh"

namespace lc {

lc_status tc_launch_tmem3(const TcArgs &a, int layout, int grid, cudaStream_t s)
{
    static void *const fns[2][2] = {
        {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 8, 0, true>),
         reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_ELEM_MAJOR, 3, 16, 0, true>)},
        {reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 8, 0, true>),
         reinterpret_cast<void *>(&tc_contract_kernel<LC_LAYOUT_NODE_MAJOR, 3, 16, 0, true>)}};
    return tc_launch_fn(fns[layout == LC_LAYOUT_NODE_MAJOR][a.chunk == 16], a, grid, s);
}

}  // namespace lc
