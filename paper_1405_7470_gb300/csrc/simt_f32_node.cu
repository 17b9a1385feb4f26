// Instances of the SIMT contraction kernel: element type float, layout node-major.
#include "simt.cuh"

namespace lc {

lc_status simt_launch_f32_node(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s)
{
    return simt_launch_impl<float, LC_LAYOUT_NODE_MAJOR>(a, g, unroll, prefetch, s);
}

}  // namespace lc
