// Instances of the SIMT contraction kernel: element type double, layout node-major.
#include "simt.cuh"

namespace lc {

lc_status simt_launch_f64_node(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s)
{
    return simt_launch_impl<double, LC_LAYOUT_NODE_MAJOR>(a, g, unroll, prefetch, s);
}

}  // namespace lc
