// Instances of the SIMT contraction kernel: element type float, layout elem-major.
#include "simt.cuh"

namespace lc {

lc_status simt_launch_f32_elem(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s)
{
    return simt_launch_impl<float, LC_LAYOUT_ELEM_MAJOR>(a, g, unroll, prefetch, s);
}

}  // namespace lc
