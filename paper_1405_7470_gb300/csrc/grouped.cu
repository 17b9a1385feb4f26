// Grouped persistent kernel: several contraction problems (groups with their own N, E,
// operators and buffers) in one launch.  The host cuts the work into (group, column
// block) units and gives each CTA a list of segments, balanced by estimated cost: a unit
// worth at least one CTA gets its own set of CTAs, which stride over its tiles (so the
// CTAs running at one time touch neighbouring tiles, as a grid-stride launch would); the
// small units are packed whole onto the remaining CTAs.  Each CTA walks its segments in
// order, staging the group's D^T block once per segment and running the SIMT tile loop of
// simt.cuh on it.  The launch can be captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include "simt.cuh"

namespace lc {

template <int RE, int RC, int UNR, int LAYOUT, bool PF>
__global__ void __launch_bounds__(simt_max_threads(RE, RC)) grouped_contract_kernel(GroupedArgs g)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int s_begin = g.cta_seg[blockIdx.x], s_end = g.cta_seg[blockIdx.x + 1];
    for (int si = s_begin; si < s_end; ++si) {
        const GroupSeg sg = g.segs[si];
        SimtArgs a = g.groups[sg.group];
        a.err = g.err;
        simt_tiles<float, RE, RC, UNR, LAYOUT, PF>(a, sg.chunk, sg.first, sg.step, sg.first + sg.count * sg.step,
                                                   smem_raw);
    }
}

template <int LAYOUT, int RE, int RC, int UNR>
static void *grouped_pick_pf(int pf)
{
    return pf ? reinterpret_cast<void *>(&grouped_contract_kernel<RE, RC, UNR, LAYOUT, true>)
              : reinterpret_cast<void *>(&grouped_contract_kernel<RE, RC, UNR, LAYOUT, false>);
}

template <int LAYOUT, int RE, int RC>
static void *grouped_pick_unr(int unr, int pf)
{
    switch (unr) {
    case 1: return grouped_pick_pf<LAYOUT, RE, RC, 1>(pf);
    case 4: return grouped_pick_pf<LAYOUT, RE, RC, 4>(pf);
    default: return nullptr;
    }
}

template <int LAYOUT>
static void *grouped_pick(int re, int rc, int unr, int pf)
{
    if (re == 4 && rc == 4) return grouped_pick_unr<LAYOUT, 4, 4>(unr, pf);
    if (re == 4 && rc == 8) return grouped_pick_unr<LAYOUT, 4, 8>(unr, pf);
    if (re == 8 && rc == 4) return grouped_pick_unr<LAYOUT, 8, 4>(unr, pf);
    if (re == 8 && rc == 8) return grouped_pick_unr<LAYOUT, 8, 8>(unr, pf);
    return nullptr;
}

void *grouped_kernel_ptr(int layout, int re, int rc, int unr, int pf)
{
    return layout == LC_LAYOUT_NODE_MAJOR ? grouped_pick<LC_LAYOUT_NODE_MAJOR>(re, rc, unr, pf)
                                          : grouped_pick<LC_LAYOUT_ELEM_MAJOR>(re, rc, unr, pf);
}

}  // namespace lc
