// Instantiates the decoder kernels for one code length, 2^PCBP_LOGN.  The
// build compiles this file once per supported n (3..11) so that the
// translation units compile in parallel.
#include "bp_kernel.cuh"
#include "bp_launch.h"

#ifndef PCBP_LOGN
#error "PCBP_LOGN must be defined"
#endif

#define PCBP_CAT2(a, b) a##b
#define PCBP_CAT(a, b) PCBP_CAT2(a, b)

namespace pcbp {

namespace {
template <bool TRACE, int FK>
cudaError_t launch_variant(const BpParams& P, const LaunchGeom& g, cudaStream_t st)
{
    constexpr int T = threads_per_slot<PCBP_LOGN>();
    auto kern = bp_decode_kernel<PCBP_LOGN, T, TRACE, FK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem));
    if (e != cudaSuccess) return e;
    kern<<<g.grid, g.slots * T, g.smem, st>>>(P);
    return cudaGetLastError();
}

template <bool TRACE, int FK>
int occupancy(const LaunchGeom& g)
{
    constexpr int T = threads_per_slot<PCBP_LOGN>();
    auto kern = bp_decode_kernel<PCBP_LOGN, T, TRACE, FK>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem)) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, g.slots * T, g.smem) != cudaSuccess) return 0;
    return blocks;
}
}  // namespace

void PCBP_CAT(bp_shape_, PCBP_LOGN)(int* threads_per_slot_out, size_t* slot_bytes_out)
{
    *threads_per_slot_out = threads_per_slot<PCBP_LOGN>();
    *slot_bytes_out = slot_bytes<PCBP_LOGN>();
}

int PCBP_CAT(bp_occupancy_, PCBP_LOGN)(const LaunchGeom& g, bool trace, int fkind)
{
    if (trace) return fkind ? occupancy<true, 1>(g) : occupancy<true, 0>(g);
    return fkind ? occupancy<false, 1>(g) : occupancy<false, 0>(g);
}

cudaError_t PCBP_CAT(bp_launch_, PCBP_LOGN)(const BpParams& P, const LaunchGeom& g, bool trace, int fkind,
                                             cudaStream_t st)
{
    if (trace) return fkind ? launch_variant<true, 1>(P, g, st) : launch_variant<true, 0>(P, g, st);
    return fkind ? launch_variant<false, 1>(P, g, st) : launch_variant<false, 0>(P, g, st);
}

}  // namespace pcbp
