// Instantiates the stage-grouped decoder kernel for one code length,
// 2^PCBP_LOGN (compiled once per n = 3..11).
#include "bp_kernel2.cuh"
#include "bp_launch.h"

#ifndef PCBP_LOGN
#error "PCBP_LOGN must be defined"
#endif

#define PCBP_CAT2(a, b) a##b
#define PCBP_CAT(a, b) PCBP_CAT2(a, b)

namespace pcbp {

namespace {
#ifndef PCBP_KB
#define PCBP_KB 2
#endif
// 2^KB positions per thread (at most n); 4 measured fastest at N=1024 (3.27 Gbit/s vs 3.09 with 8, 1.69 with 16)
constexpr int KBSEL = PCBP_LOGN < PCBP_KB ? PCBP_LOGN : PCBP_KB;
using Geo = G2<PCBP_LOGN, KBSEL>;

// pdl: programmatic dependent launch, the grid may start while the previous
// kernel of the stream still runs (for independent batches).
template <int FK>
cudaError_t launch_variant(const BpParams& P, const LaunchGeom& g, cudaStream_t st, bool pdl)
{
    auto kern = bp_decode_grouped_kernel<PCBP_LOGN, KBSEL, FK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem));
    if (e != cudaSuccess) return e;
    if (!pdl) {
        kern<<<g.grid, g.slots * Geo::T, g.smem, st>>>(P);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(g.grid));
    cfg.blockDim = dim3(unsigned(g.slots * Geo::T));
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P);
}

template <int FK>
int occupancy(const LaunchGeom& g)
{
    auto kern = bp_decode_grouped_kernel<PCBP_LOGN, KBSEL, FK>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem)) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, g.slots * Geo::T, g.smem) != cudaSuccess)
        return 0;
    return blocks;
}
}  // namespace

void PCBP_CAT(bp2_shape_, PCBP_LOGN)(int* threads_per_slot_out, size_t* slot_bytes_out, int* max_slots_out)
{
    *threads_per_slot_out = Geo::T;
    *slot_bytes_out = align16(sizeof(GroupCtl<PCBP_LOGN, KBSEL>)) + align16(2 * Geo::NW * 4) +
                      size_t(2 * Geo::NPL) * Geo::N * 4;
    const int by_threads = grouped_max_threads<KBSEL>() / Geo::T;
    *max_slots_out = Geo::T == 32 ? by_threads : (by_threads < 15 ? by_threads : 15);
}

int PCBP_CAT(bp2_occupancy_, PCBP_LOGN)(const LaunchGeom& g, int fkind)
{
    return fkind ? occupancy<1>(g) : occupancy<0>(g);
}

cudaError_t PCBP_CAT(bp2_launch_, PCBP_LOGN)(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st,
                                             bool pdl)
{
    return fkind ? launch_variant<1>(P, g, st, pdl) : launch_variant<0>(P, g, st, pdl);
}

}  // namespace pcbp
