// Instantiates the TMEM-resident stage-grouped decoder kernel for one code
// length, 2^PCBP_LOGN (compiled once per n = 7..11: every lane of a warp owns
// 2^KB positions, KB = tmem_default_kb(n) unless PCBP_KB3 sets it).
#include "bp_kernel3.cuh"
#include "bp_launch.h"

#ifndef PCBP_LOGN
#error "PCBP_LOGN must be defined"
#endif

#define PCBP_CAT2(a, b) a##b
#define PCBP_CAT(a, b) PCBP_CAT2(a, b)

namespace pcbp {

namespace {
#ifndef PCBP_KB3
#define PCBP_KB3 tmem_default_kb(PCBP_LOGN)
#endif
constexpr int KB = PCBP_KB3;   // 2^KB positions per thread
using Geo = G3<PCBP_LOGN, KB>;

// pdl: programmatic dependent launch, the grid may start while the previous
// kernel of the stream still runs (for independent batches).
template <int FK, int WG, int PO = 0>
cudaError_t launch_variant(const BpParams& P, const LaunchGeom& g, cudaStream_t st, bool pdl)
{
    auto kern = bp_decode_tmem_kernel<PCBP_LOGN, KB, FK, WG, PO>;
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
    auto kern = bp_decode_tmem_kernel<PCBP_LOGN, KB, FK, 0, 0>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem)) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, g.slots * Geo::T, g.smem) != cudaSuccess)
        return 0;
    return blocks;
}

// Frame slots a CTA can hold by threads, TMEM columns and named barriers.
constexpr int max_slots()
{
    int slots = tmem_max_threads<PCBP_LOGN, KB>() / Geo::T;
    const int by_tmem = Geo::MAX_WARPS_TMEM / (Geo::T / 32);
    slots = slots < by_tmem ? slots : by_tmem;
    if (Geo::T > 32 && slots > 15) slots = 15;   // named barriers 1..15
    return slots;
}

}  // namespace

void PCBP_CAT(bp3_shape_, PCBP_LOGN)(int* threads_per_slot_out, size_t* slot_bytes_out, int* max_slots_out)
{
    *threads_per_slot_out = Geo::T;
    *slot_bytes_out = tmem_slot_bytes<PCBP_LOGN, KB>();
    *max_slots_out = max_slots();
}

void PCBP_CAT(bp3_tables_, PCBP_LOGN)(int N, int K, size_t* bytes) { *bytes = tmem_cta_bytes<PCBP_LOGN, KB>(N, K); }

int PCBP_CAT(bp3_occupancy_, PCBP_LOGN)(const LaunchGeom& g, int fkind)
{
    return fkind ? occupancy<1>(g) : occupancy<0>(g);
}

cudaError_t PCBP_CAT(bp3_launch_, PCBP_LOGN)(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st,
                                             bool pdl)
{
    // one kernel per f and per G-matrix test, both fixed for a launch
    const bool wg = (P.job.S.stop_kind & 2) != 0;
    if (fkind) return wg ? launch_variant<1, 1>(P, g, st, pdl) : launch_variant<1, 0>(P, g, st, pdl);
    return wg ? launch_variant<0, 1>(P, g, st, pdl) : launch_variant<0, 0>(P, g, st, pdl);
}

// The same kernel with the posterior output (CRC stop or none; P.job.post set).
cudaError_t PCBP_CAT(bp3_launch_post_, PCBP_LOGN)(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st)
{
    if (P.job.S.stop_kind & 2) return cudaErrorInvalidValue;
    return fkind ? launch_variant<1, 0, 1>(P, g, st, false) : launch_variant<0, 0, 1>(P, g, st, false);
}

}  // namespace pcbp
