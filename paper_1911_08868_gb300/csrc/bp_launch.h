// Per-length launch entry points of the decoder kernels (one set per n):
// bp_* from bp_inst.cu (per-stage kernel, used for the trace entry), bp2_*
// from bp_inst2.cu (stage-grouped kernel, bp_decode for n < 7), bp3_* from
// bp_inst3.cu (stage-grouped kernel with TMEM-resident group interiors,
// bp_decode for n = 7..11).
#pragma once

#include <cuda_runtime.h>

#include "pcbp_internal.h"

namespace pcbp {

struct LaunchGeom {
    int grid;
    int slots;
    size_t smem;
};

#define PCBP_DECLARE_LEN(n)                                                                              \
    void bp_shape_##n(int* threads_per_slot_out, size_t* slot_bytes_out);                                \
    int bp_occupancy_##n(const LaunchGeom& g, bool trace, int fkind);                                    \
    cudaError_t bp_launch_##n(const BpParams& P, const LaunchGeom& g, bool trace, int fkind, cudaStream_t st); \
    void bp2_shape_##n(int* threads_per_slot_out, size_t* slot_bytes_out, int* max_slots_out);            \
    int bp2_occupancy_##n(const LaunchGeom& g, int fkind);                                                \
    cudaError_t bp2_launch_##n(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st, bool pdl);

PCBP_DECLARE_LEN(3)
PCBP_DECLARE_LEN(4)
PCBP_DECLARE_LEN(5)
PCBP_DECLARE_LEN(6)
PCBP_DECLARE_LEN(7)
PCBP_DECLARE_LEN(8)
PCBP_DECLARE_LEN(9)
PCBP_DECLARE_LEN(10)
PCBP_DECLARE_LEN(11)

#undef PCBP_DECLARE_LEN

#define PCBP_DECLARE_LEN3(n)                                                                  \
    void bp3_shape_##n(int* threads_per_slot_out, size_t* slot_bytes_out, int* max_slots_out); \
    void bp3_tables_##n(int N, int K, size_t* bytes);                                          \
    int bp3_occupancy_##n(const LaunchGeom& g, int fkind);                                     \
    cudaError_t bp3_launch_##n(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st, bool pdl); \
    cudaError_t bp3_launch_post_##n(const BpParams& P, const LaunchGeom& g, int fkind, cudaStream_t st);

PCBP_DECLARE_LEN3(7)
PCBP_DECLARE_LEN3(8)
PCBP_DECLARE_LEN3(9)
PCBP_DECLARE_LEN3(10)
PCBP_DECLARE_LEN3(11)

#undef PCBP_DECLARE_LEN3

}  // namespace pcbp
