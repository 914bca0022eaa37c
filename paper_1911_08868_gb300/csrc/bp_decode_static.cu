// bp_decode_noalloc: bp_decode for callers that cannot allocate device memory
// while they decode.  Real-time signal-processing pipelines typically
// allocate everything at start-up, because cudaMalloc synchronises the device
// and its latency is unbounded; other hosts own all device memory through
// their own allocator.  Such callers cannot hand bp_decode a workspace, so
// this entry point keeps the decoder's scratch (its frame counter) in a
// file-scope device array instead.
//
// The array is PC_STATIC_SCRATCH_BYTES long and lives on every GPU that loads
// this library until the process exits.  Host code cannot use the array's
// name as a device address (in host code it only stands in for the symbol),
// so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call therefore has to come before any stream
// capture.  Every call shares the array and its contents persist between
// calls: the decoder clears the counter on the stream at the start of each
// call, and calls that overlap on the GPU race on it.  The cached address is
// that of the device's context at the first call; after cudaDeviceReset it is
// stale, so a process that resets a device must not call this entry point on
// it again.  In a PCBP_CHECKED build the range-check status word also lands in
// the array, where callers cannot read it (bp_decode reports it).
#include <cuda_runtime.h>

#include <mutex>

#include "pcbp.h"

namespace {

static __device__ __align__(256) unsigned char g_decode_scratch[PC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_decode_scratch on the current device (looked up once).
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PC_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_decode_scratch) != cudaSuccess || !p) return PC_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PC_OK;
}

}  // namespace

extern "C" int bp_decode_noalloc(const pc_code* code, const float* d_llr, const pc_sched* sched, int32_t max_iters,
                                 int64_t B, uint32_t* d_bits, int32_t* d_iters, uint8_t* d_crc_ok, void* stream)
{
    size_t need = 0;
    int rc = bp_decode_workspace_size(code, B, &need);
    if (rc != PC_OK) return rc;
    if (need > PC_STATIC_SCRATCH_BYTES) return PC_EUNSUPPORTED;
    if (B == 0)  // validated by bp_decode; nothing is launched, no device call is made
        return bp_decode(code, d_llr, sched, max_iters, B, d_bits, d_iters, d_crc_ok, nullptr, stream);
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != PC_OK) return rc;
    return bp_decode(code, d_llr, sched, max_iters, B, d_bits, d_iters, d_crc_ok, scratch, stream);
}
