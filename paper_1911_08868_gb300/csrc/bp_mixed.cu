// Mixed-length batched decoding: one persistent launch decodes several
// batches, each with its own code (length N, rate, CRC) and schedule.
//
// Every CTA walks the batch list in order.  For each batch it loads that
// code's tables into shared memory, splits its threads into the batch's frame
// slots (threads per slot and slot size depend on N) and decodes frames
// fetched from the batch's own counter until the batch is exhausted, then
// moves on.  CTAs thus drain the batches together, with no gap between sizes
// and no tail per size.  The per-batch device descriptors (code tables,
// schedule, buffers) are prepared on the host into a caller buffer and
// uploaded once, so the launch itself is a memset and one kernel: it can be
// captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "bp_kernel2.cuh"
#include "pcbp_internal.h"

#ifndef PCBP_KB
#define PCBP_KB 2
#endif

namespace pcbp {

constexpr int kMixedKB = PCBP_KB;
constexpr int kMixedThreads = grouped_max_threads<kMixedKB>();

struct MixedBatch {
    DevCode code;
    FrameJob job;
    int32_t slots;
    int32_t pad;
};

namespace {

// One runtime-length body serves every batch (a body per length would put
// nine copies of the decoder into one kernel and exhaust its registers).
__global__ void __launch_bounds__(kMixedThreads, 1)
    bp_decode_mixed_kernel(const MixedBatch* __restrict__ batches, int nb, unsigned long long* counters)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_skip;
    for (int b = 0; b < nb; ++b) {
        const MixedBatch* mb = batches + b;
        if (threadIdx.x == 0) {
            const unsigned long long c = *reinterpret_cast<volatile unsigned long long*>(counters + b);
            s_skip = c >= (unsigned long long)mb->job.B ? 1 : 0;
        }
        __syncthreads();
        const bool skip = s_skip != 0;
        __syncthreads();
        if (skip) continue;
        const int n = mb->code.n;
        load_code_tables(mb->code, smem);
        __syncthreads();
        const int N = 1 << n;
        const int TA = N >> kMixedKB;
        const int T = TA < 32 ? 32 : TA;
        if (int(threadIdx.x) < mb->slots * T) grouped_frames<0, kMixedKB, 0>(mb->job, counters + b, smem, n);
        __syncthreads();
    }
}

void mixed_shape(int n, int* T, size_t* slot)
{
    const int N = 1 << n;
    const int TA = N >> kMixedKB;
    const int NW = N >= 32 ? N / 32 : 1;
    *T = TA < 32 ? 32 : TA;
    *slot = align16(sizeof(GroupCtl<kMaxLogN, kMixedKB>)) + align16(size_t(2 * NW * 4)) + size_t(2 * (n - 1)) * N * 4;
}

size_t mixed_tables(const pc_code* c)
{
    const size_t nw = size_t(c->N >= 32 ? c->N / 32 : 1);
    return ((nw * 4 + size_t(c->crc_len) * nw * 4 + size_t(c->K) * 2 + 15) & ~size_t(15)) + kSwzTableBytes;
}

int smem_optin(int* out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PC_ECUDA;
    if (cudaDeviceGetAttribute(out, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return PC_ECUDA;
    *out -= 1024;   // the kernel's own static shared variables
    return PC_OK;
}

// Frame slots of one batch: the requested count, else as many as fit.
int batch_slots(const pc_batch& b, int smem_limit, int* slots_out, size_t* smem_out, int* threads_out)
{
    int T = 0;
    size_t slot = 0;
    mixed_shape(b.code->n, &T, &slot);
    const size_t tab = mixed_tables(b.code);
    if (tab + slot > size_t(smem_limit)) return PC_EUNSUPPORTED;
    int max_slots = int((size_t(smem_limit) - tab) / slot);
    max_slots = std::min(max_slots, kMixedThreads / T);
    if (T > 32) max_slots = std::min(max_slots, 15);
    max_slots = std::max(max_slots, 1);
    const int slots = b.slots > 0 ? std::min(b.slots, max_slots) : max_slots;
    *slots_out = slots;
    *smem_out = tab + size_t(slots) * slot;
    *threads_out = slots * T;
    return PC_OK;
}

int validate_batch(const pc_batch& b)
{
    int rc = validate_code(b.code);
    if (rc != PC_OK) return rc;
    rc = validate_sched(b.code, &b.sched);
    if (rc != PC_OK) return rc;
    if (b.sched.fkind != 0) return PC_EUNSUPPORTED;
    if (b.max_iters < 0 || b.B < 0 || b.slots < 0) return PC_EINVAL;
    if (b.B > 0) {
        if (!b.d_llr || !b.d_bits || !b.d_iters || !b.d_crc_ok) return PC_EINVAL;
        if (reinterpret_cast<uintptr_t>(b.d_llr) & 15u) return PC_EINVAL;
    }
    return PC_OK;
}

}  // namespace

}  // namespace pcbp

using namespace pcbp;

extern "C" int bp_mixed_table_size(int32_t n_batches, size_t* bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || !bytes) return PC_EINVAL;
    *bytes = sizeof(MixedBatch) * size_t(n_batches);
    return PC_OK;
}

extern "C" int bp_mixed_prepare(const pc_batch* batches, int32_t n_batches, void* h_table, size_t bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || (n_batches > 0 && (!batches || !h_table))) return PC_EINVAL;
    if (bytes < sizeof(MixedBatch) * size_t(n_batches)) return PC_ENOMEM;
    MixedBatch* out = static_cast<MixedBatch*>(h_table);
    for (int i = 0; i < n_batches; ++i) {
        const int rc = validate_batch(batches[i]);
        if (rc != PC_OK) return rc;
    }
    int limit = 0;
    if (n_batches > 0) {
        const int rl = smem_optin(&limit);
        if (rl != PC_OK) return rl;
    }
    for (int i = 0; i < n_batches; ++i) {
        const pc_batch& b = batches[i];
        MixedBatch mb;
        std::memset(&mb, 0, sizeof(mb));
        build_dev_code(b.code, &mb.code);
        build_dev_sched(&b.sched, &mb.job.S);
        mb.job.llr = b.d_llr;
        mb.job.bits = b.d_bits;
        mb.job.iters = b.d_iters;
        mb.job.crc_ok = b.d_crc_ok;
        mb.job.B = b.B;
        mb.job.max_iters = b.max_iters;
        mb.job.K = b.code->K;
        mb.job.r = b.code->crc_len;
        int slots = 0, th = 0;
        size_t sm = 0;
        const int rs = batch_slots(b, limit, &slots, &sm, &th);
        if (rs != PC_OK) return rs;
        mb.slots = slots;
        std::memcpy(out + i, &mb, sizeof(mb));
    }
    return PC_OK;
}

extern "C" int bp_mixed_workspace_size(int32_t n_batches, size_t* bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || !bytes) return PC_EINVAL;
    *bytes = (sizeof(unsigned long long) * size_t(n_batches) + 255) & ~size_t(255);
    if (*bytes == 0) *bytes = 256;
    return PC_OK;
}

extern "C" int bp_decode_mixed(const pc_batch* batches, int32_t n_batches, void* d_table, void* d_workspace,
                               void* stream)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || (n_batches > 0 && !batches)) return PC_EINVAL;
    if (n_batches == 0) return PC_OK;
    if (!d_table || !d_workspace) return PC_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_table) & 15u) || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return PC_EINVAL;
    int rc = PC_OK;
    for (int i = 0; i < n_batches; ++i) {
        rc = validate_batch(batches[i]);
        if (rc != PC_OK) return rc;
    }
    int limit = 0;
    rc = smem_optin(&limit);
    if (rc != PC_OK) return rc;
    size_t smem = 0;
    int threads = 32;
    int slots_of[PC_MAX_BATCHES];
    for (int i = 0; i < n_batches; ++i) {
        size_t sm = 0;
        int th = 0;
        rc = batch_slots(batches[i], limit, &slots_of[i], &sm, &th);
        if (rc != PC_OK) return rc;
        smem = std::max(smem, sm);
        threads = std::max(threads, th);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    MixedBatch* d_mb = static_cast<MixedBatch*>(d_table);
    size_t ws = 0;
    bp_mixed_workspace_size(n_batches, &ws);
    if (cudaMemsetAsync(d_workspace, 0, ws, st) != cudaSuccess) return PC_ECUDA;
    if (cudaFuncSetAttribute(bp_decode_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
        cudaSuccess)
        return PC_ECUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bp_decode_mixed_kernel, threads, smem) != cudaSuccess ||
        occ < 1)
        return PC_EUNSUPPORTED;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PC_ECUDA;
    int64_t total = 0;
    for (int i = 0; i < n_batches; ++i) total += batches[i].B;
    if (total == 0) return PC_OK;
    const int grid = int(std::min<int64_t>(int64_t(sms) * occ, std::max<int64_t>(1, total)));
    bp_decode_mixed_kernel<<<grid, threads, smem, st>>>(d_mb, n_batches,
                                                         reinterpret_cast<unsigned long long*>(d_workspace));
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ECUDA;
}
