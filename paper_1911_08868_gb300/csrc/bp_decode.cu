// C-ABI entry points of libpcbp: pc_encode, bp_decode, bp_decode_trace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "bp_launch.h"
#include "pcbp_internal.h"

namespace pcbp {

namespace {

struct DeviceInfo {
    int sms = 0;
    int smem_optin = 0;
    int smem_per_sm = 0;
};

int device_info(DeviceInfo* out)
{
    static DeviceInfo cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return PC_ECUDA;
    if (dev < 64 && cache[dev].sms > 0) {
        *out = cache[dev];
        return PC_OK;
    }
    DeviceInfo d;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PC_ECUDA;
    if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return PC_ECUDA;
    if (cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return PC_ECUDA;
    if (dev < 64) cache[dev] = d;
    *out = d;
    return PC_OK;
}

void shape_of(int n, int* T, size_t* slot)
{
    switch (n) {
        case 3: bp_shape_3(T, slot); break;
        case 4: bp_shape_4(T, slot); break;
        case 5: bp_shape_5(T, slot); break;
        case 6: bp_shape_6(T, slot); break;
        case 7: bp_shape_7(T, slot); break;
        case 8: bp_shape_8(T, slot); break;
        case 9: bp_shape_9(T, slot); break;
        case 10: bp_shape_10(T, slot); break;
        default: bp_shape_11(T, slot); break;
    }
}

int occupancy_of(int n, const LaunchGeom& g, bool trace, int fk)
{
    switch (n) {
        case 3: return bp_occupancy_3(g, trace, fk);
        case 4: return bp_occupancy_4(g, trace, fk);
        case 5: return bp_occupancy_5(g, trace, fk);
        case 6: return bp_occupancy_6(g, trace, fk);
        case 7: return bp_occupancy_7(g, trace, fk);
        case 8: return bp_occupancy_8(g, trace, fk);
        case 9: return bp_occupancy_9(g, trace, fk);
        case 10: return bp_occupancy_10(g, trace, fk);
        default: return bp_occupancy_11(g, trace, fk);
    }
}

cudaError_t launch_of(int n, const BpParams& P, const LaunchGeom& g, bool trace, int fk, cudaStream_t st)
{
    switch (n) {
        case 3: return bp_launch_3(P, g, trace, fk, st);
        case 4: return bp_launch_4(P, g, trace, fk, st);
        case 5: return bp_launch_5(P, g, trace, fk, st);
        case 6: return bp_launch_6(P, g, trace, fk, st);
        case 7: return bp_launch_7(P, g, trace, fk, st);
        case 8: return bp_launch_8(P, g, trace, fk, st);
        case 9: return bp_launch_9(P, g, trace, fk, st);
        case 10: return bp_launch_10(P, g, trace, fk, st);
        default: return bp_launch_11(P, g, trace, fk, st);
    }
}

#define PCBP_SWITCH_N(n, call)                      \
    switch (n) {                                    \
        case 3: call(3); break;                     \
        case 4: call(4); break;                     \
        case 5: call(5); break;                     \
        case 6: call(6); break;                     \
        case 7: call(7); break;                     \
        case 8: call(8); break;                     \
        case 9: call(9); break;                     \
        case 10: call(10); break;                   \
        default: call(11); break;                   \
    }

void shape2_of(int n, int* T, size_t* slot, int* max_slots)
{
#define PCBP_SHAPE2(k) bp2_shape_##k(T, slot, max_slots)
    PCBP_SWITCH_N(n, PCBP_SHAPE2)
#undef PCBP_SHAPE2
}

int occupancy2_of(int n, const LaunchGeom& g, int fk)
{
    int occ = 0;
#define PCBP_OCC2(k) occ = bp2_occupancy_##k(g, fk)
    PCBP_SWITCH_N(n, PCBP_OCC2)
#undef PCBP_OCC2
    return occ;
}

cudaError_t launch2_of(int n, const BpParams& P, const LaunchGeom& g, int fk, cudaStream_t st, bool pdl)
{
    cudaError_t e = cudaSuccess;
#define PCBP_LAUNCH2(k) e = bp2_launch_##k(P, g, fk, st, pdl)
    PCBP_SWITCH_N(n, PCBP_LAUNCH2)
#undef PCBP_LAUNCH2
    return e;
}

void shape3_of(int n, int* T, size_t* slot, int* max_slots)
{
    switch (n) {
        case 7: bp3_shape_7(T, slot, max_slots); break;
        case 8: bp3_shape_8(T, slot, max_slots); break;
        case 9: bp3_shape_9(T, slot, max_slots); break;
        case 10: bp3_shape_10(T, slot, max_slots); break;
        default: bp3_shape_11(T, slot, max_slots); break;
    }
}

int occupancy3_of(int n, const LaunchGeom& g, int fk)
{
    switch (n) {
        case 7: return bp3_occupancy_7(g, fk);
        case 8: return bp3_occupancy_8(g, fk);
        case 9: return bp3_occupancy_9(g, fk);
        case 10: return bp3_occupancy_10(g, fk);
        default: return bp3_occupancy_11(g, fk);
    }
}

cudaError_t launch3_post_of(int n, const BpParams& P, const LaunchGeom& g, int fk, cudaStream_t st)
{
    switch (n) {
        case 7: return bp3_launch_post_7(P, g, fk, st);
        case 8: return bp3_launch_post_8(P, g, fk, st);
        case 9: return bp3_launch_post_9(P, g, fk, st);
        case 10: return bp3_launch_post_10(P, g, fk, st);
        default: return bp3_launch_post_11(P, g, fk, st);
    }
}

cudaError_t launch3_of(int n, const BpParams& P, const LaunchGeom& g, int fk, cudaStream_t st, bool pdl)
{
    switch (n) {
        case 7: return bp3_launch_7(P, g, fk, st, pdl);
        case 8: return bp3_launch_8(P, g, fk, st, pdl);
        case 9: return bp3_launch_9(P, g, fk, st, pdl);
        case 10: return bp3_launch_10(P, g, fk, st, pdl);
        default: return bp3_launch_11(P, g, fk, st, pdl);
    }
}

void tmem_tables_of(const pc_code* c, size_t* bytes)
{
    switch (c->n) {
        case 7: bp3_tables_7(c->N, c->K, bytes); break;
        case 8: bp3_tables_8(c->N, c->K, bytes); break;
        case 9: bp3_tables_9(c->N, c->K, bytes); break;
        case 10: bp3_tables_10(c->N, c->K, bytes); break;
        default: bp3_tables_11(c->N, c->K, bytes); break;
    }
}

// The TMEM kernel serves n = 7..11 (groups of 2 stages at n = 7, of 3 from
// n = 8) unless PCBP_DECODER=grouped selects the shared-memory-only kernel
// (both give identical outputs).
bool use_tmem_kernel(int n)
{
    if (n < 7 || n > 11) return false;
    const char* v = std::getenv("PCBP_DECODER");
    return !(v && std::strcmp(v, "grouped") == 0);
}

// Threads per frame of the TMEM kernel built for n (N / 2^KB), 0 where it has no build.
int tmem_threads_per_frame(int n)
{
    if (n < 7 || n > 11) return 0;
    int T = 0, max_slots = 0;
    size_t slot = 0;
    shape3_of(n, &T, &slot, &max_slots);
    return T;
}

// The kernel a batch asking for tpf threads per frame runs (tpf valid): at
// N = 128 both kernels take 32 threads per frame, and the choice follows
// use_tmem_kernel.
bool tmem_for(int n, int N, int tpf)
{
    if (tpf == 0) return use_tmem_kernel(n);
    if (tpf != tmem_threads_per_frame(n)) return false;
    return tpf != std::max(32, N / 4) || use_tmem_kernel(n);
}

size_t table_bytes(int N, int r, int K)
{
    const size_t nw = size_t(N >= 32 ? N / 32 : 1);
    return (nw * 4 + size_t(r) * nw * 4 + size_t(K) * 2 + 15) & ~size_t(15);
}

// Slots per CTA: as many frames as shared memory holds, at most 15 (named
// barriers 1..15) and at most 1024 threads.
int plan_launch(const pc_code* c, int64_t B, bool trace, int fk, LaunchGeom* g)
{
    DeviceInfo di;
    int rc = device_info(&di);
    if (rc != PC_OK) return rc;
    int T = 0;
    size_t slot = 0;
    shape_of(c->n, &T, &slot);
    const size_t tab = table_bytes(c->N, c->crc_len, c->K);
    if (tab + slot > size_t(di.smem_optin)) return PC_EUNSUPPORTED;
    int slots = int((size_t(di.smem_optin) - tab) / slot);
    slots = std::min(slots, 15);
    slots = std::min(slots, 1024 / T);
    slots = std::max(slots, 1);
    g->slots = slots;
    g->smem = tab + size_t(slots) * slot;
    g->grid = 1;
    int occ = occupancy_of(c->n, *g, trace, fk);
    if (occ < 1) return PC_EUNSUPPORTED;
    const int64_t need = (B + slots - 1) / slots;
    g->grid = int(std::min<int64_t>(need, int64_t(di.sms) * occ));
    return PC_OK;
}

// Stage-grouped kernel: as many slots as shared memory and the block limit
// allow (at most slots_req when that is positive).
int plan_launch2(const pc_code* c, int64_t B, int fk, LaunchGeom* g, int slots_req = 0)
{
    DeviceInfo di;
    int rc = device_info(&di);
    if (rc != PC_OK) return rc;
    int T = 0, max_slots = 0;
    size_t slot = 0;
    shape2_of(c->n, &T, &slot, &max_slots);
    const size_t tab = table_bytes(c->N, c->crc_len, c->K) + 64;   // + the 64-byte swizzle table
    if (tab + slot > size_t(di.smem_optin)) return PC_EUNSUPPORTED;
    int slots = int((size_t(di.smem_optin) - tab) / slot);
    slots = std::max(1, std::min(slots, max_slots));
    if (slots_req > 0) slots = std::min(slots, slots_req);
    g->slots = slots;
    g->smem = tab + size_t(slots) * slot;
    g->grid = 1;
    const int occ = occupancy2_of(c->n, *g, fk);
    if (occ < 1) return PC_EUNSUPPORTED;
    const int64_t need = (B + slots - 1) / slots;
    g->grid = int(std::min<int64_t>(need, int64_t(di.sms) * occ));
    return PC_OK;
}

// TMEM kernel: slots as for the stage-grouped kernel, then at least half an
// SM's shared memory per CTA, so that one CTA per SM holds all 512 TMEM
// columns and no allocation ever waits for another CTA.
int plan_launch3(const pc_code* c, int64_t B, int fk, LaunchGeom* g, int slots_req = 0)
{
    DeviceInfo di;
    int rc = device_info(&di);
    if (rc != PC_OK) return rc;
    int T = 0, max_slots = 0;
    size_t slot = 0;
    shape3_of(c->n, &T, &slot, &max_slots);
    size_t tab = 0;
    tmem_tables_of(c, &tab);
    if (tab + slot > size_t(di.smem_optin)) return PC_EUNSUPPORTED;
    int slots = int((size_t(di.smem_optin) - tab) / slot);
    slots = std::max(1, std::min(slots, max_slots));
    if (slots_req > 0) slots = std::min(slots, slots_req);
    g->slots = slots;
    g->smem = std::max(tab + size_t(slots) * slot, size_t(di.smem_per_sm) / 2 + 1024);
    if (g->smem > size_t(di.smem_optin)) return PC_EUNSUPPORTED;
    g->grid = 1;
    const int occ = occupancy3_of(c->n, *g, fk);
    if (occ != 1) return PC_EUNSUPPORTED;
    const int64_t need = (B + slots - 1) / slots;
    g->grid = int(std::min<int64_t>(need, int64_t(di.sms)));
    return PC_OK;
}

int validate_events(const pc_code* c, const pc_event* ev, int n_ev)
{
    if (n_ev < 0 || n_ev > PC_MAX_EVENTS) return PC_EINVAL;
    if (n_ev > 0 && !ev) return PC_EINVAL;
    for (int k = 0; k < n_ev; ++k) {
        const pc_event& e = ev[k];
        if (e.range < 2 || e.range > 16 || e.level < 1 || e.level + e.range - 1 > c->n) return PC_EINVAL;
        const int m = e.level + e.range - 1;
        if (e.block < 0 || e.block >= (int64_t(1) << (c->n - m))) return PC_EINVAL;
        unsigned seen = 0;
        for (int i = 0; i < e.range; ++i) {
            if (e.order[i] < 0 || e.order[i] >= e.range || ((seen >> e.order[i]) & 1u)) return PC_EINVAL;
            seen |= 1u << e.order[i];
        }
    }
    return PC_OK;
}

// Kernel parameters of one batch (no device calls).
void fill_params(const pc_code* code, const float* d_llr, const pc_sched* sched, int32_t max_iters, int64_t B,
                 uint32_t* d_bits, int32_t* d_iters, uint8_t* d_crc_ok, BpParams* P)
{
    std::memset(P, 0, sizeof(BpParams));
    build_dev_code(code, &P->code);
    build_dev_sched(sched, &P->sched);
    P->llr = d_llr;
    P->bits = d_bits;
    P->iters = d_iters;
    P->crc_ok = d_crc_ok;
    P->B = B;
    P->max_iters = max_iters;
    P->job.S = P->sched;
    P->job.llr = d_llr;
    P->job.bits = d_bits;
    P->job.iters = d_iters;
    P->job.crc_ok = d_crc_ok;
    P->job.B = B;
    P->job.max_iters = max_iters;
    P->job.K = code->K;
    P->job.r = code->crc_len;
    P->job.neg_zero = -0.0f;
}

// d_post (posterior output, nullable): the TMEM kernel's debug build that also writes L at node
// level n+1 and R at node level 1 of every frame's last iteration.
int decode_common(const pc_code* code, const float* d_llr, const pc_sched* sched, int32_t max_iters, int64_t B,
                  bool trace, const pc_event* h_events, int32_t n_events, float* d_dump, uint32_t* d_bits,
                  int32_t* d_iters, uint8_t* d_crc_ok, void* d_workspace, void* stream, float* d_post = nullptr)
{
    int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    rc = validate_sched(code, sched);
    if (rc != PC_OK) return rc;
    if (max_iters < 0 || B < 0) return PC_EINVAL;
    if (B == 0) return PC_OK;
    if (!d_llr || !d_bits || !d_iters || !d_crc_ok || !d_workspace) return PC_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_llr) & 15u) || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return PC_EINVAL;
    if (d_post) {
        if (trace || code->n < 7 || code->n > 11 || (sched->stop_kind & 2)) return PC_EUNSUPPORTED;
        if (reinterpret_cast<uintptr_t>(d_post) & 3u) return PC_EINVAL;
    }
    if (trace) {
        if (!d_dump) return PC_EINVAL;
        if (h_events) {
            rc = validate_events(code, h_events, n_events);
            if (rc != PC_OK) return rc;
        }
    }
    std::unique_ptr<BpParams> P(new BpParams);
    fill_params(code, d_llr, sched, max_iters, B, d_bits, d_iters, d_crc_ok, P.get());
    if (trace && h_events) {
        P->sched.n_explicit = n_events;
        for (int k = 0; k < n_events; ++k) {
            P->events[k].level = h_events[k].level;
            P->events[k].range = h_events[k].range;
            P->events[k].block = h_events[k].block;
            for (int i = 0; i < 16; ++i) P->events[k].order[i] = (int8_t)(i < h_events[k].range ? h_events[k].order[i] : i);
        }
    }
    P->job.S = P->sched;         // after the explicit events
    P->counter = reinterpret_cast<unsigned long long*>(d_workspace);
    P->dump = d_dump;

    P->job.post = d_post;

    LaunchGeom g;
    const bool tmem = !trace && (d_post || use_tmem_kernel(code->n));
    rc = trace ? plan_launch(code, B, trace, sched->fkind, &g)
               : (tmem ? plan_launch3(code, B, sched->fkind, &g) : plan_launch2(code, B, sched->fkind, &g));
    if (rc != PC_OK) return rc;
    P->slots = g.slots;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
#ifdef PCBP_CHECKED
    // bound-check status word at byte 16 of the workspace (read back by the caller)
    P->job.check = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(d_workspace) + 16);
    if (cudaMemsetAsync(d_workspace, 0, 32, st) != cudaSuccess) return PC_ECUDA;
#else
    if (cudaMemsetAsync(d_workspace, 0, sizeof(unsigned long long), st) != cudaSuccess) return PC_ECUDA;
#endif
    const cudaError_t e = trace    ? launch_of(code->n, *P, g, true, sched->fkind, st)
                          : d_post ? launch3_post_of(code->n, *P, g, sched->fkind, st)
                          : tmem   ? launch3_of(code->n, *P, g, sched->fkind, st, false)
                                   : launch2_of(code->n, *P, g, sched->fkind, st, false);
    if (e != cudaSuccess) return PC_ECUDA;
    return PC_OK;
}

// ---------------------------------------------------------------------------
// Encoder (Eq. 1): one CTA per frame at a time.  The CRC is the XOR of the
// per-payload-bit remainders crc_pay[i]; u is built in shared memory and the
// n butterfly layers x[t] ^= x[t + 2^p] run in place.
__global__ void __launch_bounds__(256) encode_kernel(const __grid_constant__ EncParams P)
{
    extern __shared__ uint8_t su[];
    __shared__ uint32_t red[8];
    const int N = P.N, n = P.n, K = P.K, r = P.r, Kp = P.Kp;
    for (int64_t f = blockIdx.x; f < P.B; f += gridDim.x) {
        const uint8_t* pay = P.payload + size_t(f) * Kp;
        uint32_t acc = 0;
        for (int i = threadIdx.x; i < Kp; i += blockDim.x)
            if (pay[i] & 1) acc ^= P.crc_pay[i];
        for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        for (int j = threadIdx.x; j < N; j += blockDim.x) su[j] = 0;
        __syncthreads();
        uint32_t crc = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) crc ^= red[w];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const uint8_t bit = k < Kp ? uint8_t(pay[k] & 1) : uint8_t((crc >> (r - 1 - (k - Kp))) & 1u);
            su[P.info_idx[k]] = bit;
        }
        __syncthreads();
        for (int p = 0; p < n; ++p) {
            for (int q = threadIdx.x; q < N / 2; q += blockDim.x) {
                const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                su[t] ^= su[t | (1 << p)];
            }
            __syncthreads();
        }
        uint8_t* x = P.x + size_t(f) * N;
        for (int j = threadIdx.x; j < N; j += blockDim.x) x[j] = su[j];
        __syncthreads();
    }
}

}  // namespace

}  // namespace pcbp

using namespace pcbp;

extern "C" int pc_encode(const pc_code* code, const uint8_t* d_payload, uint8_t* d_x, int64_t B, void* stream)
{
    int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    if (B < 0) return PC_EINVAL;
    if (B == 0) return PC_OK;
    if (!d_x || (!d_payload && code->K - code->crc_len > 0)) return PC_EINVAL;
    DeviceInfo di;
    rc = device_info(&di);
    if (rc != PC_OK) return rc;
    std::unique_ptr<EncParams> P(new EncParams);
    build_enc_params(code, P.get());
    P->payload = d_payload;
    P->x = d_x;
    P->B = B;
    const int grid = int(std::min<int64_t>(B, int64_t(di.sms) * 8));
    encode_kernel<<<grid, 256, size_t(code->N), reinterpret_cast<cudaStream_t>(stream)>>>(*P);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ECUDA;
}

extern "C" int bp_decode_workspace_size(const pc_code* code, int64_t B, size_t* bytes)
{
    int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    if (B < 0 || !bytes) return PC_EINVAL;
    *bytes = 256;
    return PC_OK;
}

extern "C" int bp_decode(const pc_code* code, const float* d_llr, const pc_sched* sched, int32_t max_iters,
                         int64_t B, uint32_t* d_bits, int32_t* d_iters, uint8_t* d_crc_ok, void* d_workspace,
                         void* stream)
{
    return decode_common(code, d_llr, sched, max_iters, B, false, nullptr, 0, nullptr, d_bits, d_iters, d_crc_ok,
                         d_workspace, stream);
}

extern "C" int bp_decode_posterior(const pc_code* code, const float* d_llr, const pc_sched* sched,
                                   int32_t max_iters, int64_t B, uint32_t* d_bits, int32_t* d_iters,
                                   uint8_t* d_crc_ok, float* d_post, void* d_workspace, void* stream)
{
    if (B > 0 && !d_post) return PC_EINVAL;
    return decode_common(code, d_llr, sched, max_iters, B, false, nullptr, 0, nullptr, d_bits, d_iters, d_crc_ok,
                         d_workspace, stream, B > 0 ? d_post : nullptr);
}

// ---------------------------------------------------------------------------
// Decoding in place in host memory.
namespace pcbp {
namespace {

// Device address of a buffer of `bytes` bytes that the kernels may read and
// write in place: page-locked host memory mapped into the current device's
// address space, or device or managed memory of the current device.  The
// first and the last byte must both be accessible, at device addresses
// bytes - 1 apart.  Only host-side queries; nothing is enqueued.
int mapped_address(const void* p, size_t bytes, void** dev)
{
    if (!p || bytes == 0) return PC_EINVAL;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return PC_ECUDA;
    }
    const void* last = static_cast<const char*>(p) + (bytes - 1);
    cudaPointerAttributes a0, a1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();
        return PC_EINVAL;
    }
    for (const cudaPointerAttributes* a : {&a0, &a1}) {
        if (a->type == cudaMemoryTypeUnregistered || !a->devicePointer) return PC_EINVAL;
        if (a->type == cudaMemoryTypeDevice && a->device != cur) return PC_EINVAL;
    }
    if (static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) !=
        static_cast<ptrdiff_t>(bytes - 1))
        return PC_EINVAL;
    *dev = a0.devicePointer;
    return PC_OK;
}

}  // namespace
}  // namespace pcbp

extern "C" int bp_decode_host(const pc_code* code, const float* h_llr, const pc_sched* sched, int32_t max_iters,
                              int64_t B, uint32_t* h_bits, int32_t* h_iters, uint8_t* h_crc_ok, void* d_workspace,
                              void* stream)
{
    using namespace pcbp;
    int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    if (B < 0 || max_iters < 0) return PC_EINVAL;
    if (B == 0) return PC_OK;
    if (!h_llr || !h_bits || !h_iters || !h_crc_ok || !d_workspace) return PC_EINVAL;
    const size_t KW = size_t(code->K + 31) / 32;
    if (uint64_t(B) > uint64_t(SIZE_MAX) / (size_t(code->N) * 4u)) return PC_EINVAL;
    void *llr = nullptr, *bits = nullptr, *iters = nullptr, *ok = nullptr;
    if ((rc = mapped_address(h_llr, size_t(B) * size_t(code->N) * 4u, &llr)) != PC_OK) return rc;
    if ((rc = mapped_address(h_bits, size_t(B) * KW * 4u, &bits)) != PC_OK) return rc;
    if ((rc = mapped_address(h_iters, size_t(B) * 4u, &iters)) != PC_OK) return rc;
    if ((rc = mapped_address(h_crc_ok, size_t(B), &ok)) != PC_OK) return rc;
    return decode_common(code, static_cast<const float*>(llr), sched, max_iters, B, false, nullptr, 0, nullptr,
                         static_cast<uint32_t*>(bits), static_cast<int32_t*>(iters), static_cast<uint8_t*>(ok),
                         d_workspace, stream);
}

// ---------------------------------------------------------------------------
// Mixed-length batches: each batch is launched with the kernel bp_decode
// runs for its length, all on one stream; every launch after the first is a
// programmatic dependent launch and the kernels trigger their dependents as
// they start, so a batch's CTAs take the SMs that the previous batch's CTAs
// leave while its last frames finish: one persistent sweep over all the
// batches, with no per-size tail.
namespace pcbp {
namespace {

constexpr uint32_t kMixedMagic = 0x70636278u;

struct MixedEntry {
    BpParams P;
    LaunchGeom g;
    int32_t n, tmem, fkind;
    uint32_t magic;
};

int validate_batch(const pc_batch& b)
{
    if (!b.code) return PC_EINVAL;
    int rc = validate_code(b.code);
    if (rc != PC_OK) return rc;
    rc = validate_sched(b.code, &b.sched);
    if (rc != PC_OK) return rc;
    if (b.max_iters < 0 || b.B < 0 || b.slots < 0 || b.threads_per_frame < 0 || b.reserved != 0) return PC_EINVAL;
    const int N = b.code->N;
    const int tpf = b.threads_per_frame;
    if (tpf != 0 && tpf != tmem_threads_per_frame(b.code->n) && tpf != std::max(32, N / 4))
        return PC_EUNSUPPORTED;
    if (b.B > 0) {
        if (!b.d_llr || !b.d_bits || !b.d_iters || !b.d_crc_ok) return PC_EINVAL;
        if (reinterpret_cast<uintptr_t>(b.d_llr) & 15u) return PC_EINVAL;
    }
    return PC_OK;
}

}  // namespace
}  // namespace pcbp

extern "C" int bp_mixed_table_size(int32_t n_batches, size_t* bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || !bytes) return PC_EINVAL;
    *bytes = sizeof(MixedEntry) * size_t(n_batches);
    return PC_OK;
}

extern "C" int bp_mixed_prepare(const pc_batch* batches, int32_t n_batches, void* h_table, size_t bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || (n_batches > 0 && (!batches || !h_table))) return PC_EINVAL;
    if (bytes < sizeof(MixedEntry) * size_t(n_batches)) return PC_ENOMEM;
    for (int i = 0; i < n_batches; ++i) {
        const int rc = validate_batch(batches[i]);
        if (rc != PC_OK) return rc;
    }
    for (int i = 0; i < n_batches; ++i) {
        const pc_batch& b = batches[i];
        std::unique_ptr<MixedEntry> m(new MixedEntry);
        std::memset(m.get(), 0, sizeof(MixedEntry));
        fill_params(b.code, b.d_llr, &b.sched, b.max_iters, b.B, b.d_bits, b.d_iters, b.d_crc_ok, &m->P);
        m->n = b.code->n;
        m->fkind = b.sched.fkind;
        const int tpf = b.threads_per_frame;
        m->tmem = tmem_for(b.code->n, b.code->N, tpf) ? 1 : 0;
        if (b.B > 0) {
            const int rc = m->tmem ? plan_launch3(b.code, b.B, b.sched.fkind, &m->g, b.slots)
                                   : plan_launch2(b.code, b.B, b.sched.fkind, &m->g, b.slots);
            if (rc != PC_OK) return rc;
            m->P.slots = m->g.slots;
        }
        m->magic = kMixedMagic;
        std::memcpy(static_cast<MixedEntry*>(h_table) + i, m.get(), sizeof(MixedEntry));
    }
    return PC_OK;
}

extern "C" int pc_build_info(int32_t* flags)
{
    if (!flags) return PC_EINVAL;
#ifdef PCBP_CHECKED
    *flags = 1;
#else
    *flags = 0;
#endif
    return PC_OK;
}

extern "C" int bp_kernel_threads(const pc_code* code, int32_t kernel, int32_t* threads_per_frame)
{
    using namespace pcbp;
    if (!code || !threads_per_frame || (kernel != 0 && kernel != 1)) return PC_EINVAL;
    const int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    const int t = kernel == 0 ? tmem_threads_per_frame(code->n) : std::max(32, code->N / 4);
    if (t == 0) return PC_EUNSUPPORTED;
    *threads_per_frame = t;
    return PC_OK;
}

extern "C" int bp_slot_limit(const pc_code* code, int32_t threads_per_frame, int32_t fkind, int32_t* max_slots)
{
    using namespace pcbp;
    if (!code || !max_slots) return PC_EINVAL;
    int rc = validate_code(code);
    if (rc != PC_OK) return rc;
    if (fkind != 0 && fkind != 1) return PC_EINVAL;
    const int N = code->N, tpf = threads_per_frame;
    if (tpf < 0) return PC_EINVAL;
    if (tpf != 0 && tpf != tmem_threads_per_frame(code->n) && tpf != std::max(32, N / 4))
        return PC_EUNSUPPORTED;
    const bool tmem = tmem_for(code->n, N, tpf);
    LaunchGeom g;
    rc = tmem ? plan_launch3(code, 1, fkind, &g) : plan_launch2(code, 1, fkind, &g);
    if (rc != PC_OK) return rc;
    *max_slots = g.slots;
    return PC_OK;
}

extern "C" int bp_mixed_workspace_size(int32_t n_batches, size_t* bytes)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES || !bytes) return PC_EINVAL;
    *bytes = (sizeof(unsigned long long) * size_t(n_batches) + 255) & ~size_t(255);
    if (*bytes == 0) *bytes = 256;
    return PC_OK;
}

extern "C" int bp_decode_mixed(const void* h_table, int32_t n_batches, void* d_workspace, void* stream)
{
    if (n_batches < 0 || n_batches > PC_MAX_BATCHES) return PC_EINVAL;
    if (n_batches == 0) return PC_OK;
    if (!h_table || !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return PC_EINVAL;
    std::unique_ptr<MixedEntry> m(new MixedEntry);
    for (int i = 0; i < n_batches; ++i) {
        std::memcpy(m.get(), static_cast<const MixedEntry*>(h_table) + i, sizeof(MixedEntry));
        if (m->magic != kMixedMagic) return PC_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    size_t ws = 0;
    bp_mixed_workspace_size(n_batches, &ws);
    if (cudaMemsetAsync(d_workspace, 0, ws, st) != cudaSuccess) return PC_ECUDA;
    bool first = true;
    for (int i = 0; i < n_batches; ++i) {
        std::memcpy(m.get(), static_cast<const MixedEntry*>(h_table) + i, sizeof(MixedEntry));
        if (m->P.B == 0) continue;
        m->P.counter = reinterpret_cast<unsigned long long*>(d_workspace) + i;
        const cudaError_t e = m->tmem ? launch3_of(m->n, m->P, m->g, m->fkind, st, !first)
                                      : launch2_of(m->n, m->P, m->g, m->fkind, st, !first);
        if (e != cudaSuccess) return PC_ECUDA;
        first = false;
    }
    return PC_OK;
}

extern "C" int bp_decode_trace(const pc_code* code, const float* d_llr, const pc_sched* sched, int32_t max_iters,
                               int64_t B, const pc_event* h_events, int32_t n_events, float* d_dump,
                               uint32_t* d_bits, int32_t* d_iters, uint8_t* d_crc_ok, void* d_workspace,
                               void* stream)
{
    return decode_common(code, d_llr, sched, max_iters, B, true, h_events, n_events, d_dump, d_bits, d_iters,
                         d_crc_ok, d_workspace, stream);
}
