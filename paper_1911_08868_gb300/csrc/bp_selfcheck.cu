// Verification entry points (no counterpart in the paper).  Internal
// consistency check of the TMEM kernel's two partition builders: for every event shape of N = 128..2048 and
// three orders and blocks each, the warp-parallel builder used at a switch
// must produce the packed records that build_groups + pack_groups produce,
// and every partition (the no-event one included) must have the shape the
// kernel's sweeps assume: at least two groups, and every group other than the
// first and the last either a single stage or a full KB stages.
#include <cuda_runtime.h>

#include <algorithm>

#include "bp_kernel3.cuh"

namespace pcbp {
namespace {

template <int LOGN, int KB>
__global__ void partition_selfcheck_kernel(int32_t* result)
{
    constexpr int E = 1 << KB;
    __shared__ Ctl3<LOGN, KB> A, B;
    __shared__ unsigned char tab[kSwzTableBytes];
    const int lane = int(threadIdx.x);
    for (int i = lane; i < kSwzTableBytes; i += 32) tab[i] = swz_row(i);
    __syncwarp();
    // the group shape the sweeps assume
    auto irregular = [&](const Ctl3<LOGN, KB>& c) {
        bool bad = c.g.ng < 2;
        for (int g = 1; g + 1 < c.g.ng && g < LOGN; ++g) {
            const int x = c.rec[g].x;
            bad = bad || (!((x >> 16) & 1) && ((x >> 8) & 0xff) != KB);
        }
        return bad;
    };
    if (lane == 0) {
        signed char none[16];
        build_groups<LOGN, KB>(&A.g, tab, LOGN, false, 0, 0, 0, none, true);
        pack_groups<LOGN, KB>(&A);
        atomicAdd(result + 0, 1);
        if (irregular(A)) atomicAdd(result + 2, 1);
    }
    __syncwarp();
    for (int level = 1; level < LOGN; ++level)
        for (int range = 2; range <= 16 && level + range - 1 <= LOGN; ++range)
            for (int v = 0; v < 3; ++v) {
                const int m = level + range - 1;
                const long long blk = ((1ll << (LOGN - m)) - 1) * v / 2;      // first, middle, last block
                signed char order[16];
                for (int i = 0; i < range; ++i) order[i] = (signed char)(v == 0 ? range - 1 - i : (i + v) % range);
                if (lane == 0) {
                    build_groups<LOGN, KB>(&A.g, tab, LOGN, true, level, range, blk, order, true);
                    pack_groups<LOGN, KB>(&A);
                }
                __syncwarp();
                uint64_t ord = 0;
                for (int i = 0; i < range; ++i) ord |= uint64_t(order[i]) << (4 * i);
                build_partition_warp<LOGN, KB>(&B, tab, level, range, blk, ord, lane);
                __syncwarp();
                if (lane == 0) {
                    int d = (A.g.ng != B.g.ng) + (A.g.low != B.g.low) + (A.g.beta != B.g.beta);
                    for (int s = 0; s < 16; ++s) d += A.g.pbit[s] != B.g.pbit[s];
                    for (int g = 0; g < A.g.ng && g < LOGN; ++g) {
                        const int4 a = A.rec[g], b = B.rec[g];
                        d += (a.x != b.x) + (a.y != b.y);
                        if (!((a.x >> 16) & 1)) {             // register groups: bits, offsets, cache column
                            d += (a.z != b.z) + (a.w != b.w);
                            d += (A.cmask[g].x != B.cmask[g].x) + (A.cmask[g].y != B.cmask[g].y);
                            for (int c = 0; c < 2; ++c)
                                for (int e = 0; e < E; ++e) d += A.swoff[g][c][e] != B.swoff[g][c][e];
                        }
                    }
                    atomicAdd(result + 0, 1);
                    if (d) atomicAdd(result + 1, 1);
                    if (irregular(A) || irregular(B)) atomicAdd(result + 2, 1);
                }
                __syncwarp();
            }
}

}  // namespace
}  // namespace pcbp

using namespace pcbp;

extern "C" int pc_partition_selfcheck(int32_t* d_result, void* stream)
{
    if (!d_result || (reinterpret_cast<uintptr_t>(d_result) & 3u)) return PC_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_result, 0, 3 * sizeof(int32_t), st) != cudaSuccess) return PC_ECUDA;
    // the group widths the decoder is built with
    partition_selfcheck_kernel<7, tmem_default_kb(7)><<<1, 32, 0, st>>>(d_result);
    partition_selfcheck_kernel<8, tmem_default_kb(8)><<<1, 32, 0, st>>>(d_result);
    partition_selfcheck_kernel<9, tmem_default_kb(9)><<<1, 32, 0, st>>>(d_result);
    partition_selfcheck_kernel<10, tmem_default_kb(10)><<<1, 32, 0, st>>>(d_result);
    partition_selfcheck_kernel<11, tmem_default_kb(11)><<<1, 32, 0, st>>>(d_result);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ECUDA;
}

// ---------------------------------------------------------------------------
// The processing-element function f of Sec. II-B exactly as the decoder
// kernels evaluate it, elementwise (for checking its arithmetic).
namespace pcbp {
namespace {

template <int FK>
__global__ void f_eval_kernel(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out,
                              int64_t count, float alpha)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = fnode<FK>(a[i], b[i], alpha);
}

}  // namespace
}  // namespace pcbp

extern "C" int pc_f_eval(const float* d_a, const float* d_b, float* d_out, int64_t count, int32_t fkind, float alpha,
                         void* stream)
{
    if (count < 0 || (fkind != 0 && fkind != 1)) return PC_EINVAL;
    if (count == 0) return PC_OK;
    if (!d_a || !d_b || !d_out) return PC_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_b) | reinterpret_cast<uintptr_t>(d_out)) &
        3u)
        return PC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PC_ECUDA;
    const int grid = int(std::min<int64_t>((count + 255) / 256, int64_t(sms) * 8));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (fkind) f_eval_kernel<1><<<grid, 256, 0, st>>>(d_a, d_b, d_out, count, alpha);
    else f_eval_kernel<0><<<grid, 256, 0, st>>>(d_a, d_b, d_out, count, alpha);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ECUDA;
}
