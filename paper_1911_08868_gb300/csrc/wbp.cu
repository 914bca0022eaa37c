// Weighted BP: a differentiable variant of the decoder (not in the paper).
// Unrolled round-trip BP on the original factor graph (Sec. II-B) in which
// each f evaluation has its own learnable scale w[t][s][q][k] (iteration t,
// stage s, processing element q, and k = 0 L_out1, 1 L_out2, 2 R_out1,
// 3 R_out2) in place of the fixed min-sum scale.  Forward keeps the R planes
// at every iteration boundary as checkpoints; backward runs one launch per
// iteration in reverse, recomputes that iteration from its checkpoint and
// applies the adjoint of the R sweep then of the L sweep.
//
// Derivatives of f_w(a, b) = w sign(a) sign(b) min(|a|, |b|): with a the
// minimum (|a| <= |b|: the first operand wins ties), df/da = w sign(b),
// df/db = 0, df/dw = sign(a) sign(b) |a|; symmetrically otherwise.  Frozen
// priors are +inf; an infinite message is never the minimum against a finite
// one and receives no gradient, so updates with a zero upstream gradient are
// skipped (never forming 0 * inf).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <type_traits>

#include "pcbp_internal.h"

namespace pcbp {

namespace {

template <typename Real>
struct WbpParams {
    DevCode code;
    const Real* llr;
    const Real* w;
    Real* logits;
    Real* ckpt;          // [T][B][n-1][N], R of levels 2..n after t iterations (nullable in forward)
    const Real* glogits;
    Real* gw;            // [T][n][N/2][4], accumulated
    Real* gllr;          // [B][N], accumulated over the launches (nullable)
    const Real* gin;     // [B][n-1][N] gradient of R(t+1) levels 2..n (iteration it+1)
    Real* gout;          // [B][n-1][N] gradient of R(t) levels 2..n
    unsigned long long* counter;
    int64_t B;
    int32_t T;
    int32_t it;          // backward: 0-based iteration handled by this launch
    int32_t tps;         // threads per frame slot
};

template <typename Real>
__device__ __forceinline__ Real inf_v();
template <>
__device__ __forceinline__ float inf_v<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double inf_v<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

template <typename Real>
__device__ __forceinline__ Real sgn(Real v) { return v > Real(0) ? Real(1) : (v < Real(0) ? Real(-1) : Real(0)); }

// w * sign(a) sign(b) min(|a|, |b|), the scale applied to the minimum first
template <typename Real>
__device__ __forceinline__ Real fw(Real a, Real b, Real w)
{
    const Real m = fabs(a) <= fabs(b) ? fabs(a) : fabs(b);
    const Real v = rmul(w, m);
    return (signbit(a) != signbit(b)) ? -v : v;
}

// FP32: the signed minimum from one min.xorsign.abs; w times it has exactly the
// bits of the form above for every w (a product's sign is the XOR of the signs
// and its magnitude does not depend on them)
template <>
__device__ __forceinline__ float fw<float>(float a, float b, float w)
{
    float m;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(m) : "f"(a), "f"(b));
    return __fmul_rn(w, m);
}

__device__ __forceinline__ int ins0(int q, int p) { return ((q >> p) << (p + 1)) | (q & ((1 << p) - 1)); }

__device__ __forceinline__ void bar(unsigned id, unsigned count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Synchronisation of a frame slot between the stage just done (butterfly distance 2^pd) and the
// next step (2^pn; kCross when it reads across warps).  One thread per processing element q:
// in a stage of distance 2^p <= 32 the elements q = 32w .. 32w+31 of warp w touch exactly the
// positions [64w, 64w+64), so between two such stages a warp exchanges data only with itself.
constexpr int kCross = 99;
__device__ __forceinline__ void stage_sync(int pd, int pn, unsigned id, unsigned count)
{
    if (pd <= 5 && pn <= 5) __syncwarp();
    else bar(id, count);
}

// Plane layout of the unrolled FP32 kernels: position j lives at element sw32(j), which
// complements the low five bits of j when its bit 5 is set.  A warp's element pairs of a stage of
// distance 2^p < 32 cover one block of 64 positions with bit p clear in its two halves; the
// complement sends the second half to the banks the first half leaves free (bit p set), so no
// stage has bank conflicts (in a stage of distance >= 32 all 32 positions of a warp share bit 5
// and the map permutes their banks).  The checkpoints and the gradient planes between backward
// launches keep this layout in global memory; LLRs, logits, their gradients and the LLR gradient
// are read and written at their natural positions.  Identity for N <= 32.
__device__ __forceinline__ int sw32(int j) { return j ^ (((j >> 5) & 1) * 31); }

// Copy the count = N reals of a natural-order row into a plane in the sw32 layout (4-byte
// cp.async, no register round trip); waited for with copy_wait().
__device__ __forceinline__ void copy_async_sw(float* dst, const float* src, int count, int tid, int tps)
{
    for (int j = tid; j < count; j += tps)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(uint32_t(__cvta_generic_to_shared(dst + sw32(j)))),
                     "l"(size_t(__cvta_generic_to_global(src + j)))
                     : "memory");
}

// Two consecutive weights (k, k+1) of one processing element in one load
// (the weight array is 8-byte aligned for float, 16-byte for double).
__device__ __forceinline__ float2 ld_pair(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ double2 ld_pair(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

// Copy count reals from global to shared memory with cp.async (every element
// in flight at once, no register round trip): 16-byte pieces when both ends
// are 16-byte aligned and the size is a multiple of 16, else one real each.
// The caller waits with copy_wait() and then synchronises the slot.
template <typename Real>
__device__ __forceinline__ void copy_async(Real* dst, const Real* src, int count, int tid, int tps)
{
    const uint32_t d = uint32_t(__cvta_generic_to_shared(dst));
    const size_t g = size_t(__cvta_generic_to_global(src));
    const size_t bytes = size_t(count) * sizeof(Real);
    if (((g | size_t(d) | bytes) & 15u) == 0) {
        for (int i = tid; i < int(bytes / 16); i += tps)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * uint32_t(i)), "l"(g + 16u * size_t(i))
                         : "memory");
    } else {
        for (int i = tid; i < count; i += tps)
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d + uint32_t(sizeof(Real)) * uint32_t(i)),
                         "l"(g + sizeof(Real) * size_t(i)), "n"(int(sizeof(Real)))
                         : "memory");
    }
}

__device__ __forceinline__ void copy_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename Real>
__device__ __forceinline__ Real prior_v(const uint32_t* frozen, int j)
{
    return ((frozen[j >> 5] >> (j & 31)) & 1u) ? inf_v<Real>() : Real(0);
}

// ---------------------------------------------------------------------------
// Shared memory per frame slot: L at levels 1..n+1, R at levels 2..n+1 (the
// plane of level n+1 holds the frozen priors, written once per CTA), so every
// stage reads its R operands from one plane without a per-element test.
template <typename Real>
__global__ void __launch_bounds__(1024, 1) wbp_forward_kernel(const __grid_constant__ WbpParams<Real> P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = P.code.n, N = 1 << n, NH = N / 2, K = P.code.K;
    const int NW = N >= 32 ? N / 32 : 1;
    const int tps = P.tps;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    int16_t* s_info = reinterpret_cast<int16_t*>(s_frozen + NW);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = P.code.frozen[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = P.code.info_idx[i];
    __syncthreads();
    const size_t tab = (size_t(NW) * 4 + size_t(K) * 2 + 15) & ~size_t(15);
    const int slot = threadIdx.x / tps, tid = threadIdx.x - slot * tps;
    Real* L = reinterpret_cast<Real*>(smem + tab + size_t(slot) * size_t(2 * n + 1) * N * sizeof(Real));
    Real* R = L + (n + 1) * N;                    // plane l-2 = level l, 2 <= l <= n+1
    for (int j = tid; j < N; j += tps) R[(n - 1) * N + j] = prior_v<Real>(s_frozen, j);
    __shared__ long long s_frame[32];
    const unsigned bid = 1u + unsigned(slot);
    const int wplane = n * NH * 4;                // weights of one iteration

    while (true) {
        if (tid == 0) s_frame[slot] = (long long)atomicAdd(P.counter, 1ull);
        bar(bid, tps);
        const long long f = s_frame[slot];
        if (f >= P.B) break;
        copy_async(L, P.llr + size_t(f) * N, N, tid, tps);
        for (int j = tid; j < (n - 1) * N; j += tps) R[j] = Real(0);
        if (P.ckpt)
            for (int j = tid; j < (n - 1) * N; j += tps) P.ckpt[size_t(f) * (n - 1) * N + j] = Real(0);
        copy_wait();
        bar(bid, tps);
        for (int it = 0; it < P.T; ++it) {
            const Real* wt = P.w + size_t(it) * wplane;
            for (int s = 0; s < n; ++s) {
                const int p = n - 1 - s;
                const Real* Ls = L + s * N;
                const Real* Rs = R + s * N;           // level s+2
                Real* Lo = L + (s + 1) * N;
                const Real* ws = wt + s * NH * 4;
                for (int q = tid; q < NH; q += tps) {
                    const int t = ins0(q, p), b = t | (1 << p);
                    const Real lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    const auto w2 = ld_pair(ws + q * 4);   // k = 0, 1
                    Lo[t] = fw(lt, radd(lb, rb), w2.x);
                    Lo[b] = radd(fw(rt, lt, w2.y), lb);
                }
                bar(bid, tps);
            }
            if (it == P.T - 1) break;
            for (int s = n - 1; s >= 1; --s) {
                const int p = n - 1 - s;
                const Real* Ls = L + s * N;
                const Real* Rs = R + s * N;           // level s+2
                Real* Ro = R + (s - 1) * N;           // level s+1
                const Real* ws = wt + s * NH * 4 + 2;
                for (int q = tid; q < NH; q += tps) {
                    const int t = ins0(q, p), b = t | (1 << p);
                    const Real lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    const auto w2 = ld_pair(ws + q * 4);   // k = 2, 3
                    Ro[t] = fw(rt, radd(lb, rb), w2.x);
                    Ro[b] = radd(fw(rt, lt, w2.y), rb);
                }
                bar(bid, tps);
            }
            if (P.ckpt) {
                // no barrier after the copy: the R planes are next written by the R sweep of
                // the next iteration, n slot barriers later
                Real* dst = P.ckpt + (size_t(it + 1) * P.B + size_t(f)) * (n - 1) * N;
                for (int j = tid; j < (n - 1) * N; j += tps) dst[j] = R[j];
            }
        }
        for (int k = tid; k < K; k += tps) P.logits[size_t(f) * K + k] = L[n * N + s_info[k]];
        bar(bid, tps);
    }
}

// ---------------------------------------------------------------------------
// FP32 forward for N <= 1024 with the stage loops unrolled for the length: one thread per
// processing element (tps = N/2), so every index and plane offset of a stage is a compile-time
// shift or constant.  Same planes (in the sw32 layout) and arithmetic as wbp_forward_kernel.
template <int LOGN>
__global__ void __launch_bounds__(1024, 1) wbp_forward_reg_kernel(const __grid_constant__ WbpParams<float> P)
{
    constexpr int n = LOGN, N = 1 << LOGN, NH = N / 2;
    constexpr int NW = N >= 32 ? N / 32 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = P.code.K;
    const int tps = P.tps;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    int16_t* s_info = reinterpret_cast<int16_t*>(s_frozen + NW);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = P.code.frozen[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = P.code.info_idx[i];
    __syncthreads();
    const size_t tab = (size_t(NW) * 4 + size_t(K) * 2 + 15) & ~size_t(15);
    const int slot = threadIdx.x / tps, tid = threadIdx.x - slot * tps;
    float* L = reinterpret_cast<float*>(smem + tab + size_t(slot) * size_t(2 * n + 1) * N * sizeof(float));
    float* R = L + (n + 1) * N;                   // plane l-2 = level l, 2 <= l <= n+1
    for (int j = tid; j < N; j += tps) R[(n - 1) * N + sw32(j)] = prior_v<float>(s_frozen, j);
    __shared__ long long s_frame[32];
    const unsigned bid = 1u + unsigned(slot);
    const bool act = tid < NH;                    // N < 64: fewer elements than a warp
    const int q = act ? tid : 0;

    while (true) {
        if (tid == 0) s_frame[slot] = (long long)atomicAdd(P.counter, 1ull);
        bar(bid, tps);
        const long long f = s_frame[slot];
        if (f >= P.B) break;
        copy_async_sw(L, P.llr + size_t(f) * N, N, tid, tps);
        for (int j = tid; j < (n - 1) * N; j += tps) R[j] = 0.f;
        if (P.ckpt)
            for (int j = tid; j < (n - 1) * N; j += tps) P.ckpt[size_t(f) * (n - 1) * N + j] = 0.f;
        copy_wait();
        bar(bid, tps);
        // each stage's weight pair is loaded one stage ahead (read-only, so across the barrier)
        float2 wc = ld_pair(P.w + size_t(q) * 4);
        for (int it = 0; it < P.T; ++it) {
            const float* wq = P.w + size_t(it) * n * NH * 4 + size_t(q) * 4;
#pragma unroll
            for (int s = 0; s < n; ++s) {
                const float2 w2 = wc;                              // k = 0, 1
                wc = s + 1 < n ? ld_pair(wq + (s + 1) * NH * 4) : (it + 1 < P.T ? ld_pair(wq + (n - 1) * NH * 4 + 2) : wc);
                if (act) {
                    const int p = n - 1 - s;
                    const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                    const float* Ls = L + s * N;
                    const float* Rs = R + s * N;           // level s+2
                    float* Lo = L + (s + 1) * N;
                    const float lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    Lo[t] = fw(lt, radd(lb, rb), w2.x);
                    Lo[b] = radd(fw(rt, lt, w2.y), lb);
                }
                // after the last stage: the R sweep's first stage, or the logits read across warps
                const int p = n - 1 - s;
                stage_sync(p, s < n - 1 ? p - 1 : (it == P.T - 1 ? kCross : 0), bid, tps);
            }
            if (it == P.T - 1) break;
            // the checkpoint of R after this iteration.  Every R value of levels 2..n is computed
            // by one thread at one stage of the R sweep and not changed until the next R sweep: at
            // N = 1024, where the shared-memory pipe bounds the kernel, the thread stores it to the
            // checkpoint there, from its registers (forward 0.735 -> 0.681 ms per T = 10 step at
            // batch 4096); below, the planes are copied as rows after the sweep (the scattered
            // 4-byte stores measured 3% slower at N = 256)
            constexpr bool ck_regs = LOGN >= 10;
            float* const ckp = P.ckpt ? P.ckpt + (size_t(it + 1) * P.B + size_t(f)) * (n - 1) * N : nullptr;
            float* const ck = ck_regs ? ckp : nullptr;
#pragma unroll
            for (int s = n - 1; s >= 1; --s) {
                const float2 w2 = wc;                              // k = 2, 3
                wc = s > 1 ? ld_pair(wq + (s - 1) * NH * 4 + 2) : ld_pair(wq + n * NH * 4);   // then the next iteration's stage 0
                if (act) {
                    const int p = n - 1 - s;
                    const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                    const float* Ls = L + s * N;
                    const float* Rs = R + s * N;           // level s+2
                    float* Ro = R + (s - 1) * N;           // level s+1
                    const float lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    const float ot = fw(rt, radd(lb, rb), w2.x);
                    const float ob = radd(fw(rt, lt, w2.y), rb);
                    Ro[t] = ot;
                    Ro[b] = ob;
                    if (ck) {
                        ck[(s - 1) * N + t] = ot;
                        ck[(s - 1) * N + b] = ob;
                    }
                }
                // after the last stage: the checkpoint rows or the next iteration's first stage,
                // read across warps
                const int p = n - 1 - s;
                stage_sync(p, s > 1 ? p + 1 : kCross, bid, tps);
            }
            if (!ck_regs && ckp) {
                // no barrier after the copy: the R planes are next written by the R sweep of
                // the next iteration, after the slot barrier that ends the first stage of its L
                // sweep (distance 2^(n-1) > 32 from N = 128; below, the slot is one warp)
                if ((reinterpret_cast<uintptr_t>(ckp) & 15u) == 0) {
                    float4* d4 = reinterpret_cast<float4*>(ckp);
                    const float4* s4 = reinterpret_cast<const float4*>(R);
                    for (int j = tid; j < (n - 1) * N / 4; j += tps) d4[j] = s4[j];
                } else {
                    for (int j = tid; j < (n - 1) * N; j += tps) ckp[j] = R[j];
                }
            }
        }
        for (int k = tid; k < K; k += tps) P.logits[size_t(f) * K + k] = L[n * N + sw32(s_info[k])];
        bar(bid, tps);
    }
}

// ---------------------------------------------------------------------------
// Shared memory per frame slot: L at levels 1..n+1, R at levels 2..n+1 (level
// n+1: the priors, written once per CTA), the gradient of L at levels 1..n+1
// and two planes for the gradient flowing between R levels.  The R planes hold
// R before this iteration (copied from the checkpoint with cp.async)
// for the L sweep, R after it (recomputed in place, as in the forward kernel)
// for the adjoint of the R sweep, and R before it again (a second copy) for
// the adjoint of the L sweep.
template <typename Real>
__global__ void __launch_bounds__(1024, 1) wbp_backward_kernel(const __grid_constant__ WbpParams<Real> P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = P.code.n, N = 1 << n, NH = N / 2, K = P.code.K;
    const int NW = N >= 32 ? N / 32 : 1;
    const int tps = P.tps, it = P.it;
    const bool last = it == P.T - 1;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    int16_t* s_info = reinterpret_cast<int16_t*>(s_frozen + NW);
    const size_t tab = (size_t(NW) * 4 + size_t(K) * 2 + 15) & ~size_t(15);
    Real* dw = reinterpret_cast<Real*>(smem + tab);                                   // [n][NH][4]
    const size_t dw_bytes = (size_t(n) * NH * 4 * sizeof(Real) + 15) & ~size_t(15);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = P.code.frozen[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = P.code.info_idx[i];
    for (int i = threadIdx.x; i < n * NH * 4; i += blockDim.x) dw[i] = Real(0);
    __syncthreads();
    const int slot = threadIdx.x / tps, tid = threadIdx.x - slot * tps;
    const size_t slot_reals = size_t(3 * n + 4) * N;
    Real* L = reinterpret_cast<Real*>(smem + tab + dw_bytes) + size_t(slot) * slot_reals;   // levels 1..n+1
    Real* Rt = L + (n + 1) * N;                                                              // R, levels 2..n+1
    Real* gL = Rt + n * N;                                                                   // levels 1..n+1
    Real* gA = gL + (n + 1) * N;
    Real* gB = gA + N;
    for (int j = tid; j < N; j += tps) Rt[(n - 1) * N + j] = prior_v<Real>(s_frozen, j);
    __shared__ long long s_frame[32];
    const unsigned bid = 1u + unsigned(slot);
    const Real* wt = P.w + size_t(it) * n * NH * 4;

    while (true) {
        if (tid == 0) s_frame[slot] = (long long)atomicAdd(P.counter, 1ull);
        bar(bid, tps);
        const long long f = s_frame[slot];
        if (f >= P.B) break;
        const Real* Rp = P.ckpt + (size_t(it) * P.B + size_t(f)) * (n - 1) * N;   // R(it) before this iteration
        // R(it) and the channel LLRs stream into their planes while the gradient planes are cleared
        auto load_rp = [&]() { copy_async(Rt, Rp, (n - 1) * N, tid, tps); };
        load_rp();
        copy_async(L, P.llr + size_t(f) * N, N, tid, tps);
        for (int j = tid; j < (n + 1) * N; j += tps) gL[j] = Real(0);
        for (int j = tid; j < N; j += tps) gA[j] = gB[j] = Real(0);
        copy_wait();
        bar(bid, tps);
        // forward recomputation of iteration it
        for (int s = 0; s < n; ++s) {
            const int p = n - 1 - s;
            const Real* Ls = L + s * N;
            const Real* Rs = Rt + s * N;                                   // R(it) at level s+2
            Real* Lo = L + (s + 1) * N;
            const Real* ws = wt + s * NH * 4;
            for (int q = tid; q < NH; q += tps) {
                const int t = ins0(q, p), b = t | (1 << p);
                const Real lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                const auto w2 = ld_pair(ws + q * 4);
                Lo[t] = fw(lt, radd(lb, rb), w2.x);
                Lo[b] = radd(fw(rt, lt, w2.y), lb);
            }
            bar(bid, tps);
        }
        if (!last) {
            for (int s = n - 1; s >= 1; --s) {
                const int p = n - 1 - s;
                const Real* Ls = L + s * N;
                const Real* Rs = Rt + s * N;
                Real* Ro = Rt + (s - 1) * N;
                const Real* ws = wt + s * NH * 4 + 2;
                for (int q = tid; q < NH; q += tps) {
                    const int t = ins0(q, p), b = t | (1 << p);
                    const Real lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    const auto w2 = ld_pair(ws + q * 4);
                    Ro[t] = fw(rt, radd(lb, rb), w2.x);
                    Ro[b] = radd(fw(rt, lt, w2.y), rb);
                }
                bar(bid, tps);
            }
        } else {
            for (int k = tid; k < K; k += tps) gL[n * N + s_info[k]] = P.glogits[size_t(f) * K + k];
            bar(bid, tps);
        }
        // adjoint of the R sweep: stage s makes R level s+1 from R level s+2 and L level s+1
        if (!last) {
            const Real* gin = P.gin + size_t(f) * (n - 1) * N;
            for (int s = 1; s <= n - 1; ++s) {
                const int p = n - 1 - s;
                const Real* gis = gin + (s - 1) * N;
                const Real* Rs = Rt + s * N;                                   // R level s+2
                const Real* Ls = L + s * N;
                Real* gLs = gL + s * N;
                const Real* ws = wt + s * NH * 4 + 2;
                Real* ds = dw + s * NH * 4;
                for (int q = tid; q < NH; q += tps) {
                    const int t = ins0(q, p), b = t | (1 << p);
                    const Real gt = radd(gis[t], gA[t]);                        // gradient of R level s+1
                    const Real gb = radd(gis[b], gA[b]);
                    const Real a = Rs[t], rb = Rs[b];
                    const Real lt = Ls[t], lb = Ls[b];
                    Real* d = ds + q * 4;
                    Real ct = Real(0), cb = Real(0);
                    if (gt != Real(0) || gb != Real(0)) {
                        const auto w2 = ld_pair(ws + q * 4);                    // w[2], w[3]
                        if (gt != Real(0)) {                                    // R_out1 = f(a, lb + rb; w2)
                            const Real c = radd(lb, rb);
                            const bool amin = fabs(a) <= fabs(c);
                            const Real m = amin ? fabs(a) : fabs(c);
                            atomicAdd(d + 2, rmul(gt, sgn(a) * sgn(c) * m));
                            if (amin) {
                                ct = radd(ct, rmul(rmul(gt, w2.x), sgn(c)));
                            } else {
                                const Real gc = rmul(rmul(gt, w2.x), sgn(a));
                                gLs[b] = radd(gLs[b], gc);
                                cb = radd(cb, gc);
                            }
                        }
                        if (gb != Real(0)) {                                    // R_out2 = f(a, lt; w3) + rb
                            cb = radd(cb, gb);
                            const bool amin = fabs(a) <= fabs(lt);
                            const Real m = amin ? fabs(a) : fabs(lt);
                            atomicAdd(d + 3, rmul(gb, sgn(a) * sgn(lt) * m));
                            if (amin) ct = radd(ct, rmul(rmul(gb, w2.y), sgn(lt)));
                            else gLs[t] = radd(gLs[t], rmul(rmul(gb, w2.y), sgn(a)));
                        }
                    }
                    gB[t] = ct;                                                 // contributions to R level s+2
                    gB[b] = cb;
                }
                bar(bid, tps);
                Real* tmp = gA; gA = gB; gB = tmp;
            }
        }
        // adjoint of the L sweep: stage s makes L level s+2 from L level s+1 and R(it) level s+2
        if (!last) {                  // the R planes hold R(it+1): R(it) again
            load_rp();
            copy_wait();
            bar(bid, tps);
        }
        Real* gout = P.gout + size_t(f) * (n - 1) * N;
        for (int s = n - 1; s >= 0; --s) {
            const int p = n - 1 - s;
            const Real* Ls = L + s * N;
            const Real* Rs = Rt + s * N;
            Real* gLs = gL + s * N;
            const Real* gLo = gL + (s + 1) * N;
            const Real* ws = wt + s * NH * 4;
            Real* ds = dw + s * NH * 4;
            Real* gos = gout + size_t(s) * N;
            for (int q = tid; q < NH; q += tps) {
                const int t = ins0(q, p), b = t | (1 << p);
                const Real gt = gLo[t], gb = gLo[b];
                Real gRt = Real(0), gRb = Real(0);
                Real gat = gLs[t], gab = gLs[b];
                if (gt != Real(0) || gb != Real(0)) {
                    const Real a = Ls[t], lb = Ls[b];
                    const Real rt = Rs[t], rb = Rs[b];
                    const auto w2 = ld_pair(ws + q * 4);                        // w[0], w[1]
                    Real* d = ds + q * 4;
                    if (gt != Real(0)) {                                        // L_out1 = f(a, lb + rb; w0)
                        const Real c = radd(lb, rb);
                        const bool amin = fabs(a) <= fabs(c);
                        const Real m = amin ? fabs(a) : fabs(c);
                        atomicAdd(d + 0, rmul(gt, sgn(a) * sgn(c) * m));
                        if (amin) {
                            gat = radd(gat, rmul(rmul(gt, w2.x), sgn(c)));
                        } else {
                            const Real gc = rmul(rmul(gt, w2.x), sgn(a));
                            gab = radd(gab, gc);
                            gRb = radd(gRb, gc);
                        }
                    }
                    if (gb != Real(0)) {                                        // L_out2 = f(rt, a; w1) + lb
                        gab = radd(gab, gb);
                        const bool rmin = fabs(rt) <= fabs(a);
                        const Real m = rmin ? fabs(rt) : fabs(a);
                        atomicAdd(d + 1, rmul(gb, sgn(rt) * sgn(a) * m));
                        if (rmin) gRt = radd(gRt, rmul(rmul(gb, w2.y), sgn(a)));
                        else gat = radd(gat, rmul(rmul(gb, w2.y), sgn(rt)));
                    }
                }
                gLs[t] = gat;
                gLs[b] = gab;
                if (s < n - 1) {
                    gos[t] = gRt;
                    gos[b] = gRb;
                }
            }
            bar(bid, tps);
        }
        if (P.gllr)
            for (int j = tid; j < N; j += tps) P.gllr[size_t(f) * N + j] = radd(P.gllr[size_t(f) * N + j], gL[j]);
        bar(bid, tps);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * NH * 4; i += blockDim.x)
        if (dw[i] != Real(0)) atomicAdd(P.gw + size_t(it) * n * NH * 4 + i, dw[i]);
}

// ---------------------------------------------------------------------------
// FP32 backward for N <= 1024, one thread per processing element (tps = N/2) with the stage loops
// unrolled for the length: every thread accumulates the weight gradient of its element (n x 4
// values) in registers over all the frames it handles and adds it to gw once at the end, so the
// shared memory that the accumulator takes in the kernel above holds, per frame slot, the
// incoming gradient planes (levels 2..n, copied with cp.async when the frame starts instead of
// read from global memory at every stage of the R-sweep adjoint) and a second set of R planes.
// The arithmetic of every stage is the kernel above's.
// Per slot: L levels 1..n (plane n unused: L level n+1 is not needed), R(it) (the checkpoint,
// levels 2..n), R(it+1) recomputed (levels 2..n) and the priors (level n+1), the gradient of L
// at levels 1..n+1, two gradient planes between R levels and G, the incoming gradient (levels
// 2..n): (5n+2) N floats, in the sw32 layout.  Between two stages of butterfly distance at most
// 32 a warp waits only for itself (stage_sync); the gradient planes are left zero by the stage
// that consumes them, so a frame starts without clearing them; the next frame's index and this
// frame's accumulated LLR gradient are read early and used later, so neither round trip stalls
// the slot.
template <int LOGN>
__global__ void __launch_bounds__(512, 1) wbp_backward_reg_kernel(const __grid_constant__ WbpParams<float> P)
{
    constexpr int n = LOGN, N = 1 << LOGN, NH = N / 2;
    constexpr int NW = N >= 32 ? N / 32 : 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = P.code.K;
    const int tps = P.tps, it = P.it;
    const bool last = it == P.T - 1;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    int16_t* s_info = reinterpret_cast<int16_t*>(s_frozen + NW);
    const size_t tab = (size_t(NW) * 4 + size_t(K) * 2 + 15) & ~size_t(15);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = P.code.frozen[i];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = P.code.info_idx[i];
    __syncthreads();
    const int slot = threadIdx.x / tps, tid = threadIdx.x - slot * tps;
    constexpr size_t slot_reals = size_t(5 * n + 2) * N;
    float* const L = reinterpret_cast<float*>(smem + tab) + size_t(slot) * slot_reals;   // levels 1..n
    float* const Rnw = L + (n + 1) * N;                                                 // R(it+1), levels 2..n
    float* const Pri = Rnw + (n - 1) * N;                                               // R level n+1
    float* const gL = Rnw + n * N;                                                      // levels 1..n+1
    float* gA = gL + (n + 1) * N;
    float* gB = gA + N;
    float* const G = gB + N;                                                            // incoming, levels 2..n
    float* const Rck = G + (n - 1) * N;                                                 // R(it), levels 2..n
    for (int j = tid; j < N; j += tps) Pri[sw32(j)] = prior_v<float>(s_frozen, j);
    for (int j = tid; j < (n + 1) * N; j += tps) gL[j] = 0.f;
    __shared__ long long s_frame[32], s_next[32];
    const unsigned bid = 1u + unsigned(slot);
    const float* wt = P.w + size_t(it) * n * NH * 4;
    const bool act = tid < NH;                 // N < 64: fewer elements than a warp
    const int q = act ? tid : 0;
    float dwr[n][4];
#pragma unroll
    for (int s = 0; s < n; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) dwr[s][k] = 0.f;

    // the thread's weight pairs of this iteration, each loaded one stage ahead of its use (the
    // weights are read-only and the same for every frame of the launch, so a load may be issued
    // before the barrier that ends the stage using the previous pair): w[k], w[k+1] of stage s
    auto wpair = [&](int s, int k) { return ld_pair(wt + (s * NH + q) * 4 + k); };
    // inputs of frame fx: the checkpoint R(it), the LLRs (L level 1) and (before the last
    // iteration) the incoming gradient
    auto fetch = [&](long long fx) {
        copy_async(Rck, P.ckpt + (size_t(it) * P.B + size_t(fx)) * (n - 1) * N, (n - 1) * N, tid, tps);
        copy_async_sw(L, P.llr + size_t(fx) * N, N, tid, tps);
        if (!last) copy_async(G, P.gin + size_t(fx) * (n - 1) * N, (n - 1) * N, tid, tps);
    };
    // the next frame's index is taken as a frame starts and published by the slot leader a few
    // stages later, before the slot barrier that ends the last forward stage of distance 2^6 or
    // more (or the first stage, where the slot is one warp), so the atomic's round trip overlaps
    // the stages
    constexpr int s_pub = n >= 7 ? n - 7 : 0;
    float2 wc = wpair(0, 0);
    if (tid == 0) s_frame[slot] = (long long)atomicAdd(P.counter, 1ull);
    bar(bid, tps);
    long long f = s_frame[slot];
    while (f < P.B) {
        unsigned long long nf = 0;
        if (tid == 0) nf = atomicAdd(P.counter, 1ull);
        fetch(f);
        copy_wait();
        bar(bid, tps);
        // forward recomputation of iteration it (L level n+1 is not needed)
#pragma unroll
        for (int s = 0; s < n - 1; ++s) {
            const float2 w2 = wc;
            wc = s + 1 < n - 1 ? wpair(s + 1, 0) : wpair(n - 1, last ? 0 : 2);   // next: this sweep, the R sweep or the adjoint of the L sweep
            const int p = n - 1 - s;
            if (act) {
                const float* Ls = L + s * N;
                const float* Rs = Rck + s * N;                                  // R(it) at level s+2
                float* Lo = L + (s + 1) * N;
                const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                const float lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                Lo[t] = fw(lt, radd(lb, rb), w2.x);
                Lo[b] = radd(fw(rt, lt, w2.y), lb);
            }
            if (s == s_pub && tid == 0) s_next[slot] = (long long)nf;
            stage_sync(p, p - 1, bid, tps);
        }
        const long long fn = s_next[slot];
        // this frame's accumulated LLR gradient, read now and added after the adjoint of the L sweep
        float gll[2] = {0.f, 0.f};
        if (P.gllr) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (tid + h * tps < N) gll[h] = P.gllr[size_t(f) * N + tid + h * tps];
        }
        if (!last) {
#pragma unroll
            for (int s = n - 1; s >= 1; --s) {
                const float2 w2 = wc;
                if (s > 1) wc = wpair(s - 1, 2);          // (stage 1's pair also starts the adjoint of the R sweep)
                const int p = n - 1 - s;
                if (act) {
                    const float* Ls = L + s * N;
                    const float* Rs = s == n - 1 ? Pri : Rnw + s * N;
                    float* Ro = Rnw + (s - 1) * N;
                    const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                    const float lt = Ls[t], lb = Ls[b], rt = Rs[t], rb = Rs[b];
                    Ro[t] = fw(rt, radd(lb, rb), w2.x);
                    Ro[b] = radd(fw(rt, lt, w2.y), rb);
                }
                stage_sync(p, s > 1 ? p + 1 : n - 2, bid, tps);
            }
        } else {
            for (int k = tid; k < K; k += tps) gL[n * N + sw32(s_info[k])] = P.glogits[size_t(f) * K + k];
            bar(bid, tps);
        }
        // adjoint of the R sweep: stage s makes R level s+1 from R level s+2 and L level s+1
        if (!last) {
#pragma unroll
            for (int s = 1; s <= n - 1; ++s) {
                const float2 w2 = wc;
                wc = s + 1 <= n - 1 ? wpair(s + 1, 2) : wpair(n - 1, 0);     // next: this adjoint or the L sweep's
                const int p = n - 1 - s;
                if (act) {
                    const float* gis = G + (s - 1) * N;
                    const float* Rs = s == n - 1 ? Pri : Rnw + s * N;           // R level s+2
                    const float* Ls = L + s * N;
                    float* gLs = gL + s * N;
                    const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                    // gradient of R level s+1 (stage 1 has no contribution from a previous stage)
                    const float gt = s == 1 ? gis[t] : radd(gis[t], gA[t]);
                    const float gb = s == 1 ? gis[b] : radd(gis[b], gA[b]);
                    const float a = Rs[t], rb = Rs[b];
                    const float lt = Ls[t], lb = Ls[b];
                    float ct = 0.f, cb = 0.f;
                    if (gt != 0.f || gb != 0.f) {
                        // both operand cases evaluated and the contributions of the case that does
                        // not apply replaced by exact zeros (adding 0 leaves a sum as it is), so the
                        // warp does not diverge on which operand is the minimum; a product with a
                        // zero upstream gradient is never used (it may be 0 * inf)
                        const bool g1 = gt != 0.f, g2 = gb != 0.f;
                        // R_out1 = f(a, lb + rb; w2)
                        const float c = radd(lb, rb);
                        const bool amin = fabsf(a) <= fabsf(c);
                        const float m1 = amin ? fabsf(a) : fabsf(c);
                        const float d1 = rmul(gt, sgn(a) * sgn(c) * m1);
                        dwr[s][2] = radd(dwr[s][2], g1 ? d1 : 0.f);
                        const float v1 = rmul(rmul(gt, w2.x), amin ? sgn(c) : sgn(a));
                        ct = g1 && amin ? v1 : 0.f;
                        cb = g1 && !amin ? v1 : 0.f;
                        if (g1 && !amin) gLs[b] = radd(gLs[b], v1);
                        // R_out2 = f(a, lt; w3) + rb
                        cb = radd(cb, gb);
                        const bool amin2 = fabsf(a) <= fabsf(lt);
                        const float m2 = amin2 ? fabsf(a) : fabsf(lt);
                        const float d2 = rmul(gb, sgn(a) * sgn(lt) * m2);
                        dwr[s][3] = radd(dwr[s][3], g2 ? d2 : 0.f);
                        const float v2 = rmul(rmul(gb, w2.y), amin2 ? sgn(lt) : sgn(a));
                        ct = radd(ct, g2 && amin2 ? v2 : 0.f);
                        if (g2 && !amin2) gLs[t] = radd(gLs[t], v2);
                    }
                    if (s < n - 1) {                                             // contributions to R level s+2
                        gB[t] = ct;
                        gB[b] = cb;
                    }
                }
                stage_sync(p, s < n - 1 ? p - 1 : 0, bid, tps);
                float* tmp = gA; gA = gB; gB = tmp;
            }
        }
        // adjoint of the L sweep: stage s makes L level s+2 from L level s+1 and R(it) level s+2
        float* gout = P.gout + size_t(f) * (n - 1) * N;
#pragma unroll
        for (int s = n - 1; s >= 0; --s) {
            const float2 w2 = wc;
            if (s > 0) wc = wpair(s - 1, 0);              // (stage 0's pair also starts the next frame)
            const int p = n - 1 - s;
            if (act) {
                const float* Ls = L + s * N;
                const float* Rs = s < n - 1 ? Rck + s * N : Pri;                // R(it) level s+2 (n+1: priors)
                float* gLs = gL + s * N;
                float* gLo = gL + (s + 1) * N;
                float* gos = gout + size_t(s) * N;
                const int t = sw32(ins0(q, p)), b = sw32(ins0(q, p) | (1 << p));
                const float gt = gLo[t], gb = gLo[b];
                gLo[t] = 0.f;                                                    // cleared for the next frame
                gLo[b] = 0.f;
                float gRt = 0.f, gRb = 0.f;
                float gat = gLs[t], gab = gLs[b];
                if (gt != 0.f || gb != 0.f) {
                    // both operand cases, the one that does not apply contributing exact zeros
                    // (as in the adjoint of the R sweep)
                    const float a = Ls[t], lb = Ls[b];
                    const float rt = Rs[t], rb = Rs[b];
                    const bool g1 = gt != 0.f, g2 = gb != 0.f;
                    // L_out1 = f(a, lb + rb; w0)
                    const float c = radd(lb, rb);
                    const bool amin = fabsf(a) <= fabsf(c);
                    const float m1 = amin ? fabsf(a) : fabsf(c);
                    const float d1 = rmul(gt, sgn(a) * sgn(c) * m1);
                    dwr[s][0] = radd(dwr[s][0], g1 ? d1 : 0.f);
                    const float v1 = rmul(rmul(gt, w2.x), amin ? sgn(c) : sgn(a));
                    gat = radd(gat, g1 && amin ? v1 : 0.f);
                    gab = radd(gab, g1 && !amin ? v1 : 0.f);
                    gRb = g1 && !amin ? v1 : 0.f;
                    // L_out2 = f(rt, a; w1) + lb
                    gab = radd(gab, gb);
                    const bool rmin = fabsf(rt) <= fabsf(a);
                    const float m2 = rmin ? fabsf(rt) : fabsf(a);
                    const float d2 = rmul(gb, sgn(rt) * sgn(a) * m2);
                    dwr[s][1] = radd(dwr[s][1], g2 ? d2 : 0.f);
                    const float v2 = rmul(rmul(gb, w2.y), rmin ? sgn(a) : sgn(rt));
                    gRt = g2 && rmin ? v2 : 0.f;
                    gat = radd(gat, g2 && !rmin ? v2 : 0.f);
                }
                gLs[t] = gat;
                gLs[b] = gab;
                if (s < n - 1) {
                    gos[t] = gRt;
                    gos[b] = gRb;
                }
            }
            stage_sync(p, s > 0 ? p + 1 : kCross, bid, tps);
        }
        // the gradient of the LLRs (L level 1), then level 1 cleared for the next frame
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = tid + h * tps;
            if (j < N) {
                if (P.gllr) P.gllr[size_t(f) * N + j] = radd(gll[h], gL[sw32(j)]);
                gL[sw32(j)] = 0.f;
            }
        }
        f = fn;
    }
    if (act) {
        float* g = P.gw + size_t(it) * n * NH * 4 + size_t(q) * 4;
#pragma unroll
        for (int s = 0; s < n; ++s)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (dwr[s][k] != 0.f) atomicAdd(g + size_t(s) * NH * 4 + k, dwr[s][k]);
    }
}

struct Geo {
    int tps, slots, grid;
    size_t smem;
};

// reg: the FP32 backward with the weight gradient in registers (wbp_backward_reg_kernel).
int wbp_geometry(const pc_code* c, int64_t B, size_t real_bytes, bool backward, Geo* g, bool reg = false)
{
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PC_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return PC_ECUDA;
    optin -= 1024;   // static shared variables of the kernels
    const int N = c->N, n = c->n;
    const int NW = N >= 32 ? N / 32 : 1;
    const size_t tab = (size_t(NW) * 4 + size_t(c->K) * 2 + 15) & ~size_t(15);
    const size_t fixed =
        tab + (backward && !reg ? ((size_t(n) * (N / 2) * 4 * real_bytes + 15) & ~size_t(15)) : 0);
    const size_t slot = (reg ? size_t(5 * n + 2) : (backward ? size_t(3 * n + 4) : size_t(2 * n + 1))) * N * real_bytes;
    g->tps = std::max(32, std::min(512, N / 2));
    if (fixed + slot > size_t(optin)) return PC_EUNSUPPORTED;
    int slots = int((size_t(optin) - fixed) / slot);
    slots = std::max(1, std::min({slots, 15, (reg ? 512 : 1024) / g->tps}));
    g->slots = slots;
    g->smem = fixed + size_t(slots) * slot;
    g->grid = int(std::min<int64_t>(int64_t(sms), (B + slots - 1) / slots));
    return PC_OK;
}

int validate_common(const pc_code* c, int32_t T, int64_t B)
{
    int rc = validate_code(c);
    if (rc != PC_OK) return rc;
    if (T < 1 || T > 1024 || B < 0) return PC_EINVAL;
    return PC_OK;
}

size_t workspace_bytes(const pc_code* c, int64_t B, size_t real_bytes)
{
    return 256 + 2 * size_t(B) * size_t(c->n - 1) * size_t(c->N) * real_bytes;
}

// The unrolled FP32 forward, instantiated for n = 4..10.
cudaError_t launch_forward_reg(int n, const WbpParams<float>& P, const Geo& g, cudaStream_t st)
{
#define PCBP_WBP_FWD(k)                                                                                      \
    case k: {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(wbp_forward_reg_kernel<k>,                                      \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem));      \
        if (e != cudaSuccess) return e;                                                                      \
        wbp_forward_reg_kernel<k><<<g.grid, g.slots * g.tps, g.smem, st>>>(P);                               \
        return cudaGetLastError();                                                                           \
    }
    switch (n) {
        PCBP_WBP_FWD(4)
        PCBP_WBP_FWD(5)
        PCBP_WBP_FWD(6)
        PCBP_WBP_FWD(7)
        PCBP_WBP_FWD(8)
        PCBP_WBP_FWD(9)
        PCBP_WBP_FWD(10)
        default: return cudaErrorInvalidValue;
    }
#undef PCBP_WBP_FWD
}

// The register-accumulating FP32 backward, instantiated for n = 3..10.
cudaError_t launch_backward_reg(int n, const WbpParams<float>& P, const Geo& g, cudaStream_t st)
{
#define PCBP_WBP_REG(k)                                                                                      \
    case k: {                                                                                                \
        cudaError_t e = cudaFuncSetAttribute(wbp_backward_reg_kernel<k>,                                     \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem));      \
        if (e != cudaSuccess) return e;                                                                      \
        wbp_backward_reg_kernel<k><<<g.grid, g.slots * g.tps, g.smem, st>>>(P);                              \
        return cudaGetLastError();                                                                           \
    }
    switch (n) {
        PCBP_WBP_REG(3)
        PCBP_WBP_REG(4)
        PCBP_WBP_REG(5)
        PCBP_WBP_REG(6)
        PCBP_WBP_REG(7)
        PCBP_WBP_REG(8)
        PCBP_WBP_REG(9)
        PCBP_WBP_REG(10)
        default: return cudaErrorInvalidValue;
    }
#undef PCBP_WBP_REG
}

template <typename Real>
int forward_impl(const pc_code* c, const Real* llr, const Real* w, int32_t T, int64_t B, Real* logits, Real* ckpt,
                 void* ws, void* stream)
{
    int rc = validate_common(c, T, B);
    if (rc != PC_OK) return rc;
    if (B == 0) return PC_OK;
    if (!llr || !w || !logits || !ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return PC_EINVAL;
    if (reinterpret_cast<uintptr_t>(w) & (2 * sizeof(Real) - 1)) return PC_EINVAL;   // weights are read in pairs
    Geo g;
    rc = wbp_geometry(c, B, sizeof(Real), false, &g);
    if (rc != PC_OK) return rc;
    std::unique_ptr<WbpParams<Real>> P(new WbpParams<Real>);
    std::memset(P.get(), 0, sizeof(WbpParams<Real>));
    build_dev_code(c, &P->code);
    P->llr = llr;
    P->w = w;
    P->logits = logits;
    P->ckpt = ckpt;
    P->counter = static_cast<unsigned long long*>(ws);
    P->B = B;
    P->T = T;
    P->tps = g.tps;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, 8, st) != cudaSuccess) return PC_ECUDA;
    if constexpr (std::is_same<Real, float>::value) {
        // FP32 from N = 16 to 1024 (the unrolled backward reads its checkpoints in the sw32
        // layout; at N = 8 that layout is the natural order the generic kernel writes)
        if (c->n >= 4 && c->n <= 10)
            return launch_forward_reg(c->n, *P, g, st) == cudaSuccess ? PC_OK : PC_ECUDA;
    }
    if (cudaFuncSetAttribute(wbp_forward_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem)) !=
        cudaSuccess)
        return PC_ECUDA;
    wbp_forward_kernel<Real><<<g.grid, g.slots * g.tps, g.smem, st>>>(*P);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ECUDA;
}

template <typename Real>
int backward_impl(const pc_code* c, const Real* llr, const Real* w, int32_t T, int64_t B, const Real* ckpt,
                  const Real* glogits, Real* gw, Real* gllr, void* ws, void* stream)
{
    int rc = validate_common(c, T, B);
    if (rc != PC_OK) return rc;
    if (B == 0) return PC_OK;
    if (!llr || !w || !ckpt || !glogits || !gw || !ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return PC_EINVAL;
    if (reinterpret_cast<uintptr_t>(w) & (2 * sizeof(Real) - 1)) return PC_EINVAL;   // weights are read in pairs
    // FP32 up to N = 1024: the weight gradient in registers, incoming gradients staged per frame
    const bool reg = std::is_same<Real, float>::value && c->n <= 10;
    Geo g;
    rc = wbp_geometry(c, B, sizeof(Real), true, &g, reg);
    if (rc != PC_OK) return rc;
    std::unique_ptr<WbpParams<Real>> P(new WbpParams<Real>);
    std::memset(P.get(), 0, sizeof(WbpParams<Real>));
    build_dev_code(c, &P->code);
    P->llr = llr;
    P->w = w;
    P->ckpt = const_cast<Real*>(ckpt);
    P->glogits = glogits;
    P->gw = gw;
    P->gllr = gllr;
    P->counter = static_cast<unsigned long long*>(ws);
    P->B = B;
    P->T = T;
    P->tps = g.tps;
    Real* state[2];
    state[0] = reinterpret_cast<Real*>(static_cast<unsigned char*>(ws) + 256);
    state[1] = state[0] + size_t(B) * size_t(c->n - 1) * size_t(c->N);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (gllr && cudaMemsetAsync(gllr, 0, size_t(B) * c->N * sizeof(Real), st) != cudaSuccess) return PC_ECUDA;
    if (!reg && cudaFuncSetAttribute(wbp_backward_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(g.smem)) != cudaSuccess)
        return PC_ECUDA;
    for (int it = T - 1; it >= 0; --it) {
        P->it = it;
        P->gin = state[(T - 1 - it) & 1];      // written by the launch of iteration it+1 (unused at it = T-1)
        P->gout = state[(T - it) & 1];
        if (cudaMemsetAsync(ws, 0, 8, st) != cudaSuccess) return PC_ECUDA;
        if constexpr (std::is_same<Real, float>::value) {
            if (reg) {
                if (launch_backward_reg(c->n, *P, g, st) != cudaSuccess) return PC_ECUDA;
                continue;
            }
        }
        wbp_backward_kernel<Real><<<g.grid, g.slots * g.tps, g.smem, st>>>(*P);
        if (cudaGetLastError() != cudaSuccess) return PC_ECUDA;
    }
    return PC_OK;
}

}  // namespace

}  // namespace pcbp

using namespace pcbp;

extern "C" int wbp_weights_count(const pc_code* code, int32_t T, size_t* count)
{
    int rc = validate_common(code, T, 0);
    if (rc != PC_OK) return rc;
    if (!count) return PC_EINVAL;
    *count = size_t(T) * code->n * (code->N / 2) * 4;
    return PC_OK;
}

extern "C" int wbp_ckpt_count(const pc_code* code, int32_t T, int64_t B, size_t* count)
{
    int rc = validate_common(code, T, B);
    if (rc != PC_OK) return rc;
    if (!count) return PC_EINVAL;
    *count = size_t(T) * size_t(B) * size_t(code->n - 1) * size_t(code->N);
    return PC_OK;
}

extern "C" int wbp_workspace_size(const pc_code* code, int32_t T, int64_t B, int32_t real_bytes, size_t* bytes)
{
    int rc = validate_common(code, T, B);
    if (rc != PC_OK) return rc;
    if (!bytes || (real_bytes != 4 && real_bytes != 8)) return PC_EINVAL;
    *bytes = workspace_bytes(code, B, size_t(real_bytes));
    return PC_OK;
}

extern "C" int wbp_forward(const pc_code* code, const float* d_llr, const float* d_w, int32_t T, int64_t B,
                           float* d_logits, float* d_ckpt, void* d_workspace, void* stream)
{
    return forward_impl<float>(code, d_llr, d_w, T, B, d_logits, d_ckpt, d_workspace, stream);
}

extern "C" int wbp_backward(const pc_code* code, const float* d_llr, const float* d_w, int32_t T, int64_t B,
                            const float* d_ckpt, const float* d_glogits, float* d_gw, float* d_gllr,
                            void* d_workspace, void* stream)
{
    return backward_impl<float>(code, d_llr, d_w, T, B, d_ckpt, d_glogits, d_gw, d_gllr, d_workspace, stream);
}

extern "C" int wbp_forward_f64(const pc_code* code, const double* d_llr, const double* d_w, int32_t T, int64_t B,
                               double* d_logits, double* d_ckpt, void* d_workspace, void* stream)
{
    return forward_impl<double>(code, d_llr, d_w, T, B, d_logits, d_ckpt, d_workspace, stream);
}

extern "C" int wbp_backward_f64(const pc_code* code, const double* d_llr, const double* d_w, int32_t T, int64_t B,
                                const double* d_ckpt, const double* d_glogits, double* d_gw, double* d_gllr,
                                void* d_workspace, void* stream)
{
    return backward_impl<double>(code, d_llr, d_w, T, B, d_ckpt, d_glogits, d_gw, d_gllr, d_workspace, stream);
}
