// PP-BP decoder kernel for sm_103a (Algorithm 1 of arXiv 1911.08868).
//
// Layout.  A CTA holds `slots` independent frame slots of T threads each.
// Each slot keeps one frame's message planes in shared memory:
//   L planes of node levels 1..n   (level 1 = channel LLRs, Sec. II-B),
//   R planes of node levels 2..n   (R at level n+1 is the prior: +inf frozen,
//                                   0 information, read from the frozen mask),
// plus the packed decisions of the current iteration.  L at level n+1 is
// consumed as it is produced (decision), R at level 1 only feeds the G-matrix
// test.  The CTA-wide code tables (frozen mask, CRC bit-planes, information
// positions) are copied to shared memory once.  Slots synchronise on their
// own named barrier (bar.sync 1+slot, T) and fetch frames from a global
// counter, so a frame that stops early frees its slot for the next frame
// without waiting for the rest of the CTA.
//
// Stage addressing.  Stage s (0-based; stage s+1 of the paper, counted from
// the channel) pairs indices differing in bit p = n-1-s in the original graph
// (Arikan's graph of x = u F^{(x)n}: the channel-side stage pairs the halves
// of x, the u-side stage pairs neighbours).  Processing element q of a stage
// pairs t = q with a zero inserted at bit p and b = t | 2^p.  A permutation
// event of levels level..m (m = level+range-1) acts on one of the N/2^m
// subgraphs formed by stages 1..m, the indices whose n-m low bits equal
// `block`; there stage s uses bit pbit[s].  Every bit those stages use is at
// least n-m, so inserting it into q keeps q's low bits: the PE belongs to the
// subgraph iff (q & (2^(n-m) - 1)) == block, one test per PE.
//
// Arithmetic.  Every FP32 operation is an explicitly rounded intrinsic
// (__fadd_rn, __fmul_rn): no contraction, so the decoder reproduces a
// straightforward FP32 evaluation of the PE equations bit for bit.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pcbp_internal.h"

namespace pcbp {

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

template <int LOGN>
__host__ __device__ constexpr int words_of() { return (1 << LOGN) >= 32 ? (1 << LOGN) / 32 : 1; }

// Threads per frame slot: two PEs per thread per stage, 32 .. 512.
template <int LOGN>
__host__ __device__ constexpr int threads_per_slot()
{
    return (1 << LOGN) / 4 < 32 ? 32 : ((1 << LOGN) / 4 > 512 ? 512 : (1 << LOGN) / 4);
}

constexpr int kCtlBytes = 128;

template <int LOGN>
__host__ __device__ constexpr size_t slot_bytes()
{
    return kCtlBytes + align16(2 * words_of<LOGN>() * 4) + size_t(2 * LOGN - 1) * (size_t(1) << LOGN) * 4;
}

__host__ __device__ inline size_t shared_table_bytes(int nw, int r, int K)
{
    return align16(size_t(nw) * 4 + size_t(r) * nw * 4 + size_t(K) * 2);
}

struct SlotCtl {
    long long frame;
    long long ev_blk, pv_blk;
    int crc_res, g_ok;
    int ev_level, ev_range, have_ev;
    int pv_level, pv_range, have_prev;
    int next_inc;
    signed char pbit[16];
};
static_assert(sizeof(SlotCtl) <= kCtlBytes, "slot control block");

// ---------------------------------------------------------------------------
// Counter-based draws: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), output
// for state x = finaliser(x + golden gamma); a draw keyed by (seed, frame,
// event k, draw d) chains it as sm(sm(sm(sm(seed) ^ frame) ^ k) ^ d).
__device__ __forceinline__ uint64_t splitmix_out(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t event_draw(uint64_t seed, uint64_t frame, uint64_t k, uint64_t d)
{
    return splitmix_out(splitmix_out(splitmix_out(splitmix_out(seed) ^ frame) ^ k) ^ d);
}

// The random choices of a switch (Sec. III, Algorithm 1); FP-BP
// draws a full order (level 1, range n, one block).  The stage order is a
// uniform non-identity permutation: Fisher-Yates, redrawn while identity, a
// rotation after 8 identity draws.
static __device__ __noinline__ void draw_event(const DevSched& S, int n, uint64_t frame, int k, int& level, int& range,
                                  long long& block, signed char* order)
{
    if (S.mode == 2) {
        range = n;
        level = 1;
        block = 0;
    } else {
        range = S.rho_fixed > 0 ? S.rho_fixed
                                : 2 + int(event_draw(S.seed, frame, uint64_t(k), 0) % uint64_t(S.P_range - 1));
        const int x = 1 + int(event_draw(S.seed, frame, uint64_t(k), 1) % uint64_t(S.P_level));
        level = min(x, n - range + 1);
        const int m = level + range - 1;
        block = (long long)(event_draw(S.seed, frame, uint64_t(k), 2) % (1ull << (n - m)));
    }
    for (int attempt = 0; attempt < 8; ++attempt) {
        for (int i = 0; i < range; ++i) order[i] = (signed char)i;
        for (int i = range - 1; i >= 1; --i) {
            const uint64_t d = 3 + 16 * uint64_t(attempt) + uint64_t(range - 1 - i);
            const int j = int(event_draw(S.seed, frame, uint64_t(k), d) % uint64_t(i + 1));
            const signed char t = order[i];
            order[i] = order[j];
            order[j] = t;
        }
        bool ident = true;
        for (int i = 0; i < range; ++i) ident = ident && (order[i] == i);
        if (!ident) return;
    }
    for (int i = 0; i < range; ++i) order[i] = (signed char)((i + 1) % range);
}

// ---------------------------------------------------------------------------
// f of Sec. II-B.  FK 0: scaled min-sum alpha*min(|a|,|b|) with the sign of
// a*b.  FK 1: exact box-plus; an infinite operand yields the other operand.
template <int FK>
__device__ __forceinline__ float fnode(float a, float b, float alpha);

// min(|a|,|b|) carrying the sign bit sign(a) XOR sign(b), one instruction
// (min.xorsign.abs); alpha * that value has exactly the bits of alpha *
// min(|a|,|b|) with the product sign applied afterwards, for any alpha.
__device__ __forceinline__ float signed_min(float a, float b)
{
    float m;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(m) : "f"(a), "f"(b));
    return m;
}

template <>
__device__ __forceinline__ float fnode<0>(float a, float b, float alpha)
{
    return __fmul_rn(alpha, signed_min(a, b));
}

// Hardware base-2 exponential and reciprocal (approximate, subnormals flushed).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact box-plus: f(a, b) = sign(a) sign(b) min(|a|, |b|) + c with the
// correction c = log1p(e^-|a+b|) - log1p(e^-|a-b|).  With p = e^-|a+b| and
// q = e^-|a-b|, both in [0, 1],
//   c = ln((1 + p) / (1 + q)) = 2 atanh(s),   s = (p - q) / (2 + p + q),  |s| <= 1/3,
// and 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...) is summed through s^13/13 in
// Horner form in s^2; the omitted tail is at most (1/3)^15 / 15 / (1 - 1/9),
// below 5.2e-9.  p and q come from the hardware base-2 exponential
// (e^-t = 2^(-t log2 e)), s from the hardware reciprocal.  One infinite
// operand gives p = q = 0, so c = 0 and f is the other operand's value with
// the product sign; two infinite operands return the min term directly.
template <>
__device__ __forceinline__ float fnode<1>(float a, float b, float)
{
    constexpr float kNegLog2e = -1.44269504088896341f;
    float sm;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(sm) : "f"(a), "f"(b));
    const float p = ex2_approx(__fmul_rn(fabsf(__fadd_rn(a, b)), kNegLog2e));
    const float q = ex2_approx(__fmul_rn(fabsf(__fsub_rn(a, b)), kNegLog2e));
    const float s = __fmul_rn(__fsub_rn(p, q), rcp_approx(__fadd_rn(2.f, __fadd_rn(p, q))));
    const float z = __fmul_rn(s, s);
    float h = 1.f / 13.f;
    h = __fmaf_rn(h, z, 1.f / 11.f);
    h = __fmaf_rn(h, z, 1.f / 9.f);
    h = __fmaf_rn(h, z, 1.f / 7.f);
    h = __fmaf_rn(h, z, 1.f / 5.f);
    h = __fmaf_rn(h, z, 1.f / 3.f);
    h = __fmaf_rn(h, z, 1.f);
    const float v = __fmaf_rn(__fmul_rn(2.f, s), h, sm);
    return isinf(sm) ? sm : v;
}

__device__ __forceinline__ float prior_of(const uint32_t* frozen, int j)
{
    return ((frozen[j >> 5] >> (j & 31)) & 1u) ? __int_as_float(0x7f800000) : 0.f;
}

__device__ __forceinline__ void slot_sync(unsigned id, unsigned count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// CRC residue of the decided information vector: bit i is the parity of
// (decisions & crcplane[i]) over all words.  One warp.
template <int NW>
__device__ __forceinline__ uint32_t crc_residue(const uint32_t* dec, const uint32_t* s_crc, int r, int lane)
{
    uint32_t res = 0;
    for (int i = 0; i < r; ++i) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = lane; w < NW; w += 32) acc ^= dec[w] & s_crc[i * NW + w];
        const uint32_t bal = __ballot_sync(0xffffffffu, __popc(acc) & 1);
        res |= uint32_t(__popc(bal) & 1) << i;
    }
    return res;
}

// G-matrix test (one warp): re-encode the decisions with x = u G_N over the
// original graph and compare with the hard decisions of L1 + R1.
template <int LOGN>
__device__ __forceinline__ bool g_check(const uint32_t* dec, const uint32_t* xh, int lane)
{
    constexpr int NW = words_of<LOGN>();
    constexpr int PER = NW > 32 ? NW / 32 : 1;
    uint32_t v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int w = lane + 32 * e;
        v[e] = w < NW ? dec[w] : 0u;
    }
    constexpr uint32_t masks[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
    for (int p = 0; p < (LOGN < 5 ? LOGN : 5); ++p)
#pragma unroll
        for (int e = 0; e < PER; ++e) v[e] ^= (v[e] >> (1 << p)) & masks[p];
#pragma unroll
    for (int p = 5; p < LOGN; ++p) {
        const int q = p - 5;
        if (q < 5) {
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const uint32_t other = __shfl_xor_sync(0xffffffffu, v[e], 1 << q);
                if (!((lane >> q) & 1)) v[e] ^= other;
            }
        } else {
            v[0] ^= v[PER - 1];
        }
    }
    bool ok = true;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int w = lane + 32 * e;
        if (w < NW) ok = ok && (v[e] == xh[w]);
    }
    return __all_sync(0xffffffffu, ok);
}

// ---------------------------------------------------------------------------
template <int LOGN, int T, bool TRACE, int FK>
__global__ void __launch_bounds__(1024, 1) bp_decode_kernel(const __grid_constant__ BpParams P)
{
    constexpr int N = 1 << LOGN;
    constexpr int n = LOGN;
    constexpr int NW = words_of<LOGN>();
    constexpr int NPE = N / 2;
    constexpr int PPT = NPE >= T ? NPE / T : 1;
    constexpr int NWARP = T / 32;
    extern __shared__ __align__(16) unsigned char smem[];

    const int r = P.code.r;
    const int K = P.code.K;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_crc = s_frozen + NW;
    int16_t* s_info = reinterpret_cast<int16_t*>(s_crc + r * NW);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = P.code.frozen[i];
    for (int i = threadIdx.x; i < r * NW; i += blockDim.x) s_crc[i] = P.code.crcplane[i / NW][i % NW];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = P.code.info_idx[i];
    __syncthreads();

    const int slot = threadIdx.x / T;
    const int tid = threadIdx.x - slot * T;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    unsigned char* sbase = smem + shared_table_bytes(NW, r, K) + size_t(slot) * slot_bytes<LOGN>();
    SlotCtl* ctl = reinterpret_cast<SlotCtl*>(sbase);
    uint32_t* dec = reinterpret_cast<uint32_t*>(sbase + kCtlBytes);
    uint32_t* xh = dec + NW;
    float* Lp = reinterpret_cast<float*>(sbase + kCtlBytes + align16(2 * NW * 4));
    float* Rp = Lp + n * N;
    const unsigned bar_id = 1u + unsigned(slot);

    const DevSched& S = P.sched;
    const float alpha = S.alpha;
    const int KW = (K + 31) / 32;
    const int max_iters = P.max_iters;
    const size_t plane_set = size_t(n + 1) * N;

    while (true) {
        if (tid == 0) ctl->frame = (long long)atomicAdd(P.counter, 1ull);
        slot_sync(bar_id, T);
        const long long f = ctl->frame;
        if (f >= P.B) break;

        // a1/a2: channel LLRs into L level 1, R levels 2..n to zero.
        {
            const float4* src = reinterpret_cast<const float4*>(P.llr + size_t(f) * N);
            float4* dst = reinterpret_cast<float4*>(Lp);
            for (int i = tid; i < N / 4; i += T) dst[i] = __ldcs(src + i);
            float4* rz = reinterpret_cast<float4*>(Rp);
            for (int i = tid; i < (n - 1) * N / 4; i += T) rz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = tid; i < NW; i += T) dec[i] = 0u;
            if (tid == 0) {
                ctl->have_ev = 0;
                ctl->have_prev = 0;
                ctl->ev_level = 0;
                ctl->ev_range = 0;
                ctl->ev_blk = -1;
            }
        }
        slot_sync(bar_id, T);

        int next_reset = S.mode == 1 ? S.T0 : (S.mode == 2 ? S.it_reset_full : 0);
        int kev = 0;
        int used = max_iters;
        int ev_lo = n, ev_hi = -1, ev_low = 0;
        long long ev_blk = -1;

        for (int it = 1; it <= max_iters; ++it) {
            for (int i = tid; i < NW; i += T) {
                dec[i] = 0u;
                xh[i] = 0u;
            }
            slot_sync(bar_id, T);
            float* dump_it = nullptr;
            if (TRACE) dump_it = P.dump + (size_t(f) * max_iters + size_t(it - 1)) * 2 * plane_set;

            // a3: L sweep, stages 1..n (channel side to u side).
            for (int s = 0; s < n; ++s) {
                const float* Lin = Lp + s * N;
#pragma unroll
                for (int c = 0; c < PPT; ++c) {
                    const int q = tid + c * T;
                    if (NPE < T && q >= NPE) continue;
                    int p = n - 1 - s;
                    if (s >= ev_lo && s <= ev_hi && (long long)(q & ev_low) == ev_blk) p = ctl->pbit[s];
                    const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                    const int b = t | (1 << p);
                    const float lt = Lin[t], lb = Lin[b];
                    float rt, rb;
                    if (s < n - 1) {
                        rt = Rp[s * N + t];
                        rb = Rp[s * N + b];
                    } else {
                        rt = prior_of(s_frozen, t);
                        rb = prior_of(s_frozen, b);
                    }
                    const float o1 = fnode<FK>(lt, __fadd_rn(lb, rb), alpha);
                    const float o2 = __fadd_rn(fnode<FK>(rt, lt, alpha), lb);
                    if (s < n - 1) {
                        Lp[(s + 1) * N + t] = o1;
                        Lp[(s + 1) * N + b] = o2;
                    } else {
                        // a5: decision on L[n+1] + R[n+1].
                        if (__fadd_rn(o1, rt) < 0.f) atomicOr(&dec[t >> 5], 1u << (t & 31));
                        if (__fadd_rn(o2, rb) < 0.f) atomicOr(&dec[b >> 5], 1u << (b & 31));
                        if (TRACE) {
                            dump_it[size_t(n) * N + t] = o1;
                            dump_it[size_t(n) * N + b] = o2;
                        }
                    }
                }
                slot_sync(bar_id, T);
            }

            // a5: stop test (CRC residue from the decisions).
            const bool check = S.stop_kind != 0 && it >= S.stop_from;
            if (check && (S.stop_kind & 1)) {
                if (warp == 0) {
                    const uint32_t res = crc_residue<NW>(dec, s_crc, r, lane);
                    if (lane == 0) ctl->crc_res = int(res);
                }
                slot_sync(bar_id, T);
            }
            // The decision does not depend on the R sweep, so a CRC-only stop
            // can end the frame here with identical outputs.
            if (!TRACE && check && S.stop_kind == 1 && ctl->crc_res == 0) {
                used = it;
                break;
            }

            // a4: R sweep, stages n..1 (u side to channel side).
            for (int s = n - 1; s >= 0; --s) {
                const float* Lin = Lp + s * N;
#pragma unroll
                for (int c = 0; c < PPT; ++c) {
                    const int q = tid + c * T;
                    if (NPE < T && q >= NPE) continue;
                    int p = n - 1 - s;
                    if (s >= ev_lo && s <= ev_hi && (long long)(q & ev_low) == ev_blk) p = ctl->pbit[s];
                    const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                    const int b = t | (1 << p);
                    const float lt = Lin[t], lb = Lin[b];
                    float rt, rb;
                    if (s < n - 1) {
                        rt = Rp[s * N + t];
                        rb = Rp[s * N + b];
                    } else {
                        rt = prior_of(s_frozen, t);
                        rb = prior_of(s_frozen, b);
                    }
                    const float o1 = fnode<FK>(rt, __fadd_rn(lb, rb), alpha);
                    const float o2 = __fadd_rn(fnode<FK>(rt, lt, alpha), rb);
                    if (s > 0) {
                        Rp[(s - 1) * N + t] = o1;
                        Rp[(s - 1) * N + b] = o2;
                    } else {
                        if (__fadd_rn(lt, o1) < 0.f) atomicOr(&xh[t >> 5], 1u << (t & 31));
                        if (__fadd_rn(lb, o2) < 0.f) atomicOr(&xh[b >> 5], 1u << (b & 31));
                        if (TRACE) {
                            dump_it[plane_set + t] = o1;
                            dump_it[plane_set + b] = o2;
                        }
                    }
                }
                slot_sync(bar_id, T);
            }

            bool stop = false;
            if (check) {
                bool ok = true;
                if (S.stop_kind & 1) ok = ctl->crc_res == 0;
                if (S.stop_kind & 2) {
                    if (warp == 0) {
                        const bool g = g_check<LOGN>(dec, xh, lane);
                        if (lane == 0) ctl->g_ok = g ? 1 : 0;
                    }
                    slot_sync(bar_id, T);
                    ok = ok && ctl->g_ok != 0;
                }
                stop = ok;
            }

            // a6: switch at iter == N_it,reset.
            if (!stop && S.mode != 0 && it == next_reset) {
                bool allowed = true;
                if (TRACE && S.n_explicit >= 0) allowed = kev < S.n_explicit;
                else if (S.mode == 2 && S.q_max > 0) allowed = kev < S.q_max - 1;
                if (allowed) {
                    if (tid == 0) {
                        int level, range;
                        long long blk;
                        signed char order[16];
                        if (TRACE && S.n_explicit >= 0) {
                            const DevEvent& e = P.events[kev];
                            level = e.level;
                            range = e.range;
                            blk = e.block;
                            for (int i = 0; i < 16; ++i) order[i] = e.order[i];
                        } else {
                            draw_event(S, n, S.frame_base + uint64_t(f), kev, level, range, blk, order);
                        }
                        ctl->pv_level = ctl->ev_level;
                        ctl->pv_range = ctl->ev_range;
                        ctl->pv_blk = ctl->ev_blk;
                        ctl->have_prev = ctl->have_ev;
                        ctl->ev_level = level;
                        ctl->ev_range = range;
                        ctl->ev_blk = blk;
                        ctl->have_ev = 1;
                        for (int s = 0; s < 16; ++s) ctl->pbit[s] = (signed char)(n - 1 - s);
                        for (int i = 0; i < range; ++i) ctl->pbit[level - 1 + i] = (signed char)(n - level - order[i]);
                        const long long nz = (1ll << (level + range - 1)) * (long long)(range - 1);
                        long long inc;
                        if (S.mode == 2) {
                            inc = S.it_reset_full;
                        } else {
                            const long long qz = S.D > 0 ? nz / S.D : 0;
                            inc = qz > S.N_min ? qz : S.N_min;
                        }
                        ctl->next_inc = int(inc);
                    }
                    slot_sync(bar_id, T);
                    // the message reset of Sec. III: interior levels of the previous
                    // subgraph (it reverts to the original order) and of the
                    // new one.
                    for (int pass = 0; pass < 2; ++pass) {
                        if (pass == 0 && !ctl->have_prev) continue;
                        const int lv = pass == 0 ? ctl->pv_level : ctl->ev_level;
                        const int rg = pass == 0 ? ctl->pv_range : ctl->ev_range;
                        const long long bk = pass == 0 ? ctl->pv_blk : ctl->ev_blk;
                        const int m = lv + rg - 1;
                        const int span = 1 << m;
                        for (int i = tid; i < (rg - 1) * span; i += T) {
                            const int lev = lv + 1 + i / span;  // node level, 2..n
                            const int j = int(bk) + ((i & (span - 1)) << (n - m));
                            Lp[(lev - 1) * N + j] = 0.f;
                            Rp[(lev - 2) * N + j] = 0.f;
                        }
                    }
                    ev_lo = ctl->ev_level - 1;
                    ev_hi = ctl->ev_level + ctl->ev_range - 2;
                    ev_low = (1 << (n - (ctl->ev_level + ctl->ev_range - 1))) - 1;
                    ev_blk = ctl->ev_blk;
                    next_reset = it + ctl->next_inc;
                    ++kev;
                    slot_sync(bar_id, T);
                }
            }

            if (TRACE) {
                for (int i = tid; i < n * N; i += T) dump_it[i] = Lp[i];
                for (int i = tid; i < (n - 1) * N; i += T) dump_it[plane_set + N + i] = Rp[i];
                for (int j = tid; j < N; j += T) dump_it[plane_set + size_t(n) * N + j] = prior_of(s_frozen, j);
                slot_sync(bar_id, T);
            }
            if (stop) {
                used = it;
                break;
            }
        }

        // a7: outputs.
        if (warp == 0) {
            const uint32_t res = crc_residue<NW>(dec, s_crc, r, lane);
            if (lane == 0) {
                P.crc_ok[f] = res == 0u ? 1 : 0;
                P.iters[f] = used;
            }
        }
        for (int o = warp; o < KW; o += NWARP) {
            const int kk = o * 32 + lane;
            uint32_t bit = 0;
            if (kk < K) {
                const int pos = s_info[kk];
                bit = (dec[pos >> 5] >> (pos & 31)) & 1u;
            }
            const uint32_t word = __ballot_sync(0xffffffffu, bit);
            if (lane == 0) P.bits[size_t(f) * KW + o] = word;
        }
        slot_sync(bar_id, T);
    }
}

}  // namespace pcbp
