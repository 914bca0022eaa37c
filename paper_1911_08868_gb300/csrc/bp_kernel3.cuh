// Stage-grouped PP-BP decoder kernel with group-private messages in tensor
// memory (sm_103a TMEM), the bp_decode path for N >= 256 (Algorithm 1 of
// arXiv 1911.08868).
//
// The stage partition, positions per thread, swizzled shared-memory planes,
// decisions, stop tests and switch are those of the stage-grouped kernel
// (bp_kernel2.cuh), and so is every floating-point operation: the outputs are
// bit-identical.  What changes is where the messages live between uses.
//
// A group g of stages s0 .. s0+gl-1 (0-based, counted from the channel) reads
// L at node level s0+1 and R at level s0+gl+1 from its neighbours and produces
// L at level s0+gl+1 and R at level s0+1 for them: these boundary levels stay
// in shared memory.  The levels strictly inside the group are produced and
// consumed by the same thread on the same positions, as long as the partition
// does not change:
//   L at levels s0+1 .. s0+gl    written by the L sweep, read by the R sweep
//                                of the same iteration (level 1 is the channel
//                                LLRs, kept in registers),
//   R at levels s0+2 .. s0+gl    written by the R sweep, read by the L sweep
//                                of the next iteration.
// Each thread keeps these E = 2^KB values per level in its own TMEM lane
// (tcgen05.st/ld, 32x32b shape: the warp's quarter of the 128 lanes, one
// column per value), a warp's columns at bank (warp / 4) * TCOLS.  Only the
// thread that wrote a value reads it back, so no fence orders TMEM across
// threads; tcgen05.wait::st orders a thread's stores before its next loads.
//
// Each thread also caches in TMEM, per group, the shared-memory offsets of its
// E positions and, for the last group, their priors: they depend only on the
// partition, so the sweeps read them with one tcgen05.ld instead of rebuilding
// them from the partition tables.
//
// The partition changes when a permutation event is applied (Sec. III): the
// R messages of the interior levels are then written to their canonical
// shared-memory planes with the old partition, the planes are reset as in
// the stage-grouped kernel, and the interior levels are loaded again with the
// new partition.  A new frame starts from zeroed planes the same way.
//
// One CTA per SM (its shared memory exceeds half an SM's) allocates all 512
// TMEM columns for its lifetime, so allocations never wait on one another.
#pragma once

#include <type_traits>

#include "bp_kernel2.cuh"

namespace pcbp {

// Most groups of KB stages that are not single stages, over every event
// shape the partition of build_groups can take (m = level + range - 1).
__host__ __device__ constexpr int max_register_groups(int n, int KB)
{
    auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
    int best = cdiv(n, KB);                                  // no event
    for (int level = 1; level < n; ++level)
        for (int range = 2; range <= 16 && level + range - 1 <= n; ++range) {
            const int lo = level - 1, hi = level + range - 2, m = hi + 1;
            const int g = m >= KB ? cdiv(m, KB) + cdiv(n - m, KB) : cdiv(lo, KB) + cdiv(n - 1 - hi, KB);
            best = g > best ? g : best;
        }
    return best;
}

template <int LOGN, int KB>
struct G3 {
    static constexpr int N = 1 << LOGN;
    static constexpr int n = LOGN;
    static constexpr int E = 1 << KB;
    static constexpr int T = N / E;                              // threads per slot, every one owns positions
    static constexpr int NW = words_of<LOGN>();
    static constexpr int NPL = LOGN - 1;
    static constexpr int MIN_GROUPS = (LOGN + KB - 1) / KB;
    static constexpr int COLS = (2 * LOGN - MIN_GROUPS) * E;     // interior messages: sum (2 gl - 1) E columns
    static constexpr int MAXRG = max_register_groups(LOGN, KB);
    static constexpr int ACOL = COLS;                            // E shared-memory offsets per register group
    static constexpr int PCOL = COLS + MAXRG * E;                // the last group's priors
    static constexpr int TCOLS = PCOL + E;                       // TMEM columns per thread
    static constexpr int MAX_WARPS_TMEM = 4 * (512 / TCOLS);
    static_assert(T >= 32, "every lane of a warp owns positions");
};

constexpr int kTmemCols = 512;

// Largest CTA of the TMEM kernel for a length: 512 threads, or fewer when
// shared memory or TMEM holds fewer slots (N = 1024: 3 slots of 128 threads).
template <int LOGN>
__host__ __device__ constexpr int tmem_max_threads() { return LOGN == 10 ? 384 : (LOGN >= 11 ? 256 : 512); }

// Per-slot control block: the stage partition plus a packed copy that the
// sweeps read with two 16-byte loads per group.
template <int LOGN, int KB>
struct Ctl3 {
    GroupCtl<LOGN, KB> g;
    // rec[gi] = {s0 | gl << 8 | single << 16 | local << 24, TMEM column of L level s0+1,
    //            contig(class 0) & 0xff | (contig(class 1) & 0xff) << 8,
    //            TMEM column of the group's cached shared-memory offsets}
    int4 rec[LOGN];
    uint2 cmask[LOGN];
    alignas(16) short swoff[LOGN][2][1 << KB];
};

// ---------------------------------------------------------------------------
// tcgen05 data movement between registers and this thread's TMEM lane.
template <int E>
__device__ __forceinline__ void tm_st(uint32_t a, const float* v)
{
    if constexpr (E == 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(a),
                     "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                     : "memory");
    } else {
        static_assert(E == 4, "4 or 8 positions per thread");
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]),
                     "f"(v[2]), "f"(v[3])
                     : "memory");
    }
}

// Issues the load; the values are valid after tm_wait_ld() and tm_fence(v).
template <int E>
__device__ __forceinline__ void tm_ld(uint32_t a, float* v)
{
    if constexpr (E == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                     : "r"(a)
                     : "memory");
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                     : "r"(a)
                     : "memory");
    }
}

template <int E>
__device__ __forceinline__ void tm_ld_i(uint32_t a, int* v)
{
    if constexpr (E == 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(a)
                     : "memory");
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                     : "r"(a)
                     : "memory");
    }
}

template <int E>
__device__ __forceinline__ void tm_st_i(uint32_t a, const int* v)
{
    float f[E];
#pragma unroll
    for (int e = 0; e < E; ++e) f[e] = __int_as_float(v[e]);
    tm_st<E>(a, f);
}

__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Keeps every use of v after the preceding tm_wait_ld().
template <int E>
__device__ __forceinline__ void tm_fence(float* v)
{
#pragma unroll
    for (int e = 0; e < E; ++e) asm volatile("" : "+f"(v[e]));
}

template <int E>
__device__ __forceinline__ void tm_fence(int* v)
{
#pragma unroll
    for (int e = 0; e < E; ++e) asm volatile("" : "+r"(v[e]));
}

// Packs the partition for the sweeps (slot leader, after build_groups).
template <int LOGN, int KB>
__device__ __forceinline__ void pack_groups(Ctl3<LOGN, KB>* c)
{
    constexpr int E = 1 << KB;
    int col = 0, acol = G3<LOGN, KB>::ACOL;
    for (int gi = 0; gi < c->g.ng; ++gi) {
        const int gl = c->g.g[gi], single = c->g.single_[gi];
        c->rec[gi] = make_int4(int(c->g.s0[gi]) | (gl << 8) | (single << 16) | (int(c->g.local[gi]) << 24), col,
                               (int(c->g.contig[gi][0]) & 0xff) | ((int(c->g.contig[gi][1]) & 0xff) << 8), acol);
        c->cmask[gi] = make_uint2(c->g.cmask[gi][0], c->g.cmask[gi][1]);
        for (int cls = 0; cls < 2; ++cls)
            for (int e = 0; e < E; ++e) c->swoff[gi][cls][e] = c->g.swoff[gi][cls][e];
        if (!single) {
            col += (2 * gl - 1) * E;
            acol += E;
        }
    }
}

template <int LOGN, int KB>
__device__ __forceinline__ int group_base3(const Ctl3<LOGN, KB>* c, int gi, int cls, int ctg, int tid)
{
    const int a = int((signed char)((ctg >> (8 * cls)) & 0xff));
    if (a >= 0) return (tid & ((1 << a) - 1)) | ((tid >> a) << (a + KB));
    unsigned msk = cls ? c->cmask[gi].y : c->cmask[gi].x;
    int base = 0, src = tid;
    while (msk) {
        const int b = __ffs(msk) - 1;
        if (src & 1) base |= 1 << b;
        src >>= 1;
        msk &= msk - 1;
    }
    return base;
}

// Physical (swizzled) shared-memory offsets of this thread's E positions in group gi.
template <int LOGN, int KB>
__device__ __forceinline__ void group_offsets(const Ctl3<LOGN, KB>* c, const unsigned char* s_swz, int gi, int cls,
                                              int ctg, int tid, int* ph)
{
    constexpr int E = 1 << KB;
    const int bs = swz(s_swz, group_base3<LOGN, KB>(c, gi, cls, ctg, tid));
    const int4* so = reinterpret_cast<const int4*>(&c->swoff[gi][cls][0]);
#pragma unroll
    for (int q = 0; q < E / 8 + (E % 8 ? 1 : 0); ++q) {
        int4 w;
        if constexpr (E >= 8) {
            w = so[q];
        } else {
            const int2 h = reinterpret_cast<const int2*>(so)[0];
            w = make_int4(h.x, h.y, 0, 0);
        }
        const int words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e0 = q * 8 + 2 * k;
            if (e0 < E) ph[e0] = bs ^ int(short(words[k] & 0xffff));
            if (e0 + 1 < E) ph[e0 + 1] = bs ^ int(short(words[k] >> 16));
        }
    }
}

// One PE layer inside a thread: register e pairs with e | 2^i.
template <int E, int FK>
__device__ __forceinline__ void l_layer(float* x, const float* rv, int i, float alpha)
{
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e & (1 << i)) continue;
        const int eb = e | (1 << i);
        const float lt = x[e], lb = x[eb];
        x[e] = fnode<FK>(lt, __fadd_rn(lb, rv[eb]), alpha);
        x[eb] = __fadd_rn(fnode<FK>(rv[e], lt, alpha), lb);
    }
}

template <int E, int FK>
__device__ __forceinline__ void r_layer(float* y, const float* lv, int i, float alpha)
{
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e & (1 << i)) continue;
        const int eb = e | (1 << i);
        const float rt = y[e], rb = y[eb];
        y[e] = fnode<FK>(rt, __fadd_rn(lv[eb], rb), alpha);
        y[eb] = __fadd_rn(fnode<FK>(rt, lv[e], alpha), rb);
    }
}

template <int LOGN, int KB, int FK>
__device__ __forceinline__ void tmem_frames(const FrameJob& J, unsigned long long* counter, unsigned char* smem,
                                            uint32_t tm_base)
{
    using Geo = G3<LOGN, KB>;
    using Ctl = Ctl3<LOGN, KB>;
    constexpr int n = LOGN;
    constexpr int N = Geo::N;
    constexpr int E = Geo::E;
    constexpr int T = Geo::T;
    constexpr int NW = Geo::NW;
    constexpr int NWARP = T / 32;
    constexpr int NPL = Geo::NPL;

    const int r = J.r;
    const int K = J.K;
    const uint32_t* s_frozen = reinterpret_cast<const uint32_t*>(smem);
    const uint32_t* s_crc = s_frozen + NW;
    const int16_t* s_info = reinterpret_cast<const int16_t*>(s_crc + r * NW);
    const unsigned char* s_swz = smem + shared_table_bytes(NW, r, K);
    auto sw = [&](int j) { return swz(s_swz, j); };

    const int slot = threadIdx.x / T;
    const int tid = threadIdx.x - slot * T;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    constexpr size_t ctl_bytes = align16(sizeof(Ctl));
    constexpr size_t slot_sz = ctl_bytes + align16(size_t(2 * NW * 4)) + size_t(2 * NPL) * N * 4;
    unsigned char* sbase = smem + shared_table_bytes(NW, r, K) + kSwzTableBytes + size_t(slot) * slot_sz;
    Ctl* ctl = reinterpret_cast<Ctl*>(sbase);
    uint32_t* dec = reinterpret_cast<uint32_t*>(sbase + ctl_bytes);
    uint32_t* xh = dec + NW;
    float* Lp = reinterpret_cast<float*>(sbase + ctl_bytes + align16(2 * NW * 4));   // level l at (l-2)*N
    float* Rp = Lp + NPL * N;                                                          // level l at (l-2)*N
    const int lp_off = int(reinterpret_cast<unsigned char*>(Lp) - smem);
    const unsigned bar_id = 1u + unsigned(slot);
    auto sync = [&]() {
        if (T == 32) __syncwarp();
        else slot_sync(bar_id, T);
    };
    // this thread's TMEM lane: the warp's quarter of the lanes, its column bank
    const int gwarp = int(threadIdx.x >> 5);
    const uint32_t tm = tm_base + (uint32_t(32 * (gwarp & 3)) << 16) + uint32_t((gwarp >> 2) * Geo::TCOLS);

    // Shared-memory byte offset A of a position set is that of L plane s0-1
    // (node level s0+1) of group s0; the group's other planes are at fixed
    // distances:  Lp plane s0-1+d at A + 4 d N,  Rp plane s0-1+d at A + 4 (NPL + d) N.
    auto at = [&](int a, int floats) -> float& { return *reinterpret_cast<float*>(smem + a + 4 * floats); };
    // logical position of cached offset a in group s0 (for decisions and the G-matrix bits)
    auto pos_of = [&](int a, int s0) { return sw(((a - lp_off) >> 2) - (s0 - 1) * N); };

    const DevSched& S = J.S;
    const float alpha = S.alpha;
    const int KW = (K + 31) / 32;
    const int max_iters = J.max_iters;
    const bool want_g = (S.stop_kind & 2) != 0;

    float L1[E];   // channel LLRs of the first group's positions

    auto group_class = [&](int meta) {
        const bool local = (meta >> 24) & 1;
        const int lowmask = (1 << ctl->g.low) - 1;
        return (local && ((tid & lowmask) == ctl->g.beta)) ? 1 : 0;
    };

    // After a new partition: cache every register group's offsets and the
    // last group's priors in TMEM, move the interior R messages from the
    // canonical planes to TMEM, load the channel LLRs of the first group.
    auto enter_partition = [&](const float* llr_f) {
        const int ng = ctl->g.ng;
        for (int gi = 0; gi < ng; ++gi) {
            const int4 rc = ctl->rec[gi];
            const int s0 = rc.x & 0xff, gl = (rc.x >> 8) & 0xff;
            if ((rc.x >> 16) & 1) continue;
            int ph[E], A[E];
            group_offsets<LOGN, KB>(ctl, s_swz, gi, group_class(rc.x), rc.z, tid, ph);
#pragma unroll
            for (int e = 0; e < E; ++e) A[e] = lp_off + 4 * ((s0 - 1) * N + ph[e]);
            tm_st_i<E>(tm + uint32_t(rc.w), A);
            const uint32_t colR = uint32_t(rc.y + gl * E);
            for (int i = 0; i < gl - 1; ++i) {     // R level s0+2+i: Rp plane s0+i
                float v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = at(A[e], (NPL + i + 1) * N);
                tm_st<E>(tm + colR + uint32_t(i * E), v);
            }
            if (gi == ng - 1) {
                float pr[E];
#pragma unroll
                for (int e = 0; e < E; ++e) pr[e] = prior_of(s_frozen, sw(ph[e]));
                tm_st<E>(tm + uint32_t(Geo::PCOL), pr);
            }
            if (gi == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) L1[e] = __ldcs(llr_f + sw(ph[e]));
            }
        }
        tm_wait_st();
    };

    // Before a new partition: the interior R messages back to the canonical planes.
    auto leave_partition = [&]() {
        const int ng = ctl->g.ng;
        for (int gi = 0; gi < ng; ++gi) {
            const int4 rc = ctl->rec[gi];
            const int gl = (rc.x >> 8) & 0xff;
            if ((rc.x >> 16) & 1) continue;
            if (gl < 2) continue;
            int A[E];
            tm_ld_i<E>(tm + uint32_t(rc.w), A);
            tm_wait_ld();
            tm_fence<E>(A);
            const uint32_t colR = uint32_t(rc.y + gl * E);
            for (int i = 0; i < gl - 1; ++i) {
                float v[E];
                tm_ld<E>(tm + colR + uint32_t(i * E), v);
                tm_wait_ld();
                tm_fence<E>(v);
#pragma unroll
                for (int e = 0; e < E; ++e) at(A[e], (NPL + i + 1) * N) = v[e];
            }
        }
    };

    while (true) {
        if (tid == 0) ctl->g.frame = (long long)atomicAdd(counter, 1ull);
        sync();
        const long long f = ctl->g.frame;
        if (f >= J.B) break;
        const float* llr_f = J.llr + size_t(f) * N;

        for (int i = tid; i < NPL * N / 4; i += T) reinterpret_cast<float4*>(Rp)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < NW; i += T) dec[i] = 0u;
        if (tid == 0) {
            ctl->g.have_ev = 0;
            ctl->g.have_prev = 0;
            ctl->g.ev_level = 0;
            ctl->g.ev_range = 0;
            ctl->g.ev_blk = -1;
            signed char none[16];
            build_groups<LOGN, KB>(&ctl->g, s_swz, n, false, 0, 0, 0, none);
            pack_groups<LOGN, KB>(ctl);
        }
        sync();
        enter_partition(llr_f);

        int next_reset = S.mode == 1 ? S.T0 : (S.mode == 2 ? S.it_reset_full : 0);
        int kev = 0;
        int used = max_iters;

        for (int it = 1; it <= max_iters; ++it) {
            if (tid == 0) ctl->g.crc_res = 0;
            if (want_g)
                for (int i = tid; i < NW; i += T) xh[i] = 0u;
            const int ng = ctl->g.ng;
            const int lowmask = (1 << ctl->g.low) - 1;
            const int beta = ctl->g.beta;
            tm_wait_st();

            // ---------------- L sweep, all groups but the last
            for (int gi = 0; gi < ng - 1; ++gi) {
                const int4 rc = ctl->rec[gi];
                const int s0 = rc.x & 0xff, gl = (rc.x >> 8) & 0xff;
                if ((rc.x >> 16) & 1) {
                    // one permuted stage with per-PE addressing (m < KB events)
                    const int s = s0;
                    const int lo = ctl->g.ev_level - 1, m1 = ctl->g.ev_level + ctl->g.ev_range - 2;
#pragma unroll
                    for (int c = 0; c < E / 2; ++c) {
                        const int q = tid + c * T;
                        int p = n - 1 - s;
                        if (s >= lo && s <= m1 && (q & lowmask) == beta) p = ctl->g.pbit[s];
                        const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                        const int b = t | (1 << p);
                        const float lt = s == 0 ? llr_f[t] : Lp[(s - 1) * N + sw(t)];
                        const float lb = s == 0 ? llr_f[b] : Lp[(s - 1) * N + sw(b)];
                        const float rt = Rp[s * N + sw(t)];
                        const float rb = Rp[s * N + sw(b)];
                        Lp[s * N + sw(t)] = fnode<FK>(lt, __fadd_rn(lb, rb), alpha);
                        Lp[s * N + sw(b)] = __fadd_rn(fnode<FK>(rt, lt, alpha), lb);
                    }
                    sync();
                    continue;
                }
                const uint32_t colL = uint32_t(rc.y);
                auto body = [&](auto glc) {
                    constexpr int GL = decltype(glc)::value;
                    int A[E];
                    float rp[GL > 1 ? GL - 1 : 1][E];
                    tm_ld_i<E>(tm + uint32_t(rc.w), A);
                    if constexpr (GL > 1) {
#pragma unroll
                        for (int i = 0; i < GL - 1; ++i) tm_ld<E>(tm + colL + uint32_t((GL + i) * E), rp[i]);
                    }
                    tm_wait_ld();
                    tm_fence<E>(A);
                    float x[E], rb[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        x[e] = s0 == 0 ? L1[e] : at(A[e], 0);
                        rb[e] = at(A[e], (NPL + GL) * N);                 // R level s0+GL+1 (boundary)
                    }
                    if constexpr (GL > 1) {
#pragma unroll
                        for (int i = 0; i < GL - 1; ++i) tm_fence<E>(rp[i]);
                    }
                    if (s0 > 0) tm_st<E>(tm + colL, x);                 // L level s0+1
#pragma unroll
                    for (int i = 0; i < GL; ++i) {
                        l_layer<E, FK>(x, i < GL - 1 ? rp[i < GL - 1 ? i : 0] : rb, i, alpha);
                        if (i < GL - 1) tm_st<E>(tm + colL + uint32_t((i + 1) * E), x);   // L level s0+2+i
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e) at(A[e], GL * N) = x[e];          // L level s0+GL+1
                };
                if (gl == KB) body(std::integral_constant<int, KB>{});
                else if (KB > 2 && gl == 2) body(std::integral_constant<int, (KB > 2 ? 2 : 1)>{});
                else body(std::integral_constant<int, 1>{});
                sync();
            }

            // ---------------- last group: L sweep, decisions, kept in registers
            const int gL = ng - 1;
            const int4 rcL = ctl->rec[gL];
            const int s0L = rcL.x & 0xff, glL = (rcL.x >> 8) & 0xff;
            const uint32_t colLL = uint32_t(rcL.y);
            int AL[E];
            float pr[E];     // R(n+1): the prior of the last group's positions
            float xL[KB][E];
            float x[E];
            {
                float rp[KB > 1 ? KB - 1 : 1][E];
                tm_ld_i<E>(tm + uint32_t(rcL.w), AL);
                tm_ld<E>(tm + uint32_t(Geo::PCOL), pr);
#pragma unroll
                for (int i = 0; i < KB - 1; ++i)
                    if (i < glL - 1) tm_ld<E>(tm + colLL + uint32_t((glL + i) * E), rp[i]);
                tm_wait_ld();
                tm_fence<E>(AL);
                tm_fence<E>(pr);
#pragma unroll
                for (int i = 0; i < KB - 1; ++i) tm_fence<E>(rp[i]);
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] = s0L == 0 ? L1[e] : at(AL[e], 0);
#pragma unroll
                for (int i = 0; i < KB; ++i) {
                    if (i < glL) {
#pragma unroll
                        for (int e = 0; e < E; ++e) xL[i][e] = x[e];
                        if (i < glL - 1) l_layer<E, FK>(x, rp[i < KB - 1 ? i : 0], i, alpha);
                        else l_layer<E, FK>(x, pr, i, alpha);
                    }
                }
            }
            // a5: decisions u_j = [L(n+1) + R(n+1) < 0]
            if (ctl->g.fastdec) {
                // positions base .. base+E-1, register e at offset bitreverse(e)
                uint32_t chunk = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int rev = 0;
#pragma unroll
                    for (int i = 0; i < KB; ++i) rev |= ((e >> i) & 1) << (KB - 1 - i);
                    if (__fadd_rn(x[e], pr[e]) < 0.f) chunk |= 1u << rev;
                }
                if (E >= 32) {
                    dec[(tid * E) >> 5] = chunk;
                } else {
                    constexpr int PER = 32 / E;     // threads per decision word
                    uint32_t word = chunk << ((tid % PER) * E);
#pragma unroll
                    for (int o = 1; o < PER; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
                    if ((tid % PER) == 0) dec[(tid * E) >> 5] = word;
                }
            } else {
                for (int i = tid; i < NW; i += T) dec[i] = 0u;
                sync();
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int j = pos_of(AL[e], s0L);
                    if (__fadd_rn(x[e], pr[e]) < 0.f) atomicOr(&dec[j >> 5], 1u << (j & 31));
                }
            }
            sync();

            // a5: stop test (CRC residue bits spread over the warps)
            const bool check = S.stop_kind != 0 && it >= S.stop_from;
            int res = 0;
            if (check && (S.stop_kind & 1)) {
                uint32_t part = 0;
                for (int i = warp; i < r; i += NWARP) {
                    uint32_t acc = 0;
#pragma unroll
                    for (int w = lane; w < NW; w += 32) acc ^= dec[w] & s_crc[i * NW + w];
                    const uint32_t bal = __ballot_sync(0xffffffffu, __popc(acc) & 1);
                    part |= uint32_t(__popc(bal) & 1) << i;
                }
                if (lane == 0 && part) atomicOr(reinterpret_cast<unsigned*>(&ctl->g.crc_res), part);
                sync();
                res = ctl->g.crc_res;     // read once: thread 0 clears it again next iteration
            }
            if (check && S.stop_kind == 1 && res == 0) {
                used = it;
                break;
            }

            tm_wait_st();
            // ---------------- R sweep, last group (continues from registers)
            {
                float y[E];
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = pr[e];
#pragma unroll
                for (int i = KB - 1; i >= 0; --i) {
                    if (i < glL) {
                        const int s = s0L + i;               // writes R level s+1
                        if (s == 0 && !want_g) continue;
                        r_layer<E, FK>(y, xL[i], i, alpha);
                        if (i > 0) {
                            tm_st<E>(tm + colLL + uint32_t((glL + i - 1) * E), y);   // R level s0L+1+i
                        } else if (s >= 1) {
#pragma unroll
                            for (int e = 0; e < E; ++e) at(AL[e], NPL * N) = y[e];   // R level s0L+1
                        } else {
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                const int j = pos_of(AL[e], s0L);
                                if (__fadd_rn(L1[e], y[e]) < 0.f) atomicOr(&xh[j >> 5], 1u << (j & 31));
                            }
                        }
                    }
                }
            }
            sync();

            // ---------------- R sweep, the other groups in reverse
            for (int gi = ng - 2; gi >= 0; --gi) {
                const int4 rc = ctl->rec[gi];
                const int s0 = rc.x & 0xff, gl = (rc.x >> 8) & 0xff;
                if ((rc.x >> 16) & 1) {
                    const int s = s0;
                    if (s > 0 || want_g) {
                        const int lo = ctl->g.ev_level - 1, m1 = ctl->g.ev_level + ctl->g.ev_range - 2;
#pragma unroll
                        for (int c = 0; c < E / 2; ++c) {
                            const int q = tid + c * T;
                            int p = n - 1 - s;
                            if (s >= lo && s <= m1 && (q & lowmask) == beta) p = ctl->g.pbit[s];
                            const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                            const int b = t | (1 << p);
                            const float lt = s == 0 ? llr_f[t] : Lp[(s - 1) * N + sw(t)];
                            const float lb = s == 0 ? llr_f[b] : Lp[(s - 1) * N + sw(b)];
                            const float rt = Rp[s * N + sw(t)];
                            const float rb = Rp[s * N + sw(b)];
                            const float o1 = fnode<FK>(rt, __fadd_rn(lb, rb), alpha);
                            const float o2 = __fadd_rn(fnode<FK>(rt, lt, alpha), rb);
                            if (s >= 1) {
                                Rp[(s - 1) * N + sw(t)] = o1;
                                Rp[(s - 1) * N + sw(b)] = o2;
                            } else {
                                if (__fadd_rn(lt, o1) < 0.f) atomicOr(&xh[t >> 5], 1u << (t & 31));
                                if (__fadd_rn(lb, o2) < 0.f) atomicOr(&xh[b >> 5], 1u << (b & 31));
                            }
                        }
                    }
                    sync();
                    continue;
                }
                const uint32_t colL = uint32_t(rc.y);
                auto body = [&](auto glc) {
                    constexpr int GL = decltype(glc)::value;
                    int A[E];
                    float lv[GL][E];
                    tm_ld_i<E>(tm + uint32_t(rc.w), A);
#pragma unroll
                    for (int i = 0; i < GL; ++i)
                        if (i > 0 || s0 > 0) tm_ld<E>(tm + colL + uint32_t(i * E), lv[i]);   // L level s0+1+i
                    tm_wait_ld();
                    tm_fence<E>(A);
                    float y[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) y[e] = at(A[e], (NPL + GL) * N);           // R level s0+GL+1
#pragma unroll
                    for (int i = 0; i < GL; ++i) tm_fence<E>(lv[i]);
                    if (s0 == 0) {
#pragma unroll
                        for (int e = 0; e < E; ++e) lv[0][e] = L1[e];
                    }
#pragma unroll
                    for (int i = GL - 1; i >= 0; --i) {
                        const int s = s0 + i;
                        if (s == 0 && !want_g) continue;
                        r_layer<E, FK>(y, lv[i], i, alpha);
                        if (i > 0) {
                            tm_st<E>(tm + colL + uint32_t((GL + i - 1) * E), y);            // R level s0+1+i
                        } else if (s >= 1) {
#pragma unroll
                            for (int e = 0; e < E; ++e) at(A[e], NPL * N) = y[e];           // R level s0+1
                        } else {
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                const int j = pos_of(A[e], s0);
                                if (__fadd_rn(L1[e], y[e]) < 0.f) atomicOr(&xh[j >> 5], 1u << (j & 31));
                            }
                        }
                    }
                };
                if (gl == KB) body(std::integral_constant<int, KB>{});
                else if (KB > 2 && gl == 2) body(std::integral_constant<int, (KB > 2 ? 2 : 1)>{});
                else body(std::integral_constant<int, 1>{});
                sync();
            }

            bool stop = false;
            if (check) {
                bool ok = true;
                if (S.stop_kind & 1) ok = res == 0;
                if (want_g) {
                    if (warp == 0) {
                        const bool gok = g_check<LOGN>(dec, xh, lane);
                        if (lane == 0) ctl->g.g_ok = gok ? 1 : 0;
                    }
                    sync();
                    ok = ok && ctl->g.g_ok != 0;
                    sync();             // every thread has read g_ok before it is written again
                }
                stop = ok;
            }
            if (stop) {
                used = it;
                break;
            }

            // a6: switch at iter == N_it,reset
            if (S.mode != 0 && it == next_reset) {
                bool allowed = true;
                if (S.mode == 2 && S.q_max > 0) allowed = kev < S.q_max - 1;
                if (allowed) {
                    tm_wait_st();
                    leave_partition();     // interior R of the old partition to the canonical planes
                    sync();
                    if (tid == 0) {
                        int level, range;
                        long long blk;
                        signed char order[16];
                        draw_event(S, n, S.frame_base + uint64_t(f), kev, level, range, blk, order);
                        ctl->g.pv_level = ctl->g.ev_level;
                        ctl->g.pv_range = ctl->g.ev_range;
                        ctl->g.pv_blk = ctl->g.ev_blk;
                        ctl->g.have_prev = ctl->g.have_ev;
                        ctl->g.ev_level = level;
                        ctl->g.ev_range = range;
                        ctl->g.ev_blk = blk;
                        ctl->g.have_ev = 1;
                        const long long nz = (1ll << (level + range - 1)) * (long long)(range - 1);
                        long long inc;
                        if (S.mode == 2) {
                            inc = S.it_reset_full;
                        } else {
                            const long long qz = S.D > 0 ? nz / S.D : 0;
                            inc = qz > S.N_min ? qz : S.N_min;
                        }
                        ctl->g.next_inc = int(inc);
                        build_groups<LOGN, KB>(&ctl->g, s_swz, n, true, level, range, blk, order);
                        pack_groups<LOGN, KB>(ctl);
                    }
                    sync();
                    // resetVariableNodes: R at the interior levels of the previous
                    // subgraph (reverting to the original order) and of the new one
                    for (int pass = 0; pass < 2; ++pass) {
                        if (pass == 0 && !ctl->g.have_prev) continue;
                        const int lv = pass == 0 ? ctl->g.pv_level : ctl->g.ev_level;
                        const int rg = pass == 0 ? ctl->g.pv_range : ctl->g.ev_range;
                        const long long bk = pass == 0 ? ctl->g.pv_blk : ctl->g.ev_blk;
                        const int m = lv + rg - 1;
                        const int span = 1 << m;
                        for (int i = tid; i < (rg - 1) * span; i += T) {
                            const int lev = lv + 1 + i / span;       // node level, 2..n
                            const int j = int(bk) + ((i & (span - 1)) << (n - m));
                            Rp[(lev - 2) * N + sw(j)] = 0.f;
                        }
                    }
                    next_reset = it + ctl->g.next_inc;
                    ++kev;
                    sync();
                    enter_partition(llr_f);   // interior R of the new partition to TMEM
                    sync();
                }
            }
        }

        // a7: outputs
        {
            uint32_t part = 0;
            for (int i = warp; i < r; i += NWARP) {
                uint32_t acc = 0;
#pragma unroll
                for (int w = lane; w < NW; w += 32) acc ^= dec[w] & s_crc[i * NW + w];
                const uint32_t bal = __ballot_sync(0xffffffffu, __popc(acc) & 1);
                part |= uint32_t(__popc(bal) & 1) << i;
            }
            if (tid == 0) ctl->g.crc_res = 0;
            sync();
            if (lane == 0 && part) atomicOr(reinterpret_cast<unsigned*>(&ctl->g.crc_res), part);
            for (int o = warp; o < KW; o += NWARP) {
                const int kk = o * 32 + lane;
                uint32_t bit = 0;
                if (kk < K) {
                    const int pos = s_info[kk];
                    bit = (dec[pos >> 5] >> (pos & 31)) & 1u;
                }
                const uint32_t word = __ballot_sync(0xffffffffu, bit);
                if (lane == 0) J.bits[size_t(f) * KW + o] = word;
            }
            sync();
            if (tid == 0) {
                J.crc_ok[f] = ctl->g.crc_res == 0 ? 1 : 0;
                J.iters[f] = used;
            }
            sync();
        }
    }
    tm_wait_st();
}

template <int LOGN, int KB, int FK>
__global__ void __launch_bounds__(tmem_max_threads<LOGN>(), 1) bp_decode_tmem_kernel(const __grid_constant__ BpParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tm;
    load_code_tables(P.code, smem);
    if (threadIdx.x < 32) {
        const uint32_t dst = uint32_t(__cvta_generic_to_shared(&s_tm));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm_base = s_tm;
    if (int(threadIdx.x) < P.slots * G3<LOGN, KB>::T) tmem_frames<LOGN, KB, FK>(P.job, P.counter, smem, tm_base);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_base), "n"(kTmemCols) : "memory");
}

}  // namespace pcbp
