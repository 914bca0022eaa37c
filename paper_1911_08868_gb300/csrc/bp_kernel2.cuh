// Stage-grouped PP-BP decoder kernel for sm_103a (Algorithm 1 of arXiv
// 1911.08868): the bp_decode path for N < 128 (and for every N when
// PCBP_DECODER=grouped); its stage partition and swizzled planes are also the
// base of the TMEM kernel (bp_kernel3.cuh).
//
// Same arithmetic as bp_kernel.cuh (every FP32 operation explicitly rounded,
// identical operation order per PE output), organised for fewer barriers and
// less shared-memory traffic:
//
//  * Stage groups.  The n stages of an iteration are cut into groups of at
//    most KB consecutive stages.  In a group every thread owns E = 2^KB
//    positions: a base plus every combination of KB bit positions P[0..KB-1],
//    where P[i] is the bit stage s0+i pairs on (the remaining P entries are
//    spare bits).  The group's stages then run in registers (stage s0+i pairs
//    register e with e ^ 2^i) and the block synchronises once per group.
//  * Permuted subgraph.  Inside the event's subgraph (positions whose n-m low
//    bits equal `block`) the stages level..m pair on permuted bits.  A thread
//    takes its bit list from the class of its positions: groups that contain
//    a permuted stage only contain stages 1..m and use only bits >= n-m, so
//    all positions a thread owns share their low bits and therefore their
//    class.  Group boundaries are placed after stage m for this; when m < KB
//    the permuted stages run one at a time with per-PE addressing instead.
//  * Storage.  Per frame slot: L planes of levels 2..n and R planes of levels
//    2..n in shared memory (XOR-swizzled so that the lane patterns of the
//    groups hit distinct banks), the channel LLRs (level 1) in registers of
//    the first group, the last group's L values kept in registers from its L
//    sweep to its R sweep.  R at level n+1 is the prior from the frozen mask.
//  * Decisions are packed per thread and combined with warp shuffles; the
//    CRC residue bits are spread over the slot's warps.
//  * L messages are recomputed by every L sweep before they are read, so the
//    switch only zeroes R at the interior levels of the old and new
//    subgraphs (zeroing L there, as the paper does, changes nothing that is
//    read; the trace kernel zeroes both to expose the planes).
#pragma once

#include "bp_kernel.cuh"

namespace pcbp {

// Position j is stored at j ^ h(j >> 5) in every plane, h linear over GF(2):
// bit b >= 5 of j flips the bank bits kSwzCol[b - 5].  The columns are
// chosen (by exhaustive search) so that for every group whose register bits
// are a contiguous run, the five bits that vary across a warp's lanes map to
// five independent bank bits: such accesses are free of bank conflicts.  The
// map is its own inverse.  Kernels keep h(i), i < 64, as a byte table in
// shared memory.
constexpr int kSwzTableBytes = 64;

__device__ __forceinline__ unsigned char swz_row(int i)
{
    constexpr unsigned cols = 0x04u | (0x09u << 5) | (0x12u << 10) | (0x1Cu << 15) | (0x07u << 20) | (0x0Eu << 25);
    unsigned h = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b)
        if ((i >> b) & 1) h ^= (cols >> (5 * b)) & 31u;
    return (unsigned char)h;
}

__device__ __forceinline__ int swz(const unsigned char* tab, int j) { return j ^ tab[j >> 5]; }

template <int LOGN, int KB>
struct G2 {
    static constexpr int N = 1 << LOGN;
    static constexpr int n = LOGN;
    static constexpr int E = 1 << KB;
    static constexpr int TA = N / E;                 // threads that own positions
    static constexpr int T = TA < 32 ? 32 : TA;      // threads per slot
    static constexpr int NW = words_of<LOGN>();
    static constexpr int MAXG = LOGN;                // at most one group per stage
    static constexpr int NPL = LOGN - 1;             // L planes (levels 2..n), R planes (levels 2..n)
};

// Per-slot control block of the grouped kernel.
template <int LOGN, int KB>
struct GroupCtl {
    using C = G2<LOGN, KB>;
    long long frame;
    long long ev_blk, pv_blk;
    int ev_level, ev_range, have_ev;
    int pv_level, pv_range, have_prev;
    int next_inc;
    int crc_res, g_ok;
    int ng;          // number of groups
    int low;         // n - m of the current event (class test uses tid's `low` low bits)
    int beta;        // subgraph of the current event
    int fastdec;     // the last group packs decisions with shuffles
    signed char pbit[16];
    signed char s0[C::MAXG], g[C::MAXG], single_[C::MAXG], local[C::MAXG];
    signed char P[C::MAXG][2][KB];           // [group][class: 0 original, 1 permuted subgraph][register bit]
    signed char contig[C::MAXG][2];          // a when the bit set is [a, a+KB), else -1
    unsigned cmask[C::MAXG][2];              // positions the thread index is deposited into
    short swoff[C::MAXG][2][1 << KB];        // swz(offset of register e)
};

// Partition of the stages of one iteration (slot leader).
// short_last: the last segment puts its short group at its end instead of its
// start (the TMEM kernel's choice: the no-event partition then has one group
// width before the last group).
template <int CL, int KB>
__device__ __noinline__ void build_groups(GroupCtl<CL, KB>* c, const unsigned char* swt, int n, bool have_ev,
                                          int level, int range, long long blk, const signed char* order,
                                          bool short_last = false)
{
    int lo = n, hi = -1, m = 0;
    if (have_ev) {
        lo = level - 1;
        hi = level + range - 2;
        m = hi + 1;
    }
    c->low = have_ev ? n - m : 0;
    c->beta = have_ev ? int(blk) : 0;
    for (int s = 0; s < 16; ++s) c->pbit[s] = (signed char)(n - 1 - s);
    if (have_ev)
        for (int i = 0; i < range; ++i) c->pbit[lo + i] = (signed char)(n - level - order[i]);

    // segments: [a, b, kind] kind 0 homogeneous, 1 subgraph-local blocked, 2 single stages
    int seg_a[3], seg_b[3], seg_k[3], nseg = 0;
    if (!have_ev) {
        seg_a[0] = 0; seg_b[0] = n - 1; seg_k[0] = 0; nseg = 1;
    } else if (m >= KB) {
        seg_a[nseg] = 0; seg_b[nseg] = hi; seg_k[nseg] = 1; ++nseg;
        if (hi + 1 <= n - 1) { seg_a[nseg] = hi + 1; seg_b[nseg] = n - 1; seg_k[nseg] = 0; ++nseg; }
    } else {
        if (lo >= 1) { seg_a[nseg] = 0; seg_b[nseg] = lo - 1; seg_k[nseg] = 0; ++nseg; }
        seg_a[nseg] = lo; seg_b[nseg] = hi; seg_k[nseg] = 2; ++nseg;
        if (hi + 1 <= n - 1) { seg_a[nseg] = hi + 1; seg_b[nseg] = n - 1; seg_k[nseg] = 0; ++nseg; }
    }
    int ng = 0;
    for (int sg = 0; sg < nseg; ++sg) {
        const int a = seg_a[sg], b = seg_b[sg], kind = seg_k[sg];
        if (kind == 2) {
            for (int s = a; s <= b; ++s) {
                c->s0[ng] = (signed char)s; c->g[ng] = 1; c->single_[ng] = 1; c->local[ng] = 1; ++ng;
            }
            continue;
        }
        // groups of KB from the end of the segment, the first one shorter (or,
        // short_last on the last segment, from its start, the last one shorter)
        const int len = b - a + 1;
        const int first = len % KB == 0 ? KB : len % KB;
        const bool sl = short_last && sg == nseg - 1;
        int s = a;
        for (int q = 0; s <= b; ++q) {
            const int gl = sl ? (b - s + 1 < KB ? b - s + 1 : KB) : (q == 0 ? first : KB);
            c->s0[ng] = (signed char)s; c->g[ng] = (signed char)gl; c->single_[ng] = 0;
            c->local[ng] = (signed char)(kind == 1);
            for (int cls = 0; cls < 2; ++cls) {
                unsigned used = 0;
                for (int i = 0; i < gl; ++i) {
                    const int st = s + i;
                    int bit = n - 1 - st;
                    if (cls == 1 && kind == 1 && st >= lo && st <= hi) bit = n - level - order[st - lo];
                    c->P[ng][cls][i] = (signed char)bit;
                    used |= 1u << bit;
                }
                // spare bits: below the group's stages first (bits of the next stages), then above;
                // subgraph-local groups keep every bit >= n - m
                const int floor_bit = kind == 1 ? n - m : 0;
                int nxt = gl;
                for (int bit = n - 1 - (s + gl); bit >= floor_bit && nxt < KB; --bit)
                    if (!((used >> bit) & 1u)) { c->P[ng][cls][nxt++] = (signed char)bit; used |= 1u << bit; }
                for (int bit = n - s; bit <= n - 1 && nxt < KB; ++bit)
                    if (!((used >> bit) & 1u)) { c->P[ng][cls][nxt++] = (signed char)bit; used |= 1u << bit; }
                for (int bit = floor_bit; bit <= n - 1 && nxt < KB; ++bit)
                    if (!((used >> bit) & 1u)) { c->P[ng][cls][nxt++] = (signed char)bit; used |= 1u << bit; }
                c->cmask[ng][cls] = ((1u << n) - 1u) & ~used;
                int lowb = 0;
                while (lowb < n && !((used >> lowb) & 1u)) ++lowb;
                c->contig[ng][cls] = (signed char)((used >> lowb) == ((1u << KB) - 1u) ? lowb : -1);
                for (int e = 0; e < (1 << KB); ++e) {
                    int off = 0;
                    for (int i = 0; i < KB; ++i)
                        if ((e >> i) & 1) off |= 1 << c->P[ng][cls][i];
                    c->swoff[ng][cls][e] = (short)swz(swt, off);
                }
            }
            ++ng;
            s += gl;
        }
    }
    c->ng = ng;
    // the last group packs its decisions with shuffles when it is homogeneous
    // and owns E consecutive positions in the natural register order
    const int L = ng - 1;
    bool fast = !c->single_[L] && !c->local[L] && c->g[L] == KB;
    for (int i = 0; i < KB && fast; ++i) fast = c->P[L][0][i] == KB - 1 - i;
    c->fastdec = fast ? 1 : 0;
}

template <int CL, int KB>
__device__ __forceinline__ int group_base(const GroupCtl<CL, KB>* c, int gi, int cls, int tid)
{
    const int a = c->contig[gi][cls];
    if (a >= 0) return (tid & ((1 << a) - 1)) | ((tid >> a) << (a + KB));
    unsigned msk = c->cmask[gi][cls];
    int base = 0, src = tid;
    while (msk) {
        const int b = __ffs(msk) - 1;
        if (src & 1) base |= 1 << b;
        src >>= 1;
        msk &= msk - 1;
    }
    return base;
}

// ---------------------------------------------------------------------------
// Largest block of the grouped kernel: slots x threads per slot never exceed it.
template <int KB>
__host__ __device__ constexpr int grouped_max_threads() { return KB >= 4 ? 384 : (KB == 3 ? 512 : 768); }

// Code tables in shared memory: frozen mask, CRC bit-planes, information
// positions, swizzle table; the frame slots follow.  Returns the slot area.
__device__ __forceinline__ unsigned char* load_code_tables(const DevCode& code, unsigned char* smem)
{
    const int NW = code.N >= 32 ? code.N / 32 : 1;
    const int r = code.r, K = code.K;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_crc = s_frozen + NW;
    int16_t* s_info = reinterpret_cast<int16_t*>(s_crc + r * NW);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = code.frozen[i];
    for (int i = threadIdx.x; i < r * NW; i += blockDim.x) s_crc[i] = code.crcplane[i / NW][i % NW];
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = code.info_idx[i];
    unsigned char* s_swz = smem + shared_table_bytes(NW, r, K);
    for (int i = threadIdx.x; i < kSwzTableBytes; i += blockDim.x) s_swz[i] = swz_row(i);
    return s_swz + kSwzTableBytes;
}

// Decodes frames of one job until the counter passes B.  Threads
// [0, nslots * T) take part, in slots of T threads; the code tables are
// already in shared memory (load_code_tables) and visible to all of them.
template <int LOGN, int KB, int FK>
__device__ __forceinline__ void grouped_frames(const FrameJob& J, unsigned long long* counter, unsigned char* smem)
{
    constexpr int CL = LOGN;
    using Ctl = GroupCtl<CL, KB>;
    constexpr int n = LOGN;
    constexpr int N = 1 << n;
    constexpr int E = 1 << KB;
    constexpr int TA = N / E;
    constexpr int T = TA < 32 ? 32 : TA;
    constexpr int NW = N >= 32 ? N / 32 : 1;
    constexpr int NWARP = T / 32;
    constexpr int NPL = n - 1;

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
    const bool owner = tid < TA;
    constexpr size_t ctl_bytes = align16(sizeof(Ctl));
    const size_t slot_sz = ctl_bytes + align16(size_t(2 * NW * 4)) + size_t(2 * NPL) * N * 4;
    unsigned char* sbase = smem + shared_table_bytes(NW, r, K) + kSwzTableBytes + size_t(slot) * slot_sz;
    Ctl* ctl = reinterpret_cast<Ctl*>(sbase);
    uint32_t* dec = reinterpret_cast<uint32_t*>(sbase + ctl_bytes);
    uint32_t* xh = dec + NW;
    float* Lp = reinterpret_cast<float*>(sbase + ctl_bytes + align16(2 * NW * 4));  // level l at (l-2)*N
    float* Rp = Lp + NPL * N;                                                         // level l at (l-2)*N
    const unsigned bar_id = 1u + unsigned(slot);
    auto sync = [&]() {
        if (T == 32) __syncwarp();
        else slot_sync(bar_id, T);
    };

    const DevSched& S = J.S;
    const float alpha = S.alpha;
    const int KW = (K + 31) / 32;
    const int max_iters = J.max_iters;
    const bool want_g = (S.stop_kind & 2) != 0;

    float L1[E];  // channel LLRs of the first group's positions

    while (true) {
        if (tid == 0) ctl->frame = (long long)atomicAdd(counter, 1ull);
        sync();
        const long long f = ctl->frame;
        if (f >= J.B) break;
        const float* llr_f = J.llr + size_t(f) * N;

        for (int i = tid; i < NPL * N / 4; i += T) reinterpret_cast<float4*>(Rp)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < NW; i += T) dec[i] = 0u;
        if (tid == 0) {
            ctl->have_ev = 0;
            ctl->have_prev = 0;
            ctl->ev_level = 0;
            ctl->ev_range = 0;
            ctl->ev_blk = -1;
            signed char none[16];
            build_groups<CL, KB>(ctl, s_swz, n, false, 0, 0, 0, none);
        }
        sync();

        // (re)load the channel LLRs of the first group's positions
        auto load_l1 = [&]() {
            if (!ctl->single_[0] && owner) {
                const int cls = (ctl->local[0] && ((tid & ((1 << ctl->low) - 1)) == ctl->beta)) ? 1 : 0;
                const int bs = sw(group_base<CL, KB>(ctl, 0, cls, tid));
#pragma unroll
                for (int e = 0; e < E; ++e) L1[e] = __ldcs(llr_f + sw(bs ^ ctl->swoff[0][cls][e]));
            }
        };
        load_l1();

        int next_reset = S.mode == 1 ? S.T0 : (S.mode == 2 ? S.it_reset_full : 0);
        int kev = 0;
        int used = max_iters;

        for (int it = 1; it <= max_iters; ++it) {
            if (tid == 0) ctl->crc_res = 0;
            if (want_g)
                for (int i = tid; i < NW; i += T) xh[i] = 0u;
            const int ng = ctl->ng;
            const int lowmask = (1 << ctl->low) - 1;
            const bool inb = (tid & lowmask) == ctl->beta;   // this thread's positions lie in the subgraph

            // ---------------- L sweep, all groups but the last
            for (int gi = 0; gi < ng - 1; ++gi) {
                const int s0 = ctl->s0[gi], gl = ctl->g[gi];
                if (ctl->single_[gi]) {
                    // one permuted stage with per-PE addressing (m < KB events)
                    const int s = s0;
                    const int lo = ctl->ev_level - 1, m1 = ctl->ev_level + ctl->ev_range - 2;
                    if (owner) {
#pragma unroll
                        for (int c = 0; c < E / 2; ++c) {
                            const int q = tid + c * TA;
                            int p = n - 1 - s;
                            if (s >= lo && s <= m1 && (q & lowmask) == ctl->beta) p = ctl->pbit[s];
                            const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
                            const int b = t | (1 << p);
                            const float lt = s == 0 ? llr_f[t] : Lp[(s - 1) * N + sw(t)];
                            const float lb = s == 0 ? llr_f[b] : Lp[(s - 1) * N + sw(b)];
                            const float rt = Rp[s * N + sw(t)];
                            const float rb = Rp[s * N + sw(b)];
                            Lp[s * N + sw(t)] = fnode<FK>(lt, __fadd_rn(lb, rb), alpha);
                            Lp[s * N + sw(b)] = __fadd_rn(fnode<FK>(rt, lt, alpha), lb);
                        }
                    }
                    sync();
                    continue;
                }
                if (owner) {
                    const int cls = (ctl->local[gi] && inb) ? 1 : 0;
                    const int bs = sw(group_base<CL, KB>(ctl, gi, cls, tid));
                    int ph[E];
                    float x[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        ph[e] = bs ^ ctl->swoff[gi][cls][e];
                        x[e] = s0 == 0 ? L1[e] : Lp[(s0 - 1) * N + ph[e]];
                    }
#pragma unroll
                    for (int i = 0; i < KB; ++i) {
                        if (i < gl) {
                            const int s = s0 + i;            // reads R level s+2, writes L level s+2 (<= n)
                            float rv[E];
#pragma unroll
                            for (int e = 0; e < E; ++e) rv[e] = Rp[s * N + ph[e]];
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                if (e & (1 << i)) continue;
                                const int eb = e | (1 << i);
                                const float lt = x[e], lb = x[eb];
                                x[e] = fnode<FK>(lt, __fadd_rn(lb, rv[eb]), alpha);
                                x[eb] = __fadd_rn(fnode<FK>(rv[e], lt, alpha), lb);
                            }
#pragma unroll
                            for (int e = 0; e < E; ++e) Lp[s * N + ph[e]] = x[e];
                        }
                    }
                }
                sync();
            }

            // ---------------- last group: L sweep, decisions, kept in registers
            const int gL = ng - 1;
            const int s0L = ctl->s0[gL], glL = ctl->g[gL];
            const int clsL = (ctl->local[gL] && inb) ? 1 : 0;
            float xL[KB][E];
            float x[E];
            int phL[E];
            if (owner) {
                const int bs = sw(group_base<CL, KB>(ctl, gL, clsL, tid));
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    phL[e] = bs ^ ctl->swoff[gL][clsL][e];
                    x[e] = s0L == 0 ? L1[e] : Lp[(s0L - 1) * N + phL[e]];
                }
#pragma unroll
                for (int i = 0; i < KB; ++i) {
                    if (i < glL) {
                        const int s = s0L + i;
                        float rv[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            xL[i][e] = x[e];
                            rv[e] = s < n - 1 ? Rp[s * N + phL[e]] : prior_of(s_frozen, sw(phL[e]));
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if (e & (1 << i)) continue;
                            const int eb = e | (1 << i);
                            const float lt = x[e], lb = x[eb];
                            x[e] = fnode<FK>(lt, __fadd_rn(lb, rv[eb]), alpha);
                            x[eb] = __fadd_rn(fnode<FK>(rv[e], lt, alpha), lb);
                        }
                    }
                }
            }
            // a5: decisions u_j = [L(n+1) + R(n+1) < 0]
            if (ctl->fastdec) {
                // positions base .. base+E-1, register e at offset bitreverse(e)
                uint32_t chunk = 0;
                if (owner) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        int rev = 0;
#pragma unroll
                        for (int i = 0; i < KB; ++i) rev |= ((e >> i) & 1) << (KB - 1 - i);
                        const int j = sw(phL[e]);
                        if (__fadd_rn(x[e], prior_of(s_frozen, j)) < 0.f) chunk |= 1u << rev;
                    }
                }
                if (E >= 32) {
                    if (owner) dec[(tid * E) >> 5] = chunk;
                } else {
                    constexpr int PER = 32 / E;     // threads per decision word
                    uint32_t word = owner ? chunk << ((tid % PER) * E) : 0u;
#pragma unroll
                    for (int o = 1; o < PER; o <<= 1) word |= __shfl_xor_sync(0xffffffffu, word, o);
                    if (owner && (tid % PER) == 0) dec[(tid * E) >> 5] = word;
                }
            } else {
                for (int i = tid; i < NW; i += T) dec[i] = 0u;
                sync();
                if (owner) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int j = sw(phL[e]);
                        if (__fadd_rn(x[e], prior_of(s_frozen, j)) < 0.f) atomicOr(&dec[j >> 5], 1u << (j & 31));
                    }
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
                if (lane == 0 && part) atomicOr(reinterpret_cast<unsigned*>(&ctl->crc_res), part);
                sync();
                res = ctl->crc_res;     // read once: thread 0 clears it again next iteration
            }
            if (check && S.stop_kind == 1 && res == 0) {
                used = it;
                break;
            }

            // ---------------- R sweep, last group (continues from registers)
            if (owner) {
                float y[E];
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = prior_of(s_frozen, sw(phL[e]));   // R(n+1): the last group ends at stage n
#pragma unroll
                for (int i = KB - 1; i >= 0; --i) {
                    if (i < glL) {
                        const int s = s0L + i;               // writes R level s+1
                        if (s == 0 && !want_g) continue;
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if (e & (1 << i)) continue;
                            const int eb = e | (1 << i);
                            const float rt = y[e], rb = y[eb];
                            y[e] = fnode<FK>(rt, __fadd_rn(xL[i][eb], rb), alpha);
                            y[eb] = __fadd_rn(fnode<FK>(rt, xL[i][e], alpha), rb);
                        }
                        if (s >= 1) {
#pragma unroll
                            for (int e = 0; e < E; ++e) Rp[(s - 1) * N + phL[e]] = y[e];
                        } else {
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                const int j = sw(phL[e]);
                                if (__fadd_rn(L1[e], y[e]) < 0.f) atomicOr(&xh[j >> 5], 1u << (j & 31));
                            }
                        }
                    }
                }
            }
            sync();

            // ---------------- R sweep, the other groups in reverse
            for (int gi = ng - 2; gi >= 0; --gi) {
                const int s0 = ctl->s0[gi], gl = ctl->g[gi];
                if (ctl->single_[gi]) {
                    const int s = s0;
                    if (s > 0 || want_g) {
                        const int lo = ctl->ev_level - 1, m1 = ctl->ev_level + ctl->ev_range - 2;
                        if (owner) {
#pragma unroll
                            for (int c = 0; c < E / 2; ++c) {
                                const int q = tid + c * TA;
                                int p = n - 1 - s;
                                if (s >= lo && s <= m1 && (q & lowmask) == ctl->beta) p = ctl->pbit[s];
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
                    }
                    sync();
                    continue;
                }
                if (owner) {
                    const int cls = (ctl->local[gi] && inb) ? 1 : 0;
                    const int bs = sw(group_base<CL, KB>(ctl, gi, cls, tid));
                    int ph[E];
                    float y[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        ph[e] = bs ^ ctl->swoff[gi][cls][e];
                        y[e] = Rp[(s0 + gl - 1) * N + ph[e]];                 // R level s0+gl+1
                    }
#pragma unroll
                    for (int i = KB - 1; i >= 0; --i) {
                        if (i < gl) {
                            const int s = s0 + i;
                            if (s == 0 && !want_g) continue;
                            float lv[E];
#pragma unroll
                            for (int e = 0; e < E; ++e) lv[e] = s == 0 ? L1[e] : Lp[(s - 1) * N + ph[e]];
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                if (e & (1 << i)) continue;
                                const int eb = e | (1 << i);
                                const float rt = y[e], rb = y[eb];
                                y[e] = fnode<FK>(rt, __fadd_rn(lv[eb], rb), alpha);
                                y[eb] = __fadd_rn(fnode<FK>(rt, lv[e], alpha), rb);
                            }
                            if (s >= 1) {
#pragma unroll
                                for (int e = 0; e < E; ++e) Rp[(s - 1) * N + ph[e]] = y[e];
                            } else {
#pragma unroll
                                for (int e = 0; e < E; ++e) {
                                    const int j = sw(ph[e]);
                                    if (__fadd_rn(L1[e], y[e]) < 0.f) atomicOr(&xh[j >> 5], 1u << (j & 31));
                                }
                            }
                        }
                    }
                }
                sync();
            }

            bool stop = false;
            if (check) {
                bool ok = true;
                if (S.stop_kind & 1) ok = res == 0;
                if (want_g) {
                    if (warp == 0) {
                        const bool gok = g_check<LOGN>(dec, xh, lane);
                        if (lane == 0) ctl->g_ok = gok ? 1 : 0;
                    }
                    sync();
                    ok = ok && ctl->g_ok != 0;
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
                    if (tid == 0) {
                        int level, range;
                        long long blk;
                        signed char order[16];
                        draw_event(S, n, S.frame_base + uint64_t(f), kev, level, range, blk, order);
                        ctl->pv_level = ctl->ev_level;
                        ctl->pv_range = ctl->ev_range;
                        ctl->pv_blk = ctl->ev_blk;
                        ctl->have_prev = ctl->have_ev;
                        ctl->ev_level = level;
                        ctl->ev_range = range;
                        ctl->ev_blk = blk;
                        ctl->have_ev = 1;
                        const long long nz = (1ll << (level + range - 1)) * (long long)(range - 1);
                        long long inc;
                        if (S.mode == 2) {
                            inc = S.it_reset_full;
                        } else {
                            const long long qz = S.D > 0 ? nz / S.D : 0;
                            inc = qz > S.N_min ? qz : S.N_min;
                        }
                        ctl->next_inc = int(inc);
                        build_groups<CL, KB>(ctl, s_swz, n, true, level, range, blk, order);
                    }
                    sync();
                    // the message reset of Sec. III: R at the interior levels of the previous
                    // subgraph (reverting to the original order) and of the new one
                    for (int pass = 0; pass < 2; ++pass) {
                        if (pass == 0 && !ctl->have_prev) continue;
                        const int lv = pass == 0 ? ctl->pv_level : ctl->ev_level;
                        const int rg = pass == 0 ? ctl->pv_range : ctl->ev_range;
                        const long long bk = pass == 0 ? ctl->pv_blk : ctl->ev_blk;
                        const int m = lv + rg - 1;
                        const int span = 1 << m;
                        for (int i = tid; i < (rg - 1) * span; i += T) {
                            const int lev = lv + 1 + i / span;       // node level, 2..n
                            const int j = int(bk) + ((i & (span - 1)) << (n - m));
                            Rp[(lev - 2) * N + sw(j)] = 0.f;
                        }
                    }
                    next_reset = it + ctl->next_inc;
                    ++kev;
                    load_l1();
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
            if (tid == 0) ctl->crc_res = 0;
            sync();
            if (lane == 0 && part) atomicOr(reinterpret_cast<unsigned*>(&ctl->crc_res), part);
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
                J.crc_ok[f] = ctl->crc_res == 0 ? 1 : 0;
                J.iters[f] = used;
            }
            sync();
        }
    }
}

template <int LOGN, int KB, int FK>
__global__ void __launch_bounds__(grouped_max_threads<KB>(), 1) bp_decode_grouped_kernel(const __grid_constant__ BpParams P)
{
    // a kernel launched after this one may start as soon as SMs free up
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    load_code_tables(P.code, smem);
    __syncthreads();
    grouped_frames<LOGN, KB, FK>(P.job, P.counter, smem);
}

}  // namespace pcbp
