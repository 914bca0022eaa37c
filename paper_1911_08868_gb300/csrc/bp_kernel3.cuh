// Stage-grouped PP-BP decoder kernel with group-private messages in tensor
// memory (sm_103a TMEM), the bp_decode path for N >= 128 (Algorithm 1 of
// arXiv 1911.08868).
//
// Positions per thread, swizzled shared-memory planes, stop tests and switch
// follow the stage-grouped kernel (bp_kernel2.cuh), and so does every
// floating-point operation: the outputs are bit-identical.  What changes is
// where the messages live between uses and how often the slot synchronises.
//
// Interior messages in TMEM.  A group of stages s0 .. s0+gl-1 (0-based,
// counted from the channel) reads L at node level s0+1 and R at level
// s0+gl+1 from its neighbours and produces L at level s0+gl+1 and R at level
// s0+1 for them: these boundary levels stay in shared memory.  The levels
// inside the group are produced and consumed by the same thread on the same
// positions while the partition stays:
//   L at levels s0+2 .. s0+gl    written by the L sweep, read by the R sweep
//                                (L at level s0+1 is read again from its
//                                boundary plane; the last group keeps its L
//                                in registers),
//   R at levels s0+2 .. s0+gl    written by the R sweep, read by the next
//                                L sweep.
// Each thread keeps these E = 2^KB values per level in its own TMEM lane
// (tcgen05.st/ld, 32x32b shape: the warp's quarter of the 128 lanes, one
// column per value), a warp's columns at bank (warp / 4) * TCOLS, followed by
// the shared-memory offsets of its E positions per register group (the last
// group's in registers from N = 2048 on): these depend only on the partition.
// Only the thread that wrote a value reads it back, so no fence orders TMEM
// across threads; tcgen05.wait::st orders a thread's stores before its next
// loads.
//
// Shared-memory planes (G3): R at every level 2..n in canonical planes; the
// boundary L a group reads lives in the plane of R at the level above it,
// which is interior to that group (its R messages are in TMEM while the
// partition stands), so all planes a group touches are at compile-time
// distances from its cached offsets; at a switch the interior R messages go
// back to those planes, are reset as Sec. III says and are read into TMEM
// for the new partition.  Per slot also: the priors and CRC contributions of
// the positions, and a spare plane (the channel LLRs as a frame starts; L at
// level 2 between two single stages).
//
// Fewer barriers.  The CRC residue of the decisions is linear in them: each
// thread XORs the cached contributions c_j (x^(K-1-k) mod g for the
// information bit of rank k at position j) of its positions decided 1, a
// warp reduction and one shared atomic per warp complete it.  The last
// group's R sweep runs before the stop test (wasted only in a frame's final
// iteration), so a single barrier publishes both the residue and that
// group's boundary R.  Decision words are written only when the frame stops
// or runs out of iterations, and on the iterations that run the G-matrix
// test (from stop_from on; with the combined stop only where the CRC residue
// is zero, since the frame goes on otherwise).  Group 0's R sweep writes
// nothing other threads read unless the G-matrix test runs, so no barrier
// follows it then.  Where two neighbouring
// groups deposit the thread index's warp bits into the same position bits,
// each warp owns the same positions on both sides of their boundary: that
// exchange only needs __syncwarp (with the no-event partition of N = 1024,
// two of the three group boundaries).
//
// The partition changes when a permutation event is applied (Sec. III): the
// interior R messages go back to their canonical shared-memory planes with
// the old partition, the planes are reset as in the stage-grouped kernel, and
// the caches and interior levels are loaded again with the new partition.  A
// new frame starts from zeroed planes the same way (a frame on the no-event
// partition, the usual case, zeroes only the R planes of its group boundaries
// and restarts its TMEM interiors).  At a switch the first warp builds the
// partition while the others reset the subgraph being left, and in slots of
// four warps or more the second warp draws the next switch's event ahead (the
// draws depend only on the seed, the frame and the event index).
//
// One CTA per SM (its shared memory exceeds half an SM's) allocates all 512
// TMEM columns for its lifetime, so allocations never wait on one another.
//
// Compile-time shapes.  Every partition has at least two groups; only the
// first and the last can have fewer than KB stages, and every group between
// them is a single stage or a full group (pc_partition_selfcheck checks this
// for every event shape).  So group 0, whose input is the channel LLRs held in
// registers, runs its own copy of the group step; the middle groups run the
// full-group step with no stage-count dispatch, and with no single-stage test
// unless the current event spans fewer than KB stages; the last group (never
// starting at stage 0) is dispatched once on its stage count; the G-matrix
// test is a template parameter.  Each runtime test removed from the loop that
// every iteration runs took compares, branches, convergence barriers and
// registers with it.
#pragma once

#include <type_traits>

#include "bp_kernel2.cuh"

namespace pcbp {

// Builds with PCBP_CHECKED range-check every shared-memory plane access, TMEM
// column, channel-LLR index and decision-word index of this kernel; an access
// out of range sets bit `cls` of the status word (when there is one) and is
// redirected inside the buffer, so nothing faults.
__device__ __forceinline__ void chk_fail(unsigned* status, unsigned cls)
{
    if (status) atomicOr(status, 1u << cls);
}

// Register-to-position bit maps of the two G-matrix fast paths (the register
// bits of build_partition_warp for a group of natural stage order):
// the last group of GL stages ends at stage n-1, so register bit i < GL is
// position bit GL-1-i and the filled bits GL..KB-1 are themselves; group 0's
// register bit i is position bit n-1-i.
template <int GL, int KB>
__host__ __device__ constexpr int last_group_offset(int e)
{
    int off = 0;
    for (int i = 0; i < KB; ++i)
        if ((e >> i) & 1) off |= 1 << (i < GL ? GL - 1 - i : i);
    return off;
}

// The E decision bits of a thread (bit e for register e) at their position bits in the thread's block.
template <int GL, int KB>
__device__ __forceinline__ unsigned last_group_bits(unsigned umask)
{
    unsigned v = 0u;
#pragma unroll
    for (int e = 0; e < (1 << KB); ++e) v |= ((umask >> e) & 1u) << last_group_offset<GL, KB>(e);
    return v;
}

template <int KB>
__host__ __device__ constexpr int reverse_bits(int e)
{
    int r = 0;
    for (int i = 0; i < KB; ++i)
        if ((e >> i) & 1) r |= 1 << (KB - 1 - i);
    return r;
}

// TMEM columns of one group's interior messages (E per level): L at levels
// s0+2 .. s0+gl and R at levels s0+2 .. s0+gl.  L at level s0+1 (the group's
// input) stays in its shared-memory boundary plane, where the R sweep reads it
// again (group 0: the channel LLRs, in registers); the last group keeps its L
// in registers.
__host__ __device__ constexpr int group_cols(int s0, int gl, bool single, bool last, int E)
{
    (void)s0;
    return single ? 0 : (last ? (gl - 1) * E : 2 * (gl - 1) * E);
}

// Interior columns (cols) and register groups (groups) of the partition
// build_groups<..>(short_last = true) makes for one event shape (level 0: none).
struct PartitionSize {
    int cols, groups;
};

__host__ __device__ constexpr PartitionSize partition_size(int n, int KB, int level, int range)
{
    const int E = 1 << KB;
    int sa[3] = {0, 0, 0}, sb[3] = {0, 0, 0}, sk[3] = {0, 0, 0}, ns = 0;
    if (level == 0) {
        sa[0] = 0; sb[0] = n - 1; sk[0] = 0; ns = 1;
    } else {
        const int lo = level - 1, hi = level + range - 2, m = hi + 1;
        if (m >= KB) {
            sa[ns] = 0; sb[ns] = hi; sk[ns] = 1; ++ns;
            if (hi + 1 <= n - 1) { sa[ns] = hi + 1; sb[ns] = n - 1; sk[ns] = 0; ++ns; }
        } else {
            if (lo >= 1) { sa[ns] = 0; sb[ns] = lo - 1; sk[ns] = 0; ++ns; }
            sa[ns] = lo; sb[ns] = hi; sk[ns] = 2; ++ns;
            if (hi + 1 <= n - 1) { sa[ns] = hi + 1; sb[ns] = n - 1; sk[ns] = 0; ++ns; }
        }
    }
    int s0s[32] = {}, gls[32] = {}, sing[32] = {}, ng = 0;
    for (int sg = 0; sg < ns; ++sg) {
        const int a = sa[sg], b = sb[sg];
        if (sk[sg] == 2) {
            for (int s = a; s <= b; ++s) { s0s[ng] = s; gls[ng] = 1; sing[ng] = 1; ++ng; }
            continue;
        }
        const int len = b - a + 1, first = len % KB == 0 ? KB : len % KB;
        const bool sl = sg == ns - 1;
        int s = a;
        for (int q = 0; s <= b; ++q) {
            const int gl = sl ? (b - s + 1 < KB ? b - s + 1 : KB) : (q == 0 ? first : KB);
            s0s[ng] = s; gls[ng] = gl; sing[ng] = 0; ++ng;
            s += gl;
        }
    }
    PartitionSize r{0, 0};
    for (int g = 0; g < ng; ++g) {
        r.cols += group_cols(s0s[g], gls[g], sing[g] != 0, g == ng - 1, E);
        r.groups += sing[g] ? 0 : 1;
    }
    return r;
}

// Whether plane n-1 can hold L at level 2 between two single stages: single stages exist only for
// events narrower than a group (m = level + range - 1 < KB, so at level 1 after 0 or more stages),
// and plane n-1 is free in those partitions when their last group has at least two stages (it is
// the input plane of a one-stage last group).  The last segment puts its short group last.
__host__ __device__ constexpr bool spare_is_plane_n_minus_1(int n, int KB)
{
    for (int level = 1; level < n; ++level)
        for (int range = 2; range <= 16 && level + range - 1 <= n; ++range) {
            const int hi = level + range - 2, m = hi + 1;
            if (m >= KB || hi + 1 > n - 1) continue;
            const int len = n - 1 - hi;            // the stages after the single ones
            const int last = len % KB == 0 ? KB : len % KB;
            if (last < 2) return false;
        }
    return true;
}

// From N = 2048 on, the last group keeps its shared-memory offsets in registers instead of TMEM,
// so that a thread's columns fit 128 (four threads per lane: two frame slots of 256 threads).
__host__ __device__ constexpr bool tmem_last_in_regs(int n) { return n >= 11; }

// TMEM columns one thread needs, the largest over every partition: the partition's interior
// messages followed by the offsets of its register groups (the last group's too unless
// tmem_last_in_regs).
__host__ __device__ constexpr int max_tmem_cols(int n, int KB)
{
    const int E = 1 << KB;
    const int cached_last = tmem_last_in_regs(n) ? 0 : 1;
    PartitionSize p = partition_size(n, KB, 0, 0);
    int best = p.cols + (p.groups - 1 + cached_last) * E;
    for (int level = 1; level < n; ++level)
        for (int range = 2; range <= 16 && level + range - 1 <= n; ++range) {
            p = partition_size(n, KB, level, range);
            const int need = p.cols + (p.groups - 1 + cached_last) * E;
            best = need > best ? need : best;
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
    static constexpr bool LASTREG = tmem_last_in_regs(LOGN);     // the last group's offsets in registers
    // TMEM columns per thread: a partition's interior messages, then E shared-memory offsets per
    // register group (the last group's not when LASTREG)
    static constexpr int TCOLS = max_tmem_cols(LOGN, KB);
    static constexpr int MAX_WARPS_TMEM = 4 * (512 / TCOLS);
    // Shared-memory planes of a frame slot, N floats each, in the swizzled
    // position order: plane p < n holds R at node level p+2 (p < n-1) and, while
    // level p+2 is interior to the group that starts at stage p, L at node level
    // p+1, the input boundary of that group (its canonical R copy is dead while
    // the partition stands: the group keeps those R messages in TMEM; plane n-1,
    // level n+1, holds only L, or L at level 2 between two single
    // stages where the last group then has at least two stages, so plane n-1
    // is free (else plane n+2); planes n and n+1 hold the priors R(n+1) and the
    // CRC contributions c_j of the positions.  The spare plane also receives a
    // frame's channel LLRs as the frame starts.
    static constexpr bool SPARE_SHARED = spare_is_plane_n_minus_1(LOGN, KB);
    static constexpr int NPLANES = SPARE_SHARED ? LOGN + 2 : LOGN + 3;
    static constexpr int SPARE = SPARE_SHARED ? LOGN - 1 : LOGN + 2;
    static constexpr int PRIOR = LOGN;
    static constexpr int CJ = LOGN + 1;
    static_assert(T >= 32, "every lane of a warp owns positions");
};

constexpr int kTmemCols = 512;

// Code tables of the TMEM kernel in shared memory: frozen mask, CRC
// contribution c_j of every position (bit i = bit i of x^(K-1-k) mod g for
// the information bit of rank k at j, 0 for frozen positions), information
// positions, swizzle table; the frame slots follow.
__host__ __device__ constexpr size_t tmem_table_bytes(int N, int K)
{
    const int nw = N >= 32 ? N / 32 : 1;
    return align16(size_t(nw) * 4 + size_t(N) * 4 + size_t(K) * 2) + kSwzTableBytes;
}

__device__ __forceinline__ void load_code_tables3(const DevCode& code, unsigned char* smem)
{
    const int N = code.N, K = code.K, r = code.r;
    const int NW = N >= 32 ? N / 32 : 1;
    uint32_t* s_frozen = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_cj = s_frozen + NW;
    int16_t* s_info = reinterpret_cast<int16_t*>(s_cj + N);
    for (int i = threadIdx.x; i < NW; i += blockDim.x) s_frozen[i] = code.frozen[i];
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        uint32_t c = 0;
        for (int i = 0; i < r; ++i) c |= ((code.crcplane[i][j >> 5] >> (j & 31)) & 1u) << i;
        s_cj[j] = c;
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_info[i] = code.info_idx[i];
    unsigned char* s_swz = smem + tmem_table_bytes(N, K) - kSwzTableBytes;
    for (int i = threadIdx.x; i < kSwzTableBytes; i += blockDim.x) s_swz[i] = swz_row(i);
}

// Stages per group of the TMEM kernel for a length: 2 up to N = 256 (twice the
// warps per frame, faster there: N = 256 2.13 against 2.30 ms on 65,536 PP-BP
// frames at 2.5 dB), 3 from N = 512 (N = 512 5.81 against 7.06 ms, N = 1024
// 6.93 against 9.5 ms).
__host__ __device__ constexpr int tmem_default_kb(int logn) { return logn <= 8 ? 2 : 3; }

// Largest CTA of the TMEM kernel for a length: as many frame slots as shared
// memory and TMEM hold (N = 1024: 4 slots of 128 threads; N = 2048: 2 slots
// of 256), at most 768 threads.
template <int LOGN, int KB>
__host__ __device__ constexpr int tmem_max_threads()
{
    return KB == 3 ? 512 : (LOGN >= 11 ? 512 : 768);
}

// Per-slot control block: the stage partition plus a packed copy that the
// sweeps read with one 16-byte load per group.
template <int LOGN, int KB>
struct Ctl3 {
    GroupCtl<LOGN, KB> g;
    // rec[gi] = {s0 | gl << 8 | single << 16 | local << 24 | (boundary gi|gi+1 warp-local) << 25
    //              | (boundary gi-1|gi warp-local) << 26,
    //            TMEM column of L level s0+2 (virtual for the last group;
    //            R level s0+2 is at this + (gl - 1) E),
    //            contig(class 0) & 0xff | (contig(class 1) & 0xff) << 8,
    //            TMEM column of the group's cached shared-memory offsets}
    int4 rec[LOGN];
    uint2 cmask[LOGN];
    alignas(16) short swoff[LOGN][2][1 << KB];
    unsigned crc_part[3];    // CRC residue of iteration it, accumulated in crc_part[it % 3]
    unsigned crc_final;      // the CRC test of the frame's final decisions: 2 passed, 1 failed, 0 not run
    // events drawn ahead: nx[k & 1] holds event k of frame nx[.].frame, drawn by a spare warp during
    // switch k - 1 (k = -1: none)
    struct Drawn {
        int k, level, range, frame;
        long long blk;
        unsigned long long ord;
    } nx[2];
};

// Bytes of one frame slot: control block, decision words, NPLANES planes.
template <int LOGN, int KB>
__host__ __device__ constexpr size_t tmem_slot_bytes()
{
    return align16(sizeof(Ctl3<LOGN, KB>)) + align16(size_t(2 * G3<LOGN, KB>::NW * 4)) +
           size_t(G3<LOGN, KB>::NPLANES) * (size_t(1) << LOGN) * 4;
}

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

// Packs the partition for the sweeps (one thread, after build_groups: the no-event template
// and the partition self-check; switches use build_partition_warp).
template <int LOGN, int KB>
__device__ __noinline__ void pack_groups(Ctl3<LOGN, KB>* c)
{
    constexpr int E = 1 << KB;
    constexpr int TB = LOGN - KB;        // thread-index bits: 5 lane bits, then warp bits
    const int ng = c->g.ng;
    int col = 0, acol = 0;
    for (int gi = 0; gi < ng; ++gi)       // the offsets follow this partition's interior columns
        if (!c->g.single_[gi]) acol += group_cols(c->g.s0[gi], c->g.g[gi], false, gi == ng - 1, E);
    // position bits that receive the warp bits of the thread index (the top
    // TB - 5 bits of the deposit mask), for groups that are neither single
    // stages nor subgraph-local; ~0 otherwise
    auto warp_bits = [&](int gi) -> unsigned {
        if (c->g.single_[gi] || c->g.local[gi]) return ~0u;
        unsigned m = c->g.cmask[gi][0], w = 0;
        for (int k = 0; k < TB; ++k) {
            const unsigned low = m & (0u - m);
            if (k >= 5) w |= low;
            m ^= low;
        }
        return w;
    };
    for (int gi = 0; gi < ng; ++gi) {
        const int s0 = c->g.s0[gi], gl = c->g.g[gi], single = c->g.single_[gi];
        const bool last = gi == ng - 1;
        // L level s0+2+i at colL + i E, R level s0+2+i at colL + (gl - 1 + i) E
        const int colL = last ? col - (gl - 1) * E : col;
        const bool wl_after = gi + 1 < ng && warp_bits(gi) != ~0u && warp_bits(gi) == warp_bits(gi + 1);
        const bool wl_before = gi > 0 && warp_bits(gi) != ~0u && warp_bits(gi) == warp_bits(gi - 1);
        const bool cached = !single && !(last && G3<LOGN, KB>::LASTREG);
        c->rec[gi] = make_int4(s0 | (gl << 8) | (single << 16) | (int(c->g.local[gi]) << 24) | (int(wl_after) << 25) |
                                   (int(wl_before) << 26),
                               colL,
                               (int(c->g.contig[gi][0]) & 0xff) | ((int(c->g.contig[gi][1]) & 0xff) << 8),
                               cached ? acol : 0);
        c->cmask[gi] = make_uint2(c->g.cmask[gi][0], c->g.cmask[gi][1]);
        for (int cls = 0; cls < 2; ++cls)
            for (int e = 0; e < E; ++e) c->swoff[gi][cls][e] = c->g.swoff[gi][cls][e];
        if (!single) {
            col += group_cols(s0, gl, false, last, E);
            if (cached) acol += E;
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

// alpha * m in both lanes, each lane rounded once as by __fmul_rn: a packed
// fused multiply-add whose addend nz is -0, a value the compiler cannot see
// (the exact product plus -0 is the exact product, and +0 + -0 = +0).  A
// packed multiply whose result feeds a packed add is fused into one packed
// multiply-add by ptxas (one rounding instead of two, even for mul.rn.f32x2
// and add.rn.f32x2); a product that already is a multiply-add is left alone.
__device__ __forceinline__ float2 scale2(float2 alpha2, float2 m, float2 nz2)
{
    return __ffma2_rn(alpha2, m, nz2);
}

// Two lanes of fnode<1> (exact box-plus), each lane computed with exactly the operations of
// fnode<1>: the packed additions, multiplications and fused multiply-adds round each lane as
// the scalar ones do, the exponentials, the reciprocal, the minimum and the |x| scalings stay
// scalar, and every packed product feeds only multiplications or is a multiplicand of a
// multiply-add, so none can be fused into an addition.  a - b is a + (-b), as IEEE subtraction is.
__device__ __forceinline__ float2 boxplus2(float2 a, float2 b)
{
    constexpr float kNegLog2e = -1.44269504088896341f;
    const float2 sm = make_float2(signed_min(a.x, b.x), signed_min(a.y, b.y));
    const float2 sum = __fadd2_rn(a, b), dif = __fadd2_rn(a, make_float2(-b.x, -b.y));
    const float2 p = make_float2(ex2_approx(__fmul_rn(fabsf(sum.x), kNegLog2e)),
                                 ex2_approx(__fmul_rn(fabsf(sum.y), kNegLog2e)));
    const float2 q = make_float2(ex2_approx(__fmul_rn(fabsf(dif.x), kNegLog2e)),
                                 ex2_approx(__fmul_rn(fabsf(dif.y), kNegLog2e)));
    const float2 den = __fadd2_rn(make_float2(2.f, 2.f), __fadd2_rn(p, q));
    const float2 sv = __fmul2_rn(__fadd2_rn(p, make_float2(-q.x, -q.y)),
                                 make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    const float2 z = __fmul2_rn(sv, sv);
    float2 h = make_float2(1.f / 13.f, 1.f / 13.f);
    h = __ffma2_rn(h, z, make_float2(1.f / 11.f, 1.f / 11.f));
    h = __ffma2_rn(h, z, make_float2(1.f / 9.f, 1.f / 9.f));
    h = __ffma2_rn(h, z, make_float2(1.f / 7.f, 1.f / 7.f));
    h = __ffma2_rn(h, z, make_float2(1.f / 5.f, 1.f / 5.f));
    h = __ffma2_rn(h, z, make_float2(1.f / 3.f, 1.f / 3.f));
    h = __ffma2_rn(h, z, make_float2(1.f, 1.f));
    const float2 v = __ffma2_rn(__fmul2_rn(make_float2(2.f, 2.f), sv), h, sm);
    return make_float2(isinf(sm.x) ? sm.x : v.x, isinf(sm.y) ? sm.y : v.y);
}

// f of two lanes for the packed PE layers: scaled min-sum (scale2) or exact box-plus (boxplus2).
template <int FK>
__device__ __forceinline__ float2 fnode2(float2 a, float2 b, float2 alpha2, float2 nz2)
{
    if constexpr (FK == 0) {
        return scale2(alpha2, make_float2(signed_min(a.x, b.x), signed_min(a.y, b.y)), nz2);
    } else {
        return boxplus2(a, b);
    }
}

// One PE layer inside a thread: register e pairs with e | 2^i.  For a layer
// i > 0, the elements with tops e and e+1 (e even) run together: their sums,
// f (fnode2) and final adds as packed two-lane FP32 operations, each lane
// rounded exactly as the scalar operations of fnode<FK> and __fadd_rn.
// Layer 0 pairs e with e+1 and stays scalar.
template <int E, int FK>
__device__ __forceinline__ void l_layer(float* x, const float* rv, int i, float alpha, float nz)
{
    if (i > 0) {
        const float2 a2 = make_float2(alpha, alpha), nz2 = make_float2(nz, nz);
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            if (e & (1 << i)) continue;
            const int eb = e | (1 << i);
            const float2 lt = make_float2(x[e], x[e + 1]), lb = make_float2(x[eb], x[eb + 1]);
            const float2 s = __fadd2_rn(lb, make_float2(rv[eb], rv[eb + 1]));
            const float2 top = fnode2<FK>(lt, s, a2, nz2);
            const float2 g = fnode2<FK>(make_float2(rv[e], rv[e + 1]), lt, a2, nz2);
            const float2 bot = __fadd2_rn(g, lb);
            x[e] = top.x;
            x[e + 1] = top.y;
            x[eb] = bot.x;
            x[eb + 1] = bot.y;
        }
        return;
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

template <int E, int FK>
__device__ __forceinline__ void r_layer(float* y, const float* lv, int i, float alpha, float nz)
{
    if (i > 0) {
        const float2 a2 = make_float2(alpha, alpha), nz2 = make_float2(nz, nz);
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            if (e & (1 << i)) continue;
            const int eb = e | (1 << i);
            const float2 rt = make_float2(y[e], y[e + 1]), rb = make_float2(y[eb], y[eb + 1]);
            const float2 s = __fadd2_rn(make_float2(lv[eb], lv[eb + 1]), rb);
            const float2 top = fnode2<FK>(rt, s, a2, nz2);
            const float2 g = fnode2<FK>(rt, make_float2(lv[e], lv[e + 1]), a2, nz2);
            const float2 bot = __fadd2_rn(g, rb);
            y[e] = top.x;
            y[e + 1] = top.y;
            y[eb] = bot.x;
            y[eb + 1] = bot.y;
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e & (1 << i)) continue;
        const int eb = e | (1 << i);
        const float rt = y[e], rb = y[eb];
        y[e] = fnode<FK>(rt, __fadd_rn(lv[eb], rb), alpha);
        y[eb] = __fadd_rn(fnode<FK>(rt, lv[e], alpha), rb);
    }
}

// Entry i of a stage order packed as 4-bit fields (range <= 16).
__device__ __forceinline__ int order_at(uint64_t ord, int i) { return int((ord >> (4 * i)) & 15u); }

// The partition of build_groups (short_last) plus pack_groups, computed by
// the 32 lanes of one warp: every lane walks the group list (a few dozen
// steps), lane 2g + c then builds group g's register bits for class c, and
// the lane pairs exchange what the packed record needs.  Writes g.ng, g.low,
// g.beta, g.pbit and the packed records (rec, cmask, swoff) that the TMEM
// kernel reads; the per-class bit lists of GroupCtl are not kept.  The event's
// stage order comes packed (order_at); segments, register bits and order live
// in registers (no local-memory arrays).
template <int LOGN, int KB>
__device__ __forceinline__ void build_partition_warp(Ctl3<LOGN, KB>* c, const unsigned char* swt, int level, int range,
                                                     long long blk, uint64_t ord, int lane)
{
    constexpr int n = LOGN;
    constexpr int E = 1 << KB;
    constexpr int TB = LOGN - KB;
    static_assert(5 * KB <= 32, "register bits packed 5 bits each");
    const int lo = level - 1, hi = level + range - 2, m = hi + 1;
    if (lane == 0) {
        c->g.low = n - m;
        c->g.beta = int(blk);
    }
    if (lane < 16) {
        int pb = n - 1 - lane;
        if (lane >= lo && lane <= hi) pb = n - level - order_at(ord, lane - lo);
        c->g.pbit[lane] = (signed char)pb;
    }
    // segments [a, b, kind]: 0 homogeneous, 1 subgraph-local, 2 single stages; segment sg of
    // at most 3, computed where it is used
    const bool wide = m >= KB;
    const bool head = !wide && lo >= 1;          // homogeneous stages before the single ones
    const bool tail = hi + 1 <= n - 1;           // homogeneous stages after the event
    const int nseg = (wide ? 1 : (head ? 2 : 1)) + (tail ? 1 : 0);
    auto seg = [&](int sg, int& a, int& b, int& kind) {
        if (wide) {
            if (sg == 0) { a = 0; b = hi; kind = 1; }
            else { a = hi + 1; b = n - 1; kind = 0; }
        } else {
            const int q = head ? sg : sg + 1;      // 0 head, 1 single stages, 2 tail
            if (q == 0) { a = 0; b = lo - 1; kind = 0; }
            else if (q == 1) { a = lo; b = hi; kind = 2; }
            else { a = hi + 1; b = n - 1; kind = 0; }
        }
    };
    // walk the groups: this lane's group gi = lane / 2, its columns before it
    const int gi = lane >> 1, cls = lane & 1;
    int ng = 0, my_s0 = 0, my_gl = 0, my_kind = -1, col = 0, acol = 0;
    int my_col = 0, my_acol = 0, last_gl = 0, last_col = 0;
#pragma unroll
    for (int sg = 0; sg < 3; ++sg) {
        if (sg < nseg) {
            int a = 0, b = 0, kind = 0;
            seg(sg, a, b, kind);
            const int len = b - a + 1;
            const int first = len % KB == 0 ? KB : len % KB;
            const bool sl = sg == nseg - 1;
            int st = a;
            for (int q = 0; st <= b; ++q) {
                const int gl = kind == 2 ? 1 : (sl ? (b - st + 1 < KB ? b - st + 1 : KB) : (q == 0 ? first : KB));
                if (ng == gi) {
                    my_s0 = st; my_gl = gl; my_kind = kind; my_col = col; my_acol = acol;
                }
                last_gl = gl; last_col = col;
                if (kind != 2) {
                    col += 2 * (gl - 1) * E;   // the last group's columns are counted from its R levels below
                    acol += E;
                }
                ++ng;
                st += gl;
            }
        }
    }
    const bool mine = gi < ng;
    const bool single = my_kind == 2;
    const bool last = gi == ng - 1;
    // the offsets follow this partition's interior columns (the last group stores R levels only)
    const int interior = last_col + (last_gl - 1) * E;
    const bool cached = mine && !single && !(last && G3<LOGN, KB>::LASTREG);
    // register bits of (gi, cls): position bit of register bit i in bits 5i..5i+4 of P
    unsigned used = 0, cmask = 0;
    int contig = -1;
    if (mine && !single) {
        unsigned P = 0;
        for (int i = 0; i < my_gl; ++i) {
            const int stg = my_s0 + i;
            int bit = n - 1 - stg;
            if (cls == 1 && my_kind == 1 && stg >= lo && stg <= hi) bit = n - level - order_at(ord, stg - lo);
            P |= unsigned(bit) << (5 * i);
            used |= 1u << bit;
        }
        const int floor_bit = my_kind == 1 ? n - m : 0;
        int nxt = my_gl;
        for (int bit = n - 1 - (my_s0 + my_gl); bit >= floor_bit && nxt < KB; --bit)
            if (!((used >> bit) & 1u)) { P |= unsigned(bit) << (5 * nxt++); used |= 1u << bit; }
        for (int bit = n - my_s0; bit <= n - 1 && nxt < KB; ++bit)
            if (!((used >> bit) & 1u)) { P |= unsigned(bit) << (5 * nxt++); used |= 1u << bit; }
        for (int bit = floor_bit; bit <= n - 1 && nxt < KB; ++bit)
            if (!((used >> bit) & 1u)) { P |= unsigned(bit) << (5 * nxt++); used |= 1u << bit; }
        cmask = ((1u << n) - 1u) & ~used;
        const int lowb = __ffs(used) - 1;
        contig = (used >> lowb) == ((1u << KB) - 1u) ? lowb : -1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int off = 0;
#pragma unroll
            for (int i = 0; i < KB; ++i)
                if ((e >> i) & 1) off |= 1 << ((P >> (5 * i)) & 31u);
            c->swoff[gi][cls][e] = (short)swz(swt, off);
        }
    }
    // warp bits of the thread index in group gi (class 0), ~0 for single or local groups
    unsigned wb = ~0u;
    if (mine && !single && my_kind != 1) {
        unsigned mm = cmask;
        wb = 0;
        for (int k = 0; k < TB; ++k) {
            const unsigned low = mm & (0u - mm);
            if (k >= 5) wb |= low;
            mm ^= low;
        }
    }
    const unsigned cmask1 = __shfl_down_sync(0xffffffffu, cmask, 1);
    const int contig1 = __shfl_down_sync(0xffffffffu, contig, 1);
    const unsigned wb_next = __shfl_down_sync(0xffffffffu, wb, 2);
    const unsigned wb_prev = __shfl_up_sync(0xffffffffu, wb, 2);
    if (mine && cls == 0) {
        const bool wl_after = !last && wb != ~0u && wb == wb_next;
        const bool wl_before = gi > 0 && wb != ~0u && wb == wb_prev;
        // column of L level s0+2 (virtual for the last group), as pack_groups
        const int colL = last ? my_col - (my_gl - 1) * E : my_col;
        c->rec[gi] = make_int4(my_s0 | (my_gl << 8) | (int(single) << 16) | (int(my_kind != 0) << 24) |
                                   (int(wl_after) << 25) | (int(wl_before) << 26),
                               colL, (contig & 0xff) | ((contig1 & 0xff) << 8), cached ? interior + my_acol : 0);
        c->cmask[gi] = make_uint2(cmask, cmask1);
    }
    if (lane == 0) c->g.ng = ng;
}

// x mod d for 0 < d < 2^16, equal to the 64-bit remainder: with x = hi 2^32 + lo,
// x = (hi mod d)(2^32 mod d) + (lo mod d) (mod d), and that sum is at most (d - 1)^2 + d - 1 <
// 2^32, so 32-bit remainders give it (a 64-bit remainder by a run-time divisor is a long
// serial subroutine).
__device__ __forceinline__ uint32_t mod_small(uint64_t x, uint32_t d)
{
    const uint32_t hi = uint32_t(x >> 32), lo = uint32_t(x);
    const uint32_t p = (0u - d) % d;      // 2^32 mod d
    return ((hi % d) * p + lo % d) % d;
}

// draw_event (bp_kernel.cuh) computed by the 32 lanes of a warp: lane d
// evaluates draw d of the event's counter-based stream and reduces it by the
// divisor that draw meets (lanes 0 and 1: range and level; lanes 3 + 16 a + t:
// the Fisher-Yates draw t of attempt a, modulo range - t), every lane then
// makes the same choices from those values (fetched with shuffles; draws past
// 31, needed only from the third attempt on or for ranges above 13, are
// evaluated directly).  The block draw is reduced modulo a power of two, a
// mask.  Same draws, same remainders and same choices, so the same event.
__device__ __forceinline__ void draw_event_warp(const DevSched& S, int n, uint64_t frame, int k, int lane, int& level,
                                                int& range, long long& block, uint64_t& ord)
{
    const uint64_t mine = event_draw(S.seed, frame, uint64_t(k), uint64_t(lane));
    auto draw = [&](int d) -> uint64_t {
        if (d < 32) {
            const unsigned lo32 = __shfl_sync(0xffffffffu, unsigned(mine), d);
            const unsigned hi32 = __shfl_sync(0xffffffffu, unsigned(mine >> 32), d);
            return (uint64_t(hi32) << 32) | lo32;
        }
        return event_draw(S.seed, frame, uint64_t(k), uint64_t(d));
    };
    if (S.mode == 2) {
        range = n;
        level = 1;
        block = 0;
    } else {
        const uint32_t dv = lane == 0 ? uint32_t(S.P_range > 2 ? S.P_range - 1 : 1) : uint32_t(S.P_level > 1 ? S.P_level : 1);
        const uint32_t red = mod_small(mine, dv);
        const uint32_t r0 = __shfl_sync(0xffffffffu, red, 0), r1 = __shfl_sync(0xffffffffu, red, 1);
        range = S.rho_fixed > 0 ? S.rho_fixed : 2 + int(r0);
        const int x = 1 + int(r1);
        level = min(x, n - range + 1);
        const int m = level + range - 1;
        block = (long long)(draw(2) & ((1ull << (n - m)) - 1ull));
    }
    uint32_t jr = 0;     // this lane's Fisher-Yates remainder (lanes 3 .. 31)
    {
        const int t = (lane - 3) & 15;
        if (lane >= 3 && t < range - 1) jr = mod_small(mine, uint32_t(range - t));
    }
    // the order packed 4 bits per entry (order_at); Fisher-Yates swaps exchange two fields
    uint64_t ident = 0, rot = 0;
    for (int i = 0; i < range; ++i) {
        ident |= uint64_t(i) << (4 * i);
        rot |= uint64_t((i + 1) % range) << (4 * i);
    }
    for (int attempt = 0; attempt < 8; ++attempt) {
        uint64_t v = ident;
        for (int i = range - 1; i >= 1; --i) {
            const int dl = 3 + 16 * attempt + (range - 1 - i);
            const int j = dl < 32 ? int(__shfl_sync(0xffffffffu, jr, dl))
                                  : int(mod_small(event_draw(S.seed, frame, uint64_t(k), uint64_t(dl)), uint32_t(i + 1)));
            const uint64_t x = ((v >> (4 * i)) ^ (v >> (4 * j))) & 15u;
            v ^= (x << (4 * i)) | (x << (4 * j));
        }
        if (v != ident) {
            ord = v;
            return;
        }
    }
    ord = rot;
}

// Records event (level, range, blk) of frame `frame` (Sec. III) as the current
// event (the previous one becomes the event to revert) and sets the increment
// of N_it,reset (Eq. 2).  One thread.
template <int LOGN, int KB>
__device__ __forceinline__ void apply_event(Ctl3<LOGN, KB>* ctl, const DevSched& S, int level, int range, long long blk)
{
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
}

// A switch's event and partition (Sec. III), by the first warp of a slot: the event draws
// (draw_event_warp), their record (apply_event, lane 0) and the new partition
// (build_partition_warp).  Out of line, one call per switch, so that the iteration loop stays
// compact.
template <int LOGN, int KB>
__device__ __noinline__ void switch_event_warp(Ctl3<LOGN, KB>* ctl, const DevSched& S, const unsigned char* swt,
                                               uint64_t frame, int k, int lane)
{
    int level = 0, range = 0;
    long long blk = 0;
    uint64_t ord = 0;
    const auto& d = ctl->nx[k & 1];
    if (d.k == k && d.frame == int(frame)) {      // drawn ahead during the previous switch
        level = d.level;
        range = d.range;
        blk = d.blk;
        ord = d.ord;
    } else {
        draw_event_warp(S, LOGN, frame, k, lane, level, range, blk, ord);
    }
    if (lane == 0) apply_event<LOGN, KB>(ctl, S, level, range, blk);
    build_partition_warp<LOGN, KB>(ctl, swt, level, range, blk, ord, lane);
}

// Event k of a frame drawn ahead by a warp that would otherwise wait, during switch k - 1 (the
// draws depend on the seed, the frame and k only), into nx[k & 1], which that switch does not read.
template <int LOGN, int KB>
__device__ __noinline__ void predraw_event_warp(Ctl3<LOGN, KB>* ctl, const DevSched& S, uint64_t frame, int k, int lane)
{
    int level = 0, range = 0;
    long long blk = 0;
    uint64_t ord = 0;
    draw_event_warp(S, LOGN, frame, k, lane, level, range, blk, ord);
    if (lane == 0) {
        auto& d = ctl->nx[k & 1];
        d.level = level;
        d.range = range;
        d.blk = blk;
        d.ord = ord;
        d.frame = int(frame);
        d.k = k;
    }
}

// One permuted stage s narrower than a register group (m < KB events), with
// per-PE addressing: the L sweep (r_sweep false) or the R sweep of stage s.
// L at node level s+1 comes from Lin (the channel LLRs for s = 0), L at level
// s+2 goes to Lout, R at level l is plane l-2 of Rp.  The R sweep of stage 0
// sets the hard-decision bits of L + R at node level 1 in xh, or, when post1
// is given, writes R at node level 1 there instead.  E/2 PEs per thread; out
// of line (rare).
template <int LOGN, int E, int T, int FK>
__device__ __noinline__ void single_stage(bool r_sweep, int s, int tid, int lowmask, int beta, int lo, int m1, int pbit,
                                          const float* llr_f, const float* Lin, float* Lout, float* Rp, uint32_t* xh,
                                          const unsigned char* s_swz, float alpha, unsigned* check,
                                          float* post1 = nullptr)
{
    constexpr int n = LOGN;
    constexpr int N = 1 << LOGN;
    auto sw = [&](int j) { return swz(s_swz, j); };
#pragma unroll
    for (int c = 0; c < E / 2; ++c) {
        const int q = tid + c * T;
        int p = n - 1 - s;
        if (s >= lo && s <= m1 && (q & lowmask) == beta) p = pbit;
        const int t = ((q >> p) << (p + 1)) | (q & ((1 << p) - 1));
        const int b = t | (1 << p);
#ifdef PCBP_CHECKED
        if (t >= N || b >= N || p < 0 || p >= n || s < 0 || s >= n - 1) {
            chk_fail(check, 5);
            continue;
        }
#else
        (void)check;
#endif
        const float lt = s == 0 ? llr_f[t] : Lin[sw(t)];
        const float lb = s == 0 ? llr_f[b] : Lin[sw(b)];
        const float rt = Rp[s * N + sw(t)];
        const float rb = Rp[s * N + sw(b)];
        if (!r_sweep) {
            Lout[sw(t)] = fnode<FK>(lt, __fadd_rn(lb, rb), alpha);
            Lout[sw(b)] = __fadd_rn(fnode<FK>(rt, lt, alpha), lb);
        } else {
            const float o1 = fnode<FK>(rt, __fadd_rn(lb, rb), alpha);
            const float o2 = __fadd_rn(fnode<FK>(rt, lt, alpha), rb);
            if (s >= 1) {
                Rp[(s - 1) * N + sw(t)] = o1;
                Rp[(s - 1) * N + sw(b)] = o2;
            } else if (post1) {
                post1[t] = o1;
                post1[b] = o2;
            } else {
                if (__fadd_rn(lt, o1) < 0.f) atomicOr(&xh[t >> 5], 1u << (t & 31));
                if (__fadd_rn(lb, o2) < 0.f) atomicOr(&xh[b >> 5], 1u << (b & 31));
            }
        }
    }
}

// Shared memory ahead of the frame slots: code tables, then the control
// block of the no-event partition (built once per CTA, copied into a slot
// whose previous frame switched partitions).
template <int LOGN, int KB>
__host__ __device__ constexpr size_t tmem_cta_bytes(int N, int K)
{
    return tmem_table_bytes(N, K) + align16(sizeof(Ctl3<LOGN, KB>));
}

// The no-event control block (one thread).
template <int LOGN, int KB>
__device__ __noinline__ void build_template(Ctl3<LOGN, KB>* c, const unsigned char* s_swz)
{
    c->g.frame = 0;
    c->g.have_ev = 0;
    c->g.have_prev = 0;
    c->g.ev_level = 0;
    c->g.ev_range = 0;
    c->g.ev_blk = -1;
    c->g.pv_level = 0;
    c->g.pv_range = 0;
    c->g.pv_blk = -1;
    c->g.next_inc = 0;
    c->g.crc_res = 0;
    c->g.g_ok = 0;
    c->crc_part[0] = 0u;
    c->crc_part[1] = 0u;
    c->crc_part[2] = 0u;
    c->nx[0].k = -1;
    c->nx[1].k = -1;
    signed char none[16];
    build_groups<LOGN, KB>(&c->g, s_swz, LOGN, false, 0, 0, 0, none, true);
    pack_groups<LOGN, KB>(c);
}

// PO = 1 (posterior output, a debug build of the same sweeps): every frame
// also writes L at node level n+1 and R at node level 1 after its last
// iteration to J.post, and that iteration always completes its R sweep.
template <int LOGN, int KB, int FK, int WG, int PO>
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
    const uint32_t* s_cj = s_frozen + NW;
    const int16_t* s_info = reinterpret_cast<const int16_t*>(s_cj + N);
    const unsigned char* s_swz = smem + tmem_table_bytes(N, K) - kSwzTableBytes;
    auto sw = [&](int j) { return swz(s_swz, j); };
    (void)r;

    const int slot = threadIdx.x / T;
    const int tid = threadIdx.x - slot * T;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    constexpr size_t ctl_bytes = align16(sizeof(Ctl));
    constexpr size_t slot_sz = tmem_slot_bytes<LOGN, KB>();
    const Ctl* tmpl = reinterpret_cast<const Ctl*>(smem + tmem_table_bytes(N, K));
    unsigned char* sbase = smem + tmem_cta_bytes<LOGN, KB>(N, K) + size_t(slot) * slot_sz;
    Ctl* ctl = reinterpret_cast<Ctl*>(sbase);
    uint32_t* dec = reinterpret_cast<uint32_t*>(sbase + ctl_bytes);
    uint32_t* xh = dec + NW;
    // the slot's planes (G3::NPLANES): R at node level l in plane l-2
    float* Rp = reinterpret_cast<float*>(sbase + ctl_bytes + align16(2 * NW * 4));
    float* Lspare = Rp + Geo::SPARE * N;
    const int lp_off = int(reinterpret_cast<unsigned char*>(Rp) - smem);
    const unsigned bar_id = 1u + unsigned(slot);
    auto sync = [&]() {
        if (T == 32) __syncwarp();
        else slot_sync(bar_id, T);
    };
    // this thread's TMEM lane: the warp's quarter of the lanes, its column bank
    const int gwarp = int(threadIdx.x >> 5);
    const uint32_t tm = tm_base + (uint32_t(32 * (gwarp & 3)) << 16) + uint32_t((gwarp >> 2) * Geo::TCOLS);

    // The cached offset A of a position in a group with first stage s0 is the
    // byte offset (from smem) of the position in plane s0, which holds the
    // group's input, L at node level s0+1; the other planes it touches are at
    // fixed distances, plane s0+d at A + 4 d N:
    //   R at level s0+1 (the R sweep's output)        d = -1
    //   R at level s0+2+i (interior, copied at switches) d = i
    //   R at level s0+gl+1 (the next group's output)  d = gl - 1
    //   L at level s0+gl+1 (the next group's input)   d = gl
    //   priors, CRC contributions (last group, s0 = n - gl)  d = gl, gl + 1
    auto at = [&](int a, int floats) -> float& {
        int off = a + 4 * floats;
#ifdef PCBP_CHECKED
        if (off < lp_off || off > lp_off + 4 * (Geo::NPLANES * N - 1) || (off & 3)) {
            chk_fail(J.check, 0);
            off = lp_off;
        }
#endif
        return *reinterpret_cast<float*>(smem + off);
    };
    // TMEM address of column `col` of this thread's bank
    auto tc = [&](uint32_t col) -> uint32_t {
#ifdef PCBP_CHECKED
        if (col > uint32_t(Geo::TCOLS - E)) {
            chk_fail(J.check, 1);
            col = 0;
        }
#endif
        return tm + col;
    };
    // logical position of cached offset a in a group with first stage s0
    auto pos_of = [&](int a, int s0) {
        int x = ((a - lp_off) >> 2) - s0 * N;
#ifdef PCBP_CHECKED
        if (x < 0 || x >= N) {
            chk_fail(J.check, 2);
            x = 0;
        }
#endif
        return sw(x);
    };

    const DevSched& S = J.S;
    const float alpha = S.alpha;
    const float nzero = J.neg_zero;    // -0, read at run time (scale2)
    const int KW = (K + 31) / 32;
    const int max_iters = J.max_iters;
    constexpr bool want_g = WG != 0;     // the G-matrix test is on (stop_kind & 2), fixed per launch
    static_assert(!(PO && WG), "the posterior output is built for the CRC stop only");
    const bool want_crc = (S.stop_kind & 1) != 0;

    float L1[E];   // channel LLRs of the first group's positions
    int ALr[E];    // the last group's offsets, when they are kept in registers (G3::LASTREG)
#pragma unroll
    for (int e = 0; e < E; ++e) ALr[e] = lp_off;

    auto group_class = [&](int meta) {
        const bool local = (meta >> 24) & 1;
        const int lowmask = (1 << ctl->g.low) - 1;
        return (local && ((tid & lowmask) == ctl->g.beta)) ? 1 : 0;
    };

    // Planes of a single stage's L input (level s0+1) and output (level s0+2):
    // the boundary plane of its level, or the spare plane where the
    // neighbouring stage is a single stage too (its boundary plane then holds
    // a boundary R message).  Partitions have at most KB - 1 <= 2 single stages.
    auto single_in = [&](int gi, int s0) -> const float* {
        if (s0 == 0) return nullptr;
        return ((ctl->rec[gi - 1].x >> 16) & 1) ? Lspare : Rp + s0 * N;
    };
    auto single_out = [&](int gi, int s0) -> float* {
        return ((ctl->rec[gi + 1].x >> 16) & 1) ? Lspare : Rp + (s0 + 1) * N;
    };

    // A new frame on the partition the TMEM caches already describe: zero
    // interior R messages, channel LLRs of group 0's positions (from llr_src,
    // in natural position order).
    auto restart_partition = [&](const float* llr_src) {
        // the no-event partition has (n + KB - 1) / KB groups and no single stages: the group
        // loop is unrolled, so the records and the first group's offsets load at once
        constexpr int NG0 = (LOGN + KB - 1) / KB;
#ifdef PCBP_CHECKED
        if (ctl->g.ng != NG0) chk_fail(J.check, 6);
#endif
        float z[E];
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = 0.f;
        int A[E];
        tm_ld_i<E>(tc(uint32_t(ctl->rec[0].w)), A);
#pragma unroll
        for (int gi = 0; gi < NG0; ++gi) {
            const int4 rc = ctl->rec[gi];
            const int gl = (rc.x >> 8) & 0xff;
            const uint32_t colR = uint32_t(rc.y + (gl - 1) * E);
#pragma unroll
            for (int i = 0; i < KB - 1; ++i)
                if (i < gl - 1) tm_st<E>(tc(colR + uint32_t(i * E)), z);
        }
        tm_wait_ld();
        tm_fence<E>(A);
#pragma unroll
        for (int e = 0; e < E; ++e) L1[e] = llr_src[pos_of(A[e], 0)];
        tm_wait_st();
    };

    // After a new partition: cache the register groups' offsets in TMEM, move
    // the interior R messages from the canonical planes to TMEM, load the
    // channel LLRs of the first group (from llr_src, in natural position order).
    auto enter_partition = [&](const float* llr_src) {
        const int ng = ctl->g.ng;
        #pragma unroll 1
        for (int gi = 0; gi < ng; ++gi) {
            const int4 rc = ctl->rec[gi];
            const int s0 = rc.x & 0xff, gl = (rc.x >> 8) & 0xff;
            if ((rc.x >> 16) & 1) continue;
            int ph[E], A[E];
            group_offsets<LOGN, KB>(ctl, s_swz, gi, group_class(rc.x), rc.z, tid, ph);
#ifdef PCBP_CHECKED
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (ph[e] < 0 || ph[e] >= N) {
                    chk_fail(J.check, 3);
                    ph[e] = 0;
                }
#endif
#pragma unroll
            for (int e = 0; e < E; ++e) A[e] = lp_off + 4 * (s0 * N + ph[e]);
            if (Geo::LASTREG && gi == ng - 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) ALr[e] = A[e];
            } else {
                tm_st_i<E>(tc(uint32_t(rc.w)), A);
            }
            const uint32_t colR = uint32_t(rc.y + (gl - 1) * E);
            #pragma unroll 1
            for (int i = 0; i < gl - 1; ++i) {     // R level s0+2+i: plane s0+i
                float v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = at(A[e], i * N);
                tm_st<E>(tc(colR + uint32_t(i * E)), v);
            }
            if (gi == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) L1[e] = llr_src[sw(ph[e])];
            }
        }
        tm_wait_st();
    };

    // Before a new partition: the interior R messages back to the canonical planes.
    auto leave_partition = [&]() {
        const int ng = ctl->g.ng;
        #pragma unroll 1
        for (int gi = 0; gi < ng; ++gi) {
            const int4 rc = ctl->rec[gi];
            const int gl = (rc.x >> 8) & 0xff;
            if ((rc.x >> 16) & 1) continue;
            if (gl < 2) continue;
            int A[E];
            if (Geo::LASTREG && gi == ng - 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) A[e] = ALr[e];
            } else {
                tm_ld_i<E>(tc(uint32_t(rc.w)), A);
                tm_wait_ld();
                tm_fence<E>(A);
            }
            const uint32_t colR = uint32_t(rc.y + (gl - 1) * E);
            #pragma unroll 1
            for (int i = 0; i < gl - 1; ++i) {
                float v[E];
                tm_ld<E>(tc(colR + uint32_t(i * E)), v);
                tm_wait_ld();
                tm_fence<E>(v);
#pragma unroll
                for (int e = 0; e < E; ++e) at(A[e], i * N) = v[e];
            }
        }
    };

    // Frame indices come from the launch's atomic counter.  The slot leader takes the next index
    // as soon as the current frame's last iteration is known, so the atomic's latency overlaps
    // the frame's output phase, and publishes it in s_next[slot] (outside the control block,
    // which a frame start may overwrite with the no-event template while other warps of the slot
    // have yet to read the index).
    __shared__ long long s_next[32];
    static_assert(tmem_max_threads<LOGN, KB>() / T <= 32, "one next-frame index per slot");
    long long* const next_frame = &s_next[slot];
    unsigned long long next_f = 0;
    bool have_next = false;
    auto fetch_next = [&]() {
        if (tid == 0 && !have_next) {
            next_f = atomicAdd(counter, 1ull);
            have_next = true;
        }
    };
    // the slot leader's fetched index to s_next (visible after the next slot barrier)
    auto publish_next = [&]() {
        if (tid == 0) {
            *next_frame = (long long)next_f;
            have_next = false;
        }
    };
    bool fresh = false;     // the control block holds the no-event partition and the TMEM caches match it
    // the prior R(n+1) and the CRC contribution of every position, in this slot's planes (read
    // by the last group at fixed distances from its cached offsets)
    for (int j = tid; j < N; j += T) {
        Rp[Geo::PRIOR * N + sw(j)] = prior_of(s_frozen, j);
        Rp[Geo::CJ * N + sw(j)] = __int_as_float(int(s_cj[j]));
    }
    fetch_next();
    publish_next();
    sync();
    while (true) {
        const long long f = *next_frame;     // published before a slot barrier
        if (f >= J.B) break;
        const float* llr_f = J.llr + size_t(f) * N;
        // a1: the frame's channel LLRs stream into the spare plane (free between frames) as
        // 16-byte asynchronous copies, while the planes are cleared; the first group's threads
        // then read their positions from shared memory
        float* s_llr = Rp + Geo::SPARE * N;
        {
            const uint32_t d = uint32_t(__cvta_generic_to_shared(s_llr));
            const size_t g = size_t(__cvta_generic_to_global(llr_f));
            for (int i = tid; i < N / 4; i += T)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * uint32_t(i)),
                             "l"(g + 16u * size_t(i))
                             : "memory");
        }

        if (fresh) {
            // the no-event partition (groups of KB stages from stage 0, the short one last) reads
            // R at its group boundaries, levels KB+1, 2KB+1, ... (planes KB-1, 2KB-1, ...) before
            // writing them; its interior R levels restart in TMEM, and the planes of those levels
            // hold group inputs, written before they are read
            constexpr int NBP = (LOGN - 1) / KB;
            for (int i = tid; i < NBP * N / 4; i += T) {
                const int k = i / (N / 4);
                reinterpret_cast<float4*>(Rp + ((k + 1) * KB - 1) * N)[i - k * (N / 4)] =
                    make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            // enter_partition reads the no-event partition's interior R from the planes
            for (int i = tid; i < NPL * N / 4; i += T)
                reinterpret_cast<float4*>(Rp)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int i = tid; i < NW; i += T) {
            dec[i] = 0u;
            xh[i] = 0u;
        }
        if (fresh) {
            // the partition is still the no-event one; only the residues restart
            if (tid == 0) {
                ctl->crc_part[0] = 0u;
                ctl->crc_part[1] = 0u;
                ctl->crc_part[2] = 0u;
            }
        } else {
            static_assert(sizeof(Ctl) % 16 == 0, "control block copied in 16-byte words");
            for (int i = tid; i < int(sizeof(Ctl) / 16); i += T)
                reinterpret_cast<int4*>(ctl)[i] = reinterpret_cast<const int4*>(tmpl)[i];
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        sync();
        // both read the staged LLRs and (enter_partition) the interior R planes, which the first
        // L sweep overwrites with boundary L messages: every thread's reads come first
        if (fresh) restart_partition(s_llr);
        else enter_partition(s_llr);
        if (tid == 0) ctl->crc_final = 0u;
        sync();
        fresh = true;

        int next_reset = S.mode == 1 ? S.T0 : (S.mode == 2 ? S.it_reset_full : 0);
        int kev = 0;
        int used = max_iters;

        int pb = 0;     // it % 3
        for (int it = 1; it <= max_iters; ++it) {
            pb = pb == 2 ? 0 : pb + 1;
            const int ng = ctl->g.ng;
            const int lowmask = (1 << ctl->g.low) - 1;
            const int beta = ctl->g.beta;
            tm_wait_st();

            // ---------------- L sweep, all groups but the last.  Group 0 (stages from 0;
            // never the last group, a partition has at least n / KB >= 2 groups) takes the
            // channel LLRs from registers: it runs its own copy of the group step.
            auto l_group = [&](int gi, auto firstc, auto singlesc) {
                constexpr bool FIRST = decltype(firstc)::value;
                constexpr bool SINGLES = decltype(singlesc)::value;     // the partition has single stages
                const int4 rc = ctl->rec[gi];
                const int s0 = FIRST ? 0 : (rc.x & 0xff), gl = (rc.x >> 8) & 0xff;
                if (SINGLES && ((rc.x >> 16) & 1)) {
                    // one permuted stage with per-PE addressing (m < KB events)
                    single_stage<LOGN, E, T, FK>(false, s0, tid, lowmask, beta, ctl->g.ev_level - 1,
                                                 ctl->g.ev_level + ctl->g.ev_range - 2, ctl->g.pbit[s0], llr_f,
                                                 single_in(gi, s0), single_out(gi, s0), Rp, xh, s_swz, alpha, J.check);
                } else {
                    const uint32_t colL = uint32_t(rc.y);
                    auto body = [&](auto glc) {
                        constexpr int GL = decltype(glc)::value;
                        int A[E];
                        float rp[GL > 1 ? GL - 1 : 1][E];
                        tm_ld_i<E>(tc(uint32_t(rc.w)), A);
                        if constexpr (GL > 1) {
#pragma unroll
                            for (int i = 0; i < GL - 1; ++i) tm_ld<E>(tc(colL + uint32_t((GL - 1 + i) * E)), rp[i]);
                        }
                        tm_wait_ld();
                        tm_fence<E>(A);
                        float x[E], rb[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            x[e] = FIRST ? L1[e] : at(A[e], 0);                  // L level s0+1 (boundary)
                            rb[e] = at(A[e], (GL - 1) * N);                      // R level s0+GL+1 (boundary)
                        }
                        if constexpr (GL > 1) {
#pragma unroll
                            for (int i = 0; i < GL - 1; ++i) tm_fence<E>(rp[i]);
                        }
#pragma unroll
                        for (int i = 0; i < GL; ++i) {
                            l_layer<E, FK>(x, i < GL - 1 ? rp[i < GL - 1 ? i : 0] : rb, i, alpha, nzero);
                            if (i < GL - 1) tm_st<E>(tc(colL + uint32_t(i * E)), x);   // L level s0+2+i
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e) at(A[e], GL * N) = x[e];          // L level s0+GL+1
                    };
                    // only group 0 and the last group can have fewer than KB stages: every
                    // other group is a single stage or a full KB (partition rule of
                    // build_partition_warp, checked by pc_partition_selfcheck)
                    if constexpr (FIRST) {
                        if (gl == KB) body(std::integral_constant<int, KB>{});
                        else if (KB > 2 && gl == 2) body(std::integral_constant<int, (KB > 2 ? 2 : 1)>{});
                        else body(std::integral_constant<int, 1>{});
                    } else {
                        body(std::integral_constant<int, KB>{});
                    }
                }
                if ((rc.x >> 25) & 1) __syncwarp();
                else sync();
            };
            // single stages exist only while the event spans fewer than KB stages
            const bool singles = ctl->g.have_ev && ctl->g.ev_level + ctl->g.ev_range - 1 < KB;
            if (!singles) {
                l_group(0, std::true_type{}, std::false_type{});
                #pragma unroll 1
                for (int gi = 1; gi < ng - 1; ++gi) l_group(gi, std::false_type{}, std::false_type{});
            } else {
                l_group(0, std::true_type{}, std::true_type{});
                #pragma unroll 1
                for (int gi = 1; gi < ng - 1; ++gi) l_group(gi, std::false_type{}, std::true_type{});
            }

            // ---------------- last group: L sweep, decisions, residue, R sweep
            const int gL = ng - 1;
            const int4 rcL = ctl->rec[gL];
            const int s0L = rcL.x & 0xff, glL = (rcL.x >> 8) & 0xff;
            const uint32_t colLL = uint32_t(rcL.y);
            int AL[E];
            float pr[E];     // R(n+1): the prior of the last group's positions
            unsigned umask = 0;
            unsigned pmask = 0;     // G-matrix test: the decisions at their position bits within the block
            const bool check = S.stop_kind != 0 && it >= S.stop_from;
            // the group's stage count as a compile-time constant
            auto last_body = [&](auto glc) {
                constexpr int GLL = decltype(glc)::value;
                float rp[GLL > 1 ? GLL - 1 : 1][E];
                float xL[GLL][E];
                float x[E];
                int cj[E];
                if constexpr (Geo::LASTREG) {
#pragma unroll
                    for (int e = 0; e < E; ++e) AL[e] = ALr[e];
                } else {
                    tm_ld_i<E>(tc(uint32_t(rcL.w)), AL);
                }
#pragma unroll
                for (int i = 0; i < GLL - 1; ++i) tm_ld<E>(tc(colLL + uint32_t((GLL - 1 + i) * E)), rp[i]);
                tm_wait_ld();
                tm_fence<E>(AL);
#pragma unroll
                for (int i = 0; i < GLL - 1; ++i) tm_fence<E>(rp[i]);
                // the last group ends at stage n-1, so it starts at s0 = n - GLL (never 0): its
                // input, priors and CRC contributions are planes n-GLL, n and n+1
                static_assert(Geo::PRIOR == LOGN && Geo::CJ == LOGN + 1, "plane distances below");
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    x[e] = at(AL[e], 0);
                    pr[e] = at(AL[e], GLL * N);
                    cj[e] = __float_as_int(at(AL[e], (GLL + 1) * N));
                }
#pragma unroll
                for (int i = 0; i < GLL; ++i) {
#pragma unroll
                    for (int e = 0; e < E; ++e) xL[i][e] = x[e];
                    l_layer<E, FK>(x, i < GLL - 1 ? rp[i < GLL - 1 ? i : 0] : pr, i, alpha, nzero);
                }
                if constexpr (PO != 0) {
                    // L at node level n+1, overwritten every iteration (the barriers between
                    // iterations order the writes of different threads)
                    float* po = J.post + size_t(f) * 2 * N;
#pragma unroll
                    for (int e = 0; e < E; ++e) po[pos_of(AL[e], s0L)] = x[e];
                }
                // a5: decisions u_j = [L(n+1) + R(n+1) < 0], taken as L(n+1) < -R(n+1) (a
                // rounded sum has the sign of the exact one), and their CRC residue
                unsigned part = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const bool u = x[e] < -pr[e];
                    umask |= u ? 1u << e : 0u;
                    if constexpr (want_g) pmask |= u ? 1u << last_group_offset<GLL, KB>(e) : 0u;
                    part ^= u ? unsigned(cj[e]) : 0u;
                }
                if (check && want_crc) {
                    part = __reduce_xor_sync(0xffffffffu, part);
                    if (lane == 0 && part) atomicXor(&ctl->crc_part[pb], part);
                }
                // R sweep of the last group (ahead of the stop test)
                tm_wait_st();
                float y[E];
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = pr[e];
#pragma unroll
                for (int i = GLL - 1; i >= 0; --i) {
                    r_layer<E, FK>(y, xL[i], i, alpha, nzero);
                    if (i > 0) {
                        tm_st<E>(tc(colLL + uint32_t((GLL + i - 2) * E)), y);   // R level s0L+1+i
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) at(AL[e], -N) = y[e];       // R level s0L+1
                    }
                }
            };
            if (glL == KB) last_body(std::integral_constant<int, KB>{});
            else if (KB > 2 && glL == 2) last_body(std::integral_constant<int, (KB > 2 ? 2 : 1)>{});
            else last_body(std::integral_constant<int, 1>{});
            sync();
            const unsigned res = (check && want_crc) ? ctl->crc_part[pb] : 0u;
            // every thread read the residue of iteration it-1 before this barrier; the
            // next barrier of this kind comes before anyone accumulates iteration it+2
            if (tid == 0) ctl->crc_part[pb == 0 ? 2 : pb - 1] = 0u;

            bool po_end = false;     // PO: the frame's last iteration, finished after its R sweep
            // the G-matrix test runs where it can decide: from stop_from on, and with the combined
            // stop only where the CRC residue is zero (otherwise the frame goes on either way)
            const bool gtest = want_g && check && (!want_crc || res == 0u);
            if (want_g && (gtest || it == max_iters)) {
                // the decision words of this iteration, into cleared words (every word is clear
                // except after a G-matrix test, which clears them again)
                if (!((rcL.x >> 24) & 1) && int((signed char)(rcL.z & 0xff)) == 0) {
                    // the register bits are position bits 0..KB-1 (every thread in class 0, in
                    // stage order): a thread's decisions lie in one E-bit field of the word it
                    // shares with 32/E neighbouring lanes, combined by shuffles and stored once
                    // (register e at position base + last_group_offset(e), base E-aligned)
                    const int base = pos_of(AL[0], s0L);
                    unsigned v = pmask << (base & 31);
#pragma unroll
                    for (int o = 1; o < 32 / E; o <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
                    if ((lane & (32 / E - 1)) == 0) dec[base >> 5] = v;
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((umask >> e) & 1u) {
                            const int j = pos_of(AL[e], s0L);
                            atomicOr(&dec[j >> 5], 1u << (j & 31));
                        }
                }
                if (!gtest) {
                    // the last iteration without a test: the frame ends here, without its R sweep
                    fetch_next();
                    sync();
                    break;
                }
            }
            if (!want_g) {
                const bool stop = check && res == 0u;
                if (stop || it == max_iters) {
                    if (tid == 0 && check) ctl->crc_final = stop ? 2u : 1u;    // read after the barrier below
                    fetch_next();
                    // the decision words, once per frame: where every thread's register bits are
                    // position bits 0..KB-1 (class 0, in stage order), 32/E neighbouring lanes
                    // combine one whole word by shuffles; otherwise one shared atomic per decided
                    // position into cleared words
                    if (!((rcL.x >> 24) & 1) && int((signed char)(rcL.z & 0xff)) == 0) {
                        const unsigned pm = glL == KB ? last_group_bits<KB, KB>(umask)
                                            : (KB > 2 && glL == 2) ? last_group_bits<(KB > 2 ? 2 : 1), KB>(umask)
                                                                   : last_group_bits<1, KB>(umask);
                        const int base = pos_of(AL[0], s0L);
                        unsigned v = pm << (base & 31);
#pragma unroll
                        for (int o = 1; o < 32 / E; o <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
                        if ((lane & (32 / E - 1)) == 0) dec[base >> 5] = v;
                    } else {
                        for (int i = tid; i < NW; i += T) dec[i] = 0u;
                        sync();
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if ((umask >> e) & 1u) {
                                const int j = pos_of(AL[e], s0L);
                                atomicOr(&dec[j >> 5], 1u << (j & 31));
                            }
                    }
                    sync();
                    if (stop) used = it;
                    if constexpr (PO == 0) break;
                    po_end = true;
                }
            }

            // ---------------- R sweep, the other groups in reverse (group 0 again in its own copy)
            auto r_group = [&](int gi, auto firstc, auto singlesc) {
                constexpr bool FIRST = decltype(firstc)::value;
                constexpr bool SINGLES = decltype(singlesc)::value;
                const int4 rc = ctl->rec[gi];
                const int s0 = FIRST ? 0 : (rc.x & 0xff), gl = (rc.x >> 8) & 0xff;
                if (SINGLES && ((rc.x >> 16) & 1)) {
                    if (!FIRST || gtest || PO)
                        single_stage<LOGN, E, T, FK>(true, s0, tid, lowmask, beta, ctl->g.ev_level - 1,
                                                     ctl->g.ev_level + ctl->g.ev_range - 2, ctl->g.pbit[s0], llr_f,
                                                     single_in(gi, s0), single_out(gi, s0), Rp, xh, s_swz, alpha,
                                                     J.check, (PO && FIRST) ? J.post + size_t(f) * 2 * N + N : nullptr);
                } else {
                    const uint32_t colL = uint32_t(rc.y);
                    auto body = [&](auto glc) {
                        constexpr int GL = decltype(glc)::value;
                        int A[E];
                        float lv[GL][E];
                        tm_ld_i<E>(tc(uint32_t(rc.w)), A);
#pragma unroll
                        for (int i = 1; i < GL; ++i) tm_ld<E>(tc(colL + uint32_t((i - 1) * E)), lv[i]);   // L level s0+1+i
                        tm_wait_ld();
                        tm_fence<E>(A);
                        float y[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            y[e] = at(A[e], (GL - 1) * N);                                // R level s0+GL+1
                            lv[0][e] = FIRST ? L1[e] : at(A[e], 0);                       // L level s0+1 (boundary)
                        }
#pragma unroll
                        for (int i = 1; i < GL; ++i) tm_fence<E>(lv[i]);
#pragma unroll
                        for (int i = GL - 1; i >= 0; --i) {
                            if (FIRST && i == 0 && !gtest && !PO) continue;       // stage 0 writes only the G-matrix bits
                            r_layer<E, FK>(y, lv[i], i, alpha, nzero);
                            if (i > 0) {
                                tm_st<E>(tc(colL + uint32_t((GL + i - 2) * E)), y);            // R level s0+1+i
                            } else if (!FIRST) {
#pragma unroll
                                for (int e = 0; e < E; ++e) at(A[e], -N) = y[e];                // R level s0+1
                            } else if (PO) {
                                float* po = J.post + size_t(f) * 2 * N + N;      // R at node level 1
#pragma unroll
                                for (int e = 0; e < E; ++e) po[pos_of(A[e], 0)] = y[e];
                            } else if (!((rc.x >> 24) & 1) && int((signed char)(rc.z & 0xff)) == n - KB) {
                                // the register bits are the top KB position bits (every thread in
                                // class 0), so the lanes are position bits 0..4: per register, one
                                // ballot is a whole word of the hard decisions x_j = [L1 + R1 < 0]
                                // (register e adds reverse_bits(e) << (n - KB) to the position, so
                                // reverse_bits(e) << (n - KB - 5) to lane 0's word)
                                const int w0 = pos_of(A[0], 0) >> 5;
#pragma unroll
                                for (int e = 0; e < E; ++e) {
                                    const unsigned w = __ballot_sync(0xffffffffu, __fadd_rn(L1[e], y[e]) < 0.f);
                                    if (lane == 0) xh[w0 | (reverse_bits<KB>(e) << (n - KB - 5))] = w;
                                }
                            } else {
#pragma unroll
                                for (int e = 0; e < E; ++e) {
                                    const int j = pos_of(A[e], s0);
                                    if (__fadd_rn(L1[e], y[e]) < 0.f) atomicOr(&xh[j >> 5], 1u << (j & 31));
                                }
                            }
                        }
                    };
                    // only group 0 and the last group can have fewer than KB stages: every
                    // other group is a single stage or a full KB (partition rule of
                    // build_partition_warp, checked by pc_partition_selfcheck)
                    if constexpr (FIRST) {
                        if (gl == KB) body(std::integral_constant<int, KB>{});
                        else if (KB > 2 && gl == 2) body(std::integral_constant<int, (KB > 2 ? 2 : 1)>{});
                        else body(std::integral_constant<int, 1>{});
                    } else {
                        body(std::integral_constant<int, KB>{});
                    }
                }
                // group 0 writes shared state (the G-matrix bits) only for the G-matrix test
                if (!FIRST) {
                    if ((rc.x >> 26) & 1) __syncwarp();
                    else sync();
                } else if (gtest) {
                    sync();
                }
            };
            if (!singles) {
                #pragma unroll 1
                for (int gi = ng - 2; gi >= 1; --gi) r_group(gi, std::false_type{}, std::false_type{});
                r_group(0, std::true_type{}, std::false_type{});
            } else {
                #pragma unroll 1
                for (int gi = ng - 2; gi >= 1; --gi) r_group(gi, std::false_type{}, std::true_type{});
                r_group(0, std::true_type{}, std::true_type{});
            }
            if constexpr (PO != 0) {
                if (po_end) {
                    sync();
                    break;
                }
            }

            if (gtest) {
                if (warp == 0) {
                    const bool gok = g_check<LOGN>(dec, xh, lane);
                    if (lane == 0) ctl->g.g_ok = gok ? 1 : 0;
                }
                sync();
                if (ctl->g.g_ok != 0) {
                    used = it;
                    break;
                }
                if (it == max_iters) break;
                // the decision words restart empty for the next test: their writers and readers of
                // this one are past the barriers above; the barrier below orders the clearing before
                // the next writes, and every read of g_ok before its next write
                for (int i = tid; i < NW; i += T) {
                    xh[i] = 0u;
                    dec[i] = 0u;
                }
                sync();
            }

            // a6: switch at iter == N_it,reset
            if (S.mode != 0 && it == next_reset) {
                bool allowed = true;
                if (S.mode == 2 && S.q_max > 0) allowed = kev < S.q_max - 1;
                if (allowed) {
                    // the message reset of Sec. III zeroes R at the interior levels of the subgraph
                    // being left (reverting to the original order) and of the new one.  The event
                    // being left is read before the barrier after which the first warp records the
                    // new one; the other warps reset its subgraph while the first draws the new event.
                    const int pv_lv = ctl->g.ev_level, pv_rg = ctl->g.ev_range;
                    const long long pv_bk = ctl->g.ev_blk;
                    const bool pv_have = ctl->g.have_ev != 0;
                    // zero R at node levels lv+1 .. lv+rg-1 of block bk, threads t0, t0 + nt, ...
                    // (an event over the whole graph, as in FP-BP: every R plane, 16-byte stores)
                    auto reset_block = [&](int lv, int rg, long long bk, int t0, int nt) {
                        if (lv == 1 && rg == n) {
                            for (int i = t0; i < NPL * N / 4; i += nt)
                                reinterpret_cast<float4*>(Rp)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                            return;
                        }
                        const int m = lv + rg - 1;
                        const int span = 1 << m;
                        for (int i = t0; i < (rg - 1) * span; i += nt) {
                            const int lev = lv + 1 + (i >> m);       // node level, 2..n
                            int j = int(bk) + ((i & (span - 1)) << (n - m));
                            int plane = lev - 2;
#ifdef PCBP_CHECKED
                            if (j < 0 || j >= N || plane < 0 || plane >= NPL) {
                                chk_fail(J.check, 4);
                                j = 0;
                                plane = 0;
                            }
#endif
                            Rp[plane * N + sw(j)] = 0.f;
                        }
                    };
                    tm_wait_st();
                    leave_partition();     // interior R of the old partition to the canonical planes
                    sync();
                    // the first warp draws the event (unless drawn ahead) and builds the partition;
                    // in slots of four warps or more the second draws the next switch's event
                    // ahead, and the remaining warps reset the subgraph being left (a one-warp slot
                    // does that after the partition)
                    const uint64_t fid = S.frame_base + uint64_t(f);
                    constexpr int RW = T >= 128 ? 64 : 32;     // the first thread of the resetting warps
                    if (warp == 0) {
                        switch_event_warp<LOGN, KB>(ctl, S, s_swz, fid, kev, lane);
                        if (T == 32 && pv_have) reset_block(pv_lv, pv_rg, pv_bk, tid, T);
                    } else if (T >= 128 && warp == 1) {
                        predraw_event_warp<LOGN, KB>(ctl, S, fid, kev + 1, lane);
                    } else if (pv_have) {
                        reset_block(pv_lv, pv_rg, pv_bk, tid - RW, T - RW);
                    }
                    fresh = false;
                    sync();
                    if (!(pv_have && pv_lv == 1 && pv_rg == n && ctl->g.ev_level == 1 && ctl->g.ev_range == n))
                        reset_block(ctl->g.ev_level, ctl->g.ev_range, ctl->g.ev_blk, tid, T);
                    next_reset = it + ctl->g.next_inc;
                    ++kev;
                    sync();
                    enter_partition(llr_f);   // interior R of the new partition to TMEM, LLRs from global memory
                    sync();
                }
            }
        }

        // a7: outputs
        fetch_next();
        publish_next();
        {
            // the CRC flag: from the residue of the final decisions where the last iteration
            // computed it, else from the decision words
            const unsigned crc_final = ctl->crc_final;
            const bool crc_known = crc_final != 0u;
            if (!crc_known) {
                uint32_t part = 0;
#pragma unroll
                for (int j = tid; j < N; j += T)
                    if ((dec[j >> 5] >> (j & 31)) & 1u) part ^= s_cj[j];
                part = __reduce_xor_sync(0xffffffffu, part);
                if (tid == 0) ctl->g.crc_res = 0;
                sync();
                if (lane == 0 && part) atomicXor(reinterpret_cast<unsigned*>(&ctl->g.crc_res), part);
            }
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
                J.crc_ok[f] = crc_known ? uint8_t(crc_final - 1u) : (ctl->g.crc_res == 0 ? 1 : 0);
                J.iters[f] = used;
            }
            if (!crc_known) sync();     // crc_res is read before a frame start may overwrite the control block
        }
    }
    tm_wait_st();
}

template <int LOGN, int KB, int FK, int WG, int PO>
__global__ void __launch_bounds__(tmem_max_threads<LOGN, KB>(), 1) bp_decode_tmem_kernel(const __grid_constant__ BpParams P)
{
    // a kernel launched after this one may start as soon as SMs free up
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tm;
    load_code_tables3(P.code, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int N = P.code.N, K = P.code.K;
        build_template<LOGN, KB>(reinterpret_cast<Ctl3<LOGN, KB>*>(smem + tmem_table_bytes(N, K)),
                                 smem + tmem_table_bytes(N, K) - kSwzTableBytes);
    }
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
    if (int(threadIdx.x) < P.slots * G3<LOGN, KB>::T) tmem_frames<LOGN, KB, FK, WG, PO>(P.job, P.counter, smem, tm_base);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_base), "n"(kTmemCols) : "memory");
}

}  // namespace pcbp
