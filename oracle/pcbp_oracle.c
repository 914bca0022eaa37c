/*
 * Oracle for partially permuted multi-trellis BP decoding of polar codes
 * (arXiv 1911.08868).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the
 * smoke check and the benchmark's CPU-baseline leg, never by the product
 * path.  Plain C, compiled with -ffp-contract=off so that every FP32 and FP64
 * operation is rounded exactly where it is written.
 *
 * The typed BP routines live in bp_real.inc, included twice (double, float).
 */
#define _DEFAULT_SOURCE
#include "pcbp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Code construction, Sec. II-A: Arikan's Bhattacharyya bounds of the bit
 * channels at design Eb/N0 (0 dB in the paper).  For BPSK over AWGN the
 * channel parameter is z0 = exp(-R * Eb/N0) with R = K/N (the paper counts
 * the CRC bits in the rate, Sec. IV).  One polarisation step maps z to
 * 2z - z^2 (the "minus" channel) and z^2 (the "plus" channel).  For
 * x = u F^{(x)n} in natural order the first step taken from the raw channel
 * decides the most significant bit of the index, so the recursion
 * interleaves: new[2i] = minus(old[i]), new[2i+1] = plus(old[i]).
 * Worked in log z, FP64.  log(2z - z^2) is evaluated as log1p(-(1-z)^2)
 * when z > 1/2 and as log z + log1p(1-z) otherwise, with 1 - z = -expm1(log z),
 * so that neither branch cancels.  The N-K channels with the largest z are
 * frozen; equal z freezes the lower index first. */
typedef struct { double lz; int idx; } lz_item;

static double log_minus(double lz)
{
    double one_minus_z = -expm1(lz);
    if (lz > -M_LN2) return log1p(-one_minus_z * one_minus_z);
    return lz + log1p(one_minus_z);
}

static int cmp_lz_desc(const void* pa, const void* pb)
{
    const lz_item* a = (const lz_item*)pa;
    const lz_item* b = (const lz_item*)pb;
    if (a->lz > b->lz) return -1;
    if (a->lz < b->lz) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

int orc_construct(int n, int K, double design_ebn0_db, double* lz_out, uint8_t* frozen_out)
{
    if (n < 0 || n > 20) return -1;
    int N = 1 << n;
    if (K < 0 || K > N) return -1;
    double* lz = (double*)malloc(sizeof(double) * N);
    double* nx = (double*)malloc(sizeof(double) * N);
    lz[0] = -((double)K / (double)N) * pow(10.0, design_ebn0_db / 10.0);
    for (int step = 1; step <= n; ++step) {
        int size = 1 << (step - 1);
        for (int i = 0; i < size; ++i) {
            nx[2 * i] = log_minus(lz[i]);
            nx[2 * i + 1] = 2.0 * lz[i];
        }
        double* t = lz; lz = nx; nx = t;
    }
    lz_item* items = (lz_item*)malloc(sizeof(lz_item) * N);
    for (int i = 0; i < N; ++i) { items[i].lz = lz[i]; items[i].idx = i; }
    qsort(items, N, sizeof(lz_item), cmp_lz_desc);
    for (int i = 0; i < N; ++i) frozen_out[i] = 0;
    for (int i = 0; i < N - K; ++i) frozen_out[items[i].idx] = 1;
    if (lz_out) memcpy(lz_out, lz, sizeof(double) * N);
    free(items); free(lz); free(nx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* CRC, Sec. IV ("24-bit CRC").  Polynomial long division over GF(2), most
 * significant bit first, zero initial remainder, no reflection, no final
 * XOR.  g(x) = x^r + (low terms of poly); poly may be given with or without
 * its x^r term.  residue(a) = a(x) mod g(x) with a[0] the highest power. */
uint64_t orc_crc_residue(const uint8_t* a, int len, int r, uint64_t poly)
{
    if (r <= 0) return 0;
    uint64_t g = poly | (1ull << r);
    uint64_t rem = 0;
    for (int i = 0; i < len; ++i) {
        rem = (rem << 1) | (uint64_t)(a[i] & 1);
        if ((rem >> r) & 1ull) rem ^= g;
    }
    return rem;
}

/* CRC bits of a payload: residue of payload(x) * x^r. */
uint64_t orc_crc_compute(const uint8_t* payload, int len, int r, uint64_t poly)
{
    if (r <= 0) return 0;
    uint8_t* buf = (uint8_t*)calloc((size_t)len + (size_t)r, 1);
    memcpy(buf, payload, (size_t)len);
    uint64_t c = orc_crc_residue(buf, len + r, r, poly);
    free(buf);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Encoding, Eq. 1: x = u G_N.  G_N = F^{(x)n} factors into n commuting
 * butterfly layers; the layer on bit p replaces x[i] by x[i] ^ x[i | 2^p]
 * for every i whose bit p is clear. */
void orc_encode(int n, const uint8_t* u, uint8_t* x)
{
    int N = 1 << n;
    for (int i = 0; i < N; ++i) x[i] = u[i] & 1;
    for (int p = 0; p < n; ++p)
        for (int i = 0; i < N; ++i)
            if (!((i >> p) & 1)) x[i] ^= x[i | (1 << p)];
}

/* Frozen positions carry 0 (Sec. II-B); info bits fill the remaining
 * positions in ascending index order. */
void orc_place_info(int n, const uint8_t* frozen, const uint8_t* info, uint8_t* u)
{
    int N = 1 << n, k = 0;
    for (int j = 0; j < N; ++j) u[j] = frozen[j] ? 0 : (info[k++] & 1);
}

/* Hard bits through an explicit factor graph, from level n+1 (u) down to
 * level 1 (x): at stage l, top = top ^ bottom, bottom = bottom. */
int orc_graph_encode(int n, const int8_t* stage_bit, const uint8_t* u, uint8_t* x)
{
    int N = 1 << n;
    for (int j = 0; j < N; ++j) x[j] = u[j] & 1;
    for (int l = n; l >= 1; --l) {
        const int8_t* sb = stage_bit + (size_t)(l - 1) * N;
        for (int j = 0; j < N; ++j) {
            int p = sb[j];
            if (p < 0 || p >= n) return -1;
            int partner = j ^ (1 << p);
            if (sb[partner] != p) return -1;
            if (!((j >> p) & 1)) x[j] ^= x[partner];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Factor graph of Sec. II-B/III.  Stage l joins node levels l and l+1 and,
 * in the original graph, pairs index j with j ^ 2^(n-l): the stage next to
 * the channel combines the two halves of x and the stage next to u pairs
 * neighbouring u indices (Arikan's graph of x = u F^{(x)n}).  The stages
 * 1..m, m = level + range - 1, split the indices into N / 2^m connected
 * subgraphs of 2^m indices that share their n - m low bits; `block` is that
 * low-bit value.  An event gives stage level+i of its subgraph the bit that
 * stage level+order[i] has in the original graph.  Every event is applied to
 * the original graph (at most one permuted subgraph at a time). */
void orc_graph_from_event(int n, const orc_event* ev, int8_t* stage_bit)
{
    int N = 1 << n;
    for (int l = 1; l <= n; ++l)
        for (int j = 0; j < N; ++j) stage_bit[(size_t)(l - 1) * N + j] = (int8_t)(n - l);
    if (!ev) return;
    int m = ev->level + ev->range - 1;
    int low = n - m;
    for (int j = 0; j < N; ++j) {
        if ((int64_t)(j & ((1 << low) - 1)) != ev->block) continue;
        for (int i = 0; i < ev->range; ++i)
            stage_bit[(size_t)(ev->level - 1 + i) * N + j] = (int8_t)(n - (ev->level + ev->order[i]));
    }
}

/* Counter-based random draws: SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014; constants of the
 * public-domain reference by S. Vigna).  sm(x) is the generator's output for
 * state x, i.e. the finaliser applied to x + 0x9E3779B97F4A7C15.  A draw is
 * keyed by (seed, frame, event index k, draw index d) as
 * sm(sm(sm(sm(seed) ^ frame) ^ k) ^ d). */
static uint64_t sm64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix(uint64_t state) { return sm64(state); }

uint64_t orc_hash(uint64_t seed, uint64_t frame, uint64_t k, uint64_t d)
{
    return sm64(sm64(sm64(sm64(seed) ^ frame) ^ k) ^ d);
}

/* The random choices of a switch (Sec. III, Algorithm 1):
 *   rho_range uniform on {2..P_range} (or fixed),
 *   rho_level = min(x, n - rho_range + 1), x uniform on {1..P_level},
 *   one of the N / 2^(rho_level+rho_range-1) subgraphs uniformly,
 *   a uniform non-identity order of its rho_range stages (Fisher-Yates,
 *   redrawn while it is the identity; a rotation after 8 identity draws).
 * FP-BP (Sec. II-D) draws a full order: level 1, range n, the one block.
 * Range reduction is x % m. */
int orc_draw_event(int n, const orc_sched* s, uint64_t frame_id, int k, orc_event* ev)
{
    uint64_t seed = s->seed;
    int range, level;
    int64_t block;
    if (s->mode == 2) {
        range = n; level = 1; block = 0;
    } else {
        if (s->rho_range_fixed > 0) {
            range = s->rho_range_fixed;
        } else {
            if (s->P_range < 2 || s->P_range > n) return -1;
            range = 2 + (int)(orc_hash(seed, frame_id, (uint64_t)k, 0) % (uint64_t)(s->P_range - 1));
        }
        if (range < 2 || range > n) return -1;
        if (s->P_level < 1) return -1;
        int x = 1 + (int)(orc_hash(seed, frame_id, (uint64_t)k, 1) % (uint64_t)s->P_level);
        level = x < (n - range + 1) ? x : (n - range + 1);
        int m = level + range - 1;
        uint64_t nblocks = 1ull << (n - m);
        block = (int64_t)(orc_hash(seed, frame_id, (uint64_t)k, 2) % nblocks);
    }
    ev->level = level; ev->range = range; ev->block = block;
    for (int i = 0; i < 16; ++i) ev->order[i] = i;
    for (int attempt = 0; attempt < 8; ++attempt) {
        for (int i = 0; i < range; ++i) ev->order[i] = i;
        for (int i = range - 1; i >= 1; --i) {
            uint64_t d = 3 + 16 * (uint64_t)attempt + (uint64_t)(range - 1 - i);
            int j = (int)(orc_hash(seed, frame_id, (uint64_t)k, d) % (uint64_t)(i + 1));
            int t = ev->order[i]; ev->order[i] = ev->order[j]; ev->order[j] = t;
        }
        int ident = 1;
        for (int i = 0; i < range; ++i) if (ev->order[i] != i) ident = 0;
        if (!ident) return 0;
    }
    for (int i = 0; i < range; ++i) ev->order[i] = (i + 1) % range;
    return 0;
}

/* Sec. III: N_zero = 2^(rho_level + rho_range - 1) * (rho_range - 1). */
int64_t orc_n_zero(const orc_event* ev)
{
    return ((int64_t)1 << (ev->level + ev->range - 1)) * (int64_t)(ev->range - 1);
}

/* Eq. 2: N_it,reset increment = max(N_min, floor(N_zero / D)); D = 0 stands
 * for D = infinity.  FP-BP switches every it_reset_full iterations. */
int orc_reset_increment(const orc_sched* s, const orc_event* ev)
{
    if (s->mode == 2) return s->it_reset_full;
    int64_t q = s->D > 0 ? orc_n_zero(ev) / (int64_t)s->D : 0;
    return (int)(q > s->N_min ? q : s->N_min);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
#define REAL double
#define SFX(name) name##_f64
#define RFABS fabs
#define RLOG1P log1p
#define REXP exp
#include "bp_real.inc"
#undef REAL
#undef SFX
#undef RFABS
#undef RLOG1P
#undef REXP

#define REAL float
#define SFX(name) name##_f32
#define RFABS fabsf
#define RLOG1P log1pf
#define REXP expf
#include "bp_real.inc"
#undef REAL
#undef SFX
#undef RFABS
#undef RLOG1P
#undef REXP
