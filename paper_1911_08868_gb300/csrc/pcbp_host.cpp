// Host side of libpcbp: code construction, argument validation and the
// tables the kernels read.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "pcbp_internal.h"

namespace pcbp {

static int ilog2_exact(int v)
{
    if (v <= 0 || (v & (v - 1))) return -1;
    int n = 0;
    while ((1 << n) < v) ++n;
    return n;
}

// x^e mod g over GF(2); g has bit r set.
uint32_t poly_xpow_mod(int e, int r, uint64_t g)
{
    uint64_t v = 1;
    for (int i = 0; i < e; ++i) {
        v <<= 1;
        if ((v >> r) & 1ull) v ^= g;
    }
    return (uint32_t)v;
}

// x^e mod g for e = 0 .. count-1.
static std::vector<uint32_t> xpow_table(int count, int r, uint64_t g)
{
    std::vector<uint32_t> pw((size_t)std::max(count, 0));
    uint64_t v = 1;
    for (int e = 0; e < count; ++e) {
        pw[(size_t)e] = (uint32_t)v;
        v <<= 1;
        if ((v >> r) & 1ull) v ^= g;
    }
    return pw;
}

int validate_code(const pc_code* c)
{
    if (!c) return PC_EINVAL;
    int n = ilog2_exact(c->N);
    if (n < kMinLogN || n > kMaxLogN || n != c->n) return PC_EINVAL;
    if (c->K < 1 || c->K > c->N) return PC_EINVAL;
    if (c->crc_len < 0 || c->crc_len > kMaxCrc || c->crc_len >= c->K) return PC_EINVAL;
    if (c->crc_len > 0 && (c->crc_poly >> c->crc_len) != 1ull) return PC_EINVAL;
    int prev = -1, nfree = 0;
    for (int j = 0; j < c->N; ++j)
        if (!((c->frozen_mask[j >> 5] >> (j & 31)) & 1u)) ++nfree;
    if (nfree != c->K) return PC_EINVAL;
    for (int k = 0; k < c->K; ++k) {
        int p = c->info_idx[k];
        if (p <= prev || p >= c->N) return PC_EINVAL;
        if ((c->frozen_mask[p >> 5] >> (p & 31)) & 1u) return PC_EINVAL;
        prev = p;
    }
    return PC_OK;
}

int validate_sched(const pc_code* c, const pc_sched* s)
{
    if (!s) return PC_EINVAL;
    const int n = c->n;
    if (s->mode < 0 || s->mode > 2) return PC_EINVAL;
    if (s->stop_kind < 0 || s->stop_kind > 3) return PC_EINVAL;
    if (s->fkind < 0 || s->fkind > 1) return PC_EUNSUPPORTED;
    if (s->fkind == 0 && !(std::isfinite(s->alpha) && s->alpha > 0.f)) return PC_EINVAL;
    if (s->mode == 1) {
        if (s->T0 < 1 || s->N_min < 1 || s->D < 0) return PC_EINVAL;
        if (s->P_level < 1 || s->P_level > n - 1) return PC_EINVAL;
        if (s->rho_range_fixed > 0) {
            if (s->rho_range_fixed < 2 || s->rho_range_fixed > n) return PC_EINVAL;
        } else if (s->P_range < 2 || s->P_range > n) {
            return PC_EINVAL;
        }
    }
    if (s->mode == 2 && s->it_reset_full < 1) return PC_EINVAL;
    return PC_OK;
}

void build_dev_code(const pc_code* c, DevCode* d)
{
    std::memset(d, 0, sizeof(DevCode));
    d->N = c->N;
    d->n = c->n;
    d->K = c->K;
    d->r = c->crc_len;
    const int nw = std::max(1, c->N / 32);
    for (int w = 0; w < nw; ++w) d->frozen[w] = c->frozen_mask[w];
    if (c->N < 32) d->frozen[0] &= (1u << c->N) - 1u;
    for (int k = 0; k < c->K; ++k) d->info_idx[k] = (int16_t)c->info_idx[k];
    if (c->crc_len > 0) {
        std::vector<uint32_t> pw = xpow_table(c->K, c->crc_len, c->crc_poly);
        for (int k = 0; k < c->K; ++k) {
            uint32_t ck = pw[(size_t)(c->K - 1 - k)];
            int pos = c->info_idx[k];
            for (int i = 0; i < c->crc_len; ++i)
                if ((ck >> i) & 1u) d->crcplane[i][pos >> 5] |= 1u << (pos & 31);
        }
    }
}

void build_dev_sched(const pc_sched* s, DevSched* d)
{
    d->mode = s->mode;
    d->P_range = s->P_range;
    d->P_level = s->P_level;
    d->N_min = s->N_min;
    d->D = s->D;
    d->T0 = s->T0;
    d->rho_fixed = s->rho_range_fixed;
    d->q_max = s->q_max;
    d->it_reset_full = s->it_reset_full;
    d->stop_from = s->stop_from;
    d->stop_kind = s->stop_kind;
    d->fkind = s->fkind;
    d->alpha = s->alpha;
    d->n_explicit = -1;
    d->seed = s->seed;
    d->frame_base = s->frame_base;
}

void build_enc_params(const pc_code* c, EncParams* e)
{
    std::memset(e, 0, sizeof(EncParams));
    e->N = c->N;
    e->n = c->n;
    e->K = c->K;
    e->r = c->crc_len;
    e->Kp = c->K - c->crc_len;
    for (int k = 0; k < c->K; ++k) e->info_idx[k] = (int16_t)c->info_idx[k];
    if (c->crc_len > 0) {
        std::vector<uint32_t> pw = xpow_table(c->K, c->crc_len, c->crc_poly);
        for (int i = 0; i < e->Kp; ++i) e->crc_pay[i] = pw[(size_t)(c->K - 1 - i)];
    }
}

}  // namespace pcbp

using namespace pcbp;

extern "C" int pc_construct(int32_t N, int32_t K, int32_t crc_len, uint64_t crc_poly,
                            double design_ebn0_db, pc_code* out)
{
    if (!out) return PC_EINVAL;
    const int n = ilog2_exact(N);
    if (n < kMinLogN || n > kMaxLogN) return PC_EINVAL;
    if (K < 1 || K > N) return PC_EINVAL;
    if (crc_len < 0 || crc_len > kMaxCrc || crc_len >= K) return PC_EINVAL;
    if (!std::isfinite(design_ebn0_db)) return PC_EINVAL;
    uint64_t g = 0;
    if (crc_len > 0) {
        g = crc_poly | (1ull << crc_len);
        if ((g >> (crc_len + 1)) != 0) return PC_EINVAL;
    }
    // Bhattacharyya bounds of the bit channels (Sec. II-A), log domain.  The
    // first polarisation step from the raw channel sets the most significant
    // index bit, so each step writes minus/plus children next to each other.
    std::vector<double> lz(1, -((double)K / (double)N) * std::pow(10.0, design_ebn0_db / 10.0));
    for (int step = 0; step < n; ++step) {
        std::vector<double> next(lz.size() * 2);
        for (size_t i = 0; i < lz.size(); ++i) {
            // log(2z - z^2) without cancellation on either side of z = 1/2.
            const double omz = -std::expm1(lz[i]);  // 1 - z
            next[2 * i] = lz[i] > -0.69314718055994530942 ? std::log1p(-omz * omz) : lz[i] + std::log1p(omz);
            next[2 * i + 1] = 2.0 * lz[i];  // log(z^2)
        }
        lz.swap(next);
    }
    std::vector<int> order((size_t)N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lz[(size_t)a] > lz[(size_t)b]; });

    std::memset(out, 0, sizeof(pc_code));
    out->N = N;
    out->n = n;
    out->K = K;
    out->crc_len = crc_len;
    out->crc_poly = g;
    for (int i = 0; i < N - K; ++i) {
        int j = order[(size_t)i];
        out->frozen_mask[j >> 5] |= 1u << (j & 31);
    }
    int k = 0;
    for (int j = 0; j < N; ++j)
        if (!((out->frozen_mask[j >> 5] >> (j & 31)) & 1u)) out->info_idx[k++] = j;
    return PC_OK;
}

extern "C" const char* pc_status_string(int status)
{
    switch (status) {
        case PC_OK: return "ok";
        case PC_EINVAL: return "invalid argument";
        case PC_ENOMEM: return "buffer too small";
        case PC_ECUDA: return "CUDA runtime error";
        case PC_ETIMEOUT: return "bounded device wait gave up";
        case PC_EUNSUPPORTED: return "unsupported size or mode";
        default: return "unknown status";
    }
}
