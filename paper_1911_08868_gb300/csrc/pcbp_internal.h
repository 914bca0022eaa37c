// Internal structures shared by the host code and the CUDA kernels of libpcbp.
// Plain C++ (no CUDA types) so that host-only translation units can use them.
#pragma once

#include <cstddef>
#include <cstdint>

#include "pcbp.h"

namespace pcbp {

constexpr int kMinLogN = 3;
constexpr int kMaxLogN = 11;
constexpr int kMaxN = 1 << kMaxLogN;
constexpr int kMaxWords = kMaxN / 32;
constexpr int kMaxCrc = 32;

// Code tables as the decoder reads them (passed by value as a kernel
// parameter, copied to shared memory once per CTA).
//   frozen[w]: bit j of word w = position 32w+j frozen.
//   crcplane[i][w]: bit j = bit i of x^(K-1-k) mod g, where k is the
//     information rank of position 32w+j (0 for frozen positions), so that
//     the CRC residue of the decided information vector is, bit by bit, the
//     parity of (decisions & crcplane[i]) over all words.
//   info_idx[k]: k-th information position (ascending).
struct DevCode {
    int32_t N, n, K, r;
    uint32_t frozen[kMaxWords];
    uint32_t crcplane[kMaxCrc][kMaxWords];
    int16_t info_idx[kMaxN];
};

struct DevSched {
    int32_t mode, P_range, P_level, N_min, D, T0, rho_fixed;
    int32_t q_max, it_reset_full, stop_from, stop_kind, fkind;
    float alpha;
    int32_t n_explicit;  // >= 0: explicit event list of that length; -1: counter generator
    uint64_t seed, frame_base;
};

// One batch of frames of one code: the stage-grouped decoder body's inputs
// and outputs (the frame counter is passed separately).
struct FrameJob {
    DevSched S;
    const float* llr;
    uint32_t* bits;
    int32_t* iters;
    uint8_t* crc_ok;
    int64_t B;
    int32_t max_iters;
    int32_t K, r;
    unsigned* check;   // builds with PCBP_CHECKED: bit c set when an access of class c was out of range (nullable)
    float* post;       // posterior-output kernels only: [B][2][N], L at node level n+1, R at node level 1
    float neg_zero;    // -0.0f: the addend of the packed scalings, unknown to the compiler
};

struct DevEvent {
    int32_t level, range;
    int64_t block;
    int8_t order[16];
};

struct BpParams {
    DevCode code;
    DevSched sched;
    const float* llr;
    uint32_t* bits;
    int32_t* iters;
    uint8_t* crc_ok;
    unsigned long long* counter;
    float* dump;
    int64_t B;
    int32_t max_iters;
    int32_t slots;
    DevEvent events[PC_MAX_EVENTS];
    FrameJob job;   // the same batch, as the stage-grouped kernel reads it
};

// Encoder tables: crc_pay[i] = x^(r + Kp - 1 - i) mod g for payload bit i.
struct EncParams {
    int32_t N, n, K, r, Kp;
    uint32_t crc_pay[kMaxN];
    int16_t info_idx[kMaxN];
    const uint8_t* payload;
    uint8_t* x;
    int64_t B;
};

// Host helpers (pcbp_host.cpp).
int validate_code(const pc_code* c);
int validate_sched(const pc_code* c, const pc_sched* s);
void build_dev_code(const pc_code* c, DevCode* d);
void build_dev_sched(const pc_sched* s, DevSched* d);
void build_enc_params(const pc_code* c, EncParams* e);
uint32_t poly_xpow_mod(int e, int r, uint64_t g);

}  // namespace pcbp
