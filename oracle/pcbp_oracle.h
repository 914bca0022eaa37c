/*
 * Oracle for partially permuted multi-trellis BP decoding of polar codes
 * (arXiv 1911.08868).  TEST INFRASTRUCTURE ONLY.
 *
 * This is a plain, slow CPU restatement of what the paper computes, written
 * to check the CUDA decoder against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA path under
 * paper_1911_08868_gb300/.
 *
 * Conventions (each is the paper's, or a stated reading of it):
 *   - N = 2^n, generator G_N = F^{(x)n}, F = [[1,0],[1,1]], x = u G_N (Eq. 1);
 *     in index form x_i = XOR over j that are bitwise supersets of i of u_j.
 *   - Node levels 1 (channel side) .. n+1 (u side) (Sec. II-B).  Stage l
 *     (1..n) joins levels l and l+1 and pairs index j with j ^ (1 << b), where
 *     b = stage_bit[l-1][j]; the smaller index is the "top" port.  In the
 *     original graph b = n-l: the stage next to the channel pairs the two
 *     halves of x, the stage next to u pairs neighbouring u indices (Arikan's
 *     factor graph of x = u F^{(x)n}).  The stages 1..m of that graph split
 *     the indices into N / 2^m subgraphs sharing their n-m low bits, which is
 *     the paper's subgraph count for m = rho_level + rho_range - 1 (Sec. III).
 *   - Messages are stored as planes L[(level-1)*N + j], R[(level-1)*N + j].
 *   - Bits are one per byte (0/1).
 *
 * Parity status: every function here is pinned by a "not gpu" test against
 * brute force, closed forms or the paper's stated values, except the
 * trajectory of BP on noisy frames, which the paper prints no numbers for
 * (parity unpinned beyond its invariants: noiseless recovery, valid permuted
 * graphs, FP32/FP64 agreement, first-sweep closed forms).
 */
#ifndef PCBP_ORACLE_H
#define PCBP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One partial-permutation event (Sec. III, Algorithm 1): inside the
 * subgraph `block` (indices j with j mod 2^(n-m) == block, m = level+range-1)
 * stage level+i takes the bit that stage level+order[i] has in the original
 * graph.  order is a permutation of 0..range-1. */
typedef struct {
    int32_t level;
    int32_t range;
    int64_t block;
    int32_t order[16];
} orc_event;

/* Decoder schedule.  mode: 0 plain BP, 1 PP-BP (Algorithm 1), 2 FP-BP.
 * D == 0 means D = infinity (next switch after exactly N_min iterations).
 * stop_kind: bit 0 = CRC residue, bit 1 = G-matrix test.  fkind: 0 scaled
 * min-sum (alpha), 1 exact box-plus. */
typedef struct {
    int32_t mode, P_range, P_level, N_min, D, T0, rho_range_fixed;
    int32_t q_max, it_reset_full, stop_from, stop_kind, fkind;
    double alpha;
    uint64_t seed;
    uint64_t frame_base;
} orc_sched;

/* --- code construction (Sec. II-A: Bhattacharyya bounds at design Eb/N0) */
int orc_construct(int n, int K, double design_ebn0_db, double* lz_out, uint8_t* frozen_out);

/* --- CRC (Sec. IV): plain polynomial long division over GF(2) */
uint64_t orc_crc_residue(const uint8_t* a, int len, int r, uint64_t poly);
uint64_t orc_crc_compute(const uint8_t* payload, int len, int r, uint64_t poly);

/* --- encoding (Eq. 1) */
void orc_encode(int n, const uint8_t* u, uint8_t* x);
/* u from frozen mask + K info bits (info positions ascending) */
void orc_place_info(int n, const uint8_t* frozen, const uint8_t* info, uint8_t* u);
/* propagate hard bits from level n+1 to level 1 through an explicit graph;
 * returns -1 if the stage table is not a valid pairing */
int orc_graph_encode(int n, const int8_t* stage_bit, const uint8_t* u, uint8_t* x);

/* --- factor graph and permutation events (Sec. III, Eq. 2) */
void orc_graph_from_event(int n, const orc_event* ev, int8_t* stage_bit);
uint64_t orc_splitmix(uint64_t state);
uint64_t orc_hash(uint64_t seed, uint64_t frame, uint64_t k, uint64_t d);
int orc_draw_event(int n, const orc_sched* s, uint64_t frame_id, int k, orc_event* ev);
int64_t orc_n_zero(const orc_event* ev);
int orc_reset_increment(const orc_sched* s, const orc_event* ev);

/* --- BP (Sec. II-B and Algorithm 1), in FP64 and FP32 */
double orc_f_f64(double a, double b, double alpha, int fkind);
float orc_f_f32(float a, float b, float alpha, int fkind);
void orc_bp_iteration_f64(int n, const int8_t* stage_bit, double* L, double* R, double alpha, int fkind);
void orc_bp_iteration_f32(int n, const int8_t* stage_bit, float* L, float* R, float alpha, int fkind);
int orc_decode_f64(int n, const uint8_t* frozen, int r, uint64_t poly, const double* llr,
                   const orc_sched* s, int max_iters, uint64_t frame_id,
                   const orc_event* ev_list, int n_ev,
                   uint8_t* uhat, int32_t* iters, int32_t* crc_ok, double* dump);
int orc_decode_f32(int n, const uint8_t* frozen, int r, uint64_t poly, const float* llr,
                   const orc_sched* s, int max_iters, uint64_t frame_id,
                   const orc_event* ev_list, int n_ev,
                   uint8_t* uhat, int32_t* iters, int32_t* crc_ok, float* dump);
/* frame loop over B frames (frame id = s->frame_base + b), OpenMP threads */
int orc_decode_batch_f32(int n, const uint8_t* frozen, int r, uint64_t poly, const float* llr,
                         const orc_sched* s, int max_iters, int64_t B, int nthreads,
                         uint8_t* uhat, int32_t* iters, int32_t* crc_ok);
int orc_decode_batch_f64(int n, const uint8_t* frozen, int r, uint64_t poly, const double* llr,
                         const orc_sched* s, int max_iters, int64_t B, int nthreads,
                         uint8_t* uhat, int32_t* iters, int32_t* crc_ok);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
