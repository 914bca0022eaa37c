/*
 * pcbp — GB300 (sm_103a) decoder library for polar codes with partially
 * permuted multi-trellis belief propagation (PP-BP), after Ranasinghe,
 * Rajatheva and Latva-aho, "Partially Permuted Multi-Trellis Belief
 * Propagation for Polar Codes" (arXiv 1911.08868).
 *
 * C ABI.  Conventions shared by every call:
 *   - Every call returns an int status: PC_OK (0) or a negative PC_E* code.
 *     Argument errors are detected on the host before anything is enqueued.
 *     PC_ECUDA means a CUDA runtime call failed (launch error, bad device
 *     pointer detected by the runtime); the stream may hold partial work.
 *   - All buffers are owned by the caller.  "d_" pointers are device
 *     pointers, "h_" pointers and struct pointers are host pointers.  Device
 *     calls never allocate device memory: scratch space is caller-provided
 *     and sized by the matching *_workspace_size call.
 *   - Device calls are asynchronous on the caller's stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream); outputs are valid
 *     once the stream has reached that point.  Calls that share a workspace
 *     must be ordered on one stream.
 *   - pc_code is an immutable value: it may be shared across streams and
 *     threads.
 *   - Bits are one per byte (0/1) on input; decoded information bits are
 *     packed 32 per uint32_t word, bit k of the information vector in word
 *     k/32 at bit position k%32.
 *
 * Supported sizes: N = 2^n with 3 <= n <= 11 (8 .. 2048), 1 <= K <= N,
 * CRC length 0 .. 32 (less than K).
 */
#ifndef PCBP_H
#define PCBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PC_OK 0
#define PC_EINVAL (-1)      /* an argument is out of range or a pointer is NULL */
#define PC_ENOMEM (-2)      /* a caller buffer is too small */
#define PC_ECUDA (-3)       /* a CUDA runtime call failed */
#define PC_ETIMEOUT (-4)    /* a bounded device wait gave up */
#define PC_EUNSUPPORTED (-5)/* size or mode not built into this library */

#define PC_NMAX 2048
#define PC_MAX_EVENTS 32

/* A polar code (Sec. II-A): length N = 2^n, K information positions
 * (including the crc_len CRC bits), frozen set, CRC generator.
 *   frozen_mask: bit j%32 of word j/32 is 1 when position j is frozen.
 *   info_idx[0..K-1]: the information positions in ascending order; the
 *     information vector a = payload (K - crc_len bits) || CRC (crc_len bits)
 *     goes to these positions in order.
 *   crc_poly: generator including its x^crc_len term (bit crc_len set). */
typedef struct {
    int32_t N, n, K, crc_len;
    uint64_t crc_poly;
    uint32_t frozen_mask[PC_NMAX / 32];
    int32_t info_idx[PC_NMAX];
} pc_code;

/* Decoder schedule (Algorithm 1 and Table I).
 *   mode: 0 plain BP (one trellis), 1 PP-BP (partial permutations),
 *         2 FP-BP (full permutations, Sec. II-D).
 *   PP-BP: rho_range is uniform on {2..P_range} unless rho_range_fixed > 0;
 *     rho_level = min(x, n - rho_range + 1) with x uniform on {1..P_level};
 *     first switch after T0 iterations, then after max(N_min, floor(N_zero/D))
 *     (Eq. 2), D == 0 meaning D = infinity.
 *   FP-BP: a new full stage order every it_reset_full iterations, at most
 *     q_max - 1 switches (q_max <= 0: unlimited).
 *   stop_from: first iteration at which the stop test is applied (Sec. IV
 *     skips it in an unstated number of first iterations); stop_kind bit 0 = CRC residue zero,
 *     bit 1 = G-matrix test (u G_N equals the hard decisions of L1 + R1);
 *     0 = never stop early.
 *   fkind: 0 scaled min-sum f = alpha * sign * sign * min (alpha = 1 is the
 *     paper's unscaled min-sum), 1 exact box-plus (alpha unused).
 *   seed, frame_base: frame b of a call draws its events from the counter
 *     generator keyed by (seed, frame_base + b, event index, draw index). */
typedef struct {
    int32_t mode, P_range, P_level, N_min, D, T0, rho_range_fixed;
    int32_t q_max, it_reset_full, stop_from, stop_kind, fkind;
    float alpha;
    int32_t reserved;
    uint64_t seed;
    uint64_t frame_base;
} pc_sched;

/* One explicit permutation event (Sec. III, Algorithm 1).  The
 * original factor graph is Arikan's graph of x = u F^{(x)n}: stage l (1..n,
 * counted from the channel) pairs positions that differ in bit n-l.  With
 * m = level+range-1, stages 1..m split the positions into N/2^m subgraphs of
 * positions that share their n-m low bits; `block` (0 .. N/2^m - 1) is that
 * low-bit value.  Inside the subgraph, stage level+i takes the bit that stage
 * level+order[i] has in the original graph; order[0..range-1] is a
 * permutation of 0..range-1. */
typedef struct {
    int32_t level, range;
    int64_t block;
    int32_t order[16];
} pc_event;

/* Code construction by Bhattacharyya bounds at design Eb/N0 (Sec. II-A):
 * z0 = exp(-(K/N) * 10^(design_ebn0_db/10)), worked in FP64 log domain; the
 * N-K positions with the largest bound are frozen (ties freeze the lower
 * index).  crc_poly may omit its x^crc_len term.  Host only. */
int pc_construct(int32_t N, int32_t K, int32_t crc_len, uint64_t crc_poly,
                 double design_ebn0_db, pc_code* out);

/* Encoder (Eq. 1): for each of B frames, a = payload || CRC(payload)
 * (MSB-first polynomial division, zero initial value, no reflection, no
 * final XOR), u = a on the information positions and 0 elsewhere,
 * x = u G_N.  d_payload: B x (K - crc_len) bytes; d_x: B x N bytes. */
int pc_encode(const pc_code* code, const uint8_t* d_payload, uint8_t* d_x,
              int64_t B, void* stream);

/* Bytes of device workspace bp_decode / bp_decode_trace need for B frames
 * (a frame counter; 256-byte aligned start required). */
int bp_decode_workspace_size(const pc_code* code, int64_t B, size_t* bytes);

/* PP-BP decoder, Algorithm 1, for B frames.
 *   d_llr: B x N float channel LLRs (positive favours bit 0), 16-byte
 *     aligned.  Row b is frame b.
 *   max_iters: N_it,max >= 0.
 *   d_bits: B x ceil(K/32) words, the decided information vector (payload
 *     then CRC bits) packed as described above.
 *   d_iters: B int32, the iteration at which the stop test passed, else
 *     max_iters.
 *   d_crc_ok: B bytes, 1 when the decided information vector has zero CRC
 *     residue (always 1 when crc_len == 0).
 *   d_workspace: bp_decode_workspace_size bytes, overwritten.
 * Messages are FP32; every FP32 operation is rounded as written (no fused
 * multiply-add), so results are reproducible bit for bit.  N >= 128 runs the
 * kernel that keeps each stage group's interior messages in tensor memory
 * (groups of 2 stages up to N = 256, of 3 from 512), smaller N the shared-memory
 * stage-grouped kernel (the environment variable
 * PCBP_DECODER=grouped selects the latter for every N; the outputs are the
 * same).  The frames of a call share a persistent grid: each CTA holds one
 * frame per slot and fetches the next frame index from d_workspace. */
int bp_decode(const pc_code* code, const float* d_llr, const pc_sched* sched,
              int32_t max_iters, int64_t B, uint32_t* d_bits, int32_t* d_iters,
              uint8_t* d_crc_ok, void* d_workspace, void* stream);

/* bp_decode (Algorithm 1) on buffers that stay in host memory: the decoder
 * reads each frame's LLRs once and writes its results in place across the
 * host-device link (NVLink-C2C on Grace-Blackwell systems), with no staging
 * copies.  The paper has no counterpart; the operation is bp_decode's.
 *   h_llr, h_bits, h_iters, h_crc_ok: laid out as d_llr, d_bits, d_iters,
 *     d_crc_ok of bp_decode (h_llr 16-byte aligned), each in page-locked
 *     host memory mapped into the current device's address space
 *     (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with
 *     cudaHostRegisterMapped), or in device or managed memory of the current
 *     device.  The first and the last byte of every buffer must be accessible
 *     from the device at addresses the buffer's length apart; otherwise
 *     (pageable memory, a buffer running past its allocation) the call
 *     returns PC_EINVAL before anything is enqueued.  Caller-owned.
 *   d_workspace: device memory, bp_decode_workspace_size bytes, overwritten.
 * Asynchronous on stream: synchronise it before reading the results on the
 * host.  The outputs equal bp_decode's bit for bit. */
int bp_decode_host(const pc_code* code, const float* h_llr, const pc_sched* sched,
                   int32_t max_iters, int64_t B, uint32_t* h_bits, int32_t* h_iters,
                   uint8_t* h_crc_ok, void* d_workspace, void* stream);

/* bp_decode with every message plane recorded, for verification.
 *   h_events: when not NULL, the k-th switch applies h_events[k] (for every
 *     frame) and no switch follows the n_events-th; n_events <=
 *     PC_MAX_EVENTS.  When NULL, events come from the counter generator as
 *     in bp_decode.
 *   d_dump: B x max_iters x 2 x (n+1) x N floats; after iteration i the
 *     block [b][i-1] holds the L planes of levels 1..n+1 followed by the R
 *     planes of levels 1..n+1 (after the switch of that iteration, if any).
 *     Blocks past a frame's last iteration are left untouched.
 * The final iteration is always completed in full (bp_decode may skip the
 * last R sweep when only the CRC test stops it; outputs are the same). */
int bp_decode_trace(const pc_code* code, const float* d_llr, const pc_sched* sched,
                    int32_t max_iters, int64_t B, const pc_event* h_events,
                    int32_t n_events, float* d_dump, uint32_t* d_bits,
                    int32_t* d_iters, uint8_t* d_crc_ok, void* d_workspace,
                    void* stream);

/* bp_decode (Algorithm 1) through the same production kernel, which also
 * records the messages at both ends of the factor graph after each frame's
 * last iteration, for verification of the message arithmetic (Sec. II-B)
 * where the outputs alone would hide it (the exact box-plus f).
 *   d_post: B x 2 x N floats, device memory, 4-byte aligned; block [b][0]
 *     receives L at node level n+1 (the u side), block [b][1] R at node
 *     level 1 (the channel side), both after frame b's last iteration, whose
 *     R sweep is always completed.  Left untouched when max_iters is 0.
 *   Other arguments and outputs as bp_decode (the outputs are equal).
 * Returns PC_EUNSUPPORTED for N < 128 (those lengths run another kernel) or
 * with the G-matrix stop test (stop_kind & 2). */
int bp_decode_posterior(const pc_code* code, const float* d_llr, const pc_sched* sched,
                        int32_t max_iters, int64_t B, uint32_t* d_bits, int32_t* d_iters,
                        uint8_t* d_crc_ok, float* d_post, void* d_workspace, void* stream);

/* The processing-element function f of Sec. II-B, elementwise, exactly as
 * the decoder kernels evaluate it, for verification of its arithmetic:
 * d_out[i] = f(d_a[i], d_b[i]) with fkind 0 (scaled min-sum, alpha) or 1
 * (exact box-plus, alpha unused).  Device arrays of count floats, 4-byte
 * aligned; asynchronous on stream. */
int pc_f_eval(const float* d_a, const float* d_b, float* d_out, int64_t count,
              int32_t fkind, float alpha, void* stream);

/* ---- Weighted BP (a differentiable variant; the paper has no counterpart) -
 * Unrolled round-trip BP on the original factor graph (Sec. II-B) with a
 * learnable scale per f evaluation in place of the fixed min-sum scale:
 * w[t][s][q][k] for iteration t < T, stage s < n (counted from the channel),
 * processing element q < N/2 of that stage (q with a zero inserted at bit
 * n-1-s is its top index) and k = 0 L_out1, 1 L_out2, 2 R_out1, 3 R_out2:
 *   f_w(a, b) = w * sign(a) sign(b) * min(|a|, |b|).
 * Frozen priors are +inf.  logits[b][k] = L at level n+1 of the k-th
 * information position after T iterations (no CRC, no stop test, no
 * permutation).  Gradients: the minimum takes the gradient (the first
 * operand on ties), an infinite message receives none.
 * FP32 entry points and _f64 twins (for gradient checks).  d_w must be
 * aligned to two weights (8 bytes for FP32, 16 for FP64): the kernels read a
 * processing element's (k, k+1) pair in one load; PC_EINVAL otherwise. */

/* Number of weights, T * n * (N/2) * 4. */
int wbp_weights_count(const pc_code* code, int32_t T, size_t* count);
/* Number of checkpoint values, T * B * (n-1) * N (R of levels 2..n after
 * t = 0..T-1 iterations; the values of one level are stored in an internal
 * position order, so the buffer is meant only for wbp_backward of the same
 * precision and code). */
int wbp_ckpt_count(const pc_code* code, int32_t T, int64_t B, size_t* count);
/* Device workspace bytes of wbp_forward / wbp_backward (real_bytes 4 or 8). */
int wbp_workspace_size(const pc_code* code, int32_t T, int64_t B, int32_t real_bytes, size_t* bytes);
/* d_llr [B][N], d_w (wbp_weights_count), d_logits [B][K]; d_ckpt (nullable,
 * 4-byte aligned) receives the checkpoints wbp_backward needs. */
int wbp_forward(const pc_code* code, const float* d_llr, const float* d_w, int32_t T, int64_t B,
                float* d_logits, float* d_ckpt, void* d_workspace, void* stream);
/* Given d_glogits = dLoss/dlogits [B][K]: d_gw += dLoss/dw (caller zeroes it
 * for a fresh gradient); d_gllr (nullable) = dLoss/dllr [B][N].  Runs one
 * launch per iteration, in reverse, each recomputing its iteration from the
 * checkpoint. */
int wbp_backward(const pc_code* code, const float* d_llr, const float* d_w, int32_t T, int64_t B,
                 const float* d_ckpt, const float* d_glogits, float* d_gw, float* d_gllr,
                 void* d_workspace, void* stream);
int wbp_forward_f64(const pc_code* code, const double* d_llr, const double* d_w, int32_t T, int64_t B,
                    double* d_logits, double* d_ckpt, void* d_workspace, void* stream);
int wbp_backward_f64(const pc_code* code, const double* d_llr, const double* d_w, int32_t T, int64_t B,
                     const double* d_ckpt, const double* d_glogits, double* d_gw, double* d_gllr,
                     void* d_workspace, void* stream);

/* Self-check of the decoder's internals (no counterpart in the paper): for
 * every event shape of N = 128..2048 (three orders and blocks each), the
 * partition the N >= 128 decoder builds with one warp at a switch must equal
 * the one its single-threaded builder makes, and every partition (the
 * no-event one included) must have at least two stage groups, every group but
 * the first and the last being a single stage or a full group.  Writes
 * d_result[0] = partitions checked, d_result[1] = event shapes whose two
 * builds differ, d_result[2] = partitions of another shape (device int32[3],
 * 4-byte aligned), asynchronously on the stream. */
int pc_partition_selfcheck(int32_t* d_result, void* stream);

/* ---- Mixed-length batched decoding (one persistent sweep) ------------------
 * Several batches, each with its own code (any supported N and rate), schedule
 * and buffers.  Each batch runs the kernel bp_decode runs for its length; the
 * launches after the first are programmatic dependent launches, and every
 * decoder kernel lets its dependent start as soon as it has started itself,
 * so a batch's CTAs take the SMs that the previous batch's CTAs leave while
 * its last frames finish: one persistent sweep over all batches, without the
 * tail of each separate launch.  Results are those of bp_decode on each batch
 * alone (same frame ids, same arithmetic).  Batches run in the order given:
 * put the longest work first.  Not in the paper (a throughput feature). */
#define PC_MAX_BATCHES 64

typedef struct {
    const pc_code* code;      /* host pointer */
    pc_sched sched;           /* frame b draws events with frame id sched.frame_base + b */
    int32_t max_iters;
    int32_t slots;            /* frames resident per CTA; 0 = as many as fit */
    int32_t threads_per_frame;/* 0: the bp_decode kernel for this N; otherwise the count of one
                                 kernel as bp_kernel_threads reports it (TMEM-resident stage
                                 groups: N/4 for N = 128..512, N/8 for 1024 and 2048;
                                 shared-memory groups: max(32, N/4)); anything else is
                                 PC_EUNSUPPORTED */
    int32_t reserved;         /* 0 */
    int64_t B;                /* frames in this batch */
    const float* d_llr;       /* B x N, 16-byte aligned */
    uint32_t* d_bits;         /* B x ceil(K/32) */
    int32_t* d_iters;         /* B */
    uint8_t* d_crc_ok;        /* B */
} pc_batch;

/* Bytes of the host launch table of n_batches batches. */
int bp_mixed_table_size(int32_t n_batches, size_t* bytes);
/* Validates the batches and writes, into caller-owned host memory h_table,
 * each batch's kernel parameters (code tables, schedule, buffer pointers) and
 * launch geometry for the current device.  Returns PC_EINVAL for an invalid
 * batch, PC_ENOMEM when bytes is too small; queries the device only after
 * every batch is valid. */
int bp_mixed_prepare(const pc_batch* batches, int32_t n_batches, void* h_table, size_t bytes);
/* Build flags (host only; no counterpart in the paper): bit 0 set for a
 * library built with PCBP_CHECKED, whose tensor-memory decoder kernel
 * range-checks every shared-memory plane access, TMEM column, channel-LLR
 * index and decision-word index.  In such a build bp_decode clears 32 bytes of
 * its workspace and an access out of range of class c (0 plane offset, 1 TMEM
 * column, 2 decided position, 3 position at a partition change, 4 reset
 * index, 5 single-stage index) sets bit c of the uint32 at byte 16 of the
 * workspace and is redirected inside its buffer. */
int pc_build_info(int32_t* flags);

/* Threads per frame of a decoder kernel for this code (kernel 0: the kernel
 * with TMEM-resident stage groups, N = 128..2048, groups of 2 stages up to
 * N = 256 and of 3 from N = 512, so N/4 or N/8; kernel 1: the shared-memory
 * stage-grouped kernel, max(32, N/4)), the value pc_batch.threads_per_frame
 * takes to select it; where the two are equal the TMEM kernel runs unless
 * PCBP_DECODER=grouped.  Host only, no device call.  No counterpart in the
 * paper.  PC_EUNSUPPORTED when the kernel has no build for N. */
int bp_kernel_threads(const pc_code* code, int32_t kernel, int32_t* threads_per_frame);
/* Largest number of frames one CTA of the decoder kernel keeps resident
 * (pc_batch.slots above it is clamped to it) for this code, threads_per_frame
 * (as in pc_batch) and f (fkind 0 or 1) on the current device, limited by
 * shared memory, tensor memory and registers.  No counterpart in the paper; a
 * host query for autotuners.  PC_EUNSUPPORTED for a threads_per_frame no
 * kernel has. */
int bp_slot_limit(const pc_code* code, int32_t threads_per_frame, int32_t fkind, int32_t* max_slots);
/* Bytes of device workspace of bp_decode_mixed (one frame counter per batch). */
int bp_mixed_workspace_size(int32_t n_batches, size_t* bytes);
/* Decodes all batches of a table written by bp_mixed_prepare (PC_EINVAL for
 * anything else): clears the counters in d_workspace (256-byte aligned), then
 * enqueues one launch per non-empty batch on the stream.  Enqueues only
 * device work, so the call can be captured in a CUDA graph. */
int bp_decode_mixed(const void* h_table, int32_t n_batches, void* d_workspace, void* stream);

/* bp_decode for callers that cannot allocate device memory while they decode,
 * such as real-time signal-processing pipelines that allocate everything at
 * start-up (cudaMalloc synchronises the device and has unbounded latency) or
 * hosts whose device memory belongs to another allocator.  The paper has no
 * counterpart; this is a deployment variant of bp_decode with the same
 * arguments except the workspace, and the same results.
 *   Scratch: the decoder's frame counter lives in a file-scope device array of
 *     PC_STATIC_SCRATCH_BYTES bytes that every GPU which loads this library
 *     holds until the process exits.  A call whose decode would need more
 *     scratch than that returns PC_EUNSUPPORTED.
 *   Set-up: the first call on a device looks up the array's device address
 *     (with that device current); make that first call before any stream
 *     capture.
 *   Sharing: all calls use the same array, which keeps the last call's
 *     contents; each call clears the counter on its stream before decoding.
 *     Calls that overlap on the GPU (other streams, concurrent graph
 *     replays) race on it and must be serialised by the caller.
 *   Device reset: the looked-up address belongs to the device's context at
 *     the time of the first call; after cudaDeviceReset it is stale, so do
 *     not use this entry point again in a process that reset the device.
 *   Checked build: a PCBP_CHECKED library records kernel range-check failures
 *     in the workspace's status word; here that word lies in the library's
 *     array, which callers cannot read, so use bp_decode to see it.
 *   Allocates no device memory (no cudaMalloc or cudaFree). */
#define PC_STATIC_SCRATCH_BYTES 4096
int bp_decode_noalloc(const pc_code* code, const float* d_llr, const pc_sched* sched,
                      int32_t max_iters, int64_t B, uint32_t* d_bits, int32_t* d_iters,
                      uint8_t* d_crc_ok, void* stream);

/* Short text for a status code. */
const char* pc_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
