/*
 * qsim.h — C ABI of libqsim, a compressed full-state quantum circuit simulator
 * for one GB300 (sm_103a), after BMQSim (arXiv 2410.14088).
 *
 * The problem statement follows the paper: a circuit, an SV block size and an
 * inner size are turned into stages offline (Sec. 4.1, Algorithm 1), and the
 * state is then simulated stage by stage with every SV block kept compressed
 * between stages (Sec. 4 overview, Sec. 4.2). Where the paper compresses with a
 * closed library under a point-wise relative bound (Sec. 4.3), this library
 * uses its own format, QSZ1, under the point-wise absolute bound
 * eb = eps * 2^(-n/2) on the real and imaginary part of every amplitude.
 *
 * Conventions
 *   - Qubit q is bit q of the amplitude index (little-endian, Sec. 2.1).
 *   - Amplitudes are complex64, interleaved (re, im) float32, unless stated.
 *   - Every call returns 0 (QSIM_OK) or a negative QSIM_E_* code; no C++
 *     exception crosses this boundary. qsim_last_error() gives a message for
 *     the calling thread's last failure.
 *   - Device pointers are plain CUDA device addresses (or mapped pinned host
 *     addresses) of the current device. Streams are cudaStream_t passed as
 *     void*; NULL is the legacy default stream.
 *   - The caller owns every buffer it passes in. Handles (qsim_plan,
 *     qsim_state) are owned by the library until the matching *_free.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QSIM_OK 0
#define QSIM_E_INVALID -1     /* bad argument: qubit, size, NaN/Inf, m/k range */
#define QSIM_E_NOMEM -2       /* device or pinned-host allocation failed / tiers full */
#define QSIM_E_CAPACITY -3    /* output buffer too small (needed size reported) */
#define QSIM_E_CORRUPT -4     /* malformed compressed stream */
#define QSIM_E_RANGE -5       /* |x| / 2^e >= 2^30: value out of the codec's range */
#define QSIM_E_UNSUPPORTED -6 /* non-diagonal gate with more global qubits than max(i,2) */
#define QSIM_E_TIMEOUT -7     /* a bounded device-side wait gave up */
#define QSIM_E_CUDA -8        /* CUDA runtime error */

/* ---- gates --------------------------------------------------------------- */
#define QSIM_GATE_DIAG 1u      /* optional hint; diagonality is detected from u */
#define QSIM_GATE_PHASEFLIP 2u /* amplitude |basis> times -1; u = NULL, nq/q ignored */

/*
 * One gate (Sec. 2.1 gives the 1- and 2-qubit update; any nq <= 6 is taken).
 * u: 2^nq x 2^nq row-major complex128 as (re, im) double pairs; q[0] is the
 * least-significant bit of the row/column index. u must be unitary (checked
 * to 1e-8) and is copied by qsim_plan_stages.
 */
typedef struct qsim_gate {
    uint32_t nq;
    uint32_t flags;
    uint32_t q[6];
    uint64_t basis;
    const double *u;
} qsim_gate;

/* ---- configuration -------------------------------------------------------- */
#define QSIM_PREC_FP32 0u   /* fused gates on FP32 CUDA cores */
#define QSIM_PREC_TF32 1u   /* fused gates on tensor cores, TF32 inputs, FP32 accumulate */
#define QSIM_PREC_BF16X3 2u /* tensor cores, 3-way split BF16 inputs, FP32 accumulate */

#define QSIM_MODE_STREAMS 0u    /* SV groups round-robin over CUDA streams (Sec. 4.2) */
#define QSIM_MODE_PERSISTENT 1u /* one persistent kernel per stage over a group queue */

#define QSIM_CODEC_QSZ1 0u /* compressed blocks under a point-wise absolute bound (the method) */
#define QSIM_CODEC_NONE 1u /* raw complex64 blocks: the no-compression comparison run */
#define QSIM_CODEC_QSZR 2u /* compressed blocks under a point-wise relative bound eps (Sec. 4.3,
                              Eq. 1-2, Algorithm 2); both modes, exact or learned sizing */

#define QSIM_SIZING_EXACT 0u   /* every block gets a slot of its exact size: in streams mode the encoder
                                  codes the frames in place in one read of the working vector and then
                                  reserves the exact slots; the persistent kernel sizes the frames in
                                  one read and encodes at the known offsets in a second */
#define QSIM_SIZING_PREDICT 1u /* learned size predictor reserves space; overflow re-encodes */

#define QSIM_REORDER_NONE 0u   /* Algorithm 1 over the gates in circuit order */
#define QSIM_REORDER_STAGES 1u /* commutation-aware stage partition */
#define QSIM_REORDER_PASSES 2u /* commutation-aware stages + pass-aware order within each stage, kept per
                                  stage where a model of the passes' time puts it at least 5 % lower */
#define QSIM_REORDER_PASSES_ALL 3u /* as 2, in every stage (no model; for measurements) */

typedef struct qsim_config {
    uint32_t m;           /* log2 amplitudes per SV block (the paper's b), 5..26 */
    uint32_t inner;       /* inner size i (Sec. 4.1); threshold = max(i, 2) */
    uint32_t k;           /* max fused gate width, 1..6 */
    uint32_t prec;        /* QSIM_PREC_* */
    uint32_t mode;        /* QSIM_MODE_* */
    uint32_t streams;     /* CUDA streams in QSIM_MODE_STREAMS (1..16) */
    uint32_t sizing;      /* QSIM_SIZING_* */
    uint32_t diag_exempt; /* 1: diagonal gates never count as global (off = paper) */
    uint32_t codec;       /* QSIM_CODEC_* */
    uint32_t graph;       /* 1: capture each run's stage loop in a CUDA graph (persistent mode) */
    uint32_t tile_bits;   /* log2 amplitudes per shared-memory tile, 0 = default */
    uint32_t collect;     /* 1: log (features, compressed size) of every encoded block (predictor training) */
    double eps;           /* QSZ1: eb = eps * 2^(-n/2); QSZR: the relative bound b_r, in (2^-23, 1) */
    uint64_t device_tier_cap_bytes; /* bytes of compressed blocks kept on the device; 0 = no cap */
    uint64_t init_basis;  /* initial basis state |init_basis> (Sec. 4.2 initialisation) */
    double predictor_margin; /* predictor reservation = 2^pred * (1 + margin) */
    uint32_t reorder;        /* QSIM_REORDER_*: 0 = Algorithm 1 in circuit order; 1 = commutation-
                                aware partition: a gate may be placed before earlier gates it
                                commutes with (disjoint qubits, or both diagonal) when that keeps
                                it in the current stage; 2 = that partition, and inside each stage
                                a pass-aware order: gates are gathered into shared-memory tile
                                passes (a non-diagonal gate joins a pass while the tile bits it
                                needs fit, diagonal gates join any pass) and fused pass by pass,
                                kept per stage where a model of the passes' time puts it at least
                                5 % lower; 3 = the pass-aware order in every stage */
    uint32_t tcgen05;        /* 1: TF32 and split-BF16 dense ops of width 5 on the 5th-generation
                                tensor cores (tcgen05.mma, accumulator in tensor memory) in
                                streams mode; 0: warp-level mma.sync */
    uint64_t reserved[5];    /* zero; reserved[0] bit 0 is a test hook: in persistent mode the
                                first stage's second phase waits for a count that is never
                                reached, so the run ends with QSIM_E_TIMEOUT after the
                                bounded wait (0.2 s) instead of hanging; bit 1 likewise for
                                the tcgen05 dense ops: their MMAs are neither issued nor
                                committed to the mbarrier, so each tile's wait runs out after
                                1 s with no MMA in flight */
} qsim_config;

/* Fill *cfg with defaults: m 20, inner 2, k 4, FP32, streams mode, 2 streams,
 * exact sizing, eps 1e-3, QSZ1, no cap, |0...0>. */
void qsim_config_default(qsim_config *cfg);

/* ---- planning (host only) ------------------------------------------------ */
typedef struct qsim_plan qsim_plan;

/*
 * Canonicalise the gates, cut the circuit into stages with Algorithm 1
 * (Sec. 4.1: a gate joins the current stage unless the distinct global
 * qubits — bits >= m — of stage plus gate would exceed max(inner, 2)), fuse
 * each stage's gates greedily into dense ops of at most k qubits, and lay the
 * ops out in shared-memory tile passes. Host work only; the gate matrices are
 * uploaded by qsim_run.
 * Errors: INVALID (n outside 5..40, m > n, bad qubit, non-unitary u, k < a
 * gate's width), UNSUPPORTED (a non-diagonal gate whose global qubits alone
 * exceed the threshold), NOMEM.
 */
int qsim_plan_stages(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *cfg,
                     qsim_plan **out);

/* Number of stages; if stage_inner_masks is not NULL it receives, per stage,
 * a mask whose bit j is set when global qubit m + j is an inner index. */
int qsim_plan_info(const qsim_plan *plan, size_t *nstages, uint32_t *stage_inner_masks);

/*
 * Group sharding over 2^log2_ranks ranks (Sec. 4.2: the SV groups of a stage
 * are independent, so they can run on different GPUs; Sec. 5.8 measures the
 * paper's multi-GPU runs). For every stage s the call picks log2_ranks rank
 * qubits, global qubits (>= m) outside the stage's inner set, and writes them
 * to rank_qubits[s * log2_ranks + j] (host, nstages * log2_ranks entries).
 * Block b (index bits m.. of its amplitudes) belongs during stage s to the
 * rank whose bit j is the block's bit at rank qubit j, so every SV group of
 * the stage lies on one rank. A rank qubit keeps its slot j until a stage
 * takes it as an inner qubit; it is then replaced by the free global qubit
 * whose next use as an inner qubit is farthest ahead, so blocks change ranks
 * only at the stage boundaries where a slot changes.
 * Errors: INVALID (null pointer, log2_ranks > 16, a stage that leaves fewer
 * than log2_ranks global qubits outside its inner set). log2_ranks = 0 writes
 * nothing.
 */
int qsim_plan_shards(const qsim_plan *plan, uint32_t log2_ranks, uint32_t *rank_qubits);

/* Gates [*first, *first + *count) of the input form stage `stage`. */
int qsim_plan_stage_gates(const qsim_plan *plan, size_t stage, size_t *first, size_t *count);

typedef struct qsim_plan_stats {
    uint64_t nstages, ngates, dense_ops, diag_ops, phaseflip_ops, passes;
    uint64_t max_working_log2; /* log2 amplitudes of the largest working vector */
    double plan_seconds;
} qsim_plan_stats;
int qsim_plan_get_stats(const qsim_plan *plan, qsim_plan_stats *out);

/* Introspection of a stage's fused ops (what the gate passes apply). */
typedef struct qsim_op_info {
    uint32_t type;      /* 0 dense matrix, 1 diagonal phases, 2 phase flip, 3 controlled-separable diagonal */
    uint32_t nq;        /* qubits of the op (0 for a phase flip) */
    uint32_t qubits[8]; /* full qubit ids; matrix bit j <-> qubits[j] (dense ops <= 6, diagonal ops <= 8;
                           type 3: the first 8 of qlist) */
    uint32_t ngates;    /* input gates folded into the op */
    uint32_t pass;      /* index of the shared-memory tile pass within the stage */
    uint32_t quadratic; /* diagonal op whose phase angle is a polynomial of degree <= 2 in its qubits' bits
                           (every product of one- and two-qubit diagonal gates): in passes of 4096-amplitude
                           tiles a run of such ops is applied as one phase per amplitude; else 0 */
    uint32_t reserved_; /* zero */
    uint64_t basis;     /* phase flip: the flipped basis state */
    const double *u;    /* dense: 2^nq x 2^nq complex128 row-major; diagonal: 2^nq complex128;
                           type 3: K[0], K[1], then per target D[0][0], D[0][1], D[1][0], D[1][1]
                           (complex128), phase(x) = K[b] prod_t D_t[b][x_t] with b the control bit;
                           owned by the plan */
    const uint32_t *qlist; /* type 3: nq qubits, the control then the targets; owned by the plan */
} qsim_op_info;

/* *count receives the number of ops of `stage`; if ops is not NULL it must
 * hold *count entries on input (capacity) and receives them. */
int qsim_plan_stage_ops(const qsim_plan *plan, size_t stage, size_t *count, qsim_op_info *ops);

void qsim_plan_free(qsim_plan *plan);

/* ---- simulation ------------------------------------------------------------ */
typedef struct qsim_state qsim_state;

typedef struct qsim_stats {
    double seconds;          /* device time of the run (CUDA events), init included */
    double err_norm_sum;     /* sum over stages of ||delta_s|| (codec error, FP64) */
    double err_sq_total;     /* sum over stages of ||delta_s||^2 */
    double norm_sq;          /* ||psi_sim||^2 after the last stage */
    uint64_t nstages, groups, kernel_launches;
    uint64_t peak_store_bytes;     /* max over stages of the summed stream bytes (Sec. 5.4) */
    uint64_t peak_reserved_bytes;  /* max over stages of the reserved slot bytes */
    uint64_t final_store_bytes;
    uint64_t host_tier_peak_bytes; /* max over stages of bytes placed in pinned host memory */
    uint64_t overflow_blocks;      /* predictor under-estimates that were re-encoded */
    uint64_t blocks_encoded;
    double fidelity_lower_bound;   /* (1 + |b|^2 - E^2) / (2|b|), E = err_norm_sum */
    uint64_t h2d_bytes;            /* host->device bytes copied by the run (plan upload included) */
    uint64_t d2h_bytes;            /* device->host bytes copied by the run (statistics) */
} qsim_stats;

/*
 * Run the plan from |init_basis> (Sec. 4.2: the initial store encodes the
 * block holding the basis state and one zero block, copied to every other
 * block; then, stage after stage, every SV group — the 2^|inner| blocks that
 * share their outer index bits — is decompressed, updated by the stage's
 * gates and compressed again, the groups overlapped on CUDA streams, or in
 * persistent mode inside one kernel per stage). Blocks live in the device
 * tier, then in pinned host memory once the device tier is full (Sec. 4.4).
 * Work is ordered on cuda_stream (and on the library's own streams, joined
 * back to it); the call returns once the run is complete and *stats
 * (nullable) is filled. *out receives a state handle owning the final
 * compressed store (the library's memory until qsim_state_free).
 * Errors: NOMEM (tiers full), RANGE, TIMEOUT, CUDA, INVALID.
 */
int qsim_run(const qsim_plan *plan, void *cuda_stream, qsim_state **out, qsim_stats *stats);

/* Per-stage record of a finished run: stream bytes after the stage, reserved
 * bytes, ||delta_s||^2 of the codec error injected by the stage. */
int qsim_state_stage_stats(const qsim_state *st, size_t stage, uint64_t *store_bytes,
                           uint64_t *reserved_bytes, double *err_sq);

/* ---- sharded runs: one rank's SV groups on this GPU ---------------------------
 * Sec. 4.2's groups are independent, so a run can be spread over several GPUs
 * (the paper's multi-GPU runs, Sec. 5.8): rank k holds the blocks whose bits at
 * the stage's rank qubits (qsim_plan_shards) spell k and runs the SV groups they
 * form. Between stages whose rank qubits differ, each rank exports the blocks
 * that change owner (their compressed streams, packed into a caller's device
 * buffer) and imports those it receives; the transfer itself (NCCL, or any
 * copy) is the caller's. Every call is on the current device; work is ordered
 * on the stream given to qsim_shard_begin, and the export, import and finish
 * calls synchronise it. The handle is the library's until qsim_shard_free.
 */
typedef struct qsim_shard_run qsim_shard_run;

/* Begin rank `rank` of 2^log2_ranks: the compressed store's tiers, the
 * initial store (Sec. 4.2), and the rank's SV groups of every stage. plan must
 * be in streams mode; rank_qubits: host, nstages * log2_ranks entries as from
 * qsim_plan_shards (copied). The rank starts with the blocks it owns under
 * stage 0's rank qubits. Errors: INVALID (null pointer, persistent mode, rank
 * out of range, a rank qubit that is inner or not global), NOMEM, CUDA. */
int qsim_shard_begin(const qsim_plan *plan, const uint32_t *rank_qubits, uint32_t log2_ranks, uint32_t rank,
                     void *cuda_stream, qsim_shard_run **out);

/* Run stage `stage` (stages in order, from 0) over this rank's SV groups. The
 * blocks on the rank must be exactly those its rank qubits give it for this
 * stage (INVALID otherwise). */
int qsim_shard_stage(qsim_shard_run *run, size_t stage);

/* Stream bytes of `count` blocks on this rank (host lists; each a multiple of
 * 16), as they are before the next stage. INVALID for a block not on the rank. */
int qsim_shard_block_bytes(qsim_shard_run *run, const uint64_t *blocks, size_t count, uint64_t *bytes);

/* Pack the streams of `count` blocks on this rank, in list order, into
 * d_packed (device, 16-byte aligned, cap bytes; block i at the sum of the
 * sizes before it) and remove them from the rank. CAPACITY when cap is too
 * small (nothing removed). */
int qsim_shard_export(qsim_shard_run *run, const uint64_t *blocks, size_t count, void *d_packed, size_t cap);

/* Place `count` received blocks on this rank: block ids and stream bytes
 * (host), streams packed back to back in d_packed (device, 16-byte aligned),
 * copied into the rank's current tier (device, then pinned host). Errors:
 * INVALID (a block already on the rank), CORRUPT (a size not a multiple of
 * 16), NOMEM (tiers full, reported by the device), CUDA. */
int qsim_shard_import(qsim_shard_run *run, const uint64_t *blocks, const uint64_t *bytes, size_t count,
                      const void *d_packed);

/* After the last stage: the state handle of the blocks now on this rank (the
 * others read as corrupt blocks) and the rank's statistics. */
int qsim_shard_finish(qsim_shard_run *run, qsim_state **out, qsim_stats *stats);
void qsim_shard_free(qsim_shard_run *run);

/* ---- readout -------------------------------------------------------------- */

/* Read the final state (Sec. 4.2's loop leaves it compressed, block by
 * block): gather `count` amplitudes, indices idx (host, each < 2^n), into
 * out_interleaved (HOST, 2*count floats, re then im per amplitude). Only the
 * blocks holding them are decompressed, into library scratch on the state's
 * device. Errors: INVALID (null pointer, index out of range), NOMEM, CUDA,
 * CORRUPT. */
int qsim_amplitudes(const qsim_state *st, const uint64_t *idx, size_t count, float *out_interleaved);

/* Fidelity |<ref|sim>| / (||ref|| ||sim||) (Sec. 5.3 definition, normalised),
 * reduced in FP64 on the GPU. ref: 2^n complex128 interleaved, host or
 * device pointer. */
int qsim_fidelity(const qsim_state *st, const double *ref_interleaved, double *f);

/* ||psi_sim||^2 in FP64 on the GPU. */
int qsim_state_norm(const qsim_state *st, double *norm_sq);

/* Decompress the whole state into d_out (device, 2^n complex64). */
int qsim_state_decompress(const qsim_state *st, float *d_out, void *cuda_stream);

/* Copy block `block`'s compressed stream to host_out (cap bytes); *bytes gets
 * its size (also when cap is too small: CAPACITY); 0 bytes for a block the
 * state does not hold (the other ranks' blocks after a sharded run). */
int qsim_state_block_stream(const qsim_state *st, uint64_t block, void *host_out, size_t cap,
                            size_t *bytes);

void qsim_state_free(qsim_state *st);

/* ---- single-block codec (the bit-exactness surface) --------------------- */

/* Worst-case QSZ1 stream size for a block of 2^m amplitudes:
 * 32 + pad16(4 (nframes+1)) + nframes (pad16(2C) + 8F), F = min(4096, 2^m). */
/* Largest stream of a 2^m-amplitude block: QSZ1 (absolute bound), and QSZR (relative bound). 0 if m is
 * outside 5..26. */
size_t qsim_worst_case_bytes(uint32_t m);
size_t qsim_worst_case_bytes_rel(uint32_t m);

/*
 * Compress one SV block (Sec. 4.3: error-bounded lossy compression of a
 * block, here under a point-wise ABSOLUTE bound with this library's QSZ1
 * format: quantisation to int32 on the grid 2^e with 2^e <= 2 eb, a delta
 * within 32-value chunks, zigzag and bit-plane packing at each chunk's
 * width). d_amps: 2^m complex64 amplitudes on the device, interleaved,
 * 16-byte aligned, not modified; d_out: device, cap bytes. The call
 * synchronises cuda_stream and writes the stream size to *out_bytes (host).
 * Every reconstructed component is within eb of the input.
 * Errors: INVALID (m outside 5..26, eb out of range, NaN/Inf input), RANGE,
 * CAPACITY (cap too small; *out_bytes = the size needed), CUDA.
 * Calls from several host threads are serialised inside the library.
 */
int qsim_compress_block(const float *d_amps, uint32_t m, double eb, void *d_out, size_t cap,
                        size_t *out_bytes, void *cuda_stream);

/*
 * Allocation-free variant of qsim_compress_block. This is a library
 * addition with no counterpart in the paper.
 *
 * qsim_compress_block allocates device scratch with cudaMalloc on its first
 * call on a device. Callers that cannot allow an allocation at that point —
 * an application whose framework already owns the device memory through its
 * own pool, a service that must keep a fixed footprint once started, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device — use this entry point instead. Its scratch is one fixed device
 * array inside the library image (look-back words for blocks of up to
 * 2^QSIM_NOALLOC_MAX_M amplitudes, 32 KiB, plus 256 bytes), held by every GPU
 * that loads the library until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * Arguments, output and errors are those of qsim_compress_block; in
 * addition m > QSIM_NOALLOC_MAX_M is rejected with QSIM_E_INVALID. The first
 * call on a device looks up the array's device address (once per device,
 * with that device current).
 * All calls share the one array and each call clears the parts it uses, so
 * calls must not overlap on the GPU: this call synchronises cuda_stream
 * before it returns, and calls from several host threads are serialised.
 */
#define QSIM_NOALLOC_MAX_M 24
int qsim_compress_block_noalloc(const float *d_amps, uint32_t m, double eb, void *d_out, size_t cap,
                                size_t *out_bytes, void *cuda_stream);

/*
 * Compress one block of 2^m complex64 amplitudes (d_amps, device) under the
 * point-wise RELATIVE bound rel (Sec. 4.3, Eq. 1-2; Algorithm 2's sign bitmap
 * with all-0 / all-1 chunks stored as 2-bit types) into a QSZR stream in
 * d_out (device, cap bytes). Every reconstructed component x' of a normal
 * input x satisfies |x' - x| <= rel |x| with the sign of x kept; zeros stay
 * zero; subnormal inputs get an absolute error below 2^(k-150) (k the code
 * shift, the largest integer with 2^(k-24) <= rel / (1 + rel)).
 * d_amps is not modified (the block is copied to library scratch, grown by
 * cudaMalloc when a larger m is first used). Synchronises cuda_stream and
 * writes the stream size to *out_bytes (host).
 * Errors: INVALID (m outside 5..26, rel outside (2^-23, 1), NaN/Inf input),
 * RANGE (|x| >= 2^64), CAPACITY (*out_bytes = the size needed), NOMEM, CUDA.
 */
int qsim_compress_block_rel(const float *d_amps, uint32_t m, double rel, void *d_out, size_t cap,
                            size_t *out_bytes, void *cuda_stream);

/*
 * Decompress one SV block (the inverse of the block codec of Sec. 4.3, run
 * before every stage's gate updates in Sec. 4.2): a QSZ1 or QSZR stream
 * (d_in, device, in_bytes; the format is read from its magic number) into
 * d_amps (device, 2^m complex64, interleaved; the caller's buffer).
 * Synchronises cuda_stream to report the status.
 * Errors: INVALID, CORRUPT (bad magic/header/offsets/widths/sign types), CUDA.
 */
int qsim_decompress_block(const void *d_in, size_t in_bytes, float *d_amps, uint32_t m,
                          void *cuda_stream);

/* ---- learned block-size predictor ----------------------------------------- */
/*
 * A 41 -> 64 -> 64 -> 1 ReLU MLP predicts log2 of each block's next stream
 * size from cheap statistics: the 32-bin histogram of code bit lengths as
 * decoded (fractions), the largest bit length / 32, and 8 stage
 * features. The histogram is taken over the block's SV group (the blocks a
 * stage mixes). The output is log2(bytes) - (m + 3). Parameters (6913 floats):
 * W1[64][41], b1[64], W2[64][64], b2[64], W3[64], b3. This replaces the
 * paper's reactive fall-back to a second memory level (Sec. 4.4) by a
 * reservation made before encoding; an under-estimate re-encodes the block
 * into an exactly sized slot.
 */
#define QSIM_MLP_INPUTS 41
#define QSIM_MLP_PARAMS 6913
#define QSIM_TRAIN_ROW 42 /* logged row: 41 features then the target */

/* GPU forward pass: y[b] = MLP(x[b]); device pointers; bf16_weights rounds the
 * weights to BF16 (inference precision). */
int qsim_mlp_forward(const float *d_params, const float *d_x, size_t batch, float *d_y, int bf16_weights,
                     void *cuda_stream);
/* GPU loss 0.5/B sum (y - t)^2 and its gradient (device pointers; *loss is host). */
int qsim_mlp_loss_grad(const float *d_params, const float *d_x, const float *d_t, size_t batch, float *d_grad,
                       float *loss, void *cuda_stream);
/* GPU Adam step (t is 1-based) on n parameters. */
int qsim_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, size_t n, int t, float lr,
                   float beta1, float beta2, float eps, void *cuda_stream);

typedef struct qsim_train_config {
    uint32_t epochs;        /* passes over the data */
    uint32_t batch;         /* samples per Adam step */
    float lr;               /* Adam learning rate */
    uint32_t bf16_inference;/* 1: predict with BF16-rounded weights */
    uint64_t seed;          /* initialisation and shuffling */
} qsim_train_config;

/* Train the library's predictor on the current device from logged rows (host,
 * count x QSIM_TRAIN_ROW floats) with the GPU kernels above; *final_loss
 * (nullable) receives the loss over all rows. Replaces any previous weights. */
int qsim_predictor_train(const float *rows, size_t count, const qsim_train_config *tc, double *final_loss);
/* Install / read the predictor's weights (host arrays of QSIM_MLP_PARAMS floats). */
int qsim_predictor_set(const float *params, size_t n, int bf16_inference);
int qsim_predictor_get(float *params, size_t n);

/* Rows logged by a run with cfg.collect = 1 (host, cap_rows x QSIM_TRAIN_ROW);
 * *rows receives the number available. */
int qsim_state_training_data(const qsim_state *st, float *rows_out, size_t cap_rows, size_t *rows);

/* ---- autotuner ---------------------------------------------------------------- */
/*
 * Picks the SV block size m, the fused width k, the inner size i and the
 * stream count for a circuit by timing qsim_run on a prefix of it (the paper
 * tunes inner size and block size by hand, Sec. 5.8). Coordinate search: m,
 * then k, then i, then streams, each with the others fixed at the best so
 * far. Results are cached in memory per (n, gate structure, search space,
 * precision, codec); a second call with the same key returns the cached
 * choice without running anything.
 */
typedef struct qsim_tune_space {
    uint32_t m_min, m_max;         /* SV block sizes tried */
    uint32_t k_min, k_max;         /* fused widths tried */
    uint32_t inner_min, inner_max; /* inner sizes tried */
    uint32_t streams_mask;         /* bit s set: try s streams (s = 1..16) */
    uint32_t prefix_gates;         /* gates of the circuit prefix timed (0 = all) */
    uint32_t reps;                 /* timed runs per candidate (the best is kept) */
    uint32_t max_working_log2;     /* skip candidates with m + inner above this (0: no limit), e.g. n - 2 to
                                      keep at least four SV groups per stage */
} qsim_tune_space;

/* *best receives base with m, k, inner and streams replaced by the fastest
 * candidate; *best_seconds (nullable) its prefix time; *candidates (nullable)
 * the number of configurations timed (0 on a cache hit). */
int qsim_autotune(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *base,
                  const qsim_tune_space *space, qsim_config *best, double *best_seconds, uint32_t *candidates);
void qsim_autotune_cache_clear(void);

/* ---- per-kernel timing ---------------------------------------------------- */

/* When enabled, qsim_run brackets every kernel launch with CUDA events on the
 * stream it is launched on; the per-kernel totals of a run are then read with
 * qsim_state_kernel_stats. Algorithmic bytes/flops are the run's useful
 * traffic/work per kernel (compressed bytes read or written, 8 bytes per
 * amplitude per pass over the working vector, 8 * 2^k flops per amplitude per
 * dense k-qubit op). */
void qsim_profile_enable(int on);

typedef struct qsim_kernel_stat {
    char name[32];
    uint64_t launches;
    double seconds;   /* sum of event-timed launch durations */
    double alg_bytes; /* algorithmic DRAM bytes over the run */
    double alg_flops; /* algorithmic flops over the run */
} qsim_kernel_stat;

int qsim_state_kernel_stats(const qsim_state *st, qsim_kernel_stat *out, size_t cap, size_t *count);

/* ---- a batch of independent circuits ----------------------------------------
 * Runs `count` planned circuits together: their initial stores, then ONE launch
 * of the persistent stage kernel whose work queue holds every stage of every
 * circuit. Stages are dealt round-robin over the circuits (stage 0 of each,
 * then stage 1 of each, ...); a circuit's stage waits on the device for all
 * groups of its previous stage (a bounded wait, QSIM_E_TIMEOUT), so one
 * circuit's stage boundary overlaps the other circuits' work. The paper runs
 * one circuit at a time; this extends its group pipeline (Sec. 4.2) to many
 * independent state vectors, each with its own block size, fused width and
 * error bound.
 *   plans   host array of `count` plans. Each must use codec QSZ1, k <= 5 and
 *           no row collection; all must use the same precision. Their mode and
 *           streams fields are ignored; sizing is exact or predict per plan
 *           (predict needs trained weights); the first plan's `graph` flag
 *           decides whether the launch is captured in a CUDA graph.
 *   states  out: host array of `count` handles, each freed by qsim_state_free.
 *   stats   nullable: `count` entries; `seconds` is the whole batch's time.
 *   launch  nullable: event time, algorithmic bytes and flops of the batch's
 *           persistent launch.
 * Memory: each circuit gets a share of the device and pinned-host levels in
 * proportion to its worst-case store size.
 * Errors: INVALID (empty batch, mixed precision, a plan the persistent kernel
 * cannot run), UNSUPPORTED, NOMEM, RANGE, TIMEOUT, CUDA. On error every
 * states[i] is NULL. */
int qsim_run_batch(const qsim_plan *const *plans, size_t count, void *cuda_stream, qsim_state **states,
                   qsim_stats *stats, qsim_kernel_stat *launch);

/* ---- misc ------------------------------------------------------------------ */
const char *qsim_last_error(void);

/* Number of kernels this library launched in this process so far. */
uint64_t qsim_kernel_launch_count(void);

/* Number of device (cudaMalloc) and pinned-host (cudaHostAlloc) allocations this
 * library made in this process so far; buffers it reuses from its own cache are
 * not counted again. qsim_compress_block_noalloc leaves it unchanged. */
uint64_t qsim_alloc_count(void);

/* Release cached device/pinned buffers held by the library for reuse. */
void qsim_release_cached_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
