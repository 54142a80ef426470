// Types and launchers of the block codec and the block pool (device side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsim_internal.h"

namespace qsim {

// a compressed block to read
struct BlockRef {
    const uint8_t *ptr;
    uint64_t bytes;
};

// one entry of the block table (where block b's current stream lives)
struct BlockSlot {
    uint8_t *ptr;
    uint64_t bytes;
    uint32_t tier;  // 0 device, 1 pinned host
    uint32_t pad;
};

// where an encoder writes block j of a group
struct EncTarget {
    uint8_t *ptr;
    uint64_t cap;
    uint32_t tier;
    uint32_t pad;
};

struct EncResult {
    uint64_t total;      // stream bytes (also computed when the slot overflowed)
    uint32_t overflow;   // 1 if the stream did not fit the reserved slot
    uint32_t pad;
    double err_sq;       // sum (x - x')^2 over the block
    double norm_sq;      // sum x'^2 over the block
};

// per-stage running totals, updated by the encoder
struct StageAccum {
    uint64_t store_bytes;
    uint64_t reserved_bytes;
    uint64_t host_bytes;
    uint64_t blocks;
    uint64_t overflow_blocks;
    uint64_t pad;
    double err_sq;
    double norm_sq;
};

// a bump arena (device memory, or mapped pinned host memory)
struct ArenaDev {
    uint8_t *base;
    uint64_t cap;
    uint64_t *bump;  // device counter
};

// look-back scratch of the encoder
struct LookbackScratch {
    uint64_t *state;    // one status word per frame
    uint32_t *ticket;
    uint32_t *done;
    uint32_t *epoch;
    float2 *part;       // per-frame (err_sq, norm_sq) partials, or null (then per-CTA atomics)
};

void count_launch();

// rel: the stream is QSZR (relative bound) rather than QSZ1
void launch_decode(const BlockRef *in, uint32_t nblocks, int m, float2 *wv, uint32_t *hist, int *status,
                   cudaStream_t s, bool rel = false);
void launch_encode(const float2 *wv, uint32_t nblocks, int m, int e, const EncTarget *tgt, EncResult *res,
                   int only_overflowed, const uint32_t *ids, BlockSlot *table, StageAccum *acc,
                   const LookbackScratch &scr, int *status, cudaStream_t s);
// sizing pass whose last CTA reserves every block's slot (sizes are left zeroed)
void launch_size_reserve(const float2 *wv, uint32_t nblocks, int m, int e, uint64_t *sizes, uint32_t *done_ctr,
                         const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt, EncResult *res, int *status,
                         cudaStream_t s);
// In-place exact encoder: pass 1 encodes every frame over its own amplitudes (Im-plane words to im, 4 bytes
// per amplitude), records the frames' lengths, word counts (fwords) and offsets and reserves each block's
// exact slot; pass 2 (launch_frame_copy) copies the frames into the slots. wv is overwritten.
// rel: QSZR (e is the shift k, wrec holds kQszrSideBytes per frame, fmixed one word per frame); without a
// device arena (dev.bump null) tgt is the caller's and nothing is reserved. keep_fitting: learned sizing, a
// block keeps its predicted slot (tgt, reserved beforehand) when it fits, else gets an exact one.
void launch_encode_ip(float2 *wv, uint32_t *im, uint32_t nblocks, int m, int e, uint32_t *done_ctr,
                      const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt, EncResult *res, StageAccum *acc,
                      uint8_t *wrec, uint32_t *flen, uint32_t *fwords, uint32_t *foff, float2 *part, int *status,
                      cudaStream_t s, bool rel = false, uint32_t *fmixed = nullptr, bool keep_fitting = false);
void launch_frame_copy(const float2 *wv, const uint32_t *im, uint32_t nblocks, int m, int e, const EncTarget *tgt,
                       EncResult *res, const uint32_t *ids, BlockSlot *table, StageAccum *acc, const uint8_t *wrec,
                       const uint32_t *flen, const uint32_t *fwords, const uint32_t *foff, cudaStream_t s,
                       bool rel = false, const uint32_t *fmixed = nullptr);
// leading phase ops of a stage for the decoder (count <= kMaxPreOps)
struct OpDev;
struct PreOps {
    const OpDev *ops = nullptr;
    uint32_t count = 0;
    uint32_t G = 1;                   // blocks per group
    const float2 *mats = nullptr;
    const uint64_t *gbase = nullptr;  // per group of the batch
};
// decode with the block references read from table[ids[j]]
void launch_decode_table(const BlockSlot *table, const uint32_t *ids, uint32_t nblocks, int m, float2 *wv,
                         uint32_t *hist, int *status, const PreOps &pre, cudaStream_t s, bool rel = false);
void launch_reserve(uint32_t nblocks, const uint64_t *need, uint64_t add_const, const float *pred_log2,
                    double margin, uint64_t worst, const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt,
                    EncResult *res, int retry_overflowed, int *status, cudaStream_t s);
void launch_copy_out(const float2 *wv, uint32_t nblocks, int m, const EncTarget *tgt, const uint32_t *ids,
                     BlockSlot *table, StageAccum *acc, int *status, cudaStream_t s);
void launch_copy_in(const BlockRef *in, uint32_t nblocks, int m, float2 *wv, int *status, cudaStream_t s);
// Frames frames[i] = (block id in table, frame index) decoded into out + i * min(2^m, 4096) (random access through
// the stream's frame offsets)
void launch_decode_frames(const BlockSlot *table, const uint2 *frames, uint32_t nitems, int m, float2 *out,
                          int *status, cudaStream_t s, bool rel);
void launch_gather_refs(const BlockSlot *table, const uint32_t *ids, uint32_t count, BlockRef *out,
                        cudaStream_t s);

}  // namespace qsim
