// Persistent stage kernel: work-item phases, arguments and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "gates.cuh"
#include "mlp.cuh"

namespace qsim {

enum PhaseType : uint32_t {
    PH_DECODE = 0,   // persistent_frames_per_item(um) frames per item (one warp each), leading phase ops applied
    PH_PASS = 1,     // one tile of gate pass `arg`
    PH_SIZE = 2,     // (not emitted: exact sizing uses PH_SIZE_W)
    PH_PREDICT = 3,  // one item: predicted sizes and slot reservation for the group
    PH_ENCODE = 4,   // one frame; the last item folds the group's error partials into the stage totals
    PH_FIX = 5,      // one item: exact slots for blocks whose prediction was too small
    PH_REENCODE = 6, // one frame of an overflowed block (others skip)
    PH_SIZE_W = 7,   // exact sizing, persistent_frames_per_item(um) frames per item (one warp each): widths and frame length;
                     // the last item turns the lengths into frame offsets and reserves the group's slots
    PH_ENCODE_W = 8, // exact sizing, persistent_frames_per_item(um) frames per item (one warp each) at the known offsets; the last
                     // item folds the group's error partials into the stage totals
    PH_ENCODE_IP = 9, // relative-bound codec: persistent_frames_per_item(um) frames per item (one warp each) encoded over their own
                      // amplitudes; the last item turns the lengths into frame offsets, reserves the group's
                      // exact slots (with learned sizing: keeps every predicted slot its block fits) and folds
                      // the error partials into the stage totals
    PH_COPY = 10      // relative-bound codec: persistent_frames_per_item(um) frames per item (one warp each) copied into their slots
};

struct PPhase {
    uint32_t type, count, arg, pad;
};

constexpr int kMaxPhases = 128;
// frames per work item of the frame-parallel phases (one warp each; the kernel's CTAs have 32 x this many threads):
// 4 in launches whose dense ops run on tcgen05 (128-thread CTAs, one thread per index group of a width-5 op, four
// CTAs per SM filling its TMEM), else 8 (256-thread CTAs, two per SM)
constexpr uint32_t persistent_frames_per_item(bool um) { return um ? 4u : 8u; }
constexpr uint32_t kNoGroup = 0xffffffffu;

// One segment of the work queue: one stage of one circuit. The queue holds
// ngroups x per_group items starting at item_begin; its groups take the launch's
// group numbers group_begin .. group_begin + ngroups - 1 (working-vector slot,
// look-back epoch and the done/arrive counters follow that number).
struct PSeg {
    uint64_t item_begin;
    uint32_t group_begin;
    uint32_t W, G, ngroups, m, nphases, per_group, npre, pre_begin, pbf16;
    int e;
    uint32_t stall_test;  // 1: group 0's second phase waits for a count never reached (bounded-wait test)
    PPhase ph[kMaxPhases];
    uint32_t ph_start[kMaxPhases];
    const PassDev *passes;
    const OpDev *ops;
    const float2 *mats;
    const uint4 *blob;       // the plan's pass blobs
    const uint32_t *bfr;     // B-fragment tables of the tensor-core precisions
    const uint32_t *ids;     // group-major block ids of the stage
    const uint64_t *gbase;   // per group: full-index bits of its outer qubits
    BlockSlot *tab_in, *tab_out;
    StageAccum *acc;
    ArenaDev dev, host;
    uint64_t data_start, worst;
    // per block of the stage (group-major); the kernel leaves sizes and hist zeroed for the next stage
    EncTarget *tgt;
    EncResult *res;
    uint64_t *sizes;
    uint32_t *hist;
    // predictor
    const float *pparams;
    StageFeatures sf;
    double margin;
    // stage barrier within one launch: the previous stage of the same circuit
    // (null when it ran in an earlier launch) and this stage's own counters
    const uint32_t *prev_flag;  // becomes 1 once every group of the previous stage has finished
    uint32_t *fin_count;        // groups of this stage finished
    uint32_t *fin_flag;         // set to 1 after the last group (and the arena reset below)
    uint64_t *reset_bumps;      // two bump words zeroed when the stage is complete (null: none)
};

struct PLaunch {
    const PSeg *segs;        // device array, ordered by item_begin
    uint32_t nseg;
    uint64_t total_items;    // below 2^32
    uint32_t total_groups;
    // per launch group (host-planned working-vector slots): amplitude offset of its slot in wv,
    // frame offset of its slot in lb and part, and the group that used the slot before (kNoGroup: none)
    const uint64_t *g_wv;
    const uint32_t *g_frame;
    const uint32_t *g_prev;
    float2 *wv;
    uint64_t *lb;
    float2 *part;
    uint8_t *wrec;    // per slot frame: chunk widths (256 bytes; relative codec: side record of 2048 bytes)
    uint32_t *flen;   // per slot frame: stream bytes
    uint32_t *foff;   // per slot frame: byte offset in the block's stream
    uint32_t *im;     // relative codec: Im-plane words of the in-place encoder, laid out like wv
    uint32_t *fwords; // relative codec, per slot frame: Re words | Im words << 16
    uint32_t *fmixed; // relative codec, per slot frame: Re | Im mixed sign chunks << 16
    uint32_t *done, *arrive;  // per launch group x kMaxPhases each, zero at launch
    uint32_t *ctr;            // queue head, CTAs finished, look-back epoch
    int *status;
    uint64_t wait_ns;         // limit of every dependency wait
};

// pass_bytes: the largest tile + pass blob + matrix area of the launch's passes
size_t persistent_smem_bytes(size_t pass_bytes);
// um: the launch's passes carry tcgen05 dense ops (TF32 widths 3 to 6, or split BF16 widths 3 to 5)
int prepare_stage_persistent(int prec, size_t smem, bool rel = false, bool um = false);
int launch_stage_persistent(const PLaunch &a, int prec, size_t smem, cudaStream_t s, int *grid, bool rel = false,
                            bool um = false);

}  // namespace qsim
