// Persistent stage kernel: work-item phases, arguments and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "gates.cuh"
#include "mlp.cuh"

namespace qsim {

enum PhaseType : uint32_t {
    PH_DECODE = 0,   // eight frames per item (one warp each), leading phase ops applied
    PH_PASS = 1,     // one tile of gate pass `arg`
    PH_SIZE = 2,     // one frame's exact size; the last item reserves the group's slots
    PH_PREDICT = 3,  // one item: predicted sizes and slot reservation for the group
    PH_ENCODE = 4,   // one frame; the last item folds the group's error partials into the stage totals
    PH_FIX = 5,      // one item: exact slots for blocks whose prediction was too small
    PH_REENCODE = 6  // one frame of an overflowed block (others skip)
};

struct PPhase {
    uint32_t type, count, arg, pad;
};

constexpr int kMaxPhases = 40;

struct PStageArgs {
    uint32_t W, G, ngroups, R, m, nphases, per_group, npre, pre_begin, pbf16;
    int e;
    PPhase ph[kMaxPhases];
    uint32_t ph_start[kMaxPhases];
    const PassDev *passes;
    const OpDev *ops;
    const float2 *mats;
    const uint32_t *bfr;     // B-fragment tables of the tensor-core precisions
    const uint32_t *ids;     // group-major block ids of the stage
    const uint64_t *gbase;   // per group: full-index bits of its outer qubits
    BlockSlot *tab_in, *tab_out;
    StageAccum *acc;
    ArenaDev dev, host;
    uint64_t data_start, worst;
    // per slot (R working vectors)
    float2 *wv;
    uint64_t *lb;
    float2 *part;
    // per block of the stage (group-major)
    EncTarget *tgt;
    EncResult *res;
    uint64_t *sizes;
    uint32_t *hist;
    // predictor
    const float *pparams;
    StageFeatures sf;
    double margin;
    // schedule
    uint32_t *done, *arrive;  // ngroups x nphases each
    uint32_t *ctr;            // queue head, CTAs finished, look-back epoch
    int *status;
    uint32_t stall_test;      // 1: group 0's second phase waits for a count never reached (bounded-wait test)
    uint64_t wait_ns;         // limit of every dependency wait
};

size_t persistent_smem_bytes(uint32_t T, uint32_t mat_elems);
int prepare_stage_persistent(int prec, size_t smem);
int launch_stage_persistent(const PStageArgs &a, int prec, size_t smem, cudaStream_t s, int *grid);

}  // namespace qsim
