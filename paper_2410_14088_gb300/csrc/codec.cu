// QSZ1 block codec kernels (sm_103a).
//
// The paper compresses every SV block with a GPU lossy compressor under a
// point-wise error bound (Sec. 4.3) and notes that sign runs are detected with
// warp votes. QSZ1 is this library's own absolute-bound format:
//   step s = 2^e, e = the largest integer with 2^e <= 2 eb (so s/2 <= eb);
//   q = round-half-even(x / s) in int32, |q| < 2^30;  x' = q * s exactly;
//   planes Re and Im; chunks of 32 values; d_0 = q_0, d_j = q_j - q_{j-1};
//   z = zigzag(d); w = bit length of OR z; bit planes W_b = ballot(bit b of z).
// Stream: 32-byte header (u32 magic "QSZ1", u16 version 1, u16 flags 0, u8 m,
// u8 frame_log, i8 e, u8 0, u32 nframes, u64 total_bytes, u64 0), u32
// offsets[nframes+1] padded to 16 bytes, then frames of F = min(4096, 2^m)
// amplitudes: u8 widths[2C] (C = F/32, Re then Im) padded to 16, the words of
// each chunk (Re chunks then Im chunks), padded to 16. A frame whose widths
// are all zero has length 0 (the all-zero run elision).
//
// Encoding is single-pass: each CTA encodes one frame, takes a ticket so that
// frames are processed in order, and finds its byte offset inside the block's
// stream with a decoupled look-back over the preceding frames' sizes. Every
// spin-wait is bounded and reports QSIM_E_TIMEOUT instead of hanging.
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "codec_dev.cuh"
#include "device_common.cuh"
#include "gates.cuh"

namespace qsim {

namespace {

using namespace cdev;

// NP: the most leading phase ops the kernel applies (pre.count <= NP).
template <int NP, bool REL>
__global__ void __launch_bounds__(NT, 3) k_decode(const BlockRef *__restrict__ in, const BlockSlot *__restrict__ table,
                                               const uint32_t *__restrict__ ids, uint32_t nblocks, int m,
                                               float2 *__restrict__ wv, uint32_t *__restrict__ hist,
                                               int *status, PreOps pre) {
    const FrameGeom g = geom(m);
    __shared__ OpDev s_pre[NP > 0 ? NP : 1];
    __shared__ uint2 s_pre_ab[NP > 0 ? NP : 1];
    __shared__ uint32_t s_hist[NW][32];
    if (NP > 0 && threadIdx.x < pre.count) {
        s_pre[threadIdx.x] = pre.ops[threadIdx.x];
        s_pre_ab[threadIdx.x] = pre_setup(pre.ops[threadIdx.x]);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint64_t items = uint64_t(nblocks) * g.nframes;
    for (uint64_t item = uint64_t(blockIdx.x) * NW + warp; item < items; item += uint64_t(gridDim.x) * NW) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        const uint8_t *sp;
        uint64_t bytes;
        if (table) {
            const BlockSlot sl = table[ids[j]];
            sp = sl.ptr;
            bytes = sl.bytes;
        } else {
            sp = in[j].ptr;
            bytes = in[j].bytes;
        }
        decode_frame_warp<NP, false, REL>(sp, bytes, g, m, f, wv + (uint64_t(j) << m) + uint64_t(f) * g.F,
                                         hist ? hist + uint64_t(j) * 32 : nullptr, s_hist[warp], status, s_pre,
                                         s_pre_ab, pre.count, pre.mats, pre.count ? (uint64_t(j % pre.G) << m) : 0,
                                         pre.count ? pre.gbase[j / pre.G] : 0);
    }
}

// Random access: frame frames[i].y of block frames[i].x (slot table entry) decoded into out + i * F, one warp per
// frame; no leading phase ops, no histogram.
template <bool REL>
__global__ void __launch_bounds__(NT, 3) k_decode_frames(const BlockSlot *__restrict__ table,
                                                      const uint2 *__restrict__ frames, uint32_t nitems, int m,
                                                      float2 *__restrict__ out, int *status) {
    const FrameGeom g = geom(m);
    __shared__ uint32_t s_hist[NW][32];
    const int warp = threadIdx.x >> 5;
    for (uint64_t item = uint64_t(blockIdx.x) * NW + warp; item < nitems; item += uint64_t(gridDim.x) * NW) {
        const uint2 bf = frames[item];
        const BlockSlot sl = table[bf.x];
        decode_frame_warp<0, false, REL>(sl.ptr, sl.bytes, g, m, bf.y, out + item * g.F, nullptr, s_hist[warp],
                                         status, nullptr, nullptr, 0, nullptr, 0, 0);
    }
}

__global__ void __launch_bounds__(NT) k_encode(const float2 *__restrict__ wv, uint32_t nblocks, int m, int e,
                                               const EncTarget *__restrict__ tgt, EncResult *__restrict__ res,
                                               int only_overflowed, const uint32_t *__restrict__ ids,
                                               BlockSlot *__restrict__ table, StageAccum *acc,
                                               LookbackScratch scr, int *status) {
    const FrameGeom g = geom(m);
    __shared__ __align__(16) uint32_t s_stage[kStageWords];
    __shared__ EncSmem SE;
    __shared__ uint32_t s_item, s_epoch;
    __shared__ int s_skip;
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        s_item = atomicAdd(scr.ticket, 1u);
        s_epoch = ld_relaxed_u32(scr.epoch) & kEpochMask;
    }
    __syncthreads();
    const uint32_t item = s_item, epoch = s_epoch;
    const uint32_t j = item / g.nframes, f = item % g.nframes;
    if (tid == 0) s_skip = (j >= nblocks) || (only_overflowed && res[j].overflow == 0);
    __syncthreads();
    if (!s_skip)
        encode_frame_cta(wv + (uint64_t(j) << m) + uint64_t(f) * g.F, g, m, e, f, scr.state + uint64_t(j) * g.nframes,
                         epoch, tgt[j], res + j, table ? table + ids[j] : nullptr, acc,
                         scr.part ? scr.part + item : nullptr, only_overflowed, s_stage, SE, status);
    // ---- last CTA: reduce the frame partials, reset the ticket counter, advance the epoch ----
    __syncthreads();  // the frame's writes by every thread of the CTA come before its arrival
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(scr.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (scr.part && !only_overflowed) {
        // warp per block: sum its frames' partials in FP64
        double ta = 0, tb = 0;
        for (uint32_t jb = warp; jb < nblocks; jb += NW) {
            double a = 0, b = 0;
            for (uint32_t f2 = lane; f2 < g.nframes; f2 += 32) {
                const float2 p = scr.part[uint64_t(jb) * g.nframes + f2];
                a += double(p.x);
                b += double(p.y);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                a += __shfl_xor_sync(kFull, a, o);
                b += __shfl_xor_sync(kFull, b, o);
            }
            if (lane == 0) {
                res[jb].err_sq = a;
                res[jb].norm_sq = b;
            }
            ta += a;
            tb += b;
        }
        if (lane == 0) {
            SE.red[0][warp] = ta;
            SE.red[1][warp] = tb;
        }
        __syncthreads();
        if (tid == 0 && acc) {
            double a = 0, b = 0;
            for (int w = 0; w < NW; ++w) { a += SE.red[0][w]; b += SE.red[1][w]; }
            atomicAdd(&acc->err_sq, a);
            atomicAdd(&acc->norm_sq, b);
        }
    }
    if (tid == 0) {
        *scr.ticket = 0;
        *scr.done = 0;
        __threadfence();
        atomicExch(scr.epoch, (epoch + 1) & kEpochMask);
    }
}

// Sizing pass (one CTA per frame) whose last CTA reserves every block's slot
// from the summed frame lengths; sizes are left zeroed for the next use.
__global__ void __launch_bounds__(NT, 3) k_encode_size(const float2 *__restrict__ wv, uint32_t nblocks, int m, int e,
                                                    uint64_t *__restrict__ sizes, uint32_t *done_ctr,
                                                    ArenaDev dev, ArenaDev host, EncTarget *__restrict__ tgt,
                                                    EncResult *__restrict__ res, int *status) {
    const FrameGeom g = geom(m);
    __shared__ uint32_t s_words[NW];
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const uint64_t items = uint64_t(nblocks) * g.nframes;
    for (uint64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        const uint32_t len = size_frame_cta(wv + (uint64_t(j) << m) + uint64_t(f) * g.F, g, e, s_words, status);
        if (tid == 0 && len) atomicAdd(reinterpret_cast<unsigned long long *>(&sizes[j]), uint64_t(len));
    }
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(done_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (uint32_t j = tid; j < nblocks; j += NT) {
        const uint64_t want = ld_relaxed_u64(&sizes[j]) + g.data_start;
        sizes[j] = 0;
        res[j].total = 0;
        res[j].overflow = 0;
        res[j].err_sq = 0;
        res[j].norm_sq = 0;
        reserve_slot(want, dev, host, &tgt[j], status);
    }
    if (tid == 0) *done_ctr = 0;
}

// In-place exact encoder, pass 1: one warp per frame encodes the frame over
// its own amplitudes (Im-plane words to im, F words per frame) and records
// its length and word counts; the last CTA turns the frame lengths into frame
// offsets, reserves each block's exact slot and folds the frames' error
// partials into the blocks' and the stage's totals.
// REL: the relative-bound format (e is the shift k, side records of kQszrSideBytes, mixed sign words counted
// in fmixed). Without a device arena (dev.bump null) the targets are the caller's and nothing is reserved; with
// keep_fitting (learned sizing) a block keeps the slot reserved for it beforehand when its exact size fits, and
// only a block whose prediction was too small gets an exact slot (counted as an overflowed block).
template <bool REL>
__global__ void __launch_bounds__(NT, 4) k_encode_ip(float2 *wv, uint32_t *__restrict__ im, uint32_t nblocks, int m,
                                                  int e, uint32_t *done_ctr, ArenaDev dev, ArenaDev host,
                                                  EncTarget *__restrict__ tgt, EncResult *__restrict__ res,
                                                  StageAccum *acc, uint8_t *__restrict__ wrec,
                                                  uint32_t *__restrict__ flen, uint32_t *__restrict__ fwords,
                                                  uint32_t *__restrict__ fmixed, uint32_t *__restrict__ foff,
                                                  float2 *__restrict__ part, int keep_fitting, int *status) {
    const FrameGeom g = geom(m);
    constexpr uint32_t kSide = REL ? kQszrSideBytes : 256u;
    __shared__ bool s_last;
    __shared__ double s_red[2][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t items = uint64_t(nblocks) * g.nframes;
    for (uint64_t item = uint64_t(blockIdx.x) * NW + warp; item < items; item += uint64_t(gridDim.x) * NW) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        uint32_t words, mixed;
        const uint32_t len = encode_frame_warp_ip<REL>(wv + (uint64_t(j) << m) + uint64_t(f) * g.F, im + item * g.F,
                                                       g, e, wrec + item * kSide, words, mixed, part + item, status);
        if (lane == 0) {
            flen[item] = len;
            fwords[item] = words;
            if (REL) fmixed[item] = mixed;
            __threadfence();  // the frame's records (and its error partial) before the CTA's arrival below
        }
    }
    // every warp of the CTA has written its frames' records before the CTA counts as arrived: the last CTA
    // reads all of them
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(done_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // warp per block: frame offsets = data_start + exclusive prefix of the frame lengths; exact slot;
    // the block's error sums in FP64
    double ta = 0, tb = 0;
    for (uint32_t jb = warp; jb < nblocks; jb += NW) {
        uint32_t run = uint32_t(g.data_start);
        double a = 0, b = 0;
        for (uint32_t f0 = 0; f0 < g.nframes; f0 += 32) {
            const uint64_t it = uint64_t(jb) * g.nframes + f0 + lane;
            const bool live = f0 + lane < g.nframes;
            const uint32_t v = live ? __ldcg(flen + it) : 0u;
            if (live) {
                const float2 pp = __ldcg(part + it);
                a += double(pp.x);
                b += double(pp.y);
            }
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            if (live) foff[it] = run + incl - v;
            run += __shfl_sync(kFull, incl, 31);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(kFull, a, o);
            b += __shfl_xor_sync(kFull, b, o);
        }
        if (lane == 0) {
            res[jb].total = 0;
            res[jb].overflow = 0;
            res[jb].err_sq = a;
            res[jb].norm_sq = b;
            if (dev.bump) {
                if (!keep_fitting) {
                    reserve_slot(run, dev, host, &tgt[jb], status);
                } else if (tgt[jb].ptr == nullptr || run > tgt[jb].cap) {
                    if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->overflow_blocks), 1ull);
                    reserve_slot(run, dev, host, &tgt[jb], status);
                }
            }
        }
        ta += a;
        tb += b;
    }
    if (lane == 0) {
        s_red[0][warp] = ta;
        s_red[1][warp] = tb;
    }
    __syncthreads();
    if (tid == 0) {
        if (acc) {
            double a = 0, b = 0;
            for (int w = 0; w < NW; ++w) { a += s_red[0][w]; b += s_red[1][w]; }
            atomicAdd(&acc->err_sq, a);
            atomicAdd(&acc->norm_sq, b);
        }
        *done_ctr = 0;
    }
}

// In-place exact encoder, pass 2: one warp per frame copies the frame's
// pieces to its offset in the block's slot.
template <bool REL>
__global__ void __launch_bounds__(NT) k_frame_copy(const float2 *__restrict__ wv, const uint32_t *__restrict__ im,
                                                   uint32_t nblocks, int m, int e, const EncTarget *__restrict__ tgt,
                                                   EncResult *__restrict__ res, const uint32_t *__restrict__ ids,
                                                   BlockSlot *__restrict__ table, StageAccum *acc,
                                                   const uint8_t *__restrict__ wrec, const uint32_t *__restrict__ flen,
                                                   const uint32_t *__restrict__ fwords,
                                                   const uint32_t *__restrict__ fmixed,
                                                   const uint32_t *__restrict__ foff) {
    const FrameGeom g = geom(m);
    constexpr uint32_t kSide = REL ? kQszrSideBytes : 256u;
    const int warp = threadIdx.x >> 5;
    const uint64_t items = uint64_t(nblocks) * g.nframes;
    for (uint64_t item = uint64_t(blockIdx.x) * NW + warp; item < items; item += uint64_t(gridDim.x) * NW) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        copy_frame_warp<REL>(reinterpret_cast<const uint32_t *>(wv + (uint64_t(j) << m) + uint64_t(f) * g.F),
                             im + item * g.F, wrec + item * kSide, fwords[item], REL ? fmixed[item] : 0u, flen[item],
                             foff[item], g, m, e, f, tgt[j], res + j, table ? table + ids[j] : nullptr, acc);
    }
}

// ---------------------------------------------------------------------------
// Slot reservation from the two-tier pool: device arena first, then the
// pinned host arena. need[j] bytes (plus the fixed header/offsets part when
// add_data_start is set); the slot is padded to 256 bytes.
// ---------------------------------------------------------------------------
__global__ void k_reserve(uint32_t nblocks, const uint64_t *__restrict__ need, uint64_t add_const,
                          const float *__restrict__ pred_log2, double margin, uint64_t worst,
                          ArenaDev dev, ArenaDev host, EncTarget *__restrict__ tgt, EncResult *__restrict__ res,
                          int retry_overflowed, int *status) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nblocks) return;
    uint64_t want;
    if (retry_overflowed) {
        if (res[j].overflow == 0) return;
        want = res[j].total;
    } else if (pred_log2) {
        double p = double(pred_log2[j]);
        p = p < 0 ? 0 : (p > 40 ? 40 : p);
        double b = exp2(p) * (1.0 + margin);
        want = b >= double(worst) ? worst : uint64_t(b);
    } else {
        want = (need ? need[j] : 0) + add_const;
    }
    if (!retry_overflowed) {
        res[j].total = 0;
        res[j].overflow = 0;
        res[j].err_sq = 0;
        res[j].norm_sq = 0;
    }
    reserve_slot(want, dev, host, &tgt[j], status);
}

// Raw (uncompressed) store: copy blocks, 16 bytes per thread.
__global__ void k_copy_blocks_out(const float2 *__restrict__ wv, uint32_t nblocks, int m,
                                  const EncTarget *__restrict__ tgt, const uint32_t *__restrict__ ids,
                                  BlockSlot *__restrict__ table, StageAccum *acc, int *status) {
    const uint64_t per = (8ull << m) / 16;
    const uint64_t total = per * nblocks;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t j = uint32_t(i / per);
        const uint64_t o = i % per;
        if (tgt[j].ptr == nullptr || tgt[j].cap < (8ull << m)) continue;
        reinterpret_cast<float4 *>(tgt[j].ptr)[o] = reinterpret_cast<const float4 *>(wv + (uint64_t(j) << m))[o];
        if (o == 0) {
            table[ids[j]].ptr = tgt[j].ptr;
            table[ids[j]].bytes = 8ull << m;
            table[ids[j]].tier = tgt[j].tier;
            if (acc) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), 8ull << m);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->reserved_bytes), tgt[j].cap);
                if (tgt[j].tier) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->host_bytes), tgt[j].cap);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->blocks), 1ull);
            }
        }
    }
}

__global__ void k_copy_blocks_in(const BlockRef *__restrict__ in, uint32_t nblocks, int m, float2 *__restrict__ wv,
                                 int *status) {
    const uint64_t per = (8ull << m) / 16;
    const uint64_t total = per * nblocks;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t j = uint32_t(i / per);
        const uint64_t o = i % per;
        if (in[j].ptr == nullptr || in[j].bytes < (8ull << m)) {
            if (o == 0) raise_status(status, QSIM_E_CORRUPT);
            continue;
        }
        reinterpret_cast<float4 *>(wv + (uint64_t(j) << m))[o] = reinterpret_cast<const float4 *>(in[j].ptr)[o];
    }
}

// Gather the input block references of one group from the block table.
__global__ void k_gather_refs(const BlockSlot *__restrict__ table, const uint32_t *__restrict__ ids, uint32_t count,
                              BlockRef *__restrict__ out) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) {
        out[j].ptr = table[ids[j]].ptr;
        out[j].bytes = table[ids[j]].bytes;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned grid_for(uint64_t items, unsigned cap) {
    return unsigned(items < cap ? (items ? items : 1) : cap);
}

void launch_decode(const BlockRef *in, uint32_t nblocks, int m, float2 *wv, uint32_t *hist, int *status,
                   cudaStream_t s, bool rel) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    const unsigned grid = grid_for((items + NW - 1) / NW, 152 * 8);
    if (rel)
        k_decode<0, true><<<grid, NT, 0, s>>>(in, nullptr, nullptr, nblocks, m, wv, hist, status, PreOps{});
    else
        k_decode<0, false><<<grid, NT, 0, s>>>(in, nullptr, nullptr, nblocks, m, wv, hist, status, PreOps{});
    count_launch();
}

template <bool REL>
static void decode_table(const BlockSlot *table, const uint32_t *ids, uint32_t nblocks, int m, float2 *wv,
                         uint32_t *hist, int *status, const PreOps &pre, cudaStream_t s) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    const unsigned grid = grid_for((items + NW - 1) / NW, 152 * 8);
    if (pre.count == 0)
        k_decode<0, REL><<<grid, NT, 0, s>>>(nullptr, table, ids, nblocks, m, wv, hist, status, pre);
    else if (pre.count <= 2)
        k_decode<2, REL><<<grid, NT, 0, s>>>(nullptr, table, ids, nblocks, m, wv, hist, status, pre);
    else
        k_decode<kMaxPreOps, REL><<<grid, NT, 0, s>>>(nullptr, table, ids, nblocks, m, wv, hist, status, pre);
}

void launch_decode_frames(const BlockSlot *table, const uint2 *frames, uint32_t nitems, int m, float2 *out,
                          int *status, cudaStream_t s, bool rel) {
    const unsigned grid = grid_for((uint64_t(nitems) + NW - 1) / NW, 152 * 8);
    if (rel)
        k_decode_frames<true><<<grid, NT, 0, s>>>(table, frames, nitems, m, out, status);
    else
        k_decode_frames<false><<<grid, NT, 0, s>>>(table, frames, nitems, m, out, status);
    count_launch();
}

void launch_decode_table(const BlockSlot *table, const uint32_t *ids, uint32_t nblocks, int m, float2 *wv,
                         uint32_t *hist, int *status, const PreOps &pre, cudaStream_t s, bool rel) {
    if (rel)
        decode_table<true>(table, ids, nblocks, m, wv, hist, status, pre, s);
    else
        decode_table<false>(table, ids, nblocks, m, wv, hist, status, pre, s);
    count_launch();
}

void launch_encode(const float2 *wv, uint32_t nblocks, int m, int e, const EncTarget *tgt, EncResult *res,
                   int only_overflowed, const uint32_t *ids, BlockSlot *table, StageAccum *acc,
                   const LookbackScratch &scr, int *status, cudaStream_t s) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    k_encode<<<unsigned(items), NT, 0, s>>>(wv, nblocks, m, e, tgt, res, only_overflowed, ids, table, acc, scr,
                                             status);
    count_launch();
}


void launch_size_reserve(const float2 *wv, uint32_t nblocks, int m, int e, uint64_t *sizes, uint32_t *done_ctr,
                         const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt, EncResult *res, int *status,
                         cudaStream_t s) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    k_encode_size<<<grid_for(items, 152 * 8), NT, 0, s>>>(wv, nblocks, m, e, sizes, done_ctr, dev, host, tgt, res,
                                                           status);
    count_launch();
}


void launch_encode_ip(float2 *wv, uint32_t *im, uint32_t nblocks, int m, int e, uint32_t *done_ctr,
                      const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt, EncResult *res, StageAccum *acc,
                      uint8_t *wrec, uint32_t *flen, uint32_t *fwords, uint32_t *foff, float2 *part, int *status,
                      cudaStream_t s, bool rel, uint32_t *fmixed, bool keep_fitting) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    const unsigned grid = grid_for((items + NW - 1) / NW, 152 * 8);
    if (rel)
        k_encode_ip<true><<<grid, NT, 0, s>>>(wv, im, nblocks, m, e, done_ctr, dev, host, tgt, res, acc, wrec, flen,
                                              fwords, fmixed, foff, part, keep_fitting ? 1 : 0, status);
    else
        k_encode_ip<false><<<grid, NT, 0, s>>>(wv, im, nblocks, m, e, done_ctr, dev, host, tgt, res, acc, wrec, flen,
                                               fwords, fmixed, foff, part, keep_fitting ? 1 : 0, status);
    count_launch();
}
void launch_frame_copy(const float2 *wv, const uint32_t *im, uint32_t nblocks, int m, int e, const EncTarget *tgt,
                       EncResult *res, const uint32_t *ids, BlockSlot *table, StageAccum *acc, const uint8_t *wrec,
                       const uint32_t *flen, const uint32_t *fwords, const uint32_t *foff, cudaStream_t s, bool rel,
                       const uint32_t *fmixed) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    const unsigned grid = grid_for((items + NW - 1) / NW, 152 * 16);
    if (rel)
        k_frame_copy<true><<<grid, NT, 0, s>>>(wv, im, nblocks, m, e, tgt, res, ids, table, acc, wrec, flen, fwords,
                                               fmixed, foff);
    else
        k_frame_copy<false><<<grid, NT, 0, s>>>(wv, im, nblocks, m, e, tgt, res, ids, table, acc, wrec, flen, fwords,
                                                fmixed, foff);
    count_launch();
}

void launch_reserve(uint32_t nblocks, const uint64_t *need, uint64_t add_const, const float *pred_log2,
                    double margin, uint64_t worst, const ArenaDev &dev, const ArenaDev &host, EncTarget *tgt,
                    EncResult *res, int retry_overflowed, int *status, cudaStream_t s) {
    k_reserve<<<(nblocks + 127) / 128, 128, 0, s>>>(nblocks, need, add_const, pred_log2, margin, worst, dev, host,
                                                    tgt, res, retry_overflowed, status);
    count_launch();
}

void launch_copy_out(const float2 *wv, uint32_t nblocks, int m, const EncTarget *tgt, const uint32_t *ids,
                     BlockSlot *table, StageAccum *acc, int *status, cudaStream_t s) {
    const uint64_t items = (uint64_t(nblocks) << m) / 2;
    k_copy_blocks_out<<<grid_for((items + 255) / 256, 152 * 16), 256, 0, s>>>(wv, nblocks, m, tgt, ids, table, acc,
                                                                            status);
    count_launch();
}

void launch_copy_in(const BlockRef *in, uint32_t nblocks, int m, float2 *wv, int *status, cudaStream_t s) {
    const uint64_t items = (uint64_t(nblocks) << m) / 2;
    k_copy_blocks_in<<<grid_for((items + 255) / 256, 152 * 16), 256, 0, s>>>(in, nblocks, m, wv, status);
    count_launch();
}

void launch_gather_refs(const BlockSlot *table, const uint32_t *ids, uint32_t count, BlockRef *out, cudaStream_t s) {
    k_gather_refs<<<(count + 127) / 128, 128, 0, s>>>(table, ids, count, out);
    count_launch();
}

}  // namespace qsim
