// Device functions of the QSZ1 codec (shared by the codec kernels and the
// persistent stage kernel). The format and the method are described in codec.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"

namespace qsim {
namespace cdev {


constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int NW = NT / 32;
constexpr int MAX_C = 128;       // chunks per plane per frame (F = 4096)
constexpr int MAX_CPW = MAX_C / NW;  // chunk pairs per warp
constexpr uint32_t kFlagA = 1u, kFlagP = 2u;
constexpr uint32_t kEpochMask = (1u << 30) - 1;
constexpr long long kSpinLimit = 1ll << 22;
constexpr uint64_t kLookbackWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t lb_word(uint32_t epoch, uint32_t flag, uint32_t value) {
    return (uint64_t(epoch & kEpochMask) << 34) | (uint64_t(flag) << 32) | value;
}

struct FrameGeom {
    int fl;
    uint32_t F, C, nframes;
    uint64_t data_start;
};

__device__ __forceinline__ FrameGeom geom(int m) {
    FrameGeom g;
    g.fl = m < 12 ? m : 12;
    g.F = 1u << g.fl;
    g.C = g.F / 32;
    g.nframes = 1u << (m - g.fl);
    g.data_start = 32 + ((4ull * (g.nframes + 1) + 15) & ~15ull);
    return g;
}

// QSZR (relative bound): per-frame side record of the in-place encoder (widths at 0, sign chunk types at
// kSideTypes, Re and Im stored sign words at kSideMixRe / kSideMixIm, Re and Im run records (u16) at
// kSideRunRe / kSideRunIm) and the code range (|x| < 2^64)
constexpr uint32_t kSideTypes = 256, kSideMixRe = 320, kSideMixIm = 832, kSideRunRe = 1344, kSideRunIm = 1600;
constexpr uint32_t kQszrMaxU = 0x5F800000u;

// sign chunk type: 0 all clear, 1 all set (Algorithm 2's pre-scan), 3 run-coded (the signs change 1 to 3 times
// between neighbours), 2 stored word
__device__ __forceinline__ uint32_t sign_type(uint32_t w) {
    if (w == 0u) return 0u;
    if (w == 0xFFFFFFFFu) return 1u;
    return __popc((w ^ (w >> 1)) & 0x7FFFFFFFu) <= 3 ? 3u : 2u;
}

// run record of a run-coded sign word: bit 15 = sign of value 0, bits 0-4 / 5-9 / 10-14 the run boundaries
// p1 < p2 < p3 (value p differs from value p - 1), unused fields zero
__device__ __forceinline__ uint32_t sign_run_record(uint32_t w) {
    uint32_t t = (w ^ (w >> 1)) & 0x7FFFFFFFu;
    const uint32_t p1 = __ffs(t);
    t &= t - 1u;
    const uint32_t p2 = __ffs(t);
    t &= t - 1u;
    const uint32_t p3 = __ffs(t);
    return ((w & 1u) << 15) | p1 | (p2 << 5) | (p3 << 10);
}

// sign word of a run record; ok false for a record no encoder writes
__device__ __forceinline__ uint32_t sign_run_word(uint32_t rec, bool &ok) {
    const uint32_t p1 = rec & 31u, p2 = (rec >> 5) & 31u, p3 = (rec >> 10) & 31u;
    ok = p1 != 0u && (p2 == 0u ? p3 == 0u : (p2 > p1 && (p3 == 0u || p3 > p2)));
    uint32_t w = (rec >> 15) ? 0xFFFFFFFFu : 0u;
    if (p1) w ^= 0xFFFFFFFFu << p1;
    if (p2) w ^= 0xFFFFFFFFu << p2;
    if (p3) w ^= 0xFFFFFFFFu << p3;
    return w;
}

// packed sign-section counts of a frame: stored words Re | Im << 8, run records Re << 16 | Im << 24
__device__ __forceinline__ uint32_t sign_section_bytes(uint32_t mixed) {
    const uint32_t nw = (mixed & 0xffu) + ((mixed >> 8) & 0xffu), nr = ((mixed >> 16) & 0xffu) + (mixed >> 24);
    return (4u * nw + 2u * nr + 15u) & ~15u;
}

__device__ __forceinline__ uint32_t zigzag(int32_t d) {
    return (uint32_t(d) << 1) ^ uint32_t(d >> 31);
}

__device__ __forceinline__ int32_t unzigzag(uint32_t z) {
    return int32_t((z >> 1) ^ (0u - (z & 1u)));
}

// ---------------------------------------------------------------------------
// Decode: one CTA per frame (grid-stride over all frames of all blocks).
// ---------------------------------------------------------------------------
// Leading phase ops of a stage, applied by the decoder. The phase index of a
// diagonal op splits into bits fixed for the frame (working bits >= the frame
// log, and outer qubits from the group), the lane's bits 0..4 and the chunk's
// bits 5.. ; the host builds the lane and chunk parts as byte tables (32 + 128
// bytes at float2 offset op.dlut of the phase area). pre_setup gives each op
// its launch-wide table offsets (shared memory), pre_frame its per-lane
// register for the frame, and pre_chunk applies the ops to one chunk's
// amplitude.
constexpr uint32_t kPreFlip = 0xFFFFFFFFu;  // pre_ab[o].y of a phase flip
constexpr uint32_t kPreNone = 0xFFFFFFFFu;  // register of a flip whose amplitude is not in this lane

// ab.x: byte offset of a diagonal op's chunk table in the phase area; ab.y: float2 offset of its phase
// table, or kPreFlip for a phase flip.
__device__ __forceinline__ uint2 pre_setup(const OpDev &op) {
    return op.type == OP_DIAG ? make_uint2(uint32_t(op.dlut) * 8u + 32u, uint32_t(op.mat)) : make_uint2(0u, kPreFlip);
}

// Per-lane register of each op for the frame whose first working index is w0f: a diagonal op's frame
// and lane bits of the phase index; for a phase flip, the chunk of the marked amplitude in the lane that
// holds it (kPreNone elsewhere).
template <int NP>
__device__ __forceinline__ void pre_frame(uint32_t (&cl)[NP > 0 ? NP : 1], const OpDev *ops, uint32_t nops,
                                          uint64_t w0f, uint32_t fl, uint32_t lane, uint64_t gb,
                                          const float2 *__restrict__ mats) {
#pragma unroll
    for (int o = 0; o < NP; ++o) {
        cl[o] = kPreNone;
        if (uint32_t(o) >= nops) continue;
        const OpDev &op = ops[o];
        if (op.type == OP_DIAG) {
            uint32_t idx = 0;
            for (uint32_t j = 0; j < op.k; ++j) {
                const uint32_t src = op.dsrc[j];
                if (src < fl) continue;
                const uint64_t bit = src < 64 ? (w0f >> src) & 1ull : (gb >> (src - 64)) & 1ull;
                idx |= uint32_t(bit) << j;
            }
            cl[o] = idx | __ldg(reinterpret_cast<const uint8_t *>(mats + op.dlut) + lane);
        } else if (op.basis_in_stage && gb == op.basis_outer && op.basis_w >= w0f &&
                   op.basis_w - w0f < (uint64_t(1) << fl)) {
            const uint32_t off = uint32_t(op.basis_w - w0f);
            if ((off & 31u) == lane) cl[o] = off >> 5;
        }
    }
}

template <int NP>
__device__ __forceinline__ float2 pre_chunk(float2 v, const uint32_t (&cl)[NP > 0 ? NP : 1], const uint2 *pre_ab,
                                            uint32_t nops, uint32_t c, const float2 *__restrict__ mats) {
#pragma unroll
    for (int o = 0; o < NP; ++o) {
        if (uint32_t(o) >= nops) break;
        const uint2 ab = pre_ab[o];
        if (ab.y != kPreFlip) {
            const uint32_t idx = cl[o] | __ldg(reinterpret_cast<const uint8_t *>(mats) + ab.x + c);
            const float2 ph = __ldg(mats + ab.y + idx);
            v = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
        } else if (c == cl[o]) {
            v = make_float2(-v.x, -v.y);
        }
    }
    return v;
}

// Decode frame f of one block with one warp, no block-wide barriers: the warp reads the header and
// the frame's offsets with one load per lane, the 2C width bytes with one
// 8-byte load per lane (lane l holds the widths of chunks 8l..8l+7), builds
// the chunk offsets with a warp prefix sum, then decodes the chunk pairs
// (Re chunk c, Im chunk c) eight at a time with all sixteen payload loads in
// flight: bit-plane transpose, zigzag inverse, inclusive prefix sum (the
// Lorenzo inverse), x' = q * 2^e, interleaved (re, im) stores. With REL the
// stream is QSZR: the header's exponent byte is the shift k, the frame adds
// the sign chunk types (lanes 0.. hold the types of chunks 16l..16l+15, the
// mixed chunks ranked by a warp prefix sum) and the mixed sign words, and
// x' = +-float(bits q << k).
template <int NP, bool CG = false, bool REL = false>
__device__ __forceinline__ void decode_frame_warp(const uint8_t *sp, uint64_t bytes, const FrameGeom &g, int m,
                                                  uint32_t f, float2 *__restrict__ dst, uint32_t *hist_j,
                                                  uint32_t *s_hist_w, int *status, const OpDev *pre_ops,
                                                  const uint2 *pre_ab, uint32_t npre,
                                                  const float2 *__restrict__ mats, uint64_t wbase,
                                                  uint64_t gb) {
    const int lane = threadIdx.x & 31;
    const uint32_t padw = (2u * g.C + 15u) & ~15u;
    if (hist_j) s_hist_w[lane] = 0;
    // ---- header and offsets: one load per lane ----
    const bool can = sp != nullptr && !(reinterpret_cast<uintptr_t>(sp) & 15) && bytes >= g.data_start;
    uint32_t hv = 0;
    if (can) {
        const uint32_t *h32 = reinterpret_cast<const uint32_t *>(sp);
        if (lane < 8) hv = h32[lane];
        else if (lane == 8) hv = h32[8];                    // offsets[0]
        else if (lane == 9) hv = h32[8 + f];                // offsets[f]
        else if (lane == 10) hv = h32[8 + f + 1];           // offsets[f+1]
        else if (lane == 11) hv = h32[8 + g.nframes];       // offsets[nframes]
    }
    const uint32_t magic = __shfl_sync(kFull, hv, 0), w1 = __shfl_sync(kFull, hv, 1);
    const uint32_t w2 = __shfl_sync(kFull, hv, 2), nfr = __shfl_sync(kFull, hv, 3);
    const uint64_t total = uint64_t(__shfl_sync(kFull, hv, 4)) | (uint64_t(__shfl_sync(kFull, hv, 5)) << 32);
    const uint64_t rsv = uint64_t(__shfl_sync(kFull, hv, 6)) | (uint64_t(__shfl_sync(kFull, hv, 7)) << 32);
    const uint32_t o0 = __shfl_sync(kFull, hv, 8), fa = __shfl_sync(kFull, hv, 9);
    const uint32_t fb = __shfl_sync(kFull, hv, 10), on = __shfl_sync(kFull, hv, 11);
    const int e = REL ? int(uint8_t(w2 >> 16)) : int(int8_t(uint8_t(w2 >> 16)));
    const uint32_t tbp = REL ? ((((2u * g.C + 3u) / 4u) + 15u) & ~15u) : 0u;  // sign chunk types, padded
    bool ok = can && magic == (REL ? kQszrMagic : kQszMagic) && w1 == 1u && (w2 & 0xff) == uint32_t(m) &&
              ((w2 >> 8) & 0xff) == uint32_t(g.fl) && (w2 >> 24) == 0 && nfr == g.nframes && rsv == 0 &&
              (REL ? (e >= kQszrKMin && e <= kQszrKMax) : (e >= kQszEMin && e <= kQszEMax)) && total <= bytes &&
              total >= g.data_start && o0 == g.data_start && on == total && fb >= fa && fb <= total &&
              fa >= g.data_start && !((fa | fb) & 15u) && (fb == fa || fb - fa >= padw + tbp);
    uint32_t wsum = 0, wmax = 0;
    uint2 wb = make_uint2(0, 0);
    uint32_t base_off = 0;
    uint32_t tw = 0, mbase = 0, nmix = 0, rbase = 0, nrun = 0;  // REL: sign chunk types of chunks 16 lane..,
                                                                 // ranks of stored words and run records
    if (ok && fb > fa) {
        // ---- widths: lane l holds chunks 8l .. 8l+7 (Re chunks 0..C-1, then Im chunks) ----
        if (8u * lane < 2u * g.C) wb = *reinterpret_cast<const uint2 *>(sp + fa + 8u * lane);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t a = (wb.x >> (8 * t)) & 0xff, b = (wb.y >> (8 * t)) & 0xff;
            wsum += a + b;
            wmax = max(wmax, max(a, b));
        }
        uint32_t incl = wsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        base_off = incl - wsum;
        const uint32_t words = __shfl_sync(kFull, incl, 31);
        const uint32_t maxw = __reduce_max_sync(kFull, wmax);
        if constexpr (REL) {
            if (16u * uint32_t(lane) < 2u * g.C) tw = *reinterpret_cast<const uint32_t *>(sp + fa + padw + 4u * lane);
            // odd bit of each 2-bit type: set for types 2 (stored word) and 3 (run record)
            const uint32_t hi = tw & 0xAAAAAAAAu, t3 = hi & (tw << 1);
            const uint32_t c2 = __popc(hi ^ t3), c3 = __popc(t3);
            uint32_t mi = c2, ri = c3;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, mi, o), u = __shfl_up_sync(kFull, ri, o);
                if (lane >= o) {
                    mi += t;
                    ri += u;
                }
            }
            mbase = mi - c2;
            rbase = ri - c3;
            nmix = __shfl_sync(kFull, mi, 31);
            nrun = __shfl_sync(kFull, ri, 31);
        }
        ok = maxw <= 32 && words > 0 &&
             uint64_t(fb - fa) == padw + tbp + ((4ull * nmix + 2ull * nrun + 15) & ~15ull) +
                                      ((4ull * words + 15) & ~15ull);
    }
    if (!ok) {
        if (lane == 0) raise_status(status, QSIM_E_CORRUPT);
    }
    if (!ok || fb == fa) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);  // F >= 32 amplitudes, 16-byte aligned
        for (uint32_t i = lane; i < g.F / 2; i += 32) d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (hist_j && lane == 0) atomicAdd(&hist_j[0], 2 * g.F);
        return;
    }
    const uint32_t *mixw = reinterpret_cast<const uint32_t *>(sp + fa + padw + tbp);
    const uint16_t *runw = reinterpret_cast<const uint16_t *>(sp + fa + padw + tbp + 4u * nmix);
    const uint32_t *payload = reinterpret_cast<const uint32_t *>(
        sp + fa + padw + tbp + (REL ? ((4u * nmix + 2u * nrun + 15u) & ~15u) : 0u));
    const float step = REL ? 0.f : exp2i(e);
    bool qbad = false;
    uint32_t pre[NP > 0 ? NP : 1];
    if (NP > 0 && npre) pre_frame<NP>(pre, pre_ops, npre, wbase | (uint64_t(f) * g.F), g.fl, lane, gb, mats);
    // ---- chunk pairs, eight at a time ----
    for (uint32_t c0 = 0; c0 < g.C; c0 += 8) {
        // widths/offsets of Re chunks c0.. (owner lane c0/8) and Im chunks C+c0.. (owner (C+c0)/8)
        const uint32_t lr = c0 >> 3, li = (g.C + c0) >> 3;
        const uint2 wr8 = make_uint2(__shfl_sync(kFull, wb.x, lr), __shfl_sync(kFull, wb.y, lr));
        const uint2 wi8 = make_uint2(__shfl_sync(kFull, wb.x, li), __shfl_sync(kFull, wb.y, li));
        uint32_t offr = __shfl_sync(kFull, base_off, lr), offi = __shfl_sync(kFull, base_off, li);
        // Im chunks of a small frame (C < 8) share the owner lane with the Re chunks: skip those slots
        const uint32_t si0 = (g.C + c0) & 7u;
        uint32_t xr[8], xi[8], wr[8], wi[8];
        // REL: sign chunk types of this batch (owners c0/16 and (C+c0)/16) and the mixed ranks before them
        uint32_t twr = 0, twi = 0, mbr = 0, mbi = 0, rbr = 0, rbi = 0;
        if constexpr (REL) {
            twr = __shfl_sync(kFull, tw, c0 >> 4);
            mbr = __shfl_sync(kFull, mbase, c0 >> 4);
            rbr = __shfl_sync(kFull, rbase, c0 >> 4);
            twi = __shfl_sync(kFull, tw, (g.C + c0) >> 4);
            mbi = __shfl_sync(kFull, mbase, (g.C + c0) >> 4);
            rbi = __shfl_sync(kFull, rbase, (g.C + c0) >> 4);
        }
        {
            uint32_t sr_ = 0, si_ = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const uint32_t ar = t < 4 ? (wr8.x >> (8 * t)) & 0xff : (wr8.y >> (8 * (t - 4))) & 0xff;
                const uint32_t ti = si0 + t;
                const uint32_t ai = ti < 8 ? (ti < 4 ? (wi8.x >> (8 * ti)) & 0xff : (wi8.y >> (8 * (ti - 4))) & 0xff) : 0;
                wr[t] = ar;
                wi[t] = ai;
            }
            // offsets of the Im chunks start after the skipped slots of their owner lane
            for (uint32_t t = 0; t < si0; ++t)
                offi += t < 4 ? (wi8.x >> (8 * t)) & 0xff : (wi8.y >> (8 * (t - 4))) & 0xff;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const bool live = c0 + t < g.C;
                if (wr[t] <= 16 && wi[t] <= 16) {
                    // packed: lane b < 16 loads Re plane b, lane 16 + b Im plane b (one transpose below)
                    const uint32_t b = uint32_t(lane) & 15u;
                    xr[t] = (live && b < (lane < 16 ? wr[t] : wi[t]))
                                ? __ldg(payload + (lane < 16 ? offr + sr_ : offi + si_) + b)
                                : 0u;
                    xi[t] = 0u;
                } else {
                    xr[t] = (live && lane < int(wr[t])) ? __ldg(payload + offr + sr_ + lane) : 0u;
                    xi[t] = (live && lane < int(wi[t])) ? __ldg(payload + offi + si_ + lane) : 0u;
                }
                sr_ += wr[t];
                si_ += wi[t];
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            if (c >= g.C) break;
            uint32_t zr, zi;
            if (wr[t] <= 16 && wi[t] <= 16) {
                const uint32_t y = warp_bit_transpose(xr[t], lane);
                zr = y & 0xffffu;
                zi = y >> 16;
            } else {
                zr = warp_bit_transpose(xr[t], lane);
                zi = warp_bit_transpose(xi[t], lane);
            }
            uint32_t qr = uint32_t(unzigzag(zr)), qi = uint32_t(unzigzag(zi));
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t tr = __shfl_up_sync(kFull, qr, o);
                const uint32_t ti = __shfl_up_sync(kFull, qi, o);
                if (lane >= o) { qr += tr; qi += ti; }
            }
            float2 v;
            if constexpr (REL) {
                // sign words: all clear, all set, the chunk's stored word (its rank among the type-2 chunks) or
                // the word of its run record (its rank among the type-3 chunks)
                const uint32_t pr = 2u * (c & 15u), pi = 2u * ((g.C + c) & 15u);
                const uint32_t tr = (twr >> pr) & 3u, ti = (twi >> pi) & 3u;
                const uint32_t t3r = twr & 0xAAAAAAAAu & (twr << 1), t3i = twi & 0xAAAAAAAAu & (twi << 1);
                const uint32_t t2r = (twr & 0xAAAAAAAAu) ^ t3r, t2i = (twi & 0xAAAAAAAAu) ^ t3i;
                uint32_t swr = tr == 1u ? 0xFFFFFFFFu : 0u, swi = ti == 1u ? 0xFFFFFFFFu : 0u;
                if (tr == 2u) swr = __ldg(mixw + mbr + __popc(t2r & ((1u << pr) - 1u)));
                if (ti == 2u) swi = __ldg(mixw + mbi + __popc(t2i & ((1u << pi) - 1u)));
                if (tr == 3u) {
                    bool rok;
                    swr = sign_run_word(__ldg(runw + rbr + __popc(t3r & ((1u << pr) - 1u))), rok);
                    qbad |= !rok;
                }
                if (ti == 3u) {
                    bool rok;
                    swi = sign_run_word(__ldg(runw + rbi + __popc(t3i & ((1u << pi) - 1u))), rok);
                    qbad |= !rok;
                }
                qbad |= qr > (kQszrMaxU >> e) || qi > (kQszrMaxU >> e);
                const float mr = __uint_as_float(qr << e), mi = __uint_as_float(qi << e);
                v = make_float2(((swr >> lane) & 1u) ? -mr : mr, ((swi >> lane) & 1u) ? -mi : mi);
            } else {
                const int32_t sr = int32_t(qr), si = int32_t(qi);
                v = make_float2(float(sr) * step, float(si) * step);
            }
            if (NP > 0 && npre) v = pre_chunk<NP>(v, pre, pre_ab, npre, c, mats);
            dst[c * 32 + lane] = v;
            if (hist_j && lane == 0) {  // the chunk's code widths, 32 values each
                atomicAdd(&s_hist_w[min(wr[t], 31u)], 32u);
                atomicAdd(&s_hist_w[min(wi[t], 31u)], 32u);
            }
        }
    }
    if (REL && __any_sync(kFull, qbad) && lane == 0) raise_status(status, QSIM_E_CORRUPT);
    if (hist_j) {
        __syncwarp();
        const uint32_t v = s_hist_w[lane];
        if (v) atomicAdd(&hist_j[lane], v);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Encode: one CTA per frame, ticket-ordered, decoupled look-back. The frame
// image (widths, then bit-plane words) is assembled in shared memory while
// warp 0 finds the frame's byte offset, then copied out with 16-byte stores.
// The bit planes of a chunk, W_b = ballot(bit b of z_j), are produced for all
// b at once by a 32x32 bit transpose across the warp (five shuffle stages).
// ---------------------------------------------------------------------------
constexpr uint32_t kStageWords = (256 + 8 * 4096) / 4 + 4;  // widths + worst-case payload + pad

// Shared memory of the frame encoder.
struct EncSmem {
    uint32_t w[2 * MAX_C];
    uint32_t off[2 * MAX_C];
    uint32_t warp_sums[NW];
    uint32_t total;
    uint64_t excl;
    double red[2][NW];
};

// Encode frame f of one block with the whole CTA (NT threads): src is the
// frame's amplitudes, lb_block the block's look-back words, tgt its slot,
// s_stage kStageWords words of shared memory for the frame image.
template <bool CG = false>
__device__ __forceinline__ void encode_frame_cta(const float2 *__restrict__ src, const FrameGeom &g, int m, int e,
                                                 uint32_t f, uint64_t *lb_block, uint32_t epoch, EncTarget tgt,
                                                 EncResult *res_j, BlockSlot *table_slot, StageAccum *acc,
                                                 float2 *part_item, int only_overflowed, uint32_t *s_stage,
                                                 EncSmem &SE, int *status) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *s_w = SE.w, *s_off = SE.off, *s_warp = SE.warp_sums;
    uint32_t &s_total = SE.total;
    uint64_t &s_excl = SE.excl;
    double (&s_red)[2][NW] = SE.red;
    const float inv_step = exp2i(-e);
    const float step = exp2i(e);
    // x - x' is exact in FP32 (|x - x'| <= s/2 <= |x'|/2 when q != 0, x' = 0 otherwise), so the
    // per-thread sums are FP32 and only the per-CTA totals are accumulated in FP64
    float err_sq = 0.f, norm_sq = 0.f;
    int bad = 0;
    float2 vin[MAX_CPW];
#pragma unroll
    for (int i = 0; i < MAX_CPW; ++i) {
        const uint32_t c = warp + i * NW;
        vin[i] = c < g.C ? (CG ? __ldcg(src + c * 32 + lane) : __ldcs(src + c * 32 + lane)) : make_float2(0.f, 0.f);
    }
    uint32_t zr[MAX_CPW], zi[MAX_CPW];
#pragma unroll
    for (int i = 0; i < MAX_CPW; ++i) {
        zr[i] = zi[i] = 0;
        const uint32_t c = warp + i * NW;
        if (c < g.C) {
            int32_t q[2];
            const float x[2] = {vin[i].x, vin[i].y};
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (!isfinite(x[p])) {
                    bad = QSIM_E_INVALID;
                    q[p] = 0;
                } else {
                    const float t = x[p] * inv_step;  // exact: power-of-two scaling
                    if (fabsf(t) >= 1073741824.0f) {
                        bad = bad ? bad : QSIM_E_RANGE;
                        q[p] = 0;
                    } else {
                        q[p] = __float2int_rn(t);
                    }
                }
                const float xr = float(q[p]) * step;
                const float dx = x[p] - xr;
                err_sq = fmaf(dx, dx, err_sq);
                norm_sq = fmaf(xr, xr, norm_sq);
            }
            const int32_t pr = __shfl_up_sync(kFull, q[0], 1);
            const int32_t pi = __shfl_up_sync(kFull, q[1], 1);
            zr[i] = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
            zi[i] = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
            const uint32_t wr = 32 - __clz(__reduce_or_sync(kFull, zr[i]));
            const uint32_t wi = 32 - __clz(__reduce_or_sync(kFull, zi[i]));
            if (lane == 0) {
                s_w[c] = wr;
                s_w[g.C + c] = wi;
            }
        }
    }
    if (bad) raise_status(status, bad);
    __syncthreads();
    const uint32_t my_w = tid < int(2 * g.C) ? s_w[tid] : 0;
    const uint32_t my_off = block_exclusive_scan<NT>(my_w, s_warp, &s_total);
    const uint32_t padw = (2u * g.C + 15u) & ~15u;
    if (tid < int(2 * g.C)) s_off[tid] = my_off;
    // width bytes (and their zero padding) at the head of the frame image
    if (tid < int(padw) / 4) {
        uint32_t wbytes = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t x = 4 * tid + t;
            wbytes |= (x < 2 * g.C ? s_w[x] : 0u) << (8 * t);
        }
        s_stage[tid] = wbytes;
    }
    const uint32_t words = s_total;
    const uint32_t len = words ? uint32_t(padw + ((4ull * words + 15) & ~15ull)) : 0u;
    __syncthreads();

    // ---- warp 0: decoupled look-back over the preceding frames of this block ----
    if (warp == 0) {
        uint64_t *st = lb_block;
        if (f == 0) {
            if (lane == 0) {
                st_relaxed_u64(st, lb_word(epoch, kFlagP, len));
                s_excl = 0;
            }
        } else {
            if (lane == 0) st_relaxed_u64(st + f, lb_word(epoch, kFlagA, len));
            uint64_t excl = 0;
            int64_t end = int64_t(f) - 1;
            bool timed_out = false;
            while (true) {
                const int64_t p = end - lane;
                uint32_t flag = kFlagP, val = 0;
                if (p >= 0) {
                    long long spins = 0;
                    const uint64_t t0 = global_ns();
                    while (true) {
                        const uint64_t w = ld_relaxed_u64(st + p);
                        const uint32_t fl = uint32_t(w >> 32) & 3u;
                        if (fl != 0 && uint32_t(w >> 34) == epoch) {
                            flag = fl;
                            val = uint32_t(w);
                            break;
                        }
                        if (++spins > kSpinLimit || global_ns() - t0 > kLookbackWaitNs) {
                            timed_out = true;
                            flag = kFlagP;
                            val = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                const uint32_t pmask = __ballot_sync(kFull, flag == kFlagP);
                const int first = pmask ? __ffs(pmask) - 1 : 32;
                uint64_t contrib = lane <= first ? val : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) contrib += __shfl_xor_sync(kFull, contrib, o);
                excl += contrib;
                if (pmask) break;
                end -= 32;
            }
            if (__any_sync(kFull, timed_out) && lane == 0) raise_status(status, QSIM_E_TIMEOUT);
            if (lane == 0) {
                st_relaxed_u64(st + f, lb_word(epoch, kFlagP, uint32_t(excl + len)));
                s_excl = excl;
            }
        }
    }
    // ---- bit-plane words into the frame image: W_b = ballot(bit b of z) ----
    uint32_t *stage_words = s_stage + padw / 4;
#pragma unroll
    for (int i = 0; i < MAX_CPW; ++i) {
        const uint32_t c = warp + i * NW;
        if (c < g.C) {
            const uint32_t wr = s_w[c], wi = s_w[g.C + c];
            // lane b receives W_b = ballot(bit b of z): the bit-matrix transpose of the chunk's codes
            const uint32_t word_r = warp_bit_transpose(zr[i], lane);
            const uint32_t word_i = warp_bit_transpose(zi[i], lane);
            if (lane < int(wr)) stage_words[s_off[c] + lane] = word_r;
            if (lane < int(wi)) stage_words[s_off[g.C + c] + lane] = word_i;
        }
    }
    if (words + uint32_t(tid) < (len > padw ? (len - padw) / 4 : 0u)) stage_words[words + tid] = 0;  // pad
    __syncthreads();
    const uint64_t frame_off = g.data_start + s_excl;
    uint8_t *out = tgt.ptr;
    const uint64_t cap = tgt.cap;
    const bool fits = frame_off + len <= cap;
    if (fits && len) {
        uint4 *o4 = reinterpret_cast<uint4 *>(out + frame_off);
        const uint4 *s4 = reinterpret_cast<const uint4 *>(s_stage);
        for (uint32_t i = tid; i < len / 16; i += NT) o4[i] = s4[i];
    }
    if (!fits && tid == 0) atomicOr(&res_j->overflow, 1u);
    if (tid == 0 && g.data_start <= cap)
        reinterpret_cast<uint32_t *>(out + 32)[f] = uint32_t(frame_off);
    if (f == g.nframes - 1 && tid == 0) {
        const uint64_t total = frame_off + len;
        res_j->total = total;
        if (total <= cap) {
            uint32_t *h32 = reinterpret_cast<uint32_t *>(out);
            h32[0] = kQszMagic;
            h32[1] = 1u;  // version 1, flags 0
            h32[2] = uint32_t(m) | (uint32_t(g.fl) << 8) | (uint32_t(uint8_t(int8_t(e))) << 16);
            h32[3] = g.nframes;
            reinterpret_cast<uint64_t *>(out)[2] = total;
            reinterpret_cast<uint64_t *>(out)[3] = 0;
            h32[8 + g.nframes] = uint32_t(total);
            for (uint64_t b = 32 + 4ull * (g.nframes + 1); b < g.data_start; ++b) out[b] = 0;
            if (table_slot) {
                table_slot->ptr = out;
                table_slot->bytes = total;
                table_slot->tier = tgt.tier;
            }
            if (acc) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), total);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->reserved_bytes), cap);
                if (tgt.tier) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->host_bytes), cap);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->blocks), 1ull);
            }
        } else if (acc) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc->overflow_blocks), 1ull);
        }
    }
    // error norms of this frame (only counted once: not on the overflow retry)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        err_sq += __shfl_xor_sync(kFull, err_sq, o);
        norm_sq += __shfl_xor_sync(kFull, norm_sq, o);
    }
    if (lane == 0) {
        s_red[0][warp] = double(err_sq);
        s_red[1][warp] = double(norm_sq);
    }
    __syncthreads();
    if (tid == 0 && !only_overflowed) {
        double a = 0, b = 0;
        for (int w = 0; w < NW; ++w) { a += s_red[0][w]; b += s_red[1][w]; }
        if (part_item) {
            *part_item = make_float2(float(a), float(b));  // reduced once the block's frames are done
        } else {
            atomicAdd(&res_j->err_sq, a);
            atomicAdd(&res_j->norm_sq, b);
            if (acc) {
                atomicAdd(&acc->err_sq, a);
                atomicAdd(&acc->norm_sq, b);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Reservation of one block's slot from the two-tier pool: device arena
// first, then the pinned host arena; slots are padded to 256 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reserve_slot(uint64_t want, const ArenaDev &dev, const ArenaDev &host, EncTarget *t,
                                             int *status) {
    const uint64_t sz = (want + 255) & ~255ull;
    uint64_t off = atomicAdd(reinterpret_cast<unsigned long long *>(dev.bump), sz);
    if (off + sz <= dev.cap) {
        t->ptr = dev.base + off;
        t->cap = sz;
        t->tier = 0;
        return;
    }
    if (host.base) {
        off = atomicAdd(reinterpret_cast<unsigned long long *>(host.bump), sz);
        if (off + sz <= host.cap) {
            t->ptr = host.base + off;
            t->cap = sz;
            t->tier = 1;
            return;
        }
    }
    t->ptr = nullptr;
    t->cap = 0;
    t->tier = 0;
    raise_status(status, QSIM_E_NOMEM);
}

// ---------------------------------------------------------------------------
// Sizing pass: exact stream size of every block (reads the data once more),
// then the last CTA to finish reserves each block's slot and clears the size
// counters for the next launch.
// ---------------------------------------------------------------------------
// Stream bytes of frame f (zero for an all-zero frame), computed by the whole
// CTA; the result is returned to every thread. s_words holds NW words.
template <bool CG = false>
__device__ __forceinline__ uint32_t size_frame_cta(const float2 *__restrict__ src, const FrameGeom &g, int e,
                                                   uint32_t *s_words, int *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float inv_step = exp2i(-e);
    float2 vin[MAX_CPW];
#pragma unroll
    for (int i = 0; i < MAX_CPW; ++i) {
        const uint32_t c = warp + i * NW;
        vin[i] = c < g.C ? (CG ? __ldcg(src + c * 32 + lane) : src[c * 32 + lane]) : make_float2(0.f, 0.f);
    }
    uint32_t words = 0;
    int bad = 0;
#pragma unroll
    for (int i = 0; i < MAX_CPW; ++i) {
        const uint32_t c = warp + i * NW;
        if (c >= g.C) break;
        int32_t q[2];
        const float x[2] = {vin[i].x, vin[i].y};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float t = x[p] * inv_step;  // exact: power-of-two scaling
            if (fabsf(t) < 1073741824.0f) {
                q[p] = __float2int_rn(t);
            } else {  // NaN, Inf or out of range
                q[p] = 0;
                bad = isfinite(x[p]) ? (bad ? bad : QSIM_E_RANGE) : QSIM_E_INVALID;
            }
        }
        int32_t pr = __shfl_up_sync(kFull, q[0], 1);
        int32_t pi = __shfl_up_sync(kFull, q[1], 1);
        const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
        const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
        const uint32_t wr = 32 - __clz(__reduce_or_sync(kFull, zr)), wi = 32 - __clz(__reduce_or_sync(kFull, zi));
        words += wr + wi;
    }
    if (bad) raise_status(status, bad);
    if (lane == 0) s_words[warp] = words;
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) tot += s_words[w];
    __syncthreads();
    const uint64_t padw = (2ull * g.C + 15) & ~15ull;
    return tot ? uint32_t(padw + ((4ull * tot + 15) & ~15ull)) : 0u;
}


// Chunk widths of one frame with one warp (no block-wide barrier): lane l
// receives the Re widths of chunks 4l .. 4l+3 packed in wre and the Im widths
// in wim; returns the frame's bit-plane words.
template <bool CG = false>
__device__ __forceinline__ uint32_t frame_widths_warp(const float2 *__restrict__ src, const FrameGeom &g, int e,
                                                      uint32_t &wre, uint32_t &wim, int *status) {
    const int lane = threadIdx.x & 31;
    const float inv_step = exp2i(-e);
    uint32_t words = 0;
    int bad = 0;
    wre = wim = 0;
    for (uint32_t c0 = 0; c0 < g.C; c0 += 8) {
        float2 vin[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            vin[t] = c < g.C ? (CG ? __ldcg(src + c * 32 + lane) : src[c * 32 + lane]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            if (c >= g.C) break;
            int32_t q[2];
            const float x[2] = {vin[t].x, vin[t].y};
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                const float tq = x[pl] * inv_step;  // exact: power-of-two scaling
                if (fabsf(tq) < 1073741824.0f) {
                    q[pl] = __float2int_rn(tq);
                } else {  // NaN, Inf or out of range
                    q[pl] = 0;
                    bad = isfinite(x[pl]) ? (bad ? bad : QSIM_E_RANGE) : QSIM_E_INVALID;
                }
            }
            const int32_t pr = __shfl_up_sync(kFull, q[0], 1);
            const int32_t pi = __shfl_up_sync(kFull, q[1], 1);
            const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
            const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
            const uint32_t wr = 32 - __clz(__reduce_or_sync(kFull, zr)), wi = 32 - __clz(__reduce_or_sync(kFull, zi));
            words += wr + wi;
            if (uint32_t(lane) == (c >> 2)) {
                wre |= wr << (8 * (c & 3));
                wim |= wi << (8 * (c & 3));
            }
        }
    }
    if (bad) raise_status(status, bad);
    return words;
}

// The width record (2C bytes, Re then Im) from the packed widths, as words:
// Re widths at bytes [0, C), Im widths at [C, 2C). dst may be global or shared.
__device__ __forceinline__ void store_widths_warp(uint8_t *dst, const FrameGeom &g, uint32_t wre, uint32_t wim) {
    const int lane = threadIdx.x & 31;
    if (g.C >= 4) {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(dst);
        if (4u * lane < g.C) {
            w32[lane] = wre;
            w32[g.C / 4 + lane] = wim;
        }
    } else if (lane == 0) {
        for (uint32_t c = 0; c < g.C; ++c) {
            dst[c] = uint8_t(wre >> (8 * c));
            dst[g.C + c] = uint8_t(wim >> (8 * c));
        }
    }
}

__device__ __forceinline__ uint64_t pad16d(uint64_t x) { return (x + 15u) & ~uint64_t(15); }

__device__ __forceinline__ uint32_t frame_len(const FrameGeom &g, uint32_t words) {
    const uint32_t padw = (2u * g.C + 15u) & ~15u;
    return words ? padw + ((4u * words + 15u) & ~15u) : 0u;
}

// Exact stream bytes of one frame with one warp; the chunk widths go to wrec
// (2C bytes) for encode_frame_warp_known.
template <bool CG = false>
__device__ __forceinline__ uint32_t size_frame_warp(const float2 *__restrict__ src, const FrameGeom &g, int e,
                                                    uint8_t *__restrict__ wrec, int *status) {
    uint32_t wre, wim;
    const uint32_t words = frame_widths_warp<CG>(src, g, e, wre, wim, status);
    store_widths_warp(wrec, g, wre, wim);
    return frame_len(g, words);
}

// Encode frame f of one block with one warp when the frame's chunk widths
// (wrec: 2C bytes, Re then Im, written by the sizing pass) and its byte offset
// in the block's stream are known: no look-back and no block-wide barrier.
// The words go straight to their place in the slot; lane 0 also writes the
// frame's offset-table entry and, for the block's last frame, the header.
// Width record bytes 8 lane .. 8 lane + 7 (bytes past 2C masked to zero);
// with CG the record is read through L2 (written by other CTAs of the launch).
template <bool CG>
__device__ __forceinline__ uint2 load_widths_warp(const uint8_t *wrec, const FrameGeom &g) {
    const uint32_t lane = threadIdx.x & 31;
    uint2 wb = make_uint2(0, 0);
    if (8u * lane < 2u * g.C) {
        wb = CG ? __ldcg(reinterpret_cast<const uint2 *>(wrec + 8u * lane))
                : *reinterpret_cast<const uint2 *>(wrec + 8u * lane);
        const uint32_t valid = 2u * g.C - 8u * lane;  // bytes of this lane that are widths
        if (valid < 8) {
            const uint64_t keep = (1ull << (8 * valid)) - 1;
            const uint64_t v = (uint64_t(wb.y) << 32 | wb.x) & keep;
            wb = make_uint2(uint32_t(v), uint32_t(v >> 32));
        }
    }
    return wb;
}

// Encode frame f with one warp at byte offset frame_off of the block's stream,
// given its widths (wb, as load_widths_warp) and length.
template <bool CG = false>
__device__ __forceinline__ void encode_frame_warp_core(const float2 *__restrict__ src, const FrameGeom &g, int m,
                                                       int e, uint32_t f, uint2 wb, uint32_t frame_off, uint32_t len,
                                                       EncTarget tgt, EncResult *res_j, BlockSlot *table_slot,
                                                       StageAccum *acc, float2 *part_item, int *status) {
    const int lane = threadIdx.x & 31;
    const uint32_t padw = (2u * g.C + 15u) & ~15u;
    const float inv_step = exp2i(-e), step = exp2i(e);
    uint8_t *out = tgt.ptr;
    const uint64_t cap = tgt.cap;
    const bool fits = out != nullptr && uint64_t(frame_off) + len <= cap;
    uint32_t wsum = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) wsum += ((wb.x >> (8 * t)) & 0xff) + ((wb.y >> (8 * t)) & 0xff);
    uint32_t incl = wsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t base_off = incl - wsum;
    const uint32_t words = __shfl_sync(kFull, incl, 31);
    uint32_t *payload = fits ? reinterpret_cast<uint32_t *>(out + frame_off + padw) : nullptr;
    if (fits && len && 8u * lane < padw) *reinterpret_cast<uint2 *>(out + frame_off + 8u * lane) = wb;
    float err_sq = 0.f, norm_sq = 0.f;
    int bad = 0;
    for (uint32_t c0 = 0; c0 < g.C; c0 += 8) {
        const uint32_t lr = c0 >> 3, li = (g.C + c0) >> 3;
        const uint2 wr8 = make_uint2(__shfl_sync(kFull, wb.x, lr), __shfl_sync(kFull, wb.y, lr));
        const uint2 wi8 = make_uint2(__shfl_sync(kFull, wb.x, li), __shfl_sync(kFull, wb.y, li));
        uint32_t offr = __shfl_sync(kFull, base_off, lr), offi = __shfl_sync(kFull, base_off, li);
        const uint32_t si0 = (g.C + c0) & 7u;
        for (uint32_t t = 0; t < si0; ++t) offi += t < 4 ? (wi8.x >> (8 * t)) & 0xff : (wi8.y >> (8 * (t - 4))) & 0xff;
        float2 vin[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            vin[t] = c < g.C ? (CG ? __ldcg(src + c * 32 + lane) : __ldcs(src + c * 32 + lane)) : make_float2(0.f, 0.f);
        }
        uint32_t sr_ = 0, si_ = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            if (c >= g.C) break;
            const uint32_t ti = si0 + t;
            const uint32_t wr = t < 4 ? (wr8.x >> (8 * t)) & 0xff : (wr8.y >> (8 * (t - 4))) & 0xff;
            const uint32_t wi = ti < 8 ? (ti < 4 ? (wi8.x >> (8 * ti)) & 0xff : (wi8.y >> (8 * (ti - 4))) & 0xff) : 0;
            int32_t q[2];
            const float x[2] = {vin[t].x, vin[t].y};
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                const float tq = x[pl] * inv_step;  // exact: power-of-two scaling
                if (!(fabsf(tq) < 1073741824.0f)) {  // NaN, Inf or out of range
                    bad = isfinite(x[pl]) ? (bad ? bad : QSIM_E_RANGE) : QSIM_E_INVALID;
                    q[pl] = 0;
                } else {
                    q[pl] = __float2int_rn(tq);
                }
                const float xr = float(q[pl]) * step;
                const float dx = x[pl] - xr;
                err_sq = fmaf(dx, dx, err_sq);
                norm_sq = fmaf(xr, xr, norm_sq);
            }
            const int32_t pr = __shfl_up_sync(kFull, q[0], 1);
            const int32_t pi = __shfl_up_sync(kFull, q[1], 1);
            const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
            const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
            if (wr <= 16 && wi <= 16) {
                // both planes in one transpose: lane b < 16 gets Re plane b, lane 16 + b Im plane b
                const uint32_t word = warp_bit_transpose(zr | (zi << 16), lane);
                const uint32_t b = uint32_t(lane) & 15u;
                if (payload && b < (lane < 16 ? wr : wi)) payload[(lane < 16 ? offr + sr_ : offi + si_) + b] = word;
            } else {
                const uint32_t word_r = warp_bit_transpose(zr, lane);
                const uint32_t word_i = warp_bit_transpose(zi, lane);
                if (payload) {
                    if (lane < int(wr)) payload[offr + sr_ + lane] = word_r;
                    if (lane < int(wi)) payload[offi + si_ + lane] = word_i;
                }
            }
            sr_ += wr;
            si_ += wi;
        }
    }
    if (payload && len && words + uint32_t(lane) < (len - padw) / 4) payload[words + lane] = 0;  // pad to 16 B
    if (bad) raise_status(status, bad);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        err_sq += __shfl_xor_sync(kFull, err_sq, o);
        norm_sq += __shfl_xor_sync(kFull, norm_sq, o);
    }
    if (lane == 0) {
        if (part_item) *part_item = make_float2(err_sq, norm_sq);
        if (!fits && res_j) atomicOr(&res_j->overflow, 1u);
        if (out && g.data_start <= cap) reinterpret_cast<uint32_t *>(out + 32)[f] = frame_off;
        if (f == g.nframes - 1) {
            const uint64_t total = uint64_t(frame_off) + len;
            if (res_j) res_j->total = total;
            if (out && total <= cap) {
                uint32_t *h32 = reinterpret_cast<uint32_t *>(out);
                h32[0] = kQszMagic;
                h32[1] = 1u;  // version 1, flags 0
                h32[2] = uint32_t(m) | (uint32_t(g.fl) << 8) | (uint32_t(uint8_t(int8_t(e))) << 16);
                h32[3] = g.nframes;
                reinterpret_cast<uint64_t *>(out)[2] = total;
                reinterpret_cast<uint64_t *>(out)[3] = 0;
                h32[8 + g.nframes] = uint32_t(total);
                for (uint64_t b = 32 + 4ull * (g.nframes + 1); b < g.data_start; ++b) out[b] = 0;
                if (table_slot) {
                    table_slot->ptr = out;
                    table_slot->bytes = total;
                    table_slot->tier = tgt.tier;
                }
                if (acc) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), total);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->reserved_bytes), cap);
                    if (tgt.tier) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->host_bytes), cap);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->blocks), 1ull);
                }
            } else if (acc) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->overflow_blocks), 1ull);
            }
        }
    }
}

// Exact-sizing encoder: widths (wrec) and frame offset from the sizing pass.
template <bool CG = false>
__device__ __forceinline__ void encode_frame_warp_known(const float2 *__restrict__ src, const FrameGeom &g, int m,
                                                        int e, uint32_t f, const uint8_t *__restrict__ wrec,
                                                        uint32_t frame_off, uint32_t len, EncTarget tgt,
                                                        EncResult *res_j, BlockSlot *table_slot, StageAccum *acc,
                                                        float2 *part_item, int *status) {
    encode_frame_warp_core<CG>(src, g, m, e, f, load_widths_warp<CG>(wrec, g), frame_off, len, tgt, res_j,
                               table_slot, acc, part_item, status);
}

// ---------------------------------------------------------------------------
// Relative-bound variant (QSZR, Sec. 4.3 Eq. 1-2 and Algorithm 2). The code of
// a component x is its FP32 magnitude bit pattern U = bits(|x|) (exponent plus
// linear mantissa: log2|x| up to a scale and offset) rounded to a multiple of
// 2^k: q = (U + 2^(k-1)) >> k; the sign (1 for x < 0 with q != 0) goes to a
// per-chunk sign word W = ballot(sign): chunks of all clear or all set signs
// store only their 2-bit type (0, 1: Algorithm 2's pre-scan); the others are
// coded losslessly, as a 2-byte run record when the signs change 1 to 3 times
// between neighbours (type 3), else as the raw word (type 2). Reconstruction
// |x'| = float(bits q << k).
// ---------------------------------------------------------------------------

// code of one component; bad collects QSIM_E_INVALID (non-finite, wins) or QSIM_E_RANGE
template <bool REL>
__device__ __forceinline__ int32_t quantize_one(float x, float inv_step, uint32_t k, int &bad) {
    if constexpr (REL) {
        const uint32_t U = __float_as_uint(x) & 0x7FFFFFFFu;
        if (U >= kQszrMaxU) {
            bad = U >= 0x7F800000u ? QSIM_E_INVALID : (bad ? bad : QSIM_E_RANGE);
            return 0;
        }
        return int32_t((U + (1u << (k - 1))) >> k);
    } else {
        const float tq = x * inv_step;  // exact: power-of-two scaling
        if (!(fabsf(tq) < 1073741824.0f)) {  // NaN, Inf or out of range
            bad = isfinite(x) ? (bad ? bad : QSIM_E_RANGE) : QSIM_E_INVALID;
            return 0;
        }
        return __float2int_rn(tq);
    }
}

// In-place exact encoder, first of two passes: one warp reads frame f once
// and writes its bit-plane words without knowing the frame's place in the
// stream. The Re-plane words go over the frame's own amplitudes (the words of
// chunk c end at or before byte 128 (c + 1) of the frame, and every chunk up
// to c has been read by then), the Im-plane words to im (one word per
// amplitude of scratch), the chunk widths to side (2C bytes; for REL also the
// sign chunk types, stored sign words and run records). Returns the frame's stream bytes;
// words receives its Re-plane words | Im-plane words << 16 (each at most
// 4096), mixed (REL) its stored sign words Re | Im << 8 and run records Re << 16 | Im << 24. The second pass
// (copy_frame_warp) moves the pieces to the frame's offset in the block's slot.
// e is the step exponent (QSZ1) or the shift k (REL). With CG the amplitudes are read through L2 (written by
// other CTAs of the same launch).
template <bool REL = false, bool CG = false>
__device__ __forceinline__ uint32_t encode_frame_warp_ip(float2 *frame, uint32_t *__restrict__ im,
                                                         const FrameGeom &g, int e, uint8_t *__restrict__ side,
                                                         uint32_t &words, uint32_t &mixed, float2 *part_item,
                                                         int *status) {
    const int lane = threadIdx.x & 31;
    const float inv_step = REL ? 0.f : exp2i(-e), step = REL ? 0.f : exp2i(e);
    const uint32_t k = uint32_t(e);
    uint32_t *re = reinterpret_cast<uint32_t *>(frame);  // aliases frame: no __restrict__
    uint32_t ro = 0, io = 0, wre = 0, wim = 0, tw = 0, mr = 0, mi = 0, rr = 0, ri = 0;
    float err_sq = 0.f, norm_sq = 0.f;
    int bad = 0;
    for (uint32_t c0 = 0; c0 < g.C; c0 += 8) {
        float2 vin[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            vin[t] = c < g.C ? (CG ? __ldcg(frame + c * 32 + lane) : frame[c * 32 + lane]) : make_float2(0.f, 0.f);
        }
        __syncwarp();  // every lane's reads of this batch come before the batch's in-place writes
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = c0 + t;
            if (c >= g.C) break;
            int32_t q[2];
            bool neg[2];
            const float x[2] = {vin[t].x, vin[t].y};
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                q[pl] = quantize_one<REL>(x[pl], inv_step, k, bad);
                float xr;
                if constexpr (REL) {
                    neg[pl] = x[pl] < 0.f && q[pl] != 0;
                    const float mag = __uint_as_float(uint32_t(q[pl]) << k);
                    xr = neg[pl] ? -mag : mag;
                } else {
                    xr = float(q[pl]) * step;
                }
                const float dx = x[pl] - xr;
                err_sq = fmaf(dx, dx, err_sq);
                norm_sq = fmaf(xr, xr, norm_sq);
            }
            if constexpr (REL) {
                // sign pre-scan: chunk types (owner lane t >> 4 of chunk index t = plane C + c), mixed words
                const uint32_t sr = __ballot_sync(kFull, neg[0]), si = __ballot_sync(kFull, neg[1]);
                const uint32_t tr = sign_type(sr), ti = sign_type(si);
                const uint32_t ir = c, ii = g.C + c;
                if (uint32_t(lane) == (ir >> 4)) tw |= tr << (2 * (ir & 15));
                if (uint32_t(lane) == (ii >> 4)) tw |= ti << (2 * (ii & 15));
                if (lane == 0) {
                    if (tr == 2) reinterpret_cast<uint32_t *>(side + kSideMixRe)[mr] = sr;
                    if (ti == 2) reinterpret_cast<uint32_t *>(side + kSideMixIm)[mi] = si;
                    if (tr == 3) reinterpret_cast<uint16_t *>(side + kSideRunRe)[rr] = uint16_t(sign_run_record(sr));
                    if (ti == 3) reinterpret_cast<uint16_t *>(side + kSideRunIm)[ri] = uint16_t(sign_run_record(si));
                }
                mr += tr == 2;
                mi += ti == 2;
                rr += tr == 3;
                ri += ti == 3;
            }
            const int32_t pr = __shfl_up_sync(kFull, q[0], 1);
            const int32_t pi = __shfl_up_sync(kFull, q[1], 1);
            const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
            const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
            // a plane's width is one more than its highest nonzero bit plane: taken from the transposed words
            uint32_t wr, wi;
            if (!__any_sync(kFull, (zr | zi) >> 16)) {
                // both planes in one transpose: lane b < 16 gets Re plane b, lane 16 + b Im plane b
                const uint32_t word = warp_bit_transpose(zr | (zi << 16), lane);
                const uint32_t nz = __ballot_sync(kFull, word != 0);
                wr = 32 - __clz(nz & 0xffffu);
                wi = 32 - __clz(nz >> 16);
                const uint32_t b = uint32_t(lane) & 15u;
                if (lane < 16) {
                    if (b < wr) re[ro + b] = word;
                } else if (b < wi) {
                    im[io + b] = word;
                }
            } else {
                const uint32_t word_r = warp_bit_transpose(zr, lane);
                const uint32_t word_i = warp_bit_transpose(zi, lane);
                wr = 32 - __clz(__ballot_sync(kFull, word_r != 0));
                wi = 32 - __clz(__ballot_sync(kFull, word_i != 0));
                if (lane < int(wr)) re[ro + lane] = word_r;
                if (lane < int(wi)) im[io + lane] = word_i;
            }
            if (uint32_t(lane) == (c >> 2)) {
                wre |= wr << (8 * (c & 3));
                wim |= wi << (8 * (c & 3));
            }
            ro += wr;
            io += wi;
        }
    }
    if (bad) raise_status(status, bad);
    store_widths_warp(side, g, wre, wim);
    if constexpr (REL) {
        if (16u * uint32_t(lane) < 2u * g.C) reinterpret_cast<uint32_t *>(side + kSideTypes)[lane] = tw;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        err_sq += __shfl_xor_sync(kFull, err_sq, o);
        norm_sq += __shfl_xor_sync(kFull, norm_sq, o);
    }
    if (lane == 0 && part_item) *part_item = make_float2(err_sq, norm_sq);
    words = ro | (io << 16);
    mixed = mr | (mi << 8) | (rr << 16) | (ri << 24);
    if (ro + io == 0) return 0u;
    uint32_t len = frame_len(g, ro + io);
    if constexpr (REL) len += uint32_t(pad16d((2u * g.C + 3u) / 4u)) + sign_section_bytes(mixed);
    return len;
}

// Second pass of the in-place encoder: frame f's widths (and for REL its sign
// chunk types, stored sign words and run records) from side, its Re-plane words (re, 16-byte
// aligned) and Im-plane words (im) are copied to byte offset frame_off of the
// block's slot and padded to 16 bytes; lane 0 writes the frame's offset-table
// entry and, for the block's last frame, the header, the block's table slot
// and the stage totals. words = Re words | Im words << 16, mixed = the sign-section
// counts packed as by the first pass. A slot too small (only after a failed reservation
// or a caller's short buffer) sets the block's overflow flag instead.
template <bool REL = false>
__device__ __forceinline__ void copy_frame_warp(const uint32_t *__restrict__ re, const uint32_t *__restrict__ im,
                                                const uint8_t *__restrict__ side, uint32_t words, uint32_t mixed,
                                                uint32_t len, uint32_t frame_off, const FrameGeom &g, int m, int e,
                                                uint32_t f, EncTarget tgt, EncResult *res_j, BlockSlot *table_slot,
                                                StageAccum *acc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t padw = (2u * g.C + 15u) & ~15u;
    const uint32_t nre = words & 0xffffu, nim = words >> 16;
    uint8_t *out = tgt.ptr;
    const uint64_t cap = tgt.cap;
    const bool fits = out != nullptr && uint64_t(frame_off) + len <= cap;
    if (fits && len) {
        uint8_t *dst = out + frame_off;
        const uint2 wb = load_widths_warp<true>(side, g);
        if (8u * lane < padw) *reinterpret_cast<uint2 *>(dst + 8u * lane) = wb;
        uint32_t head = padw;
        if constexpr (REL) {
            // sign chunk types, padded to 16 bytes; then the sign section: the stored words (Re chunks first),
            // then the run records (Re chunks first), padded to 16 bytes as a whole
            const uint32_t tb = uint32_t(pad16d((2u * g.C + 3u) / 4u));
            const uint32_t mre = mixed & 0xffu, mim = (mixed >> 8) & 0xffu;
            const uint32_t rre = (mixed >> 16) & 0xffu, rim = mixed >> 24;
            const uint32_t nmw = sign_section_bytes(mixed) / 4u;
            uint32_t *tdst = reinterpret_cast<uint32_t *>(dst + padw);
            if (4u * lane < tb) tdst[lane] = 16u * lane < 2u * g.C ? __ldcg(reinterpret_cast<const uint32_t *>(side + kSideTypes) + lane) : 0u;
            uint32_t *mdst = reinterpret_cast<uint32_t *>(dst + padw + tb);
            const uint16_t *rrec = reinterpret_cast<const uint16_t *>(side + kSideRunRe);
            const uint16_t *irec = reinterpret_cast<const uint16_t *>(side + kSideRunIm);
            for (uint32_t i = lane; i < nmw; i += 32) {
                uint32_t v;
                if (i < mre) {
                    v = __ldcg(reinterpret_cast<const uint32_t *>(side + kSideMixRe) + i);
                } else if (i < mre + mim) {
                    v = __ldcg(reinterpret_cast<const uint32_t *>(side + kSideMixIm) + (i - mre));
                } else {
                    // run records 2j and 2j + 1 of the section's record list (Re then Im), zero past the end
                    const uint32_t j = 2u * (i - mre - mim);
                    uint32_t h[2];
#pragma unroll
                    for (uint32_t q = 0; q < 2; ++q) {
                        const uint32_t r = j + q;
                        h[q] = r < rre ? uint32_t(__ldcg(rrec + r)) : (r - rre < rim ? uint32_t(__ldcg(irec + (r - rre))) : 0u);
                    }
                    v = h[0] | (h[1] << 16);
                }
                mdst[i] = v;
            }
            head = padw + tb + 4u * nmw;
        }
        // payload word i: Re word i (i < nre), Im word i - nre (i - nre < nim), else zero padding; written
        // as 16-byte vectors, four per lane in flight
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);  // 16-byte aligned
        const uint32_t n4 = (len - head) / 16;
        for (uint32_t k0 = lane; k0 < n4; k0 += 128) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + 32u * u, i = 4u * k;
                if (k >= n4) break;
                if (i + 4 <= nre) {
                    v[u] = __ldcg(reinterpret_cast<const uint4 *>(re) + k);
                } else if (i >= nre && !((i - nre) & 3u) && i - nre + 4 <= nim) {
                    v[u] = __ldcg(reinterpret_cast<const uint4 *>(im + (i - nre)));
                } else {
                    uint32_t w[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t ii = i + t;
                        w[t] = ii < nre ? __ldcg(re + ii) : (ii - nre < nim ? __ldcg(im + (ii - nre)) : 0u);
                    }
                    v[u] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + 32u * u;
                if (k < n4) d4[k] = v[u];
            }
        }
    }
    if (lane == 0) {
        if (!fits && res_j) atomicOr(&res_j->overflow, 1u);
        if (out && g.data_start <= cap) reinterpret_cast<uint32_t *>(out + 32)[f] = frame_off;
        if (f == g.nframes - 1) {
            const uint64_t total = uint64_t(frame_off) + len;
            if (res_j) res_j->total = total;
            if (out && total <= cap) {
                uint32_t *h32 = reinterpret_cast<uint32_t *>(out);
                h32[0] = REL ? kQszrMagic : kQszMagic;
                h32[1] = 1u;  // version 1, flags 0
                h32[2] = uint32_t(m) | (uint32_t(g.fl) << 8) | (uint32_t(uint8_t(int8_t(e))) << 16);
                h32[3] = g.nframes;
                reinterpret_cast<uint64_t *>(out)[2] = total;
                reinterpret_cast<uint64_t *>(out)[3] = 0;
                h32[8 + g.nframes] = uint32_t(total);
                for (uint64_t b = 32 + 4ull * (g.nframes + 1); b < g.data_start; ++b) out[b] = 0;
                if (table_slot) {
                    table_slot->ptr = out;
                    table_slot->bytes = total;
                    table_slot->tier = tgt.tier;
                }
                if (acc) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), total);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->reserved_bytes), cap);
                    if (tgt.tier) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->host_bytes), cap);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->blocks), 1ull);
                }
            } else if (acc) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->overflow_blocks), 1ull);
            }
        }
    }
}

// Warp look-back over the preceding frames of the block (status words of lb_block,
// tagged with epoch): publishes frame f's length, returns the bytes of frames 0..f-1.
// Every wait is time-bounded (QSIM_E_TIMEOUT).
__device__ __forceinline__ uint32_t lookback_warp(uint64_t *lb_block, uint32_t f, uint32_t epoch, uint32_t len,
                                                  int *status) {
    const int lane = threadIdx.x & 31;
    uint64_t *st = lb_block;
    if (f == 0) {
        if (lane == 0) st_relaxed_u64(st, lb_word(epoch, kFlagP, len));
        return 0;
    }
    if (lane == 0) st_relaxed_u64(st + f, lb_word(epoch, kFlagA, len));
    uint64_t excl = 0;
    int64_t end = int64_t(f) - 1;
    bool timed_out = false;
    while (true) {
        const int64_t p = end - lane;
        uint32_t flag = kFlagP, val = 0;
        if (p >= 0) {
            long long spins = 0;
            const uint64_t t0 = global_ns();
            while (true) {
                const uint64_t w = ld_relaxed_u64(st + p);
                const uint32_t fl = uint32_t(w >> 32) & 3u;
                if (fl != 0 && uint32_t(w >> 34) == epoch) {
                    flag = fl;
                    val = uint32_t(w);
                    break;
                }
                if (++spins > kSpinLimit || global_ns() - t0 > kLookbackWaitNs) {
                    timed_out = true;
                    flag = kFlagP;
                    val = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        const uint32_t pmask = __ballot_sync(kFull, flag == kFlagP);
        const int first = pmask ? __ffs(pmask) - 1 : 32;
        uint64_t contrib = lane <= first ? val : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) contrib += __shfl_xor_sync(kFull, contrib, o);
        excl += contrib;
        if (pmask) break;
        end -= 32;
    }
    if (__any_sync(kFull, timed_out) && lane == 0) raise_status(status, QSIM_E_TIMEOUT);
    if (lane == 0) st_relaxed_u64(st + f, lb_word(epoch, kFlagP, uint32_t(excl + len)));
    return uint32_t(excl);
}

// Learned-sizing encoder, one warp per frame: widths pass, look-back for the
// frame's offset, then the frame is read again (from L2) and written into the
// reserved slot if it fits (else the block's overflow flag is set and
// res.total still receives the exact size). s_wb: 64 words of shared memory
// for this warp. Frames of a block must be taken in order (ticket or queue).
template <bool CG = false>
__device__ __forceinline__ void encode_frame_warp_lb(const float2 *__restrict__ src, const FrameGeom &g, int m, int e,
                                                     uint32_t f, uint64_t *lb_block, uint32_t epoch, EncTarget tgt,
                                                     EncResult *res_j, BlockSlot *table_slot, StageAccum *acc,
                                                     float2 *part_item, uint32_t *s_wb, int *status) {
    uint32_t wre, wim;
    const uint32_t words = frame_widths_warp<CG>(src, g, e, wre, wim, status);
    const uint32_t len = frame_len(g, words);
    store_widths_warp(reinterpret_cast<uint8_t *>(s_wb), g, wre, wim);
    __syncwarp();
    const uint2 wb = load_widths_warp<false>(reinterpret_cast<const uint8_t *>(s_wb), g);
    __syncwarp();
    const uint32_t excl = lookback_warp(lb_block, f, epoch, len, status);
    encode_frame_warp_core<CG>(src, g, m, e, f, wb, uint32_t(g.data_start) + excl, len, tgt, res_j, table_slot, acc,
                               part_item, status);
}

}  // namespace cdev
}  // namespace qsim
