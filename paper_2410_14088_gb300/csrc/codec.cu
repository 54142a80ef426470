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
#include "device_common.cuh"

namespace qsim {

namespace {

constexpr int NT = 256;          // threads per CTA (8 warps)
constexpr int NW = NT / 32;
constexpr int MAX_C = 128;       // chunks per plane per frame (F = 4096)
constexpr int MAX_CPW = MAX_C / NW;  // chunk pairs per warp
constexpr uint32_t kFlagA = 1u, kFlagP = 2u;
constexpr uint32_t kEpochMask = (1u << 30) - 1;
constexpr long long kSpinLimit = 1ll << 22;

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

__device__ __forceinline__ uint32_t zigzag(int32_t d) {
    return (uint32_t(d) << 1) ^ uint32_t(d >> 31);
}

__device__ __forceinline__ int32_t unzigzag(uint32_t z) {
    return int32_t((z >> 1) ^ (0u - (z & 1u)));
}

// ---------------------------------------------------------------------------
// Decode: one CTA per frame (grid-stride over all frames of all blocks).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_decode(const BlockRef *__restrict__ in, uint32_t nblocks, int m,
                                               float2 *__restrict__ wv, uint32_t *__restrict__ hist,
                                               int *status) {
    const FrameGeom g = geom(m);
    __shared__ uint32_t s_w[2 * MAX_C];
    __shared__ uint32_t s_off[2 * MAX_C];
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_total;
    __shared__ uint64_t s_hdr[4];  // frame start, frame end, e, ok
    __shared__ uint32_t s_hist[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t items = uint64_t(nblocks) * g.nframes;

    for (uint64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        const uint8_t *s = in[j].ptr;
        const uint64_t bytes = in[j].bytes;
        float2 *dst = wv + (uint64_t(j) << m) + uint64_t(f) * g.F;
        if (tid < 32) s_hist[tid] = 0;
        if (tid == 0) {
            uint64_t ok = 1, a = 0, b = 0;
            int e = 0;
            if (bytes < 32 || s == nullptr || (reinterpret_cast<uintptr_t>(s) & 15)) {
                ok = 0;
            } else {
                const uint32_t *h32 = reinterpret_cast<const uint32_t *>(s);
                const uint64_t *h64 = reinterpret_cast<const uint64_t *>(s);
                uint32_t w1 = h32[1], w2 = h32[2];
                e = int(int8_t(uint8_t(w2 >> 16)));
                uint64_t total = h64[2];
                if (h32[0] != kQszMagic || w1 != 1u || (w2 & 0xff) != uint32_t(m) ||
                    ((w2 >> 8) & 0xff) != uint32_t(g.fl) || (w2 >> 24) != 0 || h32[3] != g.nframes ||
                    h64[3] != 0 || e < kQszEMin || e > kQszEMax || total > bytes || total < g.data_start)
                    ok = 0;
                if (ok) {
                    const uint32_t *offs = h32 + 8;
                    if (offs[0] != g.data_start || offs[g.nframes] != total) ok = 0;
                    a = offs[f];
                    b = offs[f + 1];
                    if (b < a || b > total || a < g.data_start) ok = 0;
                    if (ok && b > a && (b - a < ((2ull * g.C + 15) & ~15ull) || ((a | b) & 15))) ok = 0;
                }
            }
            s_hdr[0] = a;
            s_hdr[1] = b;
            s_hdr[2] = uint64_t(int64_t(e));
            s_hdr[3] = ok;
        }
        __syncthreads();
        const uint64_t fa = s_hdr[0], fb = s_hdr[1];
        const int e = int(int64_t(s_hdr[2]));
        bool ok = s_hdr[3] != 0;
        if (ok && fb > fa) {
            const uint8_t *fp = s + fa;
            const uint32_t wv_ = tid < int(2 * g.C) ? fp[tid] : 0;
            const uint32_t off = block_exclusive_scan<NT>(wv_, s_warp, &s_total);
            if (tid < int(2 * g.C)) {
                s_w[tid] = wv_;
                s_off[tid] = off;
            }
            __syncthreads();
            const uint64_t words = s_total;
            const uint64_t padw = (2ull * g.C + 15) & ~15ull;
            // widths > 32 make the stream corrupt (the barrier is reached by every thread)
            const bool wide = __syncthreads_or(tid < int(2 * g.C) && wv_ > 32) != 0;
            const bool bad = wide || words == 0 || (fb - fa) != padw + ((4 * words + 15) & ~15ull);
            if (bad) {
                ok = false;
            } else {
                const uint32_t *payload = reinterpret_cast<const uint32_t *>(fp + padw);
                const float step = exp2i(e);
                uint32_t my_max = 0;
                for (uint32_t c = warp; c < g.C; c += NW) {
                    const uint32_t wr = s_w[c], wi = s_w[g.C + c];
                    uint32_t xr = lane < int(wr) ? __ldg(payload + s_off[c] + lane) : 0u;
                    uint32_t xi = lane < int(wi) ? __ldg(payload + s_off[g.C + c] + lane) : 0u;
                    uint32_t zr = warp_bit_transpose(xr, lane);
                    uint32_t zi = warp_bit_transpose(xi, lane);
                    uint32_t qr = uint32_t(unzigzag(zr)), qi = uint32_t(unzigzag(zi));
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t tr = __shfl_up_sync(kFull, qr, o);
                        uint32_t ti = __shfl_up_sync(kFull, qi, o);
                        if (lane >= o) { qr += tr; qi += ti; }
                    }
                    const int32_t sr = int32_t(qr), si = int32_t(qi);
                    dst[c * 32 + lane] = make_float2(float(sr) * step, float(si) * step);
                    if (hist) {
                        uint32_t br = 32 - __clz(sr < 0 ? uint32_t(-sr) : uint32_t(sr));
                        uint32_t bi = 32 - __clz(si < 0 ? uint32_t(-si) : uint32_t(si));
                        atomicAdd(&s_hist[br & 31], 1u);
                        atomicAdd(&s_hist[bi & 31], 1u);
                        my_max = max(my_max, max(br, bi));
                    }
                }
            }
        }
        if (!ok) raise_status(status, QSIM_E_CORRUPT);
        if (!ok || fb == fa) {
            for (uint32_t i = tid; i < g.F; i += NT) dst[i] = make_float2(0.f, 0.f);
            if (hist && tid == 0) s_hist[0] += 2 * g.F;
        }
        __syncthreads();
        if (hist && tid < 32 && s_hist[tid]) atomicAdd(&hist[uint64_t(j) * 32 + tid], s_hist[tid]);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Per-frame quantisation + widths. Returns (in registers) the bit-plane words
// when KEEP is set. Used by both the encoder and the sizing pass.
// ---------------------------------------------------------------------------
struct QuantOut {
    double err_sq, norm_sq;
    int bad;  // QSIM_E_* or 0
};

// ---------------------------------------------------------------------------
// Encode: one CTA per frame, ticket-ordered, decoupled look-back.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_encode(const float2 *__restrict__ wv, uint32_t nblocks, int m, int e,
                                               const EncTarget *__restrict__ tgt, EncResult *__restrict__ res,
                                               int only_overflowed, const uint32_t *__restrict__ ids,
                                               BlockSlot *__restrict__ table, StageAccum *acc,
                                               LookbackScratch scr, int *status) {
    const FrameGeom g = geom(m);
    __shared__ uint32_t s_w[2 * MAX_C];
    __shared__ uint32_t s_off[2 * MAX_C];
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_total;
    __shared__ uint32_t s_item, s_epoch;
    __shared__ uint64_t s_excl;
    __shared__ double s_red[2][NW];
    __shared__ int s_skip;
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

    if (!s_skip) {
        if (only_overflowed && tid == 0 && f == 0) {
            // this block is encoded again into a fresh slot
        }
        const float2 *src = wv + (uint64_t(j) << m) + uint64_t(f) * g.F;
        const float inv_step = exp2i(-e);
        const float step = exp2i(e);
        uint32_t words_r[MAX_CPW], words_i[MAX_CPW];
        double err_sq = 0.0, norm_sq = 0.0;
        int bad = 0;
#pragma unroll
        for (int i = 0; i < MAX_CPW; ++i) {
            words_r[i] = 0;
            words_i[i] = 0;
            const uint32_t c = warp + i * NW;
            if (c < g.C) {
                const float2 v = src[c * 32 + lane];
                int32_t q[2];
                const float x[2] = {v.x, v.y};
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    if (!isfinite(x[p])) {
                        bad = QSIM_E_INVALID;
                        q[p] = 0;
                    } else {
                        float t = x[p] * inv_step;  // exact: power-of-two scaling
                        if (fabsf(t) >= 1073741824.0f) {
                            bad = bad ? bad : QSIM_E_RANGE;
                            q[p] = 0;
                        } else {
                            q[p] = __float2int_rn(t);
                        }
                    }
                    const float xr = float(q[p]) * step;
                    const double dx = double(x[p]) - double(xr);
                    err_sq += dx * dx;
                    norm_sq += double(xr) * double(xr);
                }
                int32_t pr = __shfl_up_sync(kFull, q[0], 1);
                int32_t pi = __shfl_up_sync(kFull, q[1], 1);
                const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
                const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
                const uint32_t wr = 32 - __clz(__reduce_or_sync(kFull, zr));
                const uint32_t wi = 32 - __clz(__reduce_or_sync(kFull, zi));
                for (uint32_t b = 0; b < wr; ++b) {
                    uint32_t bal = __ballot_sync(kFull, (zr >> b) & 1u);
                    if (lane == int(b)) words_r[i] = bal;
                }
                for (uint32_t b = 0; b < wi; ++b) {
                    uint32_t bal = __ballot_sync(kFull, (zi >> b) & 1u);
                    if (lane == int(b)) words_i[i] = bal;
                }
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
        if (tid < int(2 * g.C)) s_off[tid] = my_off;
        const uint32_t words = s_total;
        const uint64_t padw = (2ull * g.C + 15) & ~15ull;
        const uint32_t len = words ? uint32_t(padw + ((4ull * words + 15) & ~15ull)) : 0u;

        // ---- decoupled look-back over the preceding frames of this block ----
        if (warp == 0) {
            uint64_t *st = scr.state + uint64_t(j) * g.nframes;
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
                        while (true) {
                            uint64_t w = ld_relaxed_u64(st + p);
                            uint32_t fl = uint32_t(w >> 32) & 3u;
                            if (fl != 0 && uint32_t(w >> 34) == epoch) {
                                flag = fl;
                                val = uint32_t(w);
                                break;
                            }
                            if (++spins > kSpinLimit) {
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
        __syncthreads();
        const uint64_t frame_off = g.data_start + s_excl;
        uint8_t *out = tgt[j].ptr;
        const uint64_t cap = tgt[j].cap;
        const bool fits = frame_off + len <= cap;
        if (fits && len) {
            uint8_t *fp = out + frame_off;
            if (tid < int(padw)) fp[tid] = tid < int(2 * g.C) ? uint8_t(s_w[tid]) : uint8_t(0);
            uint32_t *payload = reinterpret_cast<uint32_t *>(fp + padw);
#pragma unroll
            for (int i = 0; i < MAX_CPW; ++i) {
                const uint32_t c = warp + i * NW;
                if (c < g.C) {
                    if (lane < int(s_w[c])) payload[s_off[c] + lane] = words_r[i];
                    if (lane < int(s_w[g.C + c])) payload[s_off[g.C + c] + lane] = words_i[i];
                }
            }
            const uint32_t padded = (len - uint32_t(padw)) / 4;  // words rounded up to 16 bytes
            if (words + uint32_t(tid) < padded) payload[words + tid] = 0;
        }
        if (!fits && tid == 0) atomicOr(&res[j].overflow, 1u);
        if (tid == 0 && g.data_start <= cap)
            reinterpret_cast<uint32_t *>(out + 32)[f] = uint32_t(frame_off);
        if (f == g.nframes - 1 && tid == 0) {
            const uint64_t total = frame_off + len;
            res[j].total = total;
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
                if (table) {
                    table[ids[j]].ptr = out;
                    table[ids[j]].bytes = total;
                    table[ids[j]].tier = tgt[j].tier;
                }
                if (acc) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), total);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->reserved_bytes), cap);
                    if (tgt[j].tier) atomicAdd(reinterpret_cast<unsigned long long *>(&acc->host_bytes), cap);
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
            s_red[0][warp] = err_sq;
            s_red[1][warp] = norm_sq;
        }
        __syncthreads();
        if (tid == 0 && !only_overflowed) {
            double a = 0, b = 0;
            for (int w = 0; w < NW; ++w) { a += s_red[0][w]; b += s_red[1][w]; }
            atomicAdd(&res[j].err_sq, a);
            atomicAdd(&res[j].norm_sq, b);
            if (acc) {
                atomicAdd(&acc->err_sq, a);
                atomicAdd(&acc->norm_sq, b);
            }
        }
    }
    // ---- last CTA resets the ticket counter and advances the epoch ----
    if (tid == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(scr.done, 1u);
        if (d == gridDim.x - 1) {
            *scr.ticket = 0;
            *scr.done = 0;
            __threadfence();
            atomicExch(scr.epoch, (epoch + 1) & kEpochMask);
        }
    }
}

// ---------------------------------------------------------------------------
// Sizing pass: exact stream size of every block (reads the data once more).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_encode_size(const float2 *__restrict__ wv, uint32_t nblocks, int m,
                                                    int e, uint64_t *__restrict__ sizes, int *status) {
    const FrameGeom g = geom(m);
    __shared__ uint32_t s_words[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t items = uint64_t(nblocks) * g.nframes;
    const float inv_step = exp2i(-e);
    for (uint64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const uint32_t j = uint32_t(item / g.nframes), f = uint32_t(item % g.nframes);
        const float2 *src = wv + (uint64_t(j) << m) + uint64_t(f) * g.F;
        uint32_t words = 0;
        int bad = 0;
        for (uint32_t c = warp; c < g.C; c += NW) {
            const float2 v = src[c * 32 + lane];
            int32_t q[2];
            const float x[2] = {v.x, v.y};
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float t = x[p] * inv_step;
                if (!isfinite(x[p])) { bad = QSIM_E_INVALID; q[p] = 0; }
                else if (fabsf(t) >= 1073741824.0f) { bad = bad ? bad : QSIM_E_RANGE; q[p] = 0; }
                else q[p] = __float2int_rn(t);
            }
            int32_t pr = __shfl_up_sync(kFull, q[0], 1);
            int32_t pi = __shfl_up_sync(kFull, q[1], 1);
            const uint32_t zr = zigzag(lane ? int32_t(uint32_t(q[0]) - uint32_t(pr)) : q[0]);
            const uint32_t zi = zigzag(lane ? int32_t(uint32_t(q[1]) - uint32_t(pi)) : q[1]);
            words += (32 - __clz(__reduce_or_sync(kFull, zr))) + (32 - __clz(__reduce_or_sync(kFull, zi)));
        }
        if (bad) raise_status(status, bad);
        if (lane == 0) s_words[warp] = words;
        __syncthreads();
        if (tid == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < NW; ++w) tot += s_words[w];
            const uint64_t padw = (2ull * g.C + 15) & ~15ull;
            const uint64_t len = tot ? padw + ((4ull * tot + 15) & ~15ull) : 0;
            if (len) atomicAdd(reinterpret_cast<unsigned long long *>(&sizes[j]), len);
        }
        __syncthreads();
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
    const uint64_t sz = (want + 255) & ~255ull;
    uint64_t off = atomicAdd(reinterpret_cast<unsigned long long *>(dev.bump), sz);
    if (off + sz <= dev.cap) {
        tgt[j].ptr = dev.base + off;
        tgt[j].cap = sz;
        tgt[j].tier = 0;
        return;
    }
    if (host.base) {
        off = atomicAdd(reinterpret_cast<unsigned long long *>(host.bump), sz);
        if (off + sz <= host.cap) {
            tgt[j].ptr = host.base + off;
            tgt[j].cap = sz;
            tgt[j].tier = 1;
            return;
        }
    }
    tgt[j].ptr = nullptr;
    tgt[j].cap = 0;
    tgt[j].tier = 0;
    raise_status(status, QSIM_E_NOMEM);
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
                   cudaStream_t s) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    k_decode<<<grid_for(items, 152 * 8), NT, 0, s>>>(in, nblocks, m, wv, hist, status);
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

void launch_encode_size(const float2 *wv, uint32_t nblocks, int m, int e, uint64_t *sizes, int *status,
                        cudaStream_t s) {
    const uint64_t items = uint64_t(nblocks) * qsz_nframes(m);
    k_encode_size<<<grid_for(items, 152 * 8), NT, 0, s>>>(wv, nblocks, m, e, sizes, status);
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
