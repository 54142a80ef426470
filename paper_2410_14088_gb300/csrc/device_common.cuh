// Device-side helpers shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsim {

constexpr unsigned kFull = 0xffffffffu;

// First error wins; later ones are dropped.
__device__ __forceinline__ void raise_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// nanoseconds of the GPU's global timer (for time-bounded waits)
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// 2^e as a float for e in [-126, 127] (a normal number, exact).
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// Transpose the 32x32 bit matrix held one row per lane (row = lane, column =
// bit): afterwards lane j holds the word whose bit i was bit j of lane i.
// Stage s exchanges s x s sub-blocks between lanes l and l ^ s: the lower
// lane keeps the bits under mask `left` and takes the partner's bits under
// `left` moved up by s; the upper lane keeps ~left and takes the partner's
// ~left bits moved down by s. Each lane sends its word rotated (right by s
// from the lower lane, left by s from the upper one), so that the received
// word already has the needed bits in place: one rotate, one shuffle and one
// bitwise select per stage. The masks repeat with period 2s, so the upper
// lane's mask ~left is `left` rotated by s.
__device__ __forceinline__ uint32_t warp_bit_transpose(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t left = (s == 16) ? 0x0000FFFFu
                            : (s == 8)  ? 0x00FF00FFu
                            : (s == 4)  ? 0x0F0F0F0Fu
                            : (s == 2)  ? 0x33333333u
                                        : 0x55555555u;
        const uint32_t t = uint32_t(lane) & uint32_t(s);                    // 0 (lower) or s (upper)
        const uint32_t keep = __funnelshift_r(left, left, t);                // ~left = left rotated by s
        const uint32_t sent = __funnelshift_r(x, x, uint32_t(s) - 2u * t);  // rotate right by s or 32 - s
        const uint32_t got = __shfl_xor_sync(kFull, sent, s);
        x = (x & keep) | (got & ~keep);
    }
    return x;
}

// Exclusive scan of `count` (<= blockDim.x) values held by threads 0..count-1
// in a block of `NT` threads; returns the thread's exclusive prefix and writes
// the total to *total (shared). `warp_sums` must hold NT/32 entries.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? warp_sums[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NT / 32) warp_sums[lane] = wi - w;
        if (lane == NT / 32 - 1) *total = wi;
    }
    __syncthreads();
    return warp_sums[warp] + incl - v;
}

}  // namespace qsim
