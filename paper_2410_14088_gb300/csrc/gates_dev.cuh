// Device functions of the gate passes (shared by the per-pass kernels and the
// persistent stage kernel). See gates.cu for the method.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"
#include "umma.cuh"

namespace qsim {
namespace gdev {


__device__ __forceinline__ uint32_t swz(uint32_t i) {
    return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15u);
}

// CTA-cooperative copy of a descriptor (4-byte words; src may be kernel-parameter or global memory)
template <int NT, class T>
__device__ __forceinline__ void coop_copy(T &dst, const T &src) {
    static_assert(sizeof(T) % 4 == 0, "descriptor size");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int t = threadIdx.x; t < int(sizeof(T) / 4); t += NT) d[t] = s[t];
}

struct PassSmem {
    PassDev p;
    // 4096-amplitude tiles: element tid + NT u sits at working offset thread_tile_offset(tid) + off12[u]
    uint32_t off12[32];
    uint32_t offs_sw[64];  // dense op: tile offsets of its 2^k matrix columns through the swizzle
    // dense op: swizzled base of index group g = cb[0][g & 63] ^ cb[1][g >> 6] (the swizzle is
    // linear over GF(2), so swz(b | c) = swz(b) ^ swz(c) for disjoint bit sets b, c)
    uint32_t cb[2][64];
    uint32_t dconst[kDiagRun];  // diagonal op d of a run: phase-index bits constant over the tile
    uint32_t pA[13];            // polynomial run: tile bit t's linear coefficient (t < 12) and the constant (12),
                                // angles in turns as 32-bit fixed point
    float2 ck[2];
    uint32_t cbconst;           // the branch when the control is outside the tile
    // passes with tcgen05 dense ops: the MMA-completion mbarrier and the TMEM accumulator's base address
    uint64_t mbar;
    uint32_t tmem;
};
static_assert(sizeof(OpDev) % 16 == 0, "op descriptors are copied as 16-byte words");

template <int NT, int K>
__device__ __forceinline__ void apply_dense(float2 *tile, const float2 *U, const uint32_t *cb, const uint32_t *osw,
                                            uint32_t T) {
    constexpr int D = 1 << K;
    const uint32_t ngroups = 1u << (T - K);
    for (uint32_t g = threadIdx.x; g < ngroups; g += NT) {
        const uint32_t sb = cb[g & 63u] ^ cb[64u + (g >> 6)];
        float2 x[D];
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = tile[sb ^ osw[c]];
#pragma unroll 1
        for (int r = 0; r < D; ++r) {
            const float4 *row = reinterpret_cast<const float4 *>(U + r * D);
            float ar = 0.f, ai = 0.f;
            if constexpr (D == 2) {
                float4 u = row[0];
                ar = fmaf(u.x, x[0].x, ar); ar = fmaf(-u.y, x[0].y, ar);
                ai = fmaf(u.x, x[0].y, ai); ai = fmaf(u.y, x[0].x, ai);
                ar = fmaf(u.z, x[1].x, ar); ar = fmaf(-u.w, x[1].y, ar);
                ai = fmaf(u.z, x[1].y, ai); ai = fmaf(u.w, x[1].x, ai);
            } else {
#pragma unroll
                for (int c = 0; c < D; c += 2) {
                    float4 u = row[c / 2];
                    ar = fmaf(u.x, x[c].x, ar); ar = fmaf(-u.y, x[c].y, ar);
                    ai = fmaf(u.x, x[c].y, ai); ai = fmaf(u.y, x[c].x, ai);
                    ar = fmaf(u.z, x[c + 1].x, ar); ar = fmaf(-u.w, x[c + 1].y, ar);
                    ai = fmaf(u.z, x[c + 1].y, ai); ai = fmaf(u.w, x[c + 1].x, ai);
                }
            }
            tile[sb ^ osw[r]] = make_float2(ar, ai);
        }
    }
}

template <int NT>
__device__ __forceinline__ void apply_dense_k1(float2 *tile, const float2 *U, const uint32_t *cb, const uint32_t *osw,
                                               uint32_t T) {
    const uint32_t ngroups = 1u << (T - 1);
    const float2 u00 = U[0], u01 = U[1], u10 = U[2], u11 = U[3];
    for (uint32_t g = threadIdx.x; g < ngroups; g += NT) {
        const uint32_t i0 = cb[g & 63u] ^ cb[64u + (g >> 6)], i1 = i0 ^ osw[1];
        const float2 x0 = tile[i0], x1 = tile[i1];
        tile[i0] = make_float2(u00.x * x0.x - u00.y * x0.y + u01.x * x1.x - u01.y * x1.y,
                               u00.x * x0.y + u00.y * x0.x + u01.x * x1.y + u01.y * x1.x);
        tile[i1] = make_float2(u10.x * x0.x - u10.y * x0.y + u11.x * x1.x - u11.y * x1.y,
                               u10.x * x0.y + u10.y * x0.x + u11.x * x1.y + u11.y * x1.x);
    }
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recent committed group complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }


// ---------------------------------------------------------------------------
// Tensor-core dense ops (warp-level MMA). A dense k-qubit op on the tile is the
// real GEMM  Y^T (G x 2D) = X^T (G x 2D) * U_r^T (2D x 2D), D = 2^k, G = 2^(T-k)
// index groups, with U_r = [[Re U, -Im U], [Im U, Re U]] acting on
// (re_0..re_{D-1}, im_0..im_{D-1}). Each warp owns G/4 rows (groups): it reads
// its rows' inputs from the tile into A fragments, accumulates in FP32 and
// writes its rows' outputs back in place (no other warp touches those rows).
// TF32: one m16n8k8 MMA per fragment. BF16x3: x = hi + mid + lo (BF16 each),
// the six products of order <= 2 (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi,
// mid*mid) with m16n8k16, all into the same FP32 accumulators.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// three BF16 parts of x: hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half) {
    return uint32_t(__bfloat16_as_ushort(lo_half)) | (uint32_t(__bfloat16_as_ushort(hi_half)) << 16);
}

template <int NT, int K, int PREC>
__device__ __forceinline__ void apply_dense_mma(float2 *tile, const uint32_t *__restrict__ bfr, const uint32_t *cb,
                                                const uint32_t *osw,
                                                uint32_t T) {
    // tensor-core shape: T = 12 (4096-amplitude tiles), checked by the caller
    constexpr uint32_t D = 1u << K, N2 = 2 * D;
    constexpr uint32_t KW = PREC == QSIM_PREC_TF32 ? 8 : 16;  // MMA k width
    constexpr uint32_t KS = N2 / KW;                           // k-steps; the first half reads Re, the second Im
    constexpr uint32_t NTILES = N2 / 8;                        // n8 tiles
    constexpr uint32_t ROWS = (1u << (12 - K)) / (NT / 32);    // index groups per warp
    constexpr uint32_t MT = ROWS / 16;                         // m16 tiles per warp
    static_assert(MT >= 1, "tensor-core tile needs 16 rows per warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t gq = lane >> 2, tq = lane & 3;
    const uint32_t row0 = warp * ROWS;
    uint32_t base[MT][2];  // swizzled bases of the lane's index groups
#pragma unroll
    for (uint32_t mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t g = row0 + mt * 16 + gq + 8 * h;
            base[mt][h] = cb[g & 63u] ^ cb[64u + (g >> 6)];
        }
    float acc[MT * NTILES][4];
#pragma unroll
    for (uint32_t i = 0; i < MT * NTILES; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    const uint2 *bf2 = reinterpret_cast<const uint2 *>(bfr);
    // k-step pairs (ks, ks + KS/2) read the same complex inputs: Re parts for ks, Im parts for ks + KS/2;
    // unrolled so that the next pair's operand loads overlap the current pair's MMAs
#pragma unroll
    for (uint32_t ks = 0; ks < KS / 2; ++ks) {
        if constexpr (PREC == QSIM_PREC_TF32) {
            const uint32_t c0 = osw[ks * 8 + tq], c1 = osw[ks * 8 + tq + 4];
            uint32_t are[MT][4], aim[MT][4];
#pragma unroll
            for (uint32_t mt = 0; mt < MT; ++mt) {
                const float2 v00 = tile[base[mt][0] ^ c0], v10 = tile[base[mt][1] ^ c0];
                const float2 v01 = tile[base[mt][0] ^ c1], v11 = tile[base[mt][1] ^ c1];
                are[mt][0] = f32_to_tf32(v00.x); are[mt][1] = f32_to_tf32(v10.x);
                are[mt][2] = f32_to_tf32(v01.x); are[mt][3] = f32_to_tf32(v11.x);
                aim[mt][0] = f32_to_tf32(v00.y); aim[mt][1] = f32_to_tf32(v10.y);
                aim[mt][2] = f32_to_tf32(v01.y); aim[mt][3] = f32_to_tf32(v11.y);
            }
#pragma unroll
            for (uint32_t nt = 0; nt < NTILES; ++nt) {
                const uint2 bre = __ldg(bf2 + (ks * NTILES + nt) * 32 + lane);
                const uint2 bim = __ldg(bf2 + ((ks + KS / 2) * NTILES + nt) * 32 + lane);
                const uint32_t b0[2] = {bre.x, bre.y}, b1[2] = {bim.x, bim.y};
#pragma unroll
                for (uint32_t mt = 0; mt < MT; ++mt) {
                    mma_tf32(acc[mt * NTILES + nt], are[mt], b0);
                    mma_tf32(acc[mt * NTILES + nt], aim[mt], b1);
                }
            }
        } else {
            // columns 2t, 2t+1, 2t+8, 2t+9 of the k-step
            const uint32_t cc[4] = {osw[ks * 16 + 2 * tq], osw[ks * 16 + 2 * tq + 1],
                                    osw[ks * 16 + 2 * tq + 8], osw[ks * 16 + 2 * tq + 9]};
            constexpr uint32_t PART = KS * NTILES * 32;  // uint2 entries per part
#pragma unroll
            for (int ri = 0; ri < 2; ++ri) {  // Re inputs with k-step ks, then Im inputs with ks + KS/2
#pragma unroll
                for (uint32_t mt = 0; mt < MT; ++mt) {
                    uint32_t ah[4], am[4], al[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t b = base[mt][q & 1];
                        const float2 x0 = tile[b ^ cc[(q >> 1) * 2]], x1 = tile[b ^ cc[(q >> 1) * 2 + 1]];
                        __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                        split3(ri ? x0.y : x0.x, h0, m0, l0);
                        split3(ri ? x1.y : x1.x, h1, m1, l1);
                        ah[q] = pack_bf16(h0, h1);
                        am[q] = pack_bf16(m0, m1);
                        al[q] = pack_bf16(l0, l1);
                    }
#pragma unroll
                    for (uint32_t nt = 0; nt < NTILES; ++nt) {
                        const uint32_t e = ((ks + ri * (KS / 2)) * NTILES + nt) * 32 + lane;
                        const uint2 bh = __ldg(bf2 + e), bm = __ldg(bf2 + PART + e), bl = __ldg(bf2 + 2 * PART + e);
                        const uint32_t vh[2] = {bh.x, bh.y}, vm[2] = {bm.x, bm.y}, vl[2] = {bl.x, bl.y};
                        float (&c)[4] = acc[mt * NTILES + nt];
                        mma_bf16(c, al, vh);
                        mma_bf16(c, ah, vl);
                        mma_bf16(c, am, vm);
                        mma_bf16(c, am, vh);
                        mma_bf16(c, ah, vm);
                        mma_bf16(c, ah, vh);
                    }
                }
            }
        }
    }
    __syncwarp();
    const uint32_t *offs = osw;
    // outputs: n-tile j < NTILES/2 holds Re of outputs 8j + 2tq (+1), tile j + NTILES/2 the Im parts
#pragma unroll
    for (uint32_t mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (uint32_t j = 0; j < NTILES / 2; ++j) {
            const float (&re)[4] = acc[mt * NTILES + j];
            const float (&im)[4] = acc[mt * NTILES + j + NTILES / 2];
            const uint32_t r0 = 8 * j + 2 * tq;
            tile[base[mt][0] ^ offs[r0]] = make_float2(re[0], im[0]);
            tile[base[mt][0] ^ offs[r0 + 1]] = make_float2(re[1], im[1]);
            tile[base[mt][1] ^ offs[r0]] = make_float2(re[2], im[2]);
            tile[base[mt][1] ^ offs[r0 + 1]] = make_float2(re[3], im[3]);
        }
    }
}

// Bytes of shared memory a tcgen05 pass adds: the B operand of one op (TF32 64 x 64, or split BF16 in three
// 64 x 64 parts) and the slack that aligns the tile (the A operand while the MMAs run) to 1024 bytes.
template <int PREC>
__host__ __device__ constexpr uint32_t umma_b_bytes() {
    return PREC == QSIM_PREC_BF16X3 ? 24576u : 16384u;
}
// B buffer of a tcgen05 pass from its PassDev::umma bits: 64 KB with a width-6 op, else the width-5 operand's size
__host__ __device__ constexpr uint32_t umma_pass_b_bytes(uint32_t umma_bits) {
    return (umma_bits & 8u) ? 65536u : (umma_bits & 4u) ? umma_b_bytes<QSIM_PREC_BF16X3>() : umma_b_bytes<QSIM_PREC_TF32>();
}
// TMEM columns of a tcgen05 pass: D in columns 0..63 (0..127 for width 6) and, for the width-5 TF32 form, A in
// columns kUmmaACol .. kUmmaACol + 63; 128 in every case (four resident CTAs fill the SM's 512)
__host__ __device__ constexpr uint32_t umma_pass_tmem_cols(uint32_t) { return 128u; }
constexpr uint32_t kUmmaACol = 64;
constexpr uint32_t kUmmaIdesc = umma::idesc_tf32(128, 64);
constexpr uint32_t kUmmaIdesc6 = umma::idesc_tf32(128, 128);
constexpr uint32_t kUmmaIdescBf16 = umma::idesc_bf16(128, 64);
constexpr uint64_t kUmmaWaitNs = 1000000000ull;  // bound on one MMA-completion wait

// Commit the MMAs issued by thread 0 (unless the test hook asks otherwise) and wait, bounded, for them; the
// outcome is made uniform so that every thread takes the same path. False (status set) when the wait ran out.
__device__ __forceinline__ bool umma_commit_wait(const PassSmem &S, uint32_t &phase, int *status) {
    const uint32_t bar = umma::smem_addr(&S.mbar);
    // test hook (bit 1): no MMA was issued and nothing is committed, so the wait runs out with no MMA in flight
    if (threadIdx.x == 0 && !(S.p.umma & 2u)) umma::commit(bar);
    const bool ok = __syncthreads_and(umma::mbar_wait(bar, phase, kUmmaWaitNs));
    phase ^= 1u;
    if (!ok && threadIdx.x == 0) raise_status(status, QSIM_E_TIMEOUT);
    return ok;
}

// The swizzled tile offsets of a width-5 op's 32 columns from its five basis columns: the column map and the
// swizzle are linear over GF(2), so osw[j] is the XOR of osw[2^b] over the set bits b of j (osw[0] = 0). Five
// shared-memory reads per thread instead of 32.
struct ColBasis {
    uint32_t b[5];
};
__device__ __forceinline__ ColBasis col_basis(const uint32_t *osw) {
    ColBasis c;
#pragma unroll
    for (uint32_t t = 0; t < 5; ++t) c.b[t] = osw[1u << t];
    return c;
}
// Step i of a walk over the 32 columns in Gray-code order: column gray(i) = i ^ (i >> 1), whose offset differs from
// the previous step's by basis column ctz(i) (one XOR into a running address)
__device__ __forceinline__ constexpr uint32_t gray5(uint32_t i) { return i ^ (i >> 1); }
__device__ __forceinline__ constexpr uint32_t ctz5(uint32_t i) {
    return (i & 1u) ? 0u : (i & 2u) ? 1u : (i & 4u) ? 2u : (i & 8u) ? 3u : 4u;
}

// Row g of D (TMEM lane g: Re of the 32 outputs in columns 0..31, Im in 32..63) back to the group's tile
// positions, in the gather's Gray-code order (one XOR into a running address per step, from the five basis
// offsets, instead of a table read per output) and in two halves of 16 columns: the first 16 steps of the walk
// visit columns 0..15, the last 16 columns 16..31, so each half needs only its 16 Re and 16 Im columns of D.
__device__ __forceinline__ void umma_epilogue(float2 *tile, uint32_t base, const uint32_t *osw, const PassSmem &S) {
    umma::fence_after_sync();
    const uint32_t taddr = S.tmem + ((32u * (threadIdx.x >> 5)) << 16);
    const ColBasis cbs = col_basis(osw);
    uint32_t a = base;
#pragma unroll
    for (uint32_t h = 0; h < 2; ++h) {
        uint32_t re[16], im[16];
        umma::tmem_ld16x2(taddr + 16u * h, re, taddr + 32u + 16u * h, im);
#pragma unroll
        for (uint32_t i = 16u * h; i < 16u * h + 16u; ++i) {
            if (i) a ^= cbs.b[ctz5(i)];
            const uint32_t j = gray5(i) - 16u * h;
            tile[a] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
        }
    }
    umma::fence_before_sync();  // the next op's barrier orders these TMEM reads before its MMAs
}

// Dense op of width 5 (TF32) on a 4096-amplitude tile with the 5th-generation tensor cores: the real form
// D = A * B with A = 128 index groups x 64 inputs (Re parts of the group's 32 amplitudes in K columns
// 0..31, Im parts in 32..63), B = the op's 64 x 64 real matrix (host-built, staged at `bsm` in the K-major
// 128-byte swizzled layout: B^T row n = output n, Re outputs first), D in TMEM (lane = group, 64 FP32
// columns). Thread g owns index group g: it gathers the group's amplitudes into registers and stores them,
// rounded to TF32, as row g of A in TMEM (lane g, from column kUmmaACol), so A never passes through shared
// memory; one thread issues the eight K = 8 MMAs (A from TMEM, B from shared memory) and commits them to the
// mbarrier; every thread waits (bounded), reads its D row from TMEM and writes the group's outputs back to
// their tile positions, which only it owns in this op.
// Returns false when the wait ran out (status set; the tile is then left unwritten).
template <int NT>
__device__ __forceinline__ bool apply_dense_umma(float2 *tile, uint32_t bsm, const uint32_t *cb, const uint32_t *osw,
                                                 const PassSmem &S, uint32_t &phase,
                                                 int *status);

template <int NT>
__device__ __forceinline__ bool apply_dense_umma(float2 *tile, uint32_t bsm, const uint32_t *cb, const uint32_t *osw,
                                                 const PassSmem &S, uint32_t &phase,
                                                 int *status) {
    static_assert(NT == 128, "one thread per index group");
    const uint32_t g = threadIdx.x;
    const uint32_t base = cb[g & 63u] ^ cb[64u + (g >> 6)];
    {
        const ColBasis cbs = col_basis(osw);
        uint32_t re[32], im[32];
        uint32_t a = base;
#pragma unroll
        for (uint32_t i = 0; i < 32; ++i) {
            if (i) a ^= cbs.b[ctz5(i)];
            const float2 v = tile[a];
            re[gray5(i)] = f32_to_tf32(v.x);
            im[gray5(i)] = f32_to_tf32(v.y);
        }
        // row g of A is TMEM lane g: Re parts in columns kUmmaACol.., Im parts 32 further (the tile stays as it is)
        const uint32_t ta = S.tmem + ((32u * (g >> 5)) << 16) + kUmmaACol;
        umma::tmem_st32(ta, re);
        umma::tmem_st32(ta + 32u, im);
        umma::tmem_wait_st();
    }
    cp_async_wait_all();  // this thread's share of B
    umma::fence_proxy_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    if (g == 0 && !(S.p.umma & 2u)) {  // the test hook issues nothing
        umma::fence_after_sync();
#pragma unroll
        for (uint32_t s = 0; s < 8; ++s) {
            const uint64_t db = umma::desc_kmajor_sw128(bsm + (s >> 2) * 8192u + (s & 3u) * 32u);
            umma::mma_tf32_ts(S.tmem, S.tmem + kUmmaACol + 8u * s, db, kUmmaIdesc, s);
        }
    }
    if (!umma_commit_wait(S, phase, status)) return false;
    umma_epilogue(tile, base, osw, S);
    return true;
}

// Dense op of width 6 (TF32) on a 4096-amplitude tile with tcgen05: 64 index groups, K = 128 inputs (Re parts of
// the group's 64 amplitudes, then Im parts) in four 128-byte K-chunks of 8 KB (64 rows each), N = 128 outputs, B
// (64 KB, from build_umma_b6) at `bsm`. Threads g and g + 64 share group g, each gathering 32 of its amplitudes
// into K-chunks h and 2 + h. The MMAs run at M = 128: the descriptor's rows 64..127 read the next K-chunk (the
// last one's read the B buffer after the tile), valid shared memory whose results land in TMEM lanes 64..127 and
// are never read. Warps 0 and 1 (TMEM lanes 0..63) take the 64 rows of D back, two halves of 32 outputs each.
template <int NT>
__device__ __forceinline__ bool apply_dense_umma6(float2 *tile, uint32_t bsm, const uint32_t *cb, const uint32_t *osw,
                                                  const PassSmem &S, uint32_t &phase, int *status) {
    static_assert(NT == 128, "two threads per index group");
    const uint32_t g = threadIdx.x & 63u, h = threadIdx.x >> 6;
    const uint32_t base = cb[g] ^ cb[64];
    {
        uint32_t re[32], im[32];
#pragma unroll
        for (uint32_t j = 0; j < 32; ++j) {
            const float2 v = tile[base ^ osw[32u * h + j]];
            re[j] = f32_to_tf32(v.x);
            im[j] = f32_to_tf32(v.y);
        }
        __syncthreads();  // every amplitude of the tile is in registers
        uint8_t *row = reinterpret_cast<uint8_t *>(tile) + (g >> 3) * 1024u + (g & 7u) * 128u;
#pragma unroll
        for (uint32_t c = 0; c < 8; ++c) {
            const uint32_t o = (c ^ (g & 7u)) << 4;
            *reinterpret_cast<uint4 *>(row + h * 8192u + o) =
                make_uint4(re[4 * c], re[4 * c + 1], re[4 * c + 2], re[4 * c + 3]);
            *reinterpret_cast<uint4 *>(row + (2u + h) * 8192u + o) =
                make_uint4(im[4 * c], im[4 * c + 1], im[4 * c + 2], im[4 * c + 3]);
        }
    }
    cp_async_wait_all();  // this thread's share of B
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && !(S.p.umma & 2u)) {  // the test hook issues nothing
        umma::fence_after_sync();
        const uint32_t a0 = umma::smem_addr(tile);
#pragma unroll
        for (uint32_t s = 0; s < 16; ++s) {
            const uint64_t da = umma::desc_kmajor_sw128(a0 + (s >> 2) * 8192u + (s & 3u) * 32u);
            const uint64_t db = umma::desc_kmajor_sw128(bsm + (s >> 2) * 16384u + (s & 3u) * 32u);
            umma::mma_tf32_ss(S.tmem, da, db, kUmmaIdesc6, s);
        }
    }
    if (!umma_commit_wait(S, phase, status)) return false;
    umma::fence_after_sync();
    if (threadIdx.x < 64) {
        // row g = threadIdx.x of D: Re of output j in column j, Im in column 64 + j
        const uint32_t taddr = S.tmem + ((32u * (threadIdx.x >> 5)) << 16);
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            uint32_t re[32], im[32];
            umma::tmem_ld32(taddr + 32u * half, re);
            umma::tmem_ld32(taddr + 64u + 32u * half, im);
#pragma unroll
            for (uint32_t j = 0; j < 32; ++j)
                tile[base ^ osw[32u * half + j]] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
        }
    }
    umma::fence_before_sync();  // the next op's barrier orders these TMEM reads before its MMAs
    return true;
}

// The same op in split BF16 (x = hi + mid + lo, each part BF16; the six products of order <= 2 accumulated
// in FP32) on tcgen05 (kind::f16, K = 16 per MMA). A row = 64 BF16 values = one 128-byte row per part, so
// the tile's two 16 KB halves hold two parts at a time: first A_hi and A_lo for lo x B_hi and hi x B_lo,
// then A_mid over A_lo for mid x B_mid, mid x B_hi, hi x B_mid, hi x B_hi (small terms first; each thread
// keeps its A_mid words in registers across the first wait). B: three 8 KB parts (hi, mid, lo) at bsm.
template <int NT>
__device__ __forceinline__ bool apply_dense_umma3(float2 *tile, uint32_t bsm, const uint32_t *cb, const uint32_t *osw,
                                                  const PassSmem &S, uint32_t &phase,
                                                  int *status) {
    static_assert(NT == 128, "one thread per index group");
    const uint32_t g = threadIdx.x;
    const uint32_t base = cb[g & 63u] ^ cb[64u + (g >> 6)];
    const ColBasis cbs = col_basis(osw);
    float x[64];  // K order: Re parts of inputs 0..31, then Im parts
    uint32_t a = base;
#pragma unroll
    for (uint32_t i = 0; i < 32; ++i) {
        if (i) a ^= cbs.b[ctz5(i)];
        const float2 v = tile[a];
        x[gray5(i)] = v.x;
        x[32 + gray5(i)] = v.y;
    }
    __syncthreads();  // every amplitude of the tile is in registers
    uint8_t *arow = reinterpret_cast<uint8_t *>(tile) + (g >> 3) * 1024u + (g & 7u) * 128u;
    uint32_t mid[32];
#pragma unroll
    for (uint32_t c = 0; c < 8; ++c) {  // 16-byte chunk c = K elements 8c .. 8c + 7
        uint32_t h[4], l[4];
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(x[8 * c + 2 * q], h0, m0, l0);
            split3(x[8 * c + 2 * q + 1], h1, m1, l1);
            h[q] = pack_bf16(h0, h1);
            l[q] = pack_bf16(l0, l1);
            mid[4 * c + q] = pack_bf16(m0, m1);
        }
        const uint32_t o = (c ^ (g & 7u)) << 4;
        *reinterpret_cast<uint4 *>(arow + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(arow + 16384u + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    cp_async_wait_all();  // this thread's share of B
    umma::fence_proxy_async_smem();
    __syncthreads();
    const uint32_t a0 = umma::smem_addr(tile);
    auto product = [&](uint32_t a_half, uint32_t b_part, uint32_t first) {
#pragma unroll
        for (uint32_t s = 0; s < 4; ++s) {
            const uint64_t da = umma::desc_kmajor_sw128(a0 + a_half * 16384u + s * 32u);
            const uint64_t db = umma::desc_kmajor_sw128(bsm + b_part * 8192u + s * 32u);
            umma::mma_bf16_ss(S.tmem, da, db, kUmmaIdescBf16, first && s == 0 ? 0u : 1u);
        }
    };
    if (g == 0 && !(S.p.umma & 2u)) {  // the test hook issues nothing
        umma::fence_after_sync();
        product(1, 0, 1);  // lo x B_hi (the first product overwrites D)
        product(0, 2, 0);  // hi x B_lo
    }
    if (!umma_commit_wait(S, phase, status)) return false;
#pragma unroll
    for (uint32_t c = 0; c < 8; ++c) {
        const uint32_t o = (c ^ (g & 7u)) << 4;
        *reinterpret_cast<uint4 *>(arow + 16384u + o) =
            make_uint4(mid[4 * c], mid[4 * c + 1], mid[4 * c + 2], mid[4 * c + 3]);
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (g == 0 && !(S.p.umma & 2u)) {
        umma::fence_after_sync();
        product(1, 1, 0);  // mid x B_mid
        product(1, 0, 0);  // mid x B_hi
        product(0, 1, 0);  // hi x B_mid
        product(0, 0, 0);  // hi x B_hi
    }
    if (!umma_commit_wait(S, phase, status)) return false;
    umma_epilogue(tile, base, osw, S);
    return true;
}

// Dense op of width k (<= KMAX) on the shared-memory tile; the tensor-core
// form needs 4096-amplitude tiles and at least 16 index groups per warp.
template <int NT, int KMAX, int PREC>
__device__ __forceinline__ void apply_dense_dispatch(uint32_t k, float2 *tile, const float2 *mat, const uint32_t *bfr,
                                                     const uint32_t *cb, const uint32_t *osw, uint32_t T) {
    constexpr bool TC = PREC != QSIM_PREC_FP32;
    const uint32_t min_k = PREC == QSIM_PREC_TF32 ? 3u : 4u;  // an MMA k-step must not straddle Re and Im
    const bool tc_ok = TC && k >= min_k && k <= 5 && T == 12;  // 16+ index groups per warp for NT <= 256
    switch (k) {
        case 1: apply_dense_k1<NT>(tile, mat, cb, osw, T); break;
        case 2: if constexpr (KMAX >= 2) apply_dense<NT, 2>(tile, mat, cb, osw, T); break;
        case 3:
            if constexpr (KMAX >= 3) {
                if constexpr (PREC == QSIM_PREC_TF32) {
                    if (tc_ok) { apply_dense_mma<NT, 3, PREC>(tile, bfr, cb, osw, T); break; }
                }
                apply_dense<NT, 3>(tile, mat, cb, osw, T);
            }
            break;
        case 4:
            if constexpr (KMAX >= 4) {
                if (tc_ok) apply_dense_mma<NT, 4, PREC>(tile, bfr, cb, osw, T);
                else apply_dense<NT, 4>(tile, mat, cb, osw, T);
            }
            break;
        case 5:
            if constexpr (KMAX >= 5) {
                if (tc_ok) apply_dense_mma<NT, 5, PREC>(tile, bfr, cb, osw, T);
                else apply_dense<NT, 5>(tile, mat, cb, osw, T);
            }
            break;
        default:
            if constexpr (KMAX >= 6) apply_dense<NT, 6>(tile, mat, cb, osw, T);
            break;
    }
}

// Per pass, once per CTA: the pass descriptor and the offsets of the tile's
// high part (tile bits L..T-1 placed at their working bits).
template <int NT>
__device__ __forceinline__ void pass_setup(const PassDev &pd, PassSmem &S) {
    coop_copy<NT>(S.p, pd);
    __syncthreads();
    const uint32_t T = S.p.T;
    constexpr uint32_t A = NT == 256 ? 8 : 7;
    if (T == 12) {
        // element i = tid + NT u: tile bits 0..A-1 from tid (thread_tile_offset), A..11 from u (disjoint working
        // bits)
        const uint32_t x = threadIdx.x;
        if (x < (4096u / NT)) {
            uint32_t h = 0;
            for (uint32_t t = A; t < 12; ++t) h |= ((x >> (t - A)) & 1u) << S.p.tile_pos[t];
            S.off12[x] = h;
        }
    }
    __syncthreads();
}

constexpr uint32_t kCgBatch = 16;

// Working offset of tile bits 0..A-1 taken from this thread's index (A = 7 for 128 threads, 8 for 256): the
// thread-dependent part of the 4096-amplitude tile addressing, computed where it is used rather than kept in a
// shared table
template <int NT>
__device__ __forceinline__ uint32_t thread_tile_offset(const PassSmem &S) {
    constexpr uint32_t A = NT == 256 ? 8 : 7;
    uint32_t o = 0;
#pragma unroll
    for (uint32_t t = 0; t < A; ++t) o |= ((uint32_t(threadIdx.x) >> t) & 1u) << S.p.tile_pos[t];
    return o;
}

// Fast tile addressing for T = 12: element i = tid + NT u sits at working
// offset tpart[tid] + off12[u] and at shared index (tid ^ xt) ^ xu(u) + NT u,
// the XOR swizzle split into a per-thread and a per-u part.
template <int NT>
__device__ __forceinline__ uint32_t swz_thread(uint32_t tid) {
    return tid ^ (NT == 256 ? ((tid >> 4) & 15u) : ((tid >> 4) & 7u));
}
template <int NT>
__device__ __forceinline__ constexpr uint32_t swz_u(uint32_t u) {
    return NT == 256 ? (u & 15u) : (((u & 1u) << 3) ^ ((u >> 1) & 15u));
}
template <int NT>
__device__ __forceinline__ bool fast12(const PassSmem &S) {
    return S.p.T == 12;
}

// working offset of the tile bits L..T-1 of tile element h << L (tiles other than 4096 amplitudes)
__device__ __forceinline__ uint32_t hi_off(const PassSmem &S, uint32_t h) {
    uint32_t o = 0;
    for (uint32_t t = 0; t < S.p.T - S.p.L; ++t) o |= ((h >> t) & 1u) << S.p.tile_pos[S.p.L + t];
    return o;
}

// working index of element 0 of tile `cta` (its non-tile bits)
__device__ __forceinline__ uint64_t tile_base(const PassSmem &S, uint64_t cta) {
    uint64_t base = 0;
    for (uint32_t t = 0; t < S.p.nout; ++t) base |= ((cta >> t) & 1ull) << S.p.out_pos[t];
    return base;
}

// Stage a tile in shared memory: cp.async (the caller commits and waits), or
// with CG batches of eight L2-only loads in flight per thread (data written by
// other CTAs of the same launch).
template <int NT, bool CG>
__device__ __forceinline__ void tile_load(const float2 *__restrict__ g, uint64_t base, const PassSmem &S,
                                          float2 *tile) {
    const uint32_t T = S.p.T, L = S.p.L, lmask = (1u << L) - 1;
    const int tid = threadIdx.x;
    if (fast12<NT>(S)) {
        const float2 *gt = g + (base | uint64_t(thread_tile_offset<NT>(S)));
        const uint32_t tq = swz_thread<NT>(tid);
        if constexpr (CG) {
            constexpr uint32_t B = kCgBatch;  // L2 loads in flight per thread
#pragma unroll
            for (uint32_t u0 = 0; u0 < 4096u / NT; u0 += B) {
                float2 v[B];
#pragma unroll
                for (uint32_t u = 0; u < B; ++u) v[u] = __ldcg(gt + S.off12[u0 + u]);
#pragma unroll
                for (uint32_t u = 0; u < B; ++u) tile[(tq ^ swz_u<NT>(u0 + u)) + NT * (u0 + u)] = v[u];
            }
        } else {
#pragma unroll
            for (uint32_t u = 0; u < 4096u / NT; ++u) cp_async8(&tile[(tq ^ swz_u<NT>(u)) + NT * u], gt + S.off12[u]);
        }
        return;
    }
    if constexpr (CG) {
        for (uint32_t i0 = tid; i0 < (1u << T); i0 += 8 * NT) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t i = i0 + u * NT;
                if (i < (1u << T)) v[u] = __ldcg(&g[base | (i & lmask) | hi_off(S, i >> L)]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t i = i0 + u * NT;
                if (i < (1u << T)) tile[swz(i)] = v[u];
            }
        }
    } else {
        for (uint32_t i = tid; i < (1u << T); i += NT) cp_async8(&tile[swz(i)], &g[base | (i & lmask) | hi_off(S, i >> L)]);
    }
}

template <int NT>
__device__ __forceinline__ void tile_store(float2 *__restrict__ g, uint64_t base, const PassSmem &S,
                                           const float2 *tile) {
    const uint32_t T = S.p.T, L = S.p.L, lmask = (1u << L) - 1;
    if (fast12<NT>(S)) {
        const uint32_t tid = threadIdx.x, tq = swz_thread<NT>(tid);
        float2 *gt = g + (base | uint64_t(thread_tile_offset<NT>(S)));
#pragma unroll
        for (uint32_t u = 0; u < 4096u / NT; ++u) gt[S.off12[u]] = tile[(tq ^ swz_u<NT>(u)) + NT * u];
        return;
    }
    for (uint32_t i = threadIdx.x; i < (1u << T); i += NT) g[base | (i & lmask) | hi_off(S, i >> L)] = tile[swz(i)];
}

// The pass blob (op descriptors, diagonal ops' index tables and phases, small
// dense matrices) staged in shared memory with 16-byte cp.async.
template <int NT>
__device__ __forceinline__ void blob_load(const uint4 *__restrict__ gblob, uint32_t words, uint4 *sblob) {
    for (uint32_t t = threadIdx.x; t < words; t += NT) cp_async16(sblob + t, gblob + t);
}

// The pass's ops on a staged tile; blob: the staged pass blob; mat: the matrix
// area for dense ops whose matrix is not in the blob. Starts with a CTA
// barrier, so the tile's and blob's loads need only have completed per thread.
template <int NT, int KMAX, int PREC, bool UM = false>
__device__ __forceinline__ bool tile_ops(float2 *tile, const uint4 *blob, float2 *mat,
                                         const float2 *__restrict__ mats, const uint32_t *__restrict__ bfr,
                                         uint64_t base, uint64_t gb, PassSmem &S, uint4 *bbuf, int *status,
                                         uint32_t &phase, bool b_resident = false) {
    // b_resident: the pass's only tcgen05 op has its B operand in bbuf already (staged once per CTA)
    // phase: parity of the next MMA-completion phase (tcgen05 dense ops); false after a wait ran out
    const int tid = threadIdx.x;
    const uint32_t T = S.p.T;
    const OpDev *bops = reinterpret_cast<const OpDev *>(blob);
    const float2 *bf2 = reinterpret_cast<const float2 *>(blob);
    const uint8_t *bb = reinterpret_cast<const uint8_t *>(blob);
    for (uint32_t oi = 0; oi < S.p.op_count;) {
        __syncthreads();
        const OpDev &op = bops[oi];
        const uint32_t type = op.type, k = op.k;
        uint32_t adv = 1;
        if (type == OP_DENSE) {
            const uint32_t D = 1u << k;
            // the tensor-core form reads the op's B-fragment table; the CUDA-core form its matrix
            // width 6 runs on tcgen05 too in TF32 passes that carry one (PassDev::umma bit 3)
            const bool um6 = UM && PREC == QSIM_PREC_TF32 && k == 6 && T == 12 && (S.p.umma & 8u);
            const bool tc =
                (PREC != QSIM_PREC_FP32 && k >= (PREC == QSIM_PREC_TF32 ? 3u : 4u) && k <= 5 && T == 12) || um6;
            bool um = false;  // on tcgen05: stage the op's B operand now, under the set-up below
            if constexpr (UM) {
                um = S.p.umma && (k == 5 || um6) && T == 12;
                if (um && !b_resident) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(bfr + op.bfrag);
                    const uint32_t bw = (k == 6 ? 65536u : umma_b_bytes<PREC>()) / 16;
                    for (uint32_t t = tid; t < bw; t += NT) cp_async16(bbuf + t, src + t);
                    cp_async_commit();
                }
            }
            // swizzled group bases (cb[g & 63] ^ cb[64 + (g >> 6)]) and column offsets (osw): copied from the
            // host-built tables in the blob for the tensor-core ops, else built here
            const uint32_t *cb = &S.cb[0][0], *osw = S.offs_sw;
            const float2 *M = mat;
            if (!tc) {
                if (op.tab != kNoTab) M = bf2 + op.tab;
                else
                    for (uint32_t i = tid; i < D * D; i += NT) mat[i] = mats[op.mat + i];
            }
            if (op.dlut != kNoTab) {
                // read in place from the staged blob (shared memory for the whole pass): no copy, no barrier
                const uint32_t *ht = reinterpret_cast<const uint32_t *>(blob) + op.dlut;
                cb = ht;
                osw = ht + 128;
            } else {
                if (tid < int(D)) {
                    uint32_t o = 0;
                    for (uint32_t j = 0; j < k; ++j) o |= ((uint32_t(tid) >> j) & 1u) << op.tq[j];
                    S.offs_sw[tid] = swz(o);
                }
                const uint32_t nc = T - k;
                for (uint32_t x = tid; x < 128; x += NT) {
                    const uint32_t half = x >> 6, v = x & 63u;
                    uint32_t b = 0;
                    for (uint32_t t = 0; t < 6; ++t)
                        if (6 * half + t < nc) b |= ((v >> t) & 1u) << op.comp[6 * half + t];
                    S.cb[half][v] = swz(b);
                }
            }
            if (op.dlut == kNoTab || !tc) __syncthreads();  // tables built above, or the matrix area filled
            if constexpr (UM) {
                if (um) {
                    bool done;
                    if constexpr (PREC == QSIM_PREC_BF16X3)
                        done = apply_dense_umma3<NT>(tile, umma::smem_addr(bbuf), cb, osw, S, phase, status);
                    else if (k == 6)
                        done = apply_dense_umma6<NT>(tile, umma::smem_addr(bbuf), cb, osw, S, phase, status);
                    else
                        done = apply_dense_umma<NT>(tile, umma::smem_addr(bbuf), cb, osw, S, phase, status);
                    if (!done) return false;
                    oi += adv;
                    continue;
                }
            }
            if constexpr (UM) {
                // a tcgen05 pass (T = 12) runs every dense op of width 3 to 5 above (widths 3 and 4 come widened
                // to 5), and width 6 in TF32; what is left here is width 1 or 2, or 6 in split BF16, on CUDA cores,
                // so no other dense form is compiled in
                if (k <= 2) apply_dense_dispatch<NT, 2, PREC>(k, tile, M, bfr + op.bfrag, cb, osw, T);
                else if constexpr (KMAX >= 6) apply_dense<NT, 6>(tile, M, cb, osw, T);
            } else if constexpr (KMAX >= 1) {
                apply_dense_dispatch<NT, KMAX, PREC>(k, tile, M, bfr + op.bfrag, cb, osw, T);
            }
        } else if (type == OP_DIAG) {
            // a run of r diagonal ops in one sweep; op d's phase index = bits constant over the
            // tile | lookups over the tile bits 0..6 and 7..12
            const uint32_t r = op.run;
            adv = r;
            if (tid < int(r)) {
                const OpDev &od = bops[oi + tid];
                uint32_t idx = 0;
                for (uint32_t j = 0; j < od.k; ++j) {
                    if (od.dtile[j] != 255) continue;
                    const uint32_t src = od.dsrc[j];
                    const uint64_t bit = src < 64 ? (base >> src) & 1ull : (gb >> (src - 64)) & 1ull;
                    idx |= uint32_t(bit) << j;
                }
                S.dconst[tid] = idx;
            }
            __syncthreads();
            uint32_t dc[kDiagRun], tb[kDiagRun], lb[kDiagRun];
#pragma unroll
            for (uint32_t d = 0; d < kDiagRun; ++d) {
                dc[d] = d < r ? S.dconst[d] : 0u;
                tb[d] = d < r ? bops[oi + d].tab : 0u;
                lb[d] = d < r ? 8u * bops[oi + d].dlut : 0u;
            }
            if (T == 12) {
                // element i = tid + NT u: tile bits 0..6 fixed per thread, bits 7..11 from u
                const uint32_t tq = swz_thread<NT>(tid), lo = uint32_t(tid) & 127u, hib = 128u + (uint32_t(tid) >> 7);
                uint32_t fix[kDiagRun];
#pragma unroll
                for (uint32_t d = 0; d < kDiagRun; ++d) fix[d] = d < r ? (dc[d] | bb[lb[d] + lo]) + tb[d] : 0u;
#pragma unroll
                for (uint32_t u = 0; u < 4096u / NT; ++u) {
                    float2 &a = tile[(tq ^ swz_u<NT>(u)) + NT * u];
                    float2 v = a;
#pragma unroll
                    for (uint32_t d = 0; d < kDiagRun; ++d) {
                        if (d < r) {
                            const float2 ph = bf2[fix[d] + bb[lb[d] + hib + (NT / 128) * u]];
                            v = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
                        }
                    }
                    a = v;
                }
            } else {
                for (uint32_t i = tid; i < (1u << T); i += NT) {
                    const uint32_t lo = i & 127u, hi = 128u + (i >> 7);
                    float2 &a = tile[swz(i)];
                    float2 v = a;
#pragma unroll
                    for (uint32_t d = 0; d < kDiagRun; ++d) {
                        if (d < r) {
                            const float2 ph = bf2[tb[d] + (dc[d] | bb[lb[d] + lo] | bb[lb[d] + hi])];
                            v = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
                        }
                    }
                    a = v;
                }
            }
        } else if (type == OP_POLY) {
            // a run of diagonal ops whose summed phase angle is a polynomial of degree <= 2 in the tile's bits:
            // P(x) = C + sum_t A_t x_t + sum_{t < t'} G_tt' x_t x_t', where C and A_t take the terms with bits
            // constant over the tile; one phase exp(2 pi i P) per amplitude for the whole run. Angles are turns in
            // 32-bit fixed point, so every sum wraps exactly modulo a turn; only the final angle is rounded (to FP32,
            // within 2^-26 turns) before __sincosf
            const uint32_t r = op.run;
            adv = r;
            const uint32_t *pw = reinterpret_cast<const uint32_t *>(blob) + op.tab;
            // this tile's A_t and C: the pass constants, then every term whose constant bits are 1 over this tile,
            // the records shared out over the CTA (shared atomic adds, exact modulo 2^32)
            if (tid < 13) S.pA[tid] = pw[tid < 12 ? 192 + tid : 204];
            __syncthreads();
            {
                const uint32_t *tr = pw + kPolyHeadWords;
                for (uint32_t i = tid; i < op.ncst; i += NT) {
                    const uint32_t t = tr[4 * i], s1 = tr[4 * i + 1], s2 = tr[4 * i + 2];
                    const uint64_t b1 = s1 < 64 ? (base >> s1) & 1ull : (gb >> (s1 - 64)) & 1ull;
                    const uint64_t b2 = s2 == kNoSrc ? 1ull : s2 < 64 ? (base >> s2) & 1ull : (gb >> (s2 - 64)) & 1ull;
                    if (b1 & b2) atomicAdd(&S.pA[t == kPolyConst ? 12u : t], tr[4 * i + 3]);
                }
            }
            __syncthreads();
            if (T == 12) {
                // element i = tid + NT u: tile bits 0..LB-1 from tid, LB..11 from u
                constexpr uint32_t LB = NT == 256 ? 8 : 7, HB = 12 - LB;
                const uint32_t tq = swz_thread<NT>(tid);
                uint32_t th = S.pA[12], beta[HB];
#pragma unroll
                for (uint32_t b = 0; b < HB; ++b) beta[b] = S.pA[LB + b];
#pragma unroll
                for (uint32_t t = 0; t < LB; ++t) {
                    if (!((uint32_t(tid) >> t) & 1u)) continue;
                    th += S.pA[t];
#pragma unroll
                    for (uint32_t t2 = t + 1; t2 < LB; ++t2)
                        if ((uint32_t(tid) >> t2) & 1u) th += pw[12 * t + t2];
#pragma unroll
                    for (uint32_t b = 0; b < HB; ++b) beta[b] += pw[12 * t + LB + b];
                }
                const uint32_t *q = pw + (LB == 7 ? 144 : 176);
#pragma unroll
                for (uint32_t u = 0; u < 4096u / NT; ++u) {
                    uint32_t ang = th + q[u];
#pragma unroll
                    for (uint32_t b = 0; b < HB; ++b)
                        if ((u >> b) & 1u) ang += beta[b];
                    float sn, cs;
                    __sincosf(6.28318530717958648f * 2.3283064365386963e-10f * float(int32_t(ang)), &sn, &cs);
                    float2 &a = tile[(tq ^ swz_u<NT>(u)) + NT * u];
                    const float2 v = a;
                    a = make_float2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
                }
            }
        } else if (type == OP_CSEP) {
            // phase(x) = P_lo[b][tile bits 0..6] * P_hi[b][tile bits 7..] * K_b, b = the control bit,
            // K_b from the targets outside the tile
            const float2 *plo = bf2 + op.tab, *phi = bf2 + op.dlut;
            if (tid < 2) {
                float2 kb = make_float2(1.f, 0.f);
                const float2 *rec = bf2 + op.mat;
                for (uint32_t c = 0; c < op.ncst; ++c) {
                    const uint32_t src = __float_as_uint(rec[5 * c].x);
                    const uint32_t bit = uint32_t(src < 64 ? (base >> src) & 1ull : (gb >> (src - 64)) & 1ull);
                    const float2 d = rec[5 * c + 1 + 2 * tid + bit];
                    kb = make_float2(kb.x * d.x - kb.y * d.y, kb.x * d.y + kb.y * d.x);
                }
                S.ck[tid] = kb;
                if (tid == 0) {
                    const uint32_t src = op.cctl & ~kCtlFlags;
                    S.cbconst = (op.cctl & kCtlConst)
                                    ? uint32_t(src < 64 ? (base >> src) & 1ull : (gb >> (src - 64)) & 1ull)
                                    : 0u;
                }
            }
            __syncthreads();
            // branches that are the identity (bit b of idm) leave their amplitudes as they are
            const uint32_t idm = ((op.cctl & kCtlId0) ? 1u : 0u) | ((op.cctl & kCtlId1) ? 2u : 0u);
            const bool ctile = !(op.cctl & kCtlConst);
            const uint32_t ct = op.cctl & 31u, bconst = S.cbconst;
            if (!ctile && ((idm >> bconst) & 1u)) {  // the whole tile takes an identity branch
                oi += adv;
                continue;
            }
            // per branch b, csq[64 b + h] = P_hi[b][h] * (factors of the targets outside the tile), in the pass's
            // matrix area (128 entries whenever the pass has a controlled-separable op)
            float2 *csq = mat;
            for (uint32_t x = tid; x < 128; x += NT) {
                const uint32_t b = x >> 6;
                const float2 h = phi[x], kb = S.ck[b];
                csq[x] = make_float2(h.x * kb.x - h.y * kb.y, h.x * kb.y + h.y * kb.x);
            }
            __syncthreads();
            if (T == 12) {
                const uint32_t tq = swz_thread<NT>(tid), lo = uint32_t(tid) & 127u, hib = uint32_t(tid) >> 7;
                const float2 pl0 = plo[lo], pl1 = plo[128 + lo];
#pragma unroll
                for (uint32_t u = 0; u < 4096u / NT; ++u) {
                    const uint32_t i = uint32_t(tid) + NT * u, hi = hib + (NT / 128) * u;
                    const uint32_t b = ctile ? (i >> ct) & 1u : bconst;
                    if ((idm >> b) & 1u) continue;
                    const float2 q = csq[64u * b + hi], pl = b ? pl1 : pl0;
                    const float2 ph = make_float2(pl.x * q.x - pl.y * q.y, pl.x * q.y + pl.y * q.x);
                    float2 &a = tile[(tq ^ swz_u<NT>(u)) + NT * u];
                    const float2 v = a;
                    a = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
                }
            } else {
                for (uint32_t i = tid; i < (1u << T); i += NT) {
                    const uint32_t b = ctile ? (i >> ct) & 1u : bconst;
                    if ((idm >> b) & 1u) continue;
                    const float2 q = csq[64u * b + (i >> 7)], pl = plo[128 * b + (i & 127u)];
                    const float2 ph = make_float2(pl.x * q.x - pl.y * q.y, pl.x * q.y + pl.y * q.x);
                    float2 &a = tile[swz(i)];
                    const float2 v = a;
                    a = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
                }
            }
        } else {
            if (tid == 0 && op.basis_in_stage && gb == op.basis_outer && (op.basis_w & S.p.out_mask) == base) {
                uint32_t ti = 0;
                for (uint32_t t = 0; t < T; ++t) ti |= uint32_t((op.basis_w >> S.p.tile_pos[t]) & 1ull) << t;
                float2 &a = tile[swz(ti)];
                a = make_float2(-a.x, -a.y);
            }
        }
        oi += adv;
    }
    return true;
}

// One tile of one pass: stage the pass blob and the 2^T amplitudes of tile
// `cta` of the group's working vector g in shared memory (dyn: tile, then blob,
// then matrix area), apply the pass's ops, store the tile back. CG selects
// L2-only loads in registers instead of cp.async into shared memory (L1-cached);
// a caller whose working vector was written by other CTAs of the same launch
// may still take cp.async when a gpu-scope acquire of those writes' release,
// followed by a CTA barrier, precedes the call (the persistent stage kernel).
// With phase_io the caller owns the TMEM accumulator (S.tmem, 128 columns) and the MMA mbarrier (S.mbar) across
// calls and keeps the mbarrier's phase parity in *phase_io; returns false when an MMA wait ran out.
// With cache (shared memory: cache[0] the key of the pass staged in dyn, cache[1] whether its single tcgen05
// op's B operand is staged too) a call whose key matches reuses the staged descriptor, blob and B operand; the
// caller sets cache[0] to a key no pass uses whenever something else writes dyn.
template <int NT, int KMAX, int PREC, bool CG, bool UM = false>
__device__ __forceinline__ bool pass_tile(float2 *__restrict__ g, const PassDev &pd, const uint4 *__restrict__ gblob,
                                          const float2 *__restrict__ mats, const uint32_t *__restrict__ bfr,
                                          uint64_t cta, uint64_t gb, PassSmem &S, float2 *dyn, int *status,
                                          uint32_t *phase_io = nullptr, uint32_t *cache = nullptr,
                                          uint32_t key = 0) {
    const bool hit = cache && cache[0] == key;
    // copies the descriptor only: a caller-owned S.tmem and S.mbar stay as they are
    if (!hit) pass_setup<NT>(pd, S);
    const uint32_t T = S.p.T;
    // passes with tcgen05 dense ops: the tile 1024-byte aligned (it is the A operand while the MMAs run),
    // the B operand after it, then the blob; 64 TMEM columns hold the accumulator
    static_assert(!UM || ((PREC == QSIM_PREC_TF32 || PREC == QSIM_PREC_BF16X3) && NT == 128 && KMAX >= 5),
                  "tcgen05 passes: TF32 or split BF16, 128 threads, k = 5");
    bool um = false;
    if constexpr (UM) um = S.p.umma != 0;
    float2 *tile = dyn;
    uint4 *bbuf = nullptr;
    if (um) {
        const uint32_t pad = (1024u - (umma::smem_addr(dyn) & 1023u)) & 1023u;
        tile = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(dyn) + pad);
        bbuf = reinterpret_cast<uint4 *>(tile + 4096);
        if (!phase_io) {
            if (threadIdx.x < 32) umma::tmem_alloc(umma::smem_addr(&S.tmem), umma_pass_tmem_cols(S.p.umma));
            if (threadIdx.x == 0) umma::mbar_init(umma::smem_addr(&S.mbar), 1);
        }
        umma::fence_before_sync();
    }
    uint4 *blob = reinterpret_cast<uint4 *>(tile + (1u << T)) + (um ? umma_pass_b_bytes(S.p.umma) / 16 : 0u);
    float2 *mat = reinterpret_cast<float2 *>(blob + S.p.blob_words);
    const uint64_t base = tile_base(S, cta);
    bool b_res = false;
    if (hit) {
        b_res = cache[1] != 0;
    } else {
        blob_load<NT>(gblob + S.p.blob_off, S.p.blob_words, blob);
        if (cache) {
            // a pass with a single tcgen05 op keeps that op's B operand staged for the calls that hit the cache
            if constexpr (UM) {
                if (um && T == 12) {
                    const OpDev *gops = reinterpret_cast<const OpDev *>(gblob + S.p.blob_off);
                    uint32_t n5 = 0, first = 0;
                    for (uint32_t oi = 0; oi < S.p.op_count; ++oi) {
                        const uint32_t ty = __ldg(&gops[oi].type), k = __ldg(&gops[oi].k);
                        if (ty == OP_DENSE && (k == 5 || (k == 6 && PREC == QSIM_PREC_TF32 && (S.p.umma & 8u)))) {
                            if (!n5) first = oi;
                            ++n5;
                        }
                    }
                    if (n5 == 1) {
                        const uint32_t k1 = __ldg(&gops[first].k);
                        const uint4 *src = reinterpret_cast<const uint4 *>(bfr + __ldg(&gops[first].bfrag));
                        const uint32_t bw = (k1 == 6 ? 65536u : umma_b_bytes<PREC>()) / 16;
                        for (uint32_t t = threadIdx.x; t < bw; t += NT) cp_async16(bbuf + t, src + t);
                        b_res = true;
                    }
                }
            }
            if (threadIdx.x == 0) {  // every thread read cache[0] before pass_setup's barriers
                cache[0] = key;
                cache[1] = b_res ? 1u : 0u;
            }
        }
    }
    tile_load<NT, CG>(g, base, S, tile);
    cp_async_wait_all();
    uint32_t phase = phase_io ? *phase_io : 0u;
    const bool ok =
        tile_ops<NT, KMAX, PREC, UM>(tile, blob, mat, mats, bfr, base, gb, S, bbuf, status, phase, b_res);
    __syncthreads();
    tile_store<NT>(g, base, S, tile);
    if (phase_io) {
        *phase_io = phase;
        return ok;
    }
    if (um) {
        // after a wait that ran out, wait (bounded) once more for the MMAs in flight before freeing TMEM
        if (!ok) umma::mbar_wait(umma::smem_addr(&S.mbar), phase ^ 1u, kUmmaWaitNs);
        umma::fence_before_sync();
        __syncthreads();
        if (threadIdx.x < 32) {
            umma::fence_after_sync();
            umma::tmem_dealloc(S.tmem, umma_pass_tmem_cols(S.p.umma));
        }
    }
    return ok;
}

// One pass over many tiles (streams mode): CTA c takes tiles c, c + gridDim.x, ... of the launch's groups
// (tile t: group t >> nout, tile index t & (2^nout - 1)). The pass descriptor, the pass blob, the TMEM
// accumulator and the MMA mbarrier are set up once per CTA instead of once per tile, and when the pass has a
// single tcgen05 op its B operand is staged once too; each tile is then loaded, updated and stored as in
// pass_tile, with several CTAs per SM keeping loads, ops and stores of different tiles in flight.
// Tiles are handed out in launch order from a counter (ctr[0]; ctr[1] counts the CTAs that finished, and the last
// one zeroes both for the next launch on the stream), so the tiles in flight stay a narrow window of the working
// vector: its 64-byte rows that share DRAM pages are read and written close together in time.
template <int NT, int KMAX, int PREC, bool UM = false>
__device__ __forceinline__ void pass_tiles(float2 *__restrict__ wv, uint32_t W, uint64_t ntiles, const PassDev &pd,
                                           const uint4 *__restrict__ gblob, const float2 *__restrict__ mats,
                                           const uint32_t *__restrict__ bfr, const uint64_t *__restrict__ gbase,
                                           PassSmem &S, float2 *dyn, uint32_t *ctr, int *status) {
    // the CTA's next tile, in a slot by iteration parity: thread 0 writes slot (it + 1) & 1 while a slower warp may
    // still be reading slot it & 1 after the end-of-iteration barrier; that slot is next written two barriers later
    __shared__ uint32_t s_next[2];
    pass_setup<NT>(pd, S);
    const uint32_t T = S.p.T;
    static_assert(!UM || ((PREC == QSIM_PREC_TF32 || PREC == QSIM_PREC_BF16X3) && NT == 128 && KMAX >= 5),
                  "tcgen05 passes: TF32 or split BF16, k = 5");
    bool um = false;
    if constexpr (UM) um = S.p.umma != 0;
    float2 *tile = dyn;
    uint4 *bbuf = nullptr;
    if (um) {
        const uint32_t pad = (1024u - (umma::smem_addr(dyn) & 1023u)) & 1023u;
        tile = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(dyn) + pad);
        bbuf = reinterpret_cast<uint4 *>(tile + 4096);
        if (threadIdx.x < 32) umma::tmem_alloc(umma::smem_addr(&S.tmem), umma_pass_tmem_cols(S.p.umma));
        if (threadIdx.x == 0) umma::mbar_init(umma::smem_addr(&S.mbar), 1);
        umma::fence_before_sync();
    }
    uint4 *blob = reinterpret_cast<uint4 *>(tile + (1u << T)) + (um ? umma_pass_b_bytes(S.p.umma) / 16 : 0u);
    float2 *mat = reinterpret_cast<float2 *>(blob + S.p.blob_words);
    blob_load<NT>(gblob + S.p.blob_off, S.p.blob_words, blob);
    cp_async_wait_all();
    __syncthreads();
    // a single tcgen05 op: its B operand stays in bbuf for every tile of this CTA
    bool b_res = false;
    if (um && T == 12) {
        const OpDev *bops = reinterpret_cast<const OpDev *>(blob);
        uint32_t n5 = 0, first = 0;
        for (uint32_t oi = 0; oi < S.p.op_count; ++oi)
            if (bops[oi].type == OP_DENSE &&
                (bops[oi].k == 5 || (bops[oi].k == 6 && PREC == QSIM_PREC_TF32 && (S.p.umma & 8u)))) {
                if (!n5) first = oi;
                ++n5;
            }
        if (n5 == 1) {
            const uint4 *src = reinterpret_cast<const uint4 *>(bfr + bops[first].bfrag);
            const uint32_t bw = (bops[first].k == 6 ? 65536u : umma_b_bytes<PREC>()) / 16;
            for (uint32_t t = threadIdx.x; t < bw; t += NT) cp_async16(bbuf + t, src + t);
            cp_async_commit();
            b_res = true;
        }
    }
    uint32_t phase = 0;
    bool ok = true;
    const uint64_t tmask = (1ull << S.p.nout) - 1;
    uint32_t it = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; ++it) {
        if (threadIdx.x == 0) s_next[it & 1u] = gridDim.x + atomicAdd(ctr, 1u);  // read after the barrier below
        const uint64_t grp = t >> S.p.nout, cta = t & tmask;
        float2 *g = wv + (grp << W);
        const uint64_t gb = gbase ? gbase[grp] : 0ull;
        const uint64_t base = tile_base(S, cta);
        tile_load<NT, false>(g, base, S, tile);
        cp_async_wait_all();
        ok = tile_ops<NT, KMAX, PREC, UM>(tile, blob, mat, mats, bfr, base, gb, S, bbuf, status, phase, b_res);
        __syncthreads();
        tile_store<NT>(g, base, S, tile);
        __syncthreads();  // the next tile's loads overwrite the tile; s_next[it & 1] is visible
        if (!ok) break;   // uniform: the MMA wait ran out (status set)
        t = s_next[it & 1u];
    }
    if (threadIdx.x == 0) {
        // every tile counter increment of this CTA precedes its arrival; the last CTA to arrive resets both
        __threadfence();
        if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
            atomicExch(ctr, 0u);
            atomicExch(ctr + 1, 0u);
        }
    }
    if (um) {
        // after a wait that ran out, wait (bounded) once more for the MMAs in flight before freeing TMEM
        if (!ok) umma::mbar_wait(umma::smem_addr(&S.mbar), phase ^ 1u, kUmmaWaitNs);
        umma::fence_before_sync();
        __syncthreads();
        if (threadIdx.x < 32) {
            umma::fence_after_sync();
            umma::tmem_dealloc(S.tmem, umma_pass_tmem_cols(S.p.umma));
        }
    }
}

}  // namespace gdev
}  // namespace qsim
