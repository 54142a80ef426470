// Gate passes on FP32 CUDA cores (sm_103a).
//
// The state update of Sec. 2.1 multiplies, for every index group that agrees
// outside the target bits, the 2^k amplitudes of the group by the gate matrix.
// Here a stage's gates arrive fused into dense ops of <= k qubits (plus
// diagonal phase ops and phase flips). A pass loads one tile of 2^T
// amplitudes of the working vector into shared memory (the tile's low bits
// are contiguous working-index bits, so the loads are coalesced), applies
// every op of the pass in shared memory, and stores the tile back: one read
// and one write of the working vector per pass instead of one per gate.
//
// Shared memory layout is XOR-swizzled (bits 4-7, 8-11, 12-15 folded into the
// low four bits of the float2 index) so that the lanes of a warp, which walk
// different index groups, hit different banks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"
#include "gates_dev.cuh"

namespace qsim {

namespace {

using namespace gdev;
constexpr int NT = 128;

// One wave of resident CTAs, each looping over tiles of all the launch's groups
// (one tile buffer per CTA; several resident CTAs per SM keep loads, ops and
// stores of different tiles in flight). The pass set-up, the pass blob, TMEM
// and a single tcgen05 op's B operand are staged once per CTA rather than once
// per tile. (A variant with two tile buffers per CTA and cp.async prefetch of
// the next tile ran slower on GB300: fewer resident CTAs, 3.1 against 4.3 TB/s
// on load/store-only passes.)
// UM: the pass's k = 5 dense ops run on tcgen05 (a separate instantiation, so that the warp-MMA kernels
// keep their own register allocation)
template <int KMAX, int PREC, bool UM>
__host__ __device__ constexpr int pass_threads() {
    return NT;
}
template <int KMAX, int PREC, bool UM>
__host__ __device__ constexpr int pass_min_blocks() {
    return KMAX >= 6 ? 2 : (PREC == QSIM_PREC_BF16X3 && KMAX >= 4) ? 3 : 4;
}

template <int KMAX, int PREC, bool UM>
__global__ void __launch_bounds__(pass_threads<KMAX, PREC, UM>(), pass_min_blocks<KMAX, PREC, UM>())
    k_pass(float2 *__restrict__ wv, uint32_t W, uint64_t ntiles, const __grid_constant__ PassDev P,
           const uint4 *__restrict__ blob, const float2 *__restrict__ mats, const uint32_t *__restrict__ bfr,
           const uint64_t *__restrict__ gbase, uint32_t *ctr, int *status) {
    extern __shared__ float4 dyn_smem[];
    __shared__ PassSmem S;
    pass_tiles<pass_threads<KMAX, PREC, UM>(), KMAX, PREC, UM>(wv, W, ntiles, P, blob, mats, bfr, gbase, S,
                                                                reinterpret_cast<float2 *>(dyn_smem), ctr, status);
}

// Resident CTAs per SM of one k_pass instantiation at a given dynamic shared memory size (cached), from the
// kernel's registers and static shared memory and the SM's limits (65536 registers, 2048 threads, 32 CTAs,
// 228 KB of shared memory with 1 KB reserved per CTA). (The runtime's occupancy query answered 1 here where
// 4 CTAs per SM were resident.)
template <int KMAX, int PREC, bool UM>
int pass_blocks_per_sm(size_t smem) {
    static std::mutex mu;
    static std::map<size_t, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(smem);
    if (it != cache.end()) return it->second;
    cudaFuncAttributes fa{};
    int nb = 1;
    constexpr int nt = pass_threads<KMAX, PREC, UM>();
    if (cudaFuncGetAttributes(&fa, k_pass<KMAX, PREC, UM>) == cudaSuccess) {
        const int regs = ((fa.numRegs > 0 ? fa.numRegs : 255) + 7) & ~7;
        const int by_regs = 65536 / (regs * nt);
        const int by_smem = int((228u * 1024u) / (smem + fa.sharedSizeBytes + 1024u));
        nb = std::max(1, std::min(std::min(by_regs, by_smem), std::min(2048 / nt, 32)));
    }
    cache[smem] = nb;
    return nb;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        n = v > 0 ? v : 1;
    }
    return n;
}

template <int KMAX, int PREC, bool UM>
void launch_pass_ku(dim3 grid, size_t smem, cudaStream_t s, float2 *wv, uint32_t W, const PassDev &P,
                    const uint4 *blob, const float2 *mats, const uint32_t *bfr, const uint64_t *gbase, uint32_t *ctr,
                    int *status) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_pass<KMAX, PREC, UM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        // the whole unified L1/shared array as shared memory: the resident CTAs are limited by their tiles
        cudaFuncSetAttribute(k_pass<KMAX, PREC, UM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
        attr_set = true;
    }
    // grid.x tiles per group, grid.y groups: the resident CTAs loop over all of them. The grid is twice the
    // resident count so that an underestimate of it cannot leave SMs short of CTAs (measured on the 32-qubit
    // QAOA passes: one CTA per SM 0.85 ms, one resident wave 0.41 ms, two 0.41 ms, one tile per CTA 0.46 ms);
    // CTAs that start after the tiles have run out leave at once.
    const uint64_t ntiles = uint64_t(grid.x) * grid.y;
    const uint64_t resident = 2ull * uint64_t(pass_blocks_per_sm<KMAX, PREC, UM>(smem)) * num_sms();
    const uint32_t nctas = uint32_t(ntiles < resident ? ntiles : resident);
    k_pass<KMAX, PREC, UM><<<nctas, pass_threads<KMAX, PREC, UM>(), smem, s>>>(wv, W, ntiles, P, blob, mats, bfr,
                                                                              gbase, ctr, status);
}

template <int KMAX, int PREC>
void launch_pass_k(dim3 grid, size_t smem, cudaStream_t s, float2 *wv, uint32_t W, const PassDev &P,
                   const uint4 *blob, const float2 *mats, const uint32_t *bfr, const uint64_t *gbase, uint32_t *ctr,
                   int *status) {
    if constexpr ((PREC == QSIM_PREC_TF32 || PREC == QSIM_PREC_BF16X3) && KMAX >= 5) {
        if (P.umma) {
            launch_pass_ku<KMAX, PREC, true>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status);
            return;
        }
    }
    launch_pass_ku<KMAX, PREC, false>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status);
}

template <int PREC>
void launch_pass_prec(uint32_t kmax, dim3 grid, size_t smem, cudaStream_t s, float2 *wv, uint32_t W,
                      const PassDev &P, const uint4 *blob, const float2 *mats, const uint32_t *bfr,
                      const uint64_t *gbase, uint32_t *ctr, int *status) {
    switch (kmax) {
        case 0: launch_pass_k<0, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        case 1: launch_pass_k<1, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        case 2: launch_pass_k<2, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        case 3: launch_pass_k<3, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        case 4: launch_pass_k<4, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        case 5: launch_pass_k<5, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
        default: launch_pass_k<6, PREC>(grid, smem, s, wv, W, P, blob, mats, bfr, gbase, ctr, status); break;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host: B-fragment tables
// ---------------------------------------------------------------------------
static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}
static float bits_f32(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}
// round to TF32 (10 explicit mantissa bits), nearest with ties away from zero
static uint32_t to_tf32(float x) { return (f32_bits(x) + 0x1000u) & ~0x1FFFu; }
// round to BF16, nearest even
static uint16_t to_bf16(float x) {
    const uint32_t u = f32_bits(x);
    return uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
static float from_bf16(uint16_t h) { return bits_f32(uint32_t(h) << 16); }

size_t bfrag_words(uint32_t k, int prec) {
    const size_t n2 = size_t(2) << k;
    return prec == QSIM_PREC_TF32 ? n2 * n2 : 3 * n2 * n2 / 2;
}

void build_bfrag_table(const double *u, uint32_t k, int prec, uint32_t *out) {
    const uint32_t D = 1u << k, N2 = 2 * D, NTILES = N2 / 8;
    // U_r^T[kk][n] = U_r[n][kk] as float
    auto ur = [&](uint32_t n, uint32_t kk) -> float {
        const uint32_t r = n % D, c = kk % D;
        const double re = u[2 * (size_t(r) * D + c)], im = u[2 * (size_t(r) * D + c) + 1];
        if (n < D) return float(kk < D ? re : -im);
        return float(kk < D ? im : re);
    };
    if (prec == QSIM_PREC_TF32) {
        const uint32_t KS = N2 / 8;
        for (uint32_t ks = 0; ks < KS; ++ks)
            for (uint32_t nt = 0; nt < NTILES; ++nt)
                for (uint32_t lane = 0; lane < 32; ++lane) {
                    const uint32_t g = lane / 4, t = lane % 4;
                    uint32_t *o = out + ((size_t(ks) * NTILES + nt) * 32 + lane) * 2;
                    o[0] = to_tf32(ur(nt * 8 + g, ks * 8 + t));
                    o[1] = to_tf32(ur(nt * 8 + g, ks * 8 + t + 4));
                }
        return;
    }
    const uint32_t KS = N2 / 16;
    const size_t part = size_t(KS) * NTILES * 32 * 2;
    for (uint32_t ks = 0; ks < KS; ++ks)
        for (uint32_t nt = 0; nt < NTILES; ++nt)
            for (uint32_t lane = 0; lane < 32; ++lane) {
                const uint32_t g = lane / 4, t = lane % 4;
                for (int r = 0; r < 2; ++r) {
                    uint16_t h[2], m[2], l[2];
                    for (int q = 0; q < 2; ++q) {
                        const float x = ur(nt * 8 + g, ks * 16 + 2 * t + q + 8 * r);
                        h[q] = to_bf16(x);
                        const float r1 = x - from_bf16(h[q]);
                        m[q] = to_bf16(r1);
                        l[q] = to_bf16(r1 - from_bf16(m[q]));
                    }
                    const size_t e = ((size_t(ks) * NTILES + nt) * 32 + lane) * 2 + r;
                    out[e] = uint32_t(h[0]) | (uint32_t(h[1]) << 16);
                    out[part + e] = uint32_t(m[0]) | (uint32_t(m[1]) << 16);
                    out[2 * part + e] = uint32_t(l[0]) | (uint32_t(l[1]) << 16);
                }
            }
}

size_t umma_pass_smem(uint32_t umma_bits) {
    return (umma_bits & 1u) ? size_t(umma_pass_b_bytes(umma_bits)) + 1024 : 0;
}

size_t pass_smem_bytes(const PassDev &P) {
    const size_t um = umma_pass_smem(P.umma);
    return (size_t(1) << P.T) * sizeof(float2) + um + size_t(P.blob_words) * 16 +
           size_t(P.mat_elems) * sizeof(float2);
}

void build_umma_b(const double *u, uint32_t *out) {
    constexpr uint32_t D = 32;
    for (uint32_t n = 0; n < 2 * D; ++n)
        for (uint32_t kk = 0; kk < 2 * D; ++kk) {
            const uint32_t r = n % D, c = kk % D;
            const double re = u[2 * (size_t(r) * D + c)], im = u[2 * (size_t(r) * D + c) + 1];
            const double v = n < D ? (kk < D ? re : -im) : (kk < D ? im : re);
            const uint32_t a = kk / 32, ch = (kk % 32) / 4, w = kk % 4;
            const size_t byte = size_t(a) * 8192 + (n / 8) * 1024 + (n % 8) * 128 + ((ch ^ (n % 8)) * 16) + w * 4;
            out[byte / 4] = to_tf32(float(v));
        }
}

void build_umma_b6(const double *u, uint32_t *out) {
    constexpr uint32_t D = 64;
    for (uint32_t n = 0; n < 2 * D; ++n)
        for (uint32_t kk = 0; kk < 2 * D; ++kk) {
            const uint32_t r = n % D, c = kk % D;
            const double re = u[2 * (size_t(r) * D + c)], im = u[2 * (size_t(r) * D + c) + 1];
            const double v = n < D ? (kk < D ? re : -im) : (kk < D ? im : re);
            const uint32_t a = kk / 32, ch = (kk % 32) / 4, w = kk % 4;
            const size_t byte = size_t(a) * 16384 + (n / 8) * 1024 + (n % 8) * 128 + ((ch ^ (n % 8)) * 16) + w * 4;
            out[byte / 4] = to_tf32(float(v));
        }
}

void build_umma_b3(const double *u, uint32_t *out) {
    constexpr uint32_t D = 32;
    uint16_t *o16 = reinterpret_cast<uint16_t *>(out);
    for (uint32_t n = 0; n < 2 * D; ++n)
        for (uint32_t kk = 0; kk < 2 * D; ++kk) {
            const uint32_t r = n % D, c = kk % D;
            const double re = u[2 * (size_t(r) * D + c)], im = u[2 * (size_t(r) * D + c) + 1];
            const float x = float(n < D ? (kk < D ? re : -im) : (kk < D ? im : re));
            const uint16_t h = to_bf16(x);
            const float r1 = x - from_bf16(h);
            const uint16_t m = to_bf16(r1);
            const uint16_t l = to_bf16(r1 - from_bf16(m));
            const uint32_t ch = kk / 8, w = kk % 8;
            const size_t off = (n / 8) * 1024 + (n % 8) * 128 + ((ch ^ (n % 8)) * 16) + w * 2;  // bytes in a part
            o16[(0 * 8192 + off) / 2] = h;
            o16[(1 * 8192 + off) / 2] = m;
            o16[(2 * 8192 + off) / 2] = l;
        }
}

void launch_pass(float2 *wv, uint32_t W, uint32_t ngroups, const PassDev *pass_host, const uint4 *blob_dev,
                 const float2 *mats_dev, const uint32_t *bfr_dev, const uint64_t *gbase_dev, int prec,
                 cudaStream_t s, uint32_t *ctr, int *status) {
    const PassDev &P = *pass_host;
    const size_t smem = pass_smem_bytes(P);
    dim3 grid(1u << P.nout, ngroups);
    const uint32_t kmax = P.kmax;
    if (prec == QSIM_PREC_TF32 && kmax >= 3)
        launch_pass_prec<QSIM_PREC_TF32>(kmax, grid, smem, s, wv, W, P, blob_dev, mats_dev, bfr_dev, gbase_dev, ctr, status);
    else if (prec == QSIM_PREC_BF16X3 && kmax >= 3)
        launch_pass_prec<QSIM_PREC_BF16X3>(kmax, grid, smem, s, wv, W, P, blob_dev, mats_dev, bfr_dev, gbase_dev, ctr, status);
    else
        launch_pass_prec<QSIM_PREC_FP32>(kmax, grid, smem, s, wv, W, P, blob_dev, mats_dev, bfr_dev, gbase_dev, ctr, status);
    count_launch();
}

}  // namespace qsim
