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
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"

namespace qsim {

namespace {

constexpr int NT = 128;

__device__ __forceinline__ uint32_t swz(uint32_t i) {
    return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15u);
}

struct PassSmem {
    PassDev p;
    OpDev op;
    uint32_t hi[256];
    uint32_t offs[64];
};

template <int K>
__device__ __forceinline__ void apply_dense(float2 *tile, const float2 *U, const PassSmem &S, uint32_t T) {
    constexpr int D = 1 << K;
    const uint32_t ngroups = 1u << (T - K);
    const uint32_t nc = T - K;
    for (uint32_t g = threadIdx.x; g < ngroups; g += NT) {
        uint32_t b = 0;
        for (uint32_t t = 0; t < nc; ++t) b |= ((g >> t) & 1u) << S.op.comp[t];
        float2 x[D];
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = tile[swz(b | S.offs[c])];
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
            tile[swz(b | S.offs[r])] = make_float2(ar, ai);
        }
    }
}

__device__ __forceinline__ void apply_dense_k1(float2 *tile, const float2 *U, const PassSmem &S, uint32_t T) {
    const uint32_t ngroups = 1u << (T - 1);
    const uint32_t nc = T - 1;
    const float2 u00 = U[0], u01 = U[1], u10 = U[2], u11 = U[3];
    for (uint32_t g = threadIdx.x; g < ngroups; g += NT) {
        uint32_t b = 0;
        for (uint32_t t = 0; t < nc; ++t) b |= ((g >> t) & 1u) << S.op.comp[t];
        const uint32_t i0 = swz(b), i1 = swz(b | S.offs[1]);
        const float2 x0 = tile[i0], x1 = tile[i1];
        tile[i0] = make_float2(u00.x * x0.x - u00.y * x0.y + u01.x * x1.x - u01.y * x1.y,
                               u00.x * x0.y + u00.y * x0.x + u01.x * x1.y + u01.y * x1.x);
        tile[i1] = make_float2(u10.x * x0.x - u10.y * x0.y + u11.x * x1.x - u11.y * x1.y,
                               u10.x * x0.y + u10.y * x0.x + u11.x * x1.y + u11.y * x1.x);
    }
}

__global__ void __launch_bounds__(NT) k_pass_fp32(float2 *__restrict__ wv, uint32_t W, const PassDev *__restrict__ pd,
                                                  const OpDev *__restrict__ ops, const float2 *__restrict__ mats,
                                                  const uint64_t *__restrict__ gbase) {
    extern __shared__ float4 dyn_smem[];
    __shared__ PassSmem S;
    const int tid = threadIdx.x;
    if (tid == 0) S.p = *pd;
    __syncthreads();
    const uint32_t T = S.p.T, L = S.p.L, nout = S.p.nout;
    float2 *tile = reinterpret_cast<float2 *>(dyn_smem);
    float2 *mat = tile + (1u << T);
    const uint32_t nhi = 1u << (T - L);
    for (uint32_t h = tid; h < nhi; h += NT) {
        uint32_t o = 0;
        for (uint32_t t = 0; t < T - L; ++t) o |= ((h >> t) & 1u) << S.p.tile_pos[L + t];
        S.hi[h] = o;
    }
    uint64_t base = 0;
    const uint64_t cta = blockIdx.x;
    for (uint32_t t = 0; t < nout; ++t) base |= ((cta >> t) & 1ull) << S.p.out_pos[t];
    float2 *g = wv + (uint64_t(blockIdx.y) << W);
    const uint64_t gb = gbase ? gbase[blockIdx.y] : 0ull;
    const uint32_t lmask = (1u << L) - 1;
    __syncthreads();
    for (uint32_t i = tid; i < (1u << T); i += NT) tile[swz(i)] = g[base | (i & lmask) | S.hi[i >> L]];

    for (uint32_t oi = 0; oi < S.p.op_count; ++oi) {
        __syncthreads();
        if (tid == 0) S.op = ops[S.p.op_begin + oi];
        __syncthreads();
        const uint32_t type = S.op.type, k = S.op.k;
        if (type == OP_DENSE) {
            const uint32_t D = 1u << k;
            for (uint32_t i = tid; i < D * D; i += NT) mat[i] = mats[S.op.mat + i];
            if (tid < int(D)) {
                uint32_t o = 0;
                for (uint32_t j = 0; j < k; ++j) o |= ((uint32_t(tid) >> j) & 1u) << S.op.tq[j];
                S.offs[tid] = o;
            }
            __syncthreads();
            switch (k) {
                case 1: apply_dense_k1(tile, mat, S, T); break;
                case 2: apply_dense<2>(tile, mat, S, T); break;
                case 3: apply_dense<3>(tile, mat, S, T); break;
                case 4: apply_dense<4>(tile, mat, S, T); break;
                case 5: apply_dense<5>(tile, mat, S, T); break;
                default: apply_dense<6>(tile, mat, S, T); break;
            }
        } else if (type == OP_DIAG) {
            const uint32_t D = 1u << k;
            for (uint32_t i = tid; i < D; i += NT) mat[i] = mats[S.op.mat + i];
            __syncthreads();
            for (uint32_t i = tid; i < (1u << T); i += NT) {
                const uint64_t w = base | (i & lmask) | S.hi[i >> L];
                uint32_t idx = 0;
                for (uint32_t j = 0; j < k; ++j) {
                    const uint32_t src = S.op.dsrc[j];
                    const uint64_t bit = src < 64 ? (w >> src) & 1ull : (gb >> (src - 64)) & 1ull;
                    idx |= uint32_t(bit) << j;
                }
                const float2 ph = mat[idx];
                float2 &a = tile[swz(i)];
                const float2 v = a;
                a = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
            }
        } else {
            if (tid == 0 && S.op.basis_in_stage && gb == S.op.basis_outer &&
                (S.op.basis_w & S.p.out_mask) == base) {
                uint32_t ti = 0;
                for (uint32_t t = 0; t < T; ++t) ti |= uint32_t((S.op.basis_w >> S.p.tile_pos[t]) & 1ull) << t;
                float2 &a = tile[swz(ti)];
                a = make_float2(-a.x, -a.y);
            }
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < (1u << T); i += NT) g[base | (i & lmask) | S.hi[i >> L]] = tile[swz(i)];
}

}  // namespace

void launch_pass(float2 *wv, uint32_t W, uint32_t ngroups, const PassDev *pass_host, const PassDev *pass_dev,
                 const OpDev *ops_dev, const float2 *mats_dev, const uint64_t *gbase_dev, int prec,
                 cudaStream_t s) {
    (void)prec;
    const uint32_t T = pass_host->T;
    const size_t smem = (size_t(1) << T) * sizeof(float2) + size_t(pass_host->mat_elems) * sizeof(float2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_pass_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    dim3 grid(1u << pass_host->nout, ngroups);
    k_pass_fp32<<<grid, NT, smem, s>>>(wv, W, pass_dev, ops_dev, mats_dev, gbase_dev);
    count_launch();
}

}  // namespace qsim
