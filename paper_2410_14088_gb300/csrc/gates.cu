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

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"
#include "gates_dev.cuh"

namespace qsim {

namespace {

using namespace gdev;
constexpr int NT = 128;

template <int KMAX, int PREC>
__global__ void __launch_bounds__(NT, ((KMAX >= 6 || PREC != QSIM_PREC_FP32) ? 2 : 4))
    k_pass(float2 *__restrict__ wv, uint32_t W, const PassDev *__restrict__ pd, const OpDev *__restrict__ ops,
           const float2 *__restrict__ mats, const uint64_t *__restrict__ gbase) {
    extern __shared__ float4 dyn_smem[];
    __shared__ PassSmem S;
    float2 *g = wv + (uint64_t(blockIdx.y) << W);
    const uint64_t gb = gbase ? gbase[blockIdx.y] : 0ull;
    pass_tile<NT, KMAX, PREC, false>(g, pd, ops, mats, blockIdx.x, gb, S, reinterpret_cast<float2 *>(dyn_smem));
}

template <int KMAX, int PREC>
void launch_pass_k(dim3 grid, size_t smem, cudaStream_t s, float2 *wv, uint32_t W, const PassDev *pd,
                   const OpDev *ops, const float2 *mats, const uint64_t *gbase) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_pass<KMAX, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    k_pass<KMAX, PREC><<<grid, NT, smem, s>>>(wv, W, pd, ops, mats, gbase);
}

template <int PREC>
void launch_pass_prec(uint32_t kmax, dim3 grid, size_t smem, cudaStream_t s, float2 *wv, uint32_t W,
                      const PassDev *pd, const OpDev *ops, const float2 *mats, const uint64_t *gbase) {
    switch (kmax) {
        case 0: launch_pass_k<0, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        case 1: launch_pass_k<1, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        case 2: launch_pass_k<2, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        case 3: launch_pass_k<3, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        case 4: launch_pass_k<4, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        case 5: launch_pass_k<5, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
        default: launch_pass_k<6, PREC>(grid, smem, s, wv, W, pd, ops, mats, gbase); break;
    }
}

}  // namespace

void launch_pass(float2 *wv, uint32_t W, uint32_t ngroups, const PassDev *pass_host, const PassDev *pass_dev,
                 const OpDev *ops_dev, const float2 *mats_dev, const uint64_t *gbase_dev, int prec,
                 cudaStream_t s) {
    const uint32_t T = pass_host->T;
    const size_t smem = (size_t(1) << T) * sizeof(float2) + size_t(pass_host->mat_elems) * sizeof(float2);
    dim3 grid(1u << pass_host->nout, ngroups);
    const uint32_t kmax = pass_host->kmax;
    if (prec == QSIM_PREC_TF32 && kmax >= 3)
        launch_pass_prec<QSIM_PREC_TF32>(kmax, grid, smem, s, wv, W, pass_dev, ops_dev, mats_dev, gbase_dev);
    else if (prec == QSIM_PREC_BF16X3 && kmax >= 3)
        launch_pass_prec<QSIM_PREC_BF16X3>(kmax, grid, smem, s, wv, W, pass_dev, ops_dev, mats_dev, gbase_dev);
    else
        launch_pass_prec<QSIM_PREC_FP32>(kmax, grid, smem, s, wv, W, pass_dev, ops_dev, mats_dev, gbase_dev);
    count_launch();
}

}  // namespace qsim
