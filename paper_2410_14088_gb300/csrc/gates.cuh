// Gate-pass kernels: a stage's fused ops applied to a working vector in
// shared-memory tiles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qsim {

constexpr int kMaxTileBits = 13;

// One pass: a tile is the set of 2^T amplitudes whose working indices agree
// outside the tile bits; ops whose qubits are tile bits (or are diagonal) are
// applied while the tile sits in shared memory.
struct PassDev {
    uint32_t T;              // tile bits
    uint32_t L;              // tile_pos[t] == t for t < L
    uint32_t nout;           // W - T
    uint32_t op_begin, op_count;
    uint32_t mat_elems;      // largest matrix / phase table of the pass, in float2
    uint32_t kmax;           // widest dense op of the pass (0 if none)
    uint32_t pad0;
    uint64_t out_mask;       // working-index mask of the non-tile bits
    uint32_t tile_pos[16];   // working bit of tile bit t (ascending)
    uint32_t out_pos[32];    // working bit of CTA-index bit t
};

struct OpDev {
    uint32_t type;           // 0 dense, 1 diagonal, 2 phase flip
    uint32_t k;
    uint32_t mat;            // float2 offset of the matrix (dense) or phases (diag)
    uint32_t pad0;
    uint32_t tq[6];          // dense: tile bit of matrix bit j
    uint32_t dsrc[6];        // diag: working bit (< 64) or 64 + full qubit (outer, from group base)
    uint32_t comp[16];       // dense: complement tile bits; comp[0..3] feed the lane bits
    uint64_t basis_outer;    // phase flip: basis & outer mask (full index bits)
    uint64_t basis_w;        // phase flip: working index of the basis state
    uint32_t basis_in_stage; // phase flip: 1 if the basis' outer bits can match a group
    uint32_t pad1;
};

// wv: ngroups consecutive working vectors of 2^W amplitudes; gbase[g] is the
// full-index value of group g's outer bits.
void launch_pass(float2 *wv, uint32_t W, uint32_t ngroups, const PassDev *pass_host, const PassDev *pass_dev,
                 const OpDev *ops_dev, const float2 *mats_dev, const uint64_t *gbase_dev, int prec,
                 cudaStream_t s);

}  // namespace qsim
