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
    uint32_t mat_elems;      // float2 of the matrix area (dense ops whose matrix is not in the blob)
    uint32_t kmax;           // widest dense op of the pass (0 if none)
    uint32_t blob_words;     // 16-byte words of the pass blob: op descriptors, phase tables, small matrices
    uint32_t blob_off;       // its first word in the plan's blob array
    uint32_t umma;           // bit 0: the pass's k = 5 TF32 dense ops run on tcgen05 (B operands in 128-byte
                             // swizzled form); bit 1: test hook, no MMA is issued or committed to the mbarrier;
                             // bit 2: split-BF16 B operands (three parts, 24 KB); bit 3: a TF32 width-6 op
                             // (B operand 64 KB, 128 TMEM columns)
    uint64_t out_mask;       // working-index mask of the non-tile bits
    uint32_t tile_pos[16];   // working bit of tile bit t (ascending)
    uint32_t out_pos[32];    // working bit of CTA-index bit t
};

struct __align__(16) OpDev {
    uint32_t type;           // 0 dense, 1 diagonal, 2 phase flip, 3 controlled-separable, OP_POLY (4)
    uint32_t k;
    uint32_t mat;            // float2 offset of the matrix (dense) or phases (diag) in the plan's matrix array
    uint32_t dlut;           // diag: float2 offset of its phase-index byte tables (pass: in the blob; decoder
                             // pre-op: in the matrix array); dense on tensor cores: word offset in the blob of its
                             // swizzled group-base (128) and column (32) offsets, else kNoTab
    uint32_t tq[6];          // dense: tile bit of matrix bit j
    uint32_t dsrc[8];        // diag: working bit (< 64) or 64 + full qubit (outer, from group base)
    uint32_t dtile[8];       // diag in a pass: tile bit of qubit j, or 255 when the bit is constant over a tile
    uint32_t comp[16];       // dense: complement tile bits; comp[0..3] feed the lane bits
    uint64_t basis_outer;    // phase flip: basis & outer mask (full index bits)
    uint64_t basis_w;        // phase flip: working index of the basis state
    uint32_t basis_in_stage; // phase flip: 1 if the basis' outer bits can match a group
    uint32_t bfrag;          // dense, tensor-core precisions: word offset of the op's B-fragment table
    uint32_t run;            // diag in a pass: ops applied in one sweep from here (0 inside a run)
    uint32_t tab;            // in a pass: float2 offset in the blob of the phases (diag), of the matrix (dense
                             // on CUDA cores) or of the tile-bit tables P_lo[2][128] (csep); kNoTab when not there
    uint32_t cctl;           // csep: control at tile bit cctl, or kCtlConst | source (working bit < 64 or 64 + qubit);
                             // kCtlId0 / kCtlId1: that branch is the identity
    uint32_t ncst;           // csep: targets outside the tile (records at blob offset `mat`, P_hi[2][64] at `dlut`);
                             // OP_POLY: number of term records
};

constexpr uint32_t kCtlConst = 0x80000000u;
constexpr uint32_t kCtlId0 = 0x40000000u;  // csep: branch 0 (control bit clear) is the identity
constexpr uint32_t kCtlId1 = 0x20000000u;  // csep: branch 1 is the identity
constexpr uint32_t kCtlFlags = kCtlConst | kCtlId0 | kCtlId1;

constexpr uint32_t kDiagRun = 4;            // diagonal ops applied in one sweep over a tile
// An OpDev of type OP_POLY heads a run of diagonal ops whose phases are polynomials of degree <= 2 in the index bits
// (4096-amplitude tiles): `tab` is the word offset in the pass blob of the run's summed polynomial (kPolyHeadWords
// words: G[12][12], Q7[32], Q8[16], A0[12], C0, padding; every coefficient an angle in turns as 32-bit fixed point,
// 2^32 = one turn) followed by `ncst` term records of 4 words
constexpr uint32_t OP_POLY = 4;
constexpr uint32_t kPolyHeadWords = 208;
constexpr uint32_t kPolyConst = 0xffffffffu;  // term record: adds to the constant, not to a tile bit's coefficient
constexpr uint32_t kNoSrc = 0xffffffffu;      // term record: no second source bit
constexpr uint32_t kNoTab = 0xffffffffu;
constexpr uint32_t kPassBlobMax = 40960;    // bytes of one pass blob (shared memory next to the tile)

// wv: ngroups consecutive working vectors of 2^W amplitudes; gbase[g] is the
// full-index value of group g's outer bits.
// B-fragment tables (tensor-core precisions): the real matrix U_r^T of every
// dense op, rounded to TF32 or split into BF16 hi/mid/lo, laid out in the
// register order of the warp MMA's B operand so a lane loads its fragment
// with one 8-byte load:
//   TF32 (m16n8k8):  [kstep][ntile][lane][2]      = U_r^T[8 ks + t (+4)][8 nt + g]
//   BF16 (m16n8k16): [part][kstep][ntile][lane][2] = pairs U_r^T[16 ks + 2t (+1) (+8)][8 nt + g]
// with g = lane / 4, t = lane % 4, U_r = [[Re U, -Im U], [Im U, Re U]].
void build_bfrag_table(const double *u_interleaved, uint32_t k, int prec, uint32_t *out);
size_t bfrag_words(uint32_t k, int prec);

// The B operand of a k = 5 dense op for tcgen05 (4096 words, the same count as its TF32 fragment table):
// B^T = U_r rounded to TF32, row n = output n (Re outputs 0..31, then Im), column = input (Re inputs, then
// Im), K-major in the 128-byte swizzled layout: column block a = input / 32 at byte 8192 a, row n at
// 1024 (n / 8) + 128 (n % 8), 16-byte chunk c = (input % 32) / 4 stored at chunk position c ^ (n % 8).
// Shared memory a tcgen05 pass adds (its B buffer and 1024 bytes of alignment slack) from PassDev::umma; 0 for
// a pass without tcgen05 ops.
size_t umma_pass_smem(uint32_t umma_bits);
void build_umma_b(const double *u_interleaved, uint32_t *out);
// The TF32 B operand of a width-6 op for tcgen05 (16384 words, 64 KB): U_r^T (128 x 128) K-major in four 128-byte
// K-chunks of 128 rows (16 KB each, chunk a holding inputs 32a .. 32a + 31), rows n swizzled as in build_umma_b.
void build_umma_b6(const double *u_interleaved, uint32_t *out);
// The split-BF16 form (6144 words, the count of its warp-MMA fragment table): three 8 KB parts hi, mid, lo of
// U_r (x = hi + mid + lo, each rounded to BF16 nearest-even), each part 64 rows of 64 BF16 inputs in the same
// swizzled layout (row n at 1024 (n / 8) + 128 (n % 8), 16-byte chunk c = input / 8 at position c ^ (n % 8)).
void build_umma_b3(const double *u_interleaved, uint32_t *out);

// One pass over ngroups consecutive working vectors of 2^W amplitudes. ctr: two words of device memory, zero
// before the first launch on a stream, that the launch leaves zero again; launches that overlap on the GPU
// (other streams) need their own.
void launch_pass(float2 *wv, uint32_t W, uint32_t ngroups, const PassDev *pass_host, const uint4 *blob_dev,
                 const float2 *mats_dev, const uint32_t *bfr_dev, const uint64_t *gbase_dev, int prec,
                 cudaStream_t s, uint32_t *ctr, int *status);

// dynamic shared memory of one tile pass (tile, B operand and alignment when on tcgen05, blob, matrices)
size_t pass_smem_bytes(const PassDev &P);

}  // namespace qsim
