// Internal declarations shared by the library's translation units.
#pragma once

#include <stdint.h>
#include <stddef.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// error reporting (thread-local message, no exceptions across the ABI)
// ---------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
void clear_error();

// ---------------------------------------------------------------------------
// QSZ1 format constants (block codec; the layout is spelled out in codec.cu)
// ---------------------------------------------------------------------------
constexpr uint32_t kQszMagic = 0x315A5351u;  // "QSZ1"
constexpr uint32_t kQszHeader = 32;
constexpr int kQszMaxFrameLog = 12;
constexpr int kQszMinM = 5;
constexpr int kQszMaxM = 26;
constexpr int kQszEMin = -126;
constexpr int kQszEMax = 96;

inline uint64_t pad16(uint64_t x) { return (x + 15) & ~uint64_t(15); }
inline int frame_log_for(int m) { return m < kQszMaxFrameLog ? m : kQszMaxFrameLog; }
inline uint64_t qsz_nframes(int m) { return uint64_t(1) << (m - frame_log_for(m)); }
inline uint64_t qsz_data_start(int m) { return kQszHeader + pad16(4 * (qsz_nframes(m) + 1)); }
inline uint64_t qsz_worst_case(int m) {
    uint64_t F = uint64_t(1) << frame_log_for(m), C = F / 32;
    return qsz_data_start(m) + qsz_nframes(m) * (pad16(2 * C) + 8 * F);
}
// largest e with 2^e <= 2*eb (frexp, exact); returns false when out of range
bool qsz_step_exponent(double eb, int *e);

// QSZR: the relative-bound variant (codes = FP32 magnitude bits rounded to multiples of 2^k, sign chunks)
constexpr uint32_t kQszrMagic = 0x525A5351u;  // "QSZR"
constexpr int kQszrKMin = 1;
constexpr int kQszrKMax = 22;
constexpr uint32_t kQszrSideBytes = 2048;  // per-frame side record of the in-place encoder
inline uint64_t qszr_worst_case(int m) {
    uint64_t F = uint64_t(1) << frame_log_for(m), C = F / 32;
    return qsz_data_start(m) + qsz_nframes(m) * (pad16(2 * C) + pad16((2 * C + 3) / 4) + pad16(8 * C) + 8 * F);
}
// largest k with 2^(k-24) <= rel / (1 + rel); returns false when out of range
bool qszr_shift(double rel, int *k);

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
enum OpType : uint32_t { OP_DENSE = 0, OP_DIAG = 1, OP_PHASEFLIP = 2, OP_CSEP = 3 };

struct Op {
    OpType type;
    uint32_t k;             // dense: width; diag: number of qubits
    uint32_t wq[6];         // dense: working-index bit of matrix bit j
    uint32_t fq[8];         // diag: full qubit ids (matrix bit j)
    uint64_t basis;         // phaseflip
    std::vector<cd> u;      // dense: 2^k x 2^k row-major; diag: 2^k phases; csep: see below
    uint32_t ngates;        // input gates folded into this op
    // csep (controlled-separable diagonal): phase(x) = K[b] * prod_t D_t[b][x_t] with b = x_c;
    // csep_q = {c, t_1, t_2, ...} (full qubits), u = {K[0], K[1], then per target D[0][0], D[0][1], D[1][0], D[1][1]}
    std::vector<uint32_t> csep_q;
    bool quad = false;      // diag: its phase is a polynomial of degree <= 2 in its bits (diag_quadratic)
};

// A diagonal op whose phase angle is a polynomial of degree at most 2 in its qubits' bits, which every product
// of one- and two-qubit diagonal gates is: phase(x) = exp(2 pi i (c + sum_j a[j] x_j + sum_{j<l} g[j][l] x_j x_l))
// with x_j the bit of qubit j of the op; angles in turns, each reduced to [-1/2, 1/2).
struct DiagPoly {
    double c = 0;
    double a[8] = {};
    double g[8][8] = {};
};
// true (and *out filled) when op is an OP_DIAG op of unit-modulus phases whose angles match such a polynomial to
// 1e-9 turns at every one of its 2^k indices
bool diag_quadratic(const Op &op, DiagPoly *out);

struct Pass {
    uint32_t T;                   // tile bits
    uint32_t tile_pos[16];        // working bit of tile bit t, ascending
    std::vector<uint32_t> ops;    // indices into Stage::ops
};

struct Stage {
    size_t first_gate = 0, ngates = 0;
    std::vector<uint32_t> inner;  // ascending global qubits that are local in this stage
    uint32_t W = 0;               // working vector = 2^W amplitudes (m + |inner|)
    std::vector<Op> ops;
    std::vector<uint32_t> pre_ops;  // leading diagonal ops applied while decoding (no pass needed)
    std::vector<Pass> passes;
    bool pass_order = false;  // the stage's gates were reordered pass by pass (QSIM_REORDER_PASSES)
};

constexpr uint32_t kMaxPreOps = 8;
constexpr uint32_t kMaxDiagQubits = 8;  // widest fused diagonal op (phase index fits a byte)
constexpr size_t kOpDescBytes = 208;    // device descriptor of an op in a pass
constexpr size_t kPassOpBytes = 32768;  // op data of one pass held in shared memory next to its tile
constexpr size_t kCsepTableBytes = 3072; // controlled-separable op: tile-bit tables P_lo[2][128], P_hi[2][64]

struct Gate {
    uint32_t nq = 0;
    uint32_t q[6] = {0, 0, 0, 0, 0, 0};
    bool diag = false;
    bool phaseflip = false;
    uint64_t basis = 0;
    std::vector<cd> u;  // 2^nq x 2^nq
};

}  // namespace qsim

struct qsim_plan {
    uint32_t n = 0;
    qsim_config cfg{};
    std::vector<qsim::Gate> gates;
    std::vector<qsim::Stage> stages;
    qsim_plan_stats stats{};
};

namespace qsim {
// planner.cpp
int build_plan(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *cfg,
               qsim_plan **out);
int plan_shards(const qsim_plan *p, uint32_t log2_ranks, uint32_t *rank_qubits);
}  // namespace qsim
