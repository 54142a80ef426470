// Stage engine, two-tier block pool, readout and the C ABI (host side).
//
// Execution follows the paper's transfer-concealed workflow (Sec. 4.2): every
// SV group of a stage goes through decompress -> update -> compress on one CUDA
// stream, and groups are dealt round-robin to the streams so that the codec,
// the gate passes and (for the pinned-host tier) the link traffic of different
// groups overlap. A group is the 2^|inner| blocks sharing the stage's outer
// global bits (Sec. 4.1); consecutive groups are batched into one launch per
// kernel so that small blocks still fill the GPU.
//
// Compressed blocks live in bump arenas: a device arena and, when the device
// tier is capped or full, a mapped pinned-host arena (the two memory levels of
// Sec. 4.4, with pinned host memory standing in for the SSD tier). Each stage
// reads the arena written by the previous stage and writes the other one, so
// the memory held is the compressed input plus output of one stage. Slots are
// reserved on the device (atomic bump), so no host round trip is needed
// between the sizing and the encoding of a block.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "codec.cuh"
#include "device_common.cuh"
#include "gates.cuh"
#include "mlp.cuh"
#include "persistent.cuh"
#include "qsim_internal.h"

namespace qsim {

// ---------------------------------------------------------------------------
// errors, counters
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_allocs{0};  // successful cudaMalloc / cudaHostAlloc calls of the library

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}
void clear_error() { g_err[0] = 0; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// optional per-kernel event timing (events reused across runs)
// ---------------------------------------------------------------------------
static std::atomic<int> g_profile{0};
enum ProfCat { P_DECODE = 0, P_PASS, P_ENCODE_SIZE, P_RESERVE, P_ENCODE, P_GATHER, P_COPY_IN, P_COPY_OUT, P_INIT,
               P_PREDICT, P_REENCODE, P_STAGE, P_FRAME_COPY, P_NCAT };
static const char *kProfNames[P_NCAT] = {"decode", "gate_pass", "encode_size", "reserve", "encode",
                                         "gather_refs", "copy_in", "copy_out", "init", "predict", "reencode",
                                         "stage_persistent", "frame_copy"};

struct Profiler {
    bool on = false;
    struct Rec {
        int cat;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    size_t used = 0;
    static std::vector<cudaEvent_t> &pool() {
        static std::vector<cudaEvent_t> *p = new std::vector<cudaEvent_t>();
        return *p;
    }
    cudaEvent_t get() {
        auto &P = pool();
        if (used < P.size()) return P[used++];
        cudaEvent_t e;
        cudaEventCreate(&e);
        P.push_back(e);
        ++used;
        return e;
    }
    void begin(int cat, cudaStream_t s) {
        if (!on) return;
        Rec r{cat, get(), nullptr};
        cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end(cudaStream_t s) {
        if (!on) return;
        recs.back().b = get();
        cudaEventRecord(recs.back().b, s);
    }
    // after synchronisation
    void collect(double secs[P_NCAT], uint64_t launches[P_NCAT]) {
        for (int c = 0; c < P_NCAT; ++c) { secs[c] = 0; launches[c] = 0; }
        for (const Rec &r : recs) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                secs[r.cat] += ms * 1e-3;
                launches[r.cat] += 1;
            }
        }
        cudaGetLastError();
    }
};

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess)                                                              \
            return set_error(_e == cudaErrorMemoryAllocation ? QSIM_E_NOMEM : QSIM_E_CUDA,  \
                             "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
    } while (0)

// NVTX range for timeline tools (a no-op when none is attached)
struct NvtxRange {
    explicit NvtxRange(const char *fmt, ...) {
        char buf[96];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
};

// ---------------------------------------------------------------------------
// caching allocator (device and pinned host), exact-size reuse
// ---------------------------------------------------------------------------
struct Cache {
    std::mutex mu;
    std::multimap<size_t, void *> dev_free, host_free;
    std::map<void *, size_t> dev_live, host_live;
};
static Cache &cache() {
    static Cache *c = new Cache();
    return *c;
}

static int dev_alloc(void **p, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    Cache &c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.dev_free.find(bytes);
        if (it != c.dev_free.end()) {
            *p = it->second;
            c.dev_free.erase(it);
            c.dev_live[*p] = bytes;
            return QSIM_OK;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // drop cached blocks and retry once
        qsim_release_cached_memory();
        e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(QSIM_E_NOMEM, "cudaMalloc(%zu) failed", bytes);
        }
    }
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(c.mu);
    c.dev_live[*p] = bytes;
    return QSIM_OK;
}

// bytes of device memory held by the cache for reuse (free for a new run's sizing)
static uint64_t cached_dev_bytes() {
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    uint64_t b = 0;
    for (const auto &kv : c.dev_free) b += kv.first;
    return b;
}

static void dev_free(void *p) {
    if (!p) return;
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.dev_live.find(p);
    if (it == c.dev_live.end()) return;
    c.dev_free.emplace(it->second, p);
    c.dev_live.erase(it);
}

static int host_alloc(void **p, size_t bytes) {
    bytes = (bytes + 4095) & ~size_t(4095);
    Cache &c = cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.host_free.find(bytes);
        if (it != c.host_free.end()) {
            *p = it->second;
            c.host_free.erase(it);
            c.host_live[*p] = bytes;
            return QSIM_OK;
        }
    }
    cudaError_t e = cudaHostAlloc(p, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(QSIM_E_NOMEM, "cudaHostAlloc(%zu) failed", bytes);
    }
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(c.mu);
    c.host_live[*p] = bytes;
    return QSIM_OK;
}

static void host_free(void *p) {
    if (!p) return;
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.host_live.find(p);
    if (it == c.host_live.end()) return;
    c.host_free.emplace(it->second, p);
    c.host_live.erase(it);
}

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    int alloc(size_t count) {
        release();
        n = count;
        if (!count) return QSIM_OK;
        return dev_alloc(reinterpret_cast<void **>(&p), count * sizeof(T));
    }
    void release() {
        dev_free(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
};

// ---------------------------------------------------------------------------
// per-device context: status word and the single-block codec scratch
// ---------------------------------------------------------------------------
struct DeviceCtx {
    std::mutex mu;  // serialises the single-block entry points
    // relative-bound block compression: a copy of the block, the Im-plane scratch and the per-frame records
    uint8_t *rel_buf = nullptr;
    size_t rel_cap = 0;
    int *status = nullptr;
    uint64_t *lb_state = nullptr;
    uint32_t *lb_ctr = nullptr;  // ticket, done, epoch
    EncTarget *tgt = nullptr;
    EncResult *res = nullptr;
    BlockRef *ref = nullptr;
    bool ready = false;
    // learned size predictor of this device
    float *pred_params = nullptr;
    bool pred_ready = false;
    int pred_bf16 = 0;
};

static DeviceCtx &device_ctx(int dev) {
    static DeviceCtx ctx[16];
    return ctx[dev & 15];
}

static int ensure_device_ctx(DeviceCtx &c) {
    if (c.ready) return QSIM_OK;
    const size_t max_frames = size_t(1) << (kQszMaxM - kQszMaxFrameLog);
    auto alloc = [](auto **p, size_t bytes) {
        const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
        if (e == cudaSuccess) g_allocs.fetch_add(1, std::memory_order_relaxed);
        return e;
    };
    CUDA_TRY(alloc(&c.status, 256));
    CUDA_TRY(alloc(&c.lb_state, max_frames * sizeof(uint64_t)));
    CUDA_TRY(alloc(&c.lb_ctr, 256));
    CUDA_TRY(alloc(&c.tgt, sizeof(EncTarget)));
    CUDA_TRY(alloc(&c.res, sizeof(EncResult)));
    CUDA_TRY(alloc(&c.ref, sizeof(BlockRef)));
    CUDA_TRY(alloc(&c.pred_params, kMlpParams * sizeof(float)));
    CUDA_TRY(cudaMemset(c.status, 0, 256));
    CUDA_TRY(cudaMemset(c.lb_state, 0, max_frames * sizeof(uint64_t)));
    CUDA_TRY(cudaMemset(c.lb_ctr, 0, 256));
    c.ready = true;
    return QSIM_OK;
}

static LookbackScratch make_scratch(uint64_t *state, uint32_t *ctr, float2 *part = nullptr) {
    LookbackScratch s{};
    s.part = part;
    s.state = state;
    s.ticket = ctr;
    s.done = ctr + 1;
    s.epoch = ctr + 2;
    return s;
}

static int read_status(int *d_status, cudaStream_t s) {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    return h;
}

static const char *status_text(int code) {
    switch (code) {
        case QSIM_E_INVALID: return "non-finite input value";
        case QSIM_E_RANGE: return "value out of the codec range (|x|/2^e >= 2^30)";
        case QSIM_E_CORRUPT: return "corrupt compressed stream";
        case QSIM_E_NOMEM: return "compressed-block tiers are full";
        case QSIM_E_TIMEOUT: return "a bounded device wait gave up";
        default: return "device error";
    }
}

// ---------------------------------------------------------------------------
// plan upload: pass/op descriptors, matrices, group layouts
// ---------------------------------------------------------------------------
struct StageDev {
    uint32_t W, G;              // working bits, blocks per group
    uint32_t ngroups;
    uint32_t pass_begin, npasses;
    uint32_t pre_begin, npre;   // leading phase ops applied by the decoder
    std::vector<PassDev> passes_host;
};

static_assert(sizeof(OpDev) == kOpDescBytes, "the planner sizes pass blobs by the descriptor size");

struct PlanDev {
    bool ready = false;
    int device = -1;
    DevBuf<PassDev> passes;
    DevBuf<OpDev> ops;
    DevBuf<float2> mats;
    DevBuf<uint32_t> bfr;     // B-fragment tables of the dense ops (tensor-core precisions)
    DevBuf<uint4> blob;       // per pass: op descriptors, phase tables and index tables, small matrices
    DevBuf<uint32_t> ids;     // per stage: 2^c block ids, group-major
    DevBuf<uint64_t> gbase;   // per stage: per group outer bits
    std::vector<StageDev> stages;
    std::vector<size_t> ids_off, gbase_off;
    uint64_t upload_bytes = 0;
    bool counted = false;  // upload bytes reported by the first run that used it
};

static std::mutex g_plan_mu;
static std::map<const qsim_plan *, PlanDev *> g_plan_dev;

// Order the op's complement tile bits (the bits that enumerate its index
// groups). Tile bit t lands on bank-pair bit t % 4 of the swizzled layout; a
// half-warp's 16 accesses are conflict-free when the 4 tile bits that vary
// across them fall on 4 different residues. SIMT ops: lanes are consecutive
// groups, so the first 4 complement bits take distinct residues. Tensor-core
// ops: a half-warp spans 2 row bits (complement bits 0, 1) and 2 column bits
// (the op's matrix bits 0, 1), so the first 2 complement bits avoid the
// residues of those columns.
static void order_complement(OpDev &od, uint32_t T, bool mma) {
    bool is_t[16] = {false};
    for (uint32_t j = 0; j < od.k; ++j) is_t[od.tq[j]] = true;
    std::vector<uint32_t> comp;
    for (uint32_t t = 0; t < T; ++t)
        if (!is_t[t]) comp.push_back(t);
    std::vector<uint32_t> first, rest;
    bool have[4] = {false, false, false, false};
    uint32_t want = 4;
    if (mma && od.k >= 2) {
        have[od.tq[0] % 4] = true;
        have[od.tq[1] % 4] = true;
        want = 2;
    }
    for (uint32_t t : comp) {
        if (!have[t % 4] && first.size() < want) {
            have[t % 4] = true;
            first.push_back(t);
        } else {
            rest.push_back(t);
        }
    }
    uint32_t i = 0;
    for (uint32_t t : first) od.comp[i++] = t;
    for (uint32_t t : rest) od.comp[i++] = t;
    for (; i < 16; ++i) od.comp[i] = 0;
}

// Dense op `op` (width k <= kw, all of its working bits tile bits of pass ps) as a width-kw op: matrix bits
// k..kw-1 are the lowest tile bits the op does not touch, and the matrix is I (x) U (the identity on those
// bits): U'[r][c] = U[r mod 2^k][c mod 2^k] when r and c agree above bit k, else 0.
static Op widen_dense(const Op &op, const Pass &ps, uint32_t kw) {
    Op w = op;
    const uint32_t k = op.k, D = 1u << k, DW = 1u << kw;
    for (uint32_t t = 0, j = k; j < kw && t < ps.T; ++t) {
        const uint32_t b = ps.tile_pos[t];
        bool used = false;
        for (uint32_t i = 0; i < j; ++i) used |= w.wq[i] == b;
        if (!used) w.wq[j++] = b;
    }
    w.k = kw;
    w.u.assign(size_t(DW) * DW, cd(0, 0));
    for (uint32_t r = 0; r < DW; ++r)
        for (uint32_t c = 0; c < DW; ++c)
            if ((r >> k) == (c >> k)) w.u[size_t(r) * DW + c] = op.u[size_t(r & (D - 1)) * D + (c & (D - 1))];
    return w;
}

static int upload_plan(const qsim_plan *p, PlanDev **out) {
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plan_dev.find(p);
    if (it != g_plan_dev.end() && it->second->device == dev) {
        *out = it->second;
        return QSIM_OK;
    }
    PlanDev *pd = new PlanDev();
    pd->device = dev;
    const uint32_t n = p->n, m = p->cfg.m, c = n - m;
    std::vector<PassDev> passes;
    std::vector<uint4> blob;
    std::vector<OpDev> ops;
    std::vector<float2> mats;
    std::vector<uint32_t> bfr;
    std::vector<uint32_t> ids;
    std::vector<uint64_t> gbases;
    for (const Stage &st : p->stages) {
        StageDev sd;
        sd.W = st.W;
        sd.G = 1u << st.inner.size();
        sd.ngroups = 1u << (c - st.inner.size());
        sd.pass_begin = passes.size();
        sd.npasses = st.passes.size();
        std::vector<uint32_t> outer;
        uint64_t outer_mask = 0;
        for (uint32_t q = m; q < n; ++q)
            if (std::find(st.inner.begin(), st.inner.end(), q) == st.inner.end()) {
                outer.push_back(q);
                outer_mask |= 1ull << q;
            }
        pd->ids_off.push_back(ids.size());
        pd->gbase_off.push_back(gbases.size());
        for (uint64_t g = 0; g < sd.ngroups; ++g) {
            uint64_t gb = 0;
            for (size_t t = 0; t < outer.size(); ++t) gb |= ((g >> t) & 1ull) << outer[t];
            gbases.push_back(gb);
            for (uint64_t j = 0; j < sd.G; ++j) {
                uint64_t full = gb;
                for (size_t t = 0; t < st.inner.size(); ++t) full |= ((j >> t) & 1ull) << st.inner[t];
                ids.push_back(uint32_t(full >> m));
            }
        }
        auto diag_opdev = [&](const Op &op) {
            OpDev od{};
            od.type = op.type;
            od.k = op.k;
            for (int j = 0; j < 8; ++j) od.dtile[j] = 255;
            if (op.type == OP_DIAG) {
                for (uint32_t j = 0; j < op.k; ++j) {
                    uint32_t q = op.fq[j];
                    if (q < m) {
                        od.dsrc[j] = q;
                    } else {
                        auto f = std::find(st.inner.begin(), st.inner.end(), q);
                        od.dsrc[j] = f != st.inner.end() ? uint32_t(m + (f - st.inner.begin())) : 64 + q;
                    }
                }
                od.mat = mats.size();
                for (const cd &v : op.u) mats.push_back(make_float2(float(v.real()), float(v.imag())));
            } else {
                od.basis_in_stage = 1;
                od.basis_outer = op.basis & outer_mask;
                uint64_t w = op.basis & ((1ull << m) - 1);
                for (size_t t = 0; t < st.inner.size(); ++t) w |= ((op.basis >> st.inner[t]) & 1ull) << (m + t);
                od.basis_w = w;
            }
            return od;
        };
        sd.pre_begin = ops.size();
        sd.npre = st.pre_ops.size();
        for (uint32_t oi : st.pre_ops) {
            OpDev od = diag_opdev(st.ops[oi]);
            if (od.type == OP_DIAG) {
                // decoder tables: phase-index bits from the lane (working bits 0..4, 32 bytes) and from the
                // chunk within the frame (working bits 5..fl-1, 128 bytes)
                const uint32_t fl = uint32_t(frame_log_for(int(m)));
                uint8_t lut[160] = {0};
                for (uint32_t j = 0; j < od.k; ++j) {
                    const uint32_t src = od.dsrc[j];
                    if (src < 5) {
                        for (uint32_t x = 0; x < 32; ++x) lut[x] |= uint8_t(((x >> src) & 1u) << j);
                    } else if (src < fl) {
                        for (uint32_t x = 0; x < 128; ++x) lut[32 + x] |= uint8_t(((x >> (src - 5)) & 1u) << j);
                    }
                }
                while (mats.size() & 1) mats.push_back(make_float2(0, 0));
                od.dlut = mats.size();
                for (uint32_t w = 0; w < 20; ++w) {
                    float2 fv;
                    memcpy(&fv, lut + 8 * w, 8);
                    mats.push_back(fv);
                }
            }
            ops.push_back(od);
        }
        for (const Pass &ps : st.passes) {
            PassDev P{};
            P.T = ps.T;
            uint32_t L = 0;
            while (L < ps.T && ps.tile_pos[L] == L) ++L;
            P.L = L;
            P.nout = st.W - ps.T;
            for (uint32_t t = 0; t < ps.T; ++t) P.tile_pos[t] = ps.tile_pos[t];
            uint32_t o = 0;
            uint64_t om = 0;
            for (uint32_t b = 0; b < st.W; ++b) {
                bool in_tile = false;
                for (uint32_t t = 0; t < ps.T; ++t) in_tile |= ps.tile_pos[t] == b;
                if (!in_tile) {
                    P.out_pos[o++] = b;
                    om |= 1ull << b;
                }
            }
            P.out_mask = om;
            if (ps.T > kMaxTileBits || o != P.nout)
                return set_error(QSIM_E_INVALID, "internal: pass tile layout out of range");
            for (uint32_t t = 0; t < ps.T; ++t)
                if (ps.tile_pos[t] >= st.W) return set_error(QSIM_E_INVALID, "internal: tile bit outside the working vector");
            P.op_begin = ops.size();
            P.op_count = ps.ops.size();
            P.mat_elems = 0;
            for (uint32_t oi : ps.ops) {
                // in passes whose width-5 dense ops run on tcgen05, dense ops of width 3 and 4 run there too,
                // as width-5 ops: the op's matrix times the identity on the lowest tile bits it does not touch
                // (the same operator, so the same result up to the FP32 accumulation order)
                Op wide;
                const Op *opp = &st.ops[oi];
                if (opp->type == OP_DENSE && (opp->k == 3 || opp->k == 4) && ps.T == 12 && p->cfg.tcgen05 &&
                    (p->cfg.prec == QSIM_PREC_TF32 || p->cfg.prec == QSIM_PREC_BF16X3)) {
                    wide = widen_dense(*opp, ps, 5);
                    opp = &wide;
                }
                const Op &op = *opp;
                OpDev od{};
                od.type = op.type;
                od.k = op.k;
                if (op.type == OP_DENSE) {
                    od.dlut = kNoTab;  // set for tensor-core ops when the pass blob is laid out
                    for (uint32_t j = 0; j < op.k; ++j) {
                        uint32_t t = 0;
                        while (ps.tile_pos[t] != op.wq[j]) ++t;
                        od.tq[j] = t;
                    }
                    const uint32_t min_k = p->cfg.prec == QSIM_PREC_TF32 ? 3u : 4u;
                    // dense ops of 4096-amplitude passes on tcgen05 when asked for (one thread per index group of a
                    // 128-thread CTA, in both modes: the complement ordered for that gather): width 5 (and the
                    // widened 3 and 4) in TF32 or split BF16, width 6 in TF32
                    const bool um6 = p->cfg.tcgen05 && p->cfg.prec == QSIM_PREC_TF32 && op.k == 6 && ps.T == 12;
                    const bool um = um6 || (p->cfg.tcgen05 && op.k == 5 && ps.T == 12 &&
                                            (p->cfg.prec == QSIM_PREC_TF32 || p->cfg.prec == QSIM_PREC_BF16X3));
                    order_complement(od, ps.T,
                                     !um && p->cfg.prec != QSIM_PREC_FP32 && op.k >= min_k && op.k <= 5 &&
                                         ps.T == 12);
                    od.mat = mats.size();
                    for (const cd &v : op.u) mats.push_back(make_float2(float(v.real()), float(v.imag())));
                    // the matrix area serves the CUDA-core form only (the tensor-core forms read B tables)
                    if (!um && !(p->cfg.prec != QSIM_PREC_FP32 && op.k >= min_k && op.k <= 5 && ps.T == 12))
                        P.mat_elems = std::max<uint32_t>(P.mat_elems, 1u << (2 * op.k));
                    if (p->cfg.prec != QSIM_PREC_FP32 && ((op.k >= 3 && op.k <= 5) || um6)) {
                        bfr.resize((bfr.size() + 3) & ~size_t(3));  // 16-byte aligned tables
                        od.bfrag = bfr.size();
                        bfr.resize(bfr.size() + bfrag_words(op.k, int(p->cfg.prec)));
                        if (um6)
                            build_umma_b6(reinterpret_cast<const double *>(op.u.data()), bfr.data() + od.bfrag);
                        else if (um && p->cfg.prec == QSIM_PREC_BF16X3)
                            build_umma_b3(reinterpret_cast<const double *>(op.u.data()), bfr.data() + od.bfrag);
                        else if (um)
                            build_umma_b(reinterpret_cast<const double *>(op.u.data()), bfr.data() + od.bfrag);
                        else
                            build_bfrag_table(reinterpret_cast<const double *>(op.u.data()), op.k, int(p->cfg.prec),
                                              bfr.data() + od.bfrag);
                        if (um)  // bit 1: wait-limit test hook; bit 2: split-BF16 operands; bit 3: a width-6 op
                            P.umma |= 1u | ((p->cfg.reserved[0] & 2) ? 2u : 0u) |
                                      (p->cfg.prec == QSIM_PREC_BF16X3 ? 4u : 0u) | (um6 ? 8u : 0u);
                    }
                    P.kmax = std::max<uint32_t>(P.kmax, op.k);
                } else if (op.type == OP_CSEP) {
                    // control and targets: tile bits, or bits constant over a tile (working bit or outer qubit)
                    auto source = [&](uint32_t q) -> uint32_t {
                        if (q < m) return q;
                        auto f = std::find(st.inner.begin(), st.inner.end(), q);
                        return f != st.inner.end() ? uint32_t(m + (f - st.inner.begin())) : 64 + q;
                    };
                    auto tile_bit = [&](uint32_t src) -> int32_t {
                        if (src >= 64) return -1;
                        for (uint32_t t = 0; t < ps.T; ++t)
                            if (ps.tile_pos[t] == src) return int32_t(t);
                        return -1;
                    };
                    od.k = uint32_t(op.csep_q.size());
                    const uint32_t cs = source(op.csep_q[0]);
                    const int32_t ctb = tile_bit(cs);
                    od.cctl = ctb >= 0 ? uint32_t(ctb) : (kCtlConst | cs);
                    // a branch whose factors are all exactly 1 leaves its amplitudes unchanged: skipped
                    for (uint32_t b = 0; b < 2; ++b) {
                        bool id = op.u[b] == cd(1, 0);
                        for (size_t t = 1; t < op.csep_q.size() && id; ++t)
                            id = op.u[2 + 4 * (t - 1) + 2 * b] == cd(1, 0) && op.u[2 + 4 * (t - 1) + 2 * b + 1] == cd(1, 0);
                        if (id) od.cctl |= b ? kCtlId1 : kCtlId0;
                    }
                } else {
                    od = diag_opdev(op);
                    if (op.type == OP_DIAG) {
                        P.mat_elems = std::max<uint32_t>(P.mat_elems, 1u << op.k);
                        for (uint32_t j = 0; j < op.k; ++j) {
                            od.dtile[j] = 255;
                            if (od.dsrc[j] < 64)
                                for (uint32_t t = 0; t < ps.T; ++t)
                                    if (ps.tile_pos[t] == od.dsrc[j]) od.dtile[j] = t;
                        }
                    }
                }
                ops.push_back(od);
            }
            // diagonal ops whose phase is a polynomial of degree <= 2 in their bits (4096-amplitude tiles only)
            std::vector<char> quad(P.op_count, 0);
            std::vector<DiagPoly> qpoly(P.op_count);
            if (ps.T == 12)
                for (uint32_t a = 0; a < P.op_count; ++a)
                    if (ops[P.op_begin + a].type == OP_DIAG) quad[a] = diag_quadratic(st.ops[ps.ops[a]], &qpoly[a]);
            // runs of consecutive diagonal ops applied in one sweep: up to kDiagRun table ops, or any number of
            // polynomial ops (one phase per amplitude for the whole run; the head becomes an OP_POLY descriptor)
            for (uint32_t a = P.op_begin; a < P.op_begin + P.op_count;) {
                if (ops[a].type != OP_DIAG) {
                    ++a;
                    continue;
                }
                const bool pq = quad[a - P.op_begin];
                uint32_t b = a;
                while (b < P.op_begin + P.op_count && ops[b].type == OP_DIAG && bool(quad[b - P.op_begin]) == pq &&
                       (pq || b - a < kDiagRun))
                    ops[b++].run = 0;
                ops[a].run = b - a;
                if (pq) ops[a].type = OP_POLY;
                a = b;
            }
            // the pass blob: descriptors, then per diagonal op its index tables (tile bits 0..6 and
            // 7..12, 192 bytes) and its phases, then CUDA-core dense matrices while they fit
            {
                std::vector<uint8_t> pb(size_t(P.op_count) * sizeof(OpDev));
                auto align16 = [&]() { pb.resize((pb.size() + 15) & ~size_t(15), 0); };
                const uint32_t min_k = p->cfg.prec == QSIM_PREC_TF32 ? 3u : 4u;
                P.mat_elems = 0;
                for (uint32_t a = 0; a < P.op_count; ++a) {
                    OpDev &od = ops[P.op_begin + a];
                    const Op &op = st.ops[ps.ops[a]];
                    od.tab = kNoTab;
                    if (od.type == OP_POLY) {
                        // the run's summed phase polynomial (angles in turns, 32-bit fixed point) over the tile bits t (the bits of a
                        // 4096-amplitude tile): G[t][t'] (t < t'), the run's quadratic part over tile bits 7..11
                        // (Q7, 32 values) and 8..11 (Q8, 16), the linear coefficients A0[t], the constant C0, then
                        // records {t or -1, source, source or kNoSrc, coefficient} of the terms with bits constant
                        // over the tile (a working bit outside the tile, or 64 + an outer qubit): tile bit t's linear
                        // coefficient, or (t = -1) the constant, gains the coefficient when those bits are 1
                        const uint32_t r = od.run;
                        double G[12][12] = {}, A0[12] = {}, C0 = 0;
                        std::map<std::array<uint32_t, 3>, double> terms;
                        for (uint32_t d = 0; d < r; ++d) {
                            const OpDev &rd = ops[P.op_begin + a + d];
                            const DiagPoly &q = qpoly[a + d];
                            C0 += q.c;
                            for (uint32_t j = 0; j < rd.k; ++j) {
                                if (rd.dtile[j] != 255) A0[rd.dtile[j]] += q.a[j];
                                else terms[{kPolyConst, rd.dsrc[j], kNoSrc}] += q.a[j];
                                for (uint32_t l = j + 1; l < rd.k; ++l) {
                                    const uint32_t tj = rd.dtile[j], tl = rd.dtile[l];
                                    if (tj != 255 && tl != 255) G[std::min(tj, tl)][std::max(tj, tl)] += q.g[j][l];
                                    else if (tj != 255) terms[{tj, rd.dsrc[l], kNoSrc}] += q.g[j][l];
                                    else if (tl != 255) terms[{tl, rd.dsrc[j], kNoSrc}] += q.g[j][l];
                                    else
                                        terms[{kPolyConst, std::min(rd.dsrc[j], rd.dsrc[l]),
                                               std::max(rd.dsrc[j], rd.dsrc[l])}] += q.g[j][l];
                                }
                            }
                        }
                        // angles as 32-bit fixed point in turns (2^32 = one turn): sums wrap exactly modulo a turn
                        auto red = [](double t) {
                            const double f = t - std::floor(t);
                            return uint32_t(uint64_t(std::llround(f * 4294967296.0)) & 0xffffffffull);
                        };
                        std::vector<uint32_t> w(kPolyHeadWords, 0u);
                        for (uint32_t t = 0; t < 12; ++t)
                            for (uint32_t t2 = t + 1; t2 < 12; ++t2) w[12 * t + t2] = red(G[t][t2]);
                        for (uint32_t u = 0; u < 32; ++u) {
                            double qv = 0, qv8 = 0;
                            for (uint32_t b = 7; b < 12; ++b)
                                for (uint32_t b2 = b + 1; b2 < 12; ++b2) {
                                    const bool on = ((u >> (b - 7)) & 1u) && ((u >> (b2 - 7)) & 1u);
                                    if (on) qv += G[b][b2];
                                    if (b >= 8 && u < 16 && ((u >> (b - 8)) & 1u) && ((u >> (b2 - 8)) & 1u)) qv8 += G[b][b2];
                                }
                            w[144 + u] = red(qv);
                            if (u < 16) w[176 + u] = red(qv8);
                        }
                        for (uint32_t t = 0; t < 12; ++t) w[192 + t] = red(A0[t]);
                        w[204] = red(C0);
                        align16();
                        od.tab = uint32_t(pb.size() / 4);
                        od.ncst = uint32_t(terms.size());
                        const uint8_t *wb = reinterpret_cast<const uint8_t *>(w.data());
                        pb.insert(pb.end(), wb, wb + 4 * w.size());
                        for (const auto &kv : terms) {
                            const uint32_t rec[4] = {kv.first[0], kv.first[1], kv.first[2], red(kv.second)};
                            const uint8_t *rb = reinterpret_cast<const uint8_t *>(rec);
                            pb.insert(pb.end(), rb, rb + 16);
                        }
                    } else if (od.type == OP_DIAG && quad[a]) {
                        // inside a polynomial run: nothing of its own in the blob
                    } else if (od.type == OP_DIAG) {
                        align16();
                        od.dlut = uint32_t(pb.size() / 8);
                        for (uint32_t v = 0; v < 192; ++v) {
                            const bool lo = v < 128;
                            const uint32_t x = lo ? v : v - 128;
                            uint32_t idx = 0;
                            for (uint32_t j = 0; j < od.k; ++j) {
                                const uint32_t t = od.dtile[j];
                                if (t == 255) continue;
                                if (lo && t < 7) idx |= ((x >> t) & 1u) << j;
                                if (!lo && t >= 7) idx |= ((x >> (t - 7)) & 1u) << j;
                            }
                            pb.push_back(uint8_t(idx));
                        }
                        align16();
                        od.tab = uint32_t(pb.size() / 8);
                        for (const cd &v : op.u) {
                            const float2 f = make_float2(float(v.real()), float(v.imag()));
                            const uint8_t *fb = reinterpret_cast<const uint8_t *>(&f);
                            pb.insert(pb.end(), fb, fb + 8);
                        }
                    } else if (od.type == OP_CSEP) {
                        P.mat_elems = std::max<uint32_t>(P.mat_elems, 128u);  // the per-tile branch table
                        // P_lo[b][x] over tile bits 0..6, P_hi[b][y] over tile bits 7.. (with K[b]), and the
                        // records {source, D[0][0], D[0][1], D[1][0], D[1][1]} of the targets outside the tile
                        auto source = [&](uint32_t q) -> uint32_t {
                            if (q < m) return q;
                            auto f = std::find(st.inner.begin(), st.inner.end(), q);
                            return f != st.inner.end() ? uint32_t(m + (f - st.inner.begin())) : 64 + q;
                        };
                        std::vector<cd> plo(256, cd(1, 0)), phi(128, cd(1, 0));
                        for (uint32_t b = 0; b < 2; ++b)
                            for (uint32_t y = 0; y < 64; ++y) phi[64 * b + y] = op.u[b];
                        std::vector<float2> recs;
                        for (size_t t = 1; t < op.csep_q.size(); ++t) {
                            const cd *D = op.u.data() + 2 + 4 * (t - 1);
                            const uint32_t src = source(op.csep_q[t]);
                            int32_t tb = -1;
                            if (src < 64)
                                for (uint32_t x = 0; x < ps.T; ++x)
                                    if (ps.tile_pos[x] == src) tb = int32_t(x);
                            if (tb >= 0 && tb < 7) {
                                for (uint32_t b = 0; b < 2; ++b)
                                    for (uint32_t x = 0; x < 128; ++x) plo[128 * b + x] *= D[2 * b + ((x >> tb) & 1u)];
                            } else if (tb >= 7) {
                                for (uint32_t b = 0; b < 2; ++b)
                                    for (uint32_t y = 0; y < 64; ++y) phi[64 * b + y] *= D[2 * b + ((y >> (tb - 7)) & 1u)];
                            } else {
                                float2 r0;
                                const uint32_t srcw = src;
                                memcpy(&r0.x, &srcw, 4);
                                r0.y = 0.f;
                                recs.push_back(r0);
                                for (int v = 0; v < 4; ++v)
                                    recs.push_back(make_float2(float(D[v].real()), float(D[v].imag())));
                            }
                        }
                        auto put = [&](const float2 &f) {
                            const uint8_t *fb = reinterpret_cast<const uint8_t *>(&f);
                            pb.insert(pb.end(), fb, fb + 8);
                        };
                        align16();
                        od.tab = uint32_t(pb.size() / 8);
                        for (const cd &v : plo) put(make_float2(float(v.real()), float(v.imag())));
                        align16();
                        od.dlut = uint32_t(pb.size() / 8);
                        for (const cd &v : phi) put(make_float2(float(v.real()), float(v.imag())));
                        align16();
                        od.mat = uint32_t(pb.size() / 8);
                        od.ncst = uint32_t(recs.size() / 5);
                        for (const float2 &f : recs) put(f);
                    } else if (od.type == OP_DENSE) {
                        const bool tc6 = od.k == 6 && (P.umma & 8u) && p->cfg.prec == QSIM_PREC_TF32;
                        const bool tc = (p->cfg.prec != QSIM_PREC_FP32 && od.k >= min_k && od.k <= 5 && ps.T == 12) ||
                                        tc6;
                        if (tc) {
                            // swizzled tile offsets of the op's index groups (128 words: the group bits 0..5 and
                            // 6.. through the complement) and of its matrix columns (2^k words), read by the
                            // tensor-core forms in place of a per-tile set-up
                            auto swz = [](uint32_t i) { return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15u); };
                            uint32_t t[192] = {};
                            const uint32_t nc = ps.T - od.k;
                            for (uint32_t x = 0; x < 128; ++x) {
                                const uint32_t half = x >> 6, v = x & 63u;
                                uint32_t bits = 0;
                                for (uint32_t j = 0; j < 6; ++j)
                                    if (6 * half + j < nc) bits |= ((v >> j) & 1u) << od.comp[6 * half + j];
                                t[x] = swz(bits);
                            }
                            for (uint32_t c = 0; c < (1u << od.k); ++c) {
                                uint32_t o = 0;
                                for (uint32_t j = 0; j < od.k; ++j) o |= ((c >> j) & 1u) << od.tq[j];
                                t[128 + c] = swz(o);
                            }
                            align16();
                            od.dlut = uint32_t(pb.size() / 4);
                            const uint8_t *tb = reinterpret_cast<const uint8_t *>(t);
                            pb.insert(pb.end(), tb, tb + 4 * (128 + (1u << od.k)));
                            continue;
                        }
                        const size_t mb = size_t(8) << (2 * od.k);
                        if (((pb.size() + 15) & ~size_t(15)) + mb <= kPassBlobMax) {
                            align16();
                            od.tab = uint32_t(pb.size() / 8);
                            for (const cd &v : op.u) {
                                const float2 f = make_float2(float(v.real()), float(v.imag()));
                                const uint8_t *fb = reinterpret_cast<const uint8_t *>(&f);
                                pb.insert(pb.end(), fb, fb + 8);
                            }
                        } else {
                            P.mat_elems = std::max<uint32_t>(P.mat_elems, 1u << (2 * od.k));
                        }
                    }
                }
                align16();
                memcpy(pb.data(), ops.data() + P.op_begin, size_t(P.op_count) * sizeof(OpDev));
                P.blob_off = uint32_t(blob.size());
                P.blob_words = uint32_t(pb.size() / 16);
                const size_t w0 = blob.size();
                blob.resize(w0 + P.blob_words);
                memcpy(blob.data() + w0, pb.data(), pb.size());
            }
            P.mat_elems = (P.mat_elems + 1) & ~1u;
            sd.passes_host.push_back(P);
            passes.push_back(P);
        }
        pd->stages.push_back(std::move(sd));
    }
    if (mats.empty()) mats.push_back(make_float2(0, 0));
    if (bfr.empty()) bfr.push_back(0);
    if (blob.empty()) blob.push_back(make_uint4(0, 0, 0, 0));
    int rc;
    if ((rc = pd->passes.alloc(passes.size())) || (rc = pd->ops.alloc(ops.size())) ||
        (rc = pd->mats.alloc(mats.size())) || (rc = pd->ids.alloc(ids.size())) || (rc = pd->bfr.alloc(bfr.size())) ||
        (rc = pd->gbase.alloc(gbases.size())) || (rc = pd->blob.alloc(blob.size()))) {
        delete pd;
        return rc;
    }
    CUDA_TRY(cudaMemcpy(pd->passes.p, passes.data(), passes.size() * sizeof(PassDev), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->ops.p, ops.data(), ops.size() * sizeof(OpDev), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->mats.p, mats.data(), mats.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->bfr.p, bfr.data(), bfr.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->ids.p, ids.data(), ids.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->gbase.p, gbases.data(), gbases.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pd->blob.p, blob.data(), blob.size() * sizeof(uint4), cudaMemcpyHostToDevice));
    pd->upload_bytes = passes.size() * sizeof(PassDev) + ops.size() * sizeof(OpDev) + mats.size() * sizeof(float2) +
                       bfr.size() * sizeof(uint32_t) + blob.size() * sizeof(uint4) +
                       ids.size() * sizeof(uint32_t) + gbases.size() * sizeof(uint64_t);
    pd->ready = true;
    if (it != g_plan_dev.end()) delete it->second;
    g_plan_dev[p] = pd;
    *out = pd;
    return QSIM_OK;
}

static void drop_plan_dev(const qsim_plan *p) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plan_dev.find(p);
    if (it != g_plan_dev.end()) {
        delete it->second;
        g_plan_dev.erase(it);
    }
}

}  // namespace qsim

// ---------------------------------------------------------------------------
// state handle
// ---------------------------------------------------------------------------
struct qsim_state {
    int device = 0;
    uint32_t n = 0, m = 0, codec = 0;
    int e = 0;
    uint8_t *dev_arena = nullptr;
    uint8_t *host_arena = nullptr;
    qsim::BlockSlot *table = nullptr;  // device, 2^(n-m) entries
    std::vector<qsim::StageAccum> stage_acc;
    std::vector<qsim_kernel_stat> kstats;
    std::vector<float> train_rows;  // collect mode: rows of 41 features + target
};

namespace qsim {

// small kernels used by the engine and readout
__global__ void k_init_blocks(float2 *wv, int m, uint64_t local_index) {
    // wv holds two blocks: [0] with the basis amplitude, [1] all zero
    const uint64_t N = 2ull << m;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < N; i += uint64_t(gridDim.x) * blockDim.x)
        wv[i] = make_float2(i == local_index ? 1.f : 0.f, 0.f);
}

// every block except b0 gets its own copy of the zero stream (Sec. 4.2)
__global__ void k_replicate_zero(BlockSlot *table, uint32_t nblocks, uint32_t b0, const BlockSlot *zero_slot,
                                 ArenaDev dev, ArenaDev host, int *status) {
    __shared__ uint8_t *dst;
    __shared__ uint32_t tier;
    const uint64_t bytes = zero_slot->bytes;
    for (uint32_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        if (b == b0) continue;
        if (threadIdx.x == 0) {
            const uint64_t sz = (bytes + 255) & ~255ull;
            uint64_t off = atomicAdd(reinterpret_cast<unsigned long long *>(dev.bump), sz);
            dst = nullptr;
            tier = 0;
            if (off + sz <= dev.cap) {
                dst = dev.base + off;
            } else if (host.base) {
                off = atomicAdd(reinterpret_cast<unsigned long long *>(host.bump), sz);
                if (off + sz <= host.cap) {
                    dst = host.base + off;
                    tier = 1;
                }
            }
            if (!dst) raise_status(status, QSIM_E_NOMEM);
            table[b].ptr = dst;
            table[b].bytes = bytes;
            table[b].tier = tier;
        }
        __syncthreads();
        if (dst) {
            const uint4 *s = reinterpret_cast<const uint4 *>(zero_slot->ptr);
            uint4 *d = reinterpret_cast<uint4 *>(dst);
            for (uint64_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
        }
        __syncthreads();
    }
}

__global__ void k_set_slot(BlockSlot *table, uint32_t b, const EncTarget *tgt, const EncResult *res) {
    table[b].ptr = tgt->ptr;
    table[b].bytes = res->total;
    table[b].tier = tgt->tier;
}

__global__ void k_copy_slot(BlockSlot *dst, const BlockSlot *src) { *dst = *src; }

__global__ void k_sum_table(const BlockSlot *table, uint64_t nblocks, StageAccum *acc) {
    uint64_t s = 0;
    for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nblocks; b += uint64_t(gridDim.x) * blockDim.x)
        s += table[b].bytes;
    atomicAdd(reinterpret_cast<unsigned long long *>(&acc->store_bytes), s);
}

// FP64 reductions for readout: <ref|sim>, ||ref||^2, ||sim||^2 over count amplitudes
__global__ void k_reduce_fid(const double2 *__restrict__ ref, const float2 *__restrict__ sim, uint64_t count,
                             double *acc) {
    double ip_r = 0, ip_i = 0, nr = 0, ns = 0;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < count; i += uint64_t(gridDim.x) * blockDim.x) {
        const double2 a = ref ? ref[i] : make_double2(0, 0);
        const float2 b = sim[i];
        const double br = b.x, bi = b.y;
        ip_r += a.x * br + a.y * bi;
        ip_i += a.x * bi - a.y * br;
        nr += a.x * a.x + a.y * a.y;
        ns += br * br + bi * bi;
    }
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ip_r += __shfl_xor_sync(kFull, ip_r, o);
        ip_i += __shfl_xor_sync(kFull, ip_i, o);
        nr += __shfl_xor_sync(kFull, nr, o);
        ns += __shfl_xor_sync(kFull, ns, o);
    }
    if (lane == 0) {
        red[0][w] = ip_r;
        red[1][w] = ip_i;
        red[2][w] = nr;
        red[3][w] = ns;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int i = 0; i < int(blockDim.x / 32); ++i) s += red[threadIdx.x][i];
        atomicAdd(&acc[threadIdx.x], s);
    }
}

__global__ void k_gather_amps(const float2 *__restrict__ blocks, const uint32_t *__restrict__ slot_of,
                              const uint32_t *__restrict__ local, uint64_t count, int m, float2 *out) {
    const uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    if (i < count) out[i] = blocks[(uint64_t(slot_of[i]) << m) + local[i]];
}

// ---------------------------------------------------------------------------
// the run
// ---------------------------------------------------------------------------
struct StreamWork {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf<float2> wv;
    DevBuf<BlockRef> refs;
    DevBuf<EncTarget> tgt;
    DevBuf<EncResult> res;
    DevBuf<uint64_t> sizes;
    DevBuf<uint64_t> lb_state;
    DevBuf<uint32_t> lb_ctr;
    DevBuf<float2> part;
    DevBuf<uint32_t> hist;   // per block: 32-bin histogram of code bit lengths (decoder)
    DevBuf<float> pred;      // per block: predicted log2 stream bytes
    DevBuf<uint8_t> wrec;    // per frame: chunk widths recorded by the sizing pass
    DevBuf<uint32_t> flen, foff;  // per frame: stream bytes and offset
    DevBuf<uint32_t> fwords;      // per frame: Re words | Im words << 16 (in-place encoder)
    DevBuf<uint32_t> fmixed;      // per frame: Re | Im mixed sign chunks << 16 (relative-bound codec)
    DevBuf<uint32_t> imsc;        // Im-plane words of the in-place encoder, one word per amplitude
};

static StageFeatures stage_features(const qsim_plan *p, size_t si, int e) {
    const Stage &st = p->stages[si];
    uint32_t dense = 0, diag = 0, kmax = 0, nondiag = 0;
    for (const Op &op : st.ops) {
        if (op.type == OP_DENSE) {
            ++dense;
            kmax = std::max(kmax, op.k);
        } else {
            ++diag;
        }
    }
    for (size_t gi = st.first_gate; gi < st.first_gate + st.ngates; ++gi) nondiag += p->gates[gi].diag ? 0 : 1;
    StageFeatures sf{};
    sf.v[0] = float(p->cfg.m) / 32.f;
    sf.v[1] = float(st.inner.size()) / 8.f;
    sf.v[2] = float(dense) / 16.f;
    sf.v[3] = float(diag) / 16.f;
    sf.v[4] = float(kmax) / 6.f;
    sf.v[5] = float(-e) / 64.f;
    sf.v[6] = float(st.ngates) / 64.f;
    sf.v[7] = st.ngates ? float(nondiag) / float(st.ngates) : 0.f;
    return sf;
}

// ---------------------------------------------------------------------------
// one circuit's run: validation, compressed store, tables and statistics
// ---------------------------------------------------------------------------
struct RunCtx {
    const qsim_plan *p = nullptr;
    PlanDev *pd = nullptr;
    uint32_t n = 0, m = 0;
    uint64_t nblocks = 0, nframes = 1;
    size_t nst = 0;
    bool raw = false, predict = false, collect = false, persistent = false;
    bool rel = false;  // QSZR: point-wise relative bound; e is then the code shift k
    int e = 0;
    uint64_t worst = 0, slot_worst = 0;
    uint64_t need_per_parity = 0;  // every block at its worst-case size, plus the zero template
    uint64_t raw_need = 0;         // the same for uncompressed blocks
    uint64_t dev_cap = 0, host_cap = 0;
    uint8_t *dev_arena[2] = {nullptr, nullptr}, *host_arena[2] = {nullptr, nullptr};
    uint8_t *host_arena_dev[2] = {nullptr, nullptr};
    DevBuf<uint64_t> bumps;      // per parity: device and host bump offsets
    DevBuf<BlockSlot> tables;    // per parity: block table
    DevBuf<StageAccum> accs;     // per stage, then the initial store
    DevBuf<float> log_rows;      // collect mode: predictor training rows
    DevBuf<uint32_t> init_ids;   // initial store: the two encoded blocks
    DevBuf<BlockSlot> tmpl;
    uint64_t log_next = 0;
    ArenaDev arena_dev(int parity) const {
        ArenaDev a;
        a.base = dev_arena[parity];
        a.cap = dev_arena[parity] ? dev_cap : 0;
        a.bump = bumps.p + 2 * parity;
        return a;
    }
    ArenaDev arena_host(int parity) const {
        ArenaDev a;
        a.base = host_arena_dev[parity];
        a.cap = host_arena[parity] ? host_cap : 0;
        a.bump = bumps.p + 2 * parity + 1;
        return a;
    }
    void free_arenas() {
        for (int i = 0; i < 2; ++i) {
            dev_free(dev_arena[i]);
            host_free(host_arena[i]);
            dev_arena[i] = host_arena[i] = host_arena_dev[i] = nullptr;
        }
    }
    ~RunCtx() { free_arenas(); }
};

static uint64_t host_phys_bytes() {
    const long pages = sysconf(_SC_PHYS_PAGES), page = sysconf(_SC_PAGE_SIZE);
    return (pages > 0 && page > 0) ? uint64_t(pages) * uint64_t(page) : (64ull << 30);
}

static int prepare_run(RunCtx &R, const qsim_plan *p, const DeviceCtx &dctx) {
    const qsim_config &cfg = p->cfg;
    R.p = p;
    R.persistent = cfg.mode == QSIM_MODE_PERSISTENT;
    if (R.persistent && cfg.codec == QSIM_CODEC_NONE)
        return set_error(QSIM_E_INVALID, "persistent mode runs the compressed store (codec QSZ1 or QSZR)");
    if (R.persistent && cfg.collect)
        return set_error(QSIM_E_INVALID, "training-row collection runs in streams mode");
    int rc = upload_plan(p, &R.pd);
    if (rc) return rc;
    R.n = p->n;
    R.m = cfg.m;
    R.nblocks = 1ull << (R.n - R.m);
    R.nst = p->stages.size();
    R.raw = cfg.codec == QSIM_CODEC_NONE;
    R.rel = cfg.codec == QSIM_CODEC_QSZR;
    if (R.rel ? !qszr_shift(cfg.eps, &R.e)
              : (!R.raw && !qsz_step_exponent(cfg.eps * std::pow(2.0, -double(R.n) / 2.0), &R.e)))
        return set_error(QSIM_E_INVALID, "error bound out of range");
    R.predict = cfg.sizing == QSIM_SIZING_PREDICT && !R.raw;
    R.collect = cfg.collect != 0 && !R.raw;
    if (R.predict && !dctx.pred_ready)
        return set_error(QSIM_E_INVALID, "predictor sizing needs trained weights (qsim_predictor_train/set)");
    R.worst = R.raw ? (8ull << R.m) : (R.rel ? qszr_worst_case(R.m) : qsz_worst_case(R.m));
    R.slot_worst = (R.worst + 255) & ~255ull;
    R.nframes = R.raw ? 1 : qsz_nframes(R.m);
    R.need_per_parity = (R.nblocks + 1) * R.slot_worst;
    R.raw_need = (R.nblocks + 1) * (((8ull << R.m) + qsz_data_start(int(R.m)) + 255) & ~255ull);
    return QSIM_OK;
}

// Pool sizing: device arenas first (both parities within dev_budget), pinned
// host for the rest (at most host_limit per parity). The host level is only set
// up when the device level is capped or cannot hold a raw-sized store.
static int alloc_run(RunCtx &R, uint64_t dev_budget, uint64_t host_limit, cudaStream_t main) {
    const qsim_config &cfg = R.p->cfg;
    if (cfg.device_tier_cap_bytes) dev_budget = std::min<uint64_t>(dev_budget, cfg.device_tier_cap_bytes);
    R.dev_cap = std::min<uint64_t>(R.need_per_parity, dev_budget / 2) & ~uint64_t(255);
    R.host_cap = 0;
    if (R.need_per_parity > R.dev_cap && (cfg.device_tier_cap_bytes || R.raw_need > R.dev_cap)) {
        R.host_cap = std::min<uint64_t>(R.need_per_parity - R.dev_cap, host_limit);
        R.host_cap = (R.host_cap + 4095) & ~uint64_t(4095);
    }
    int rc;
    for (int i = 0; i < 2; ++i) {
        if (R.dev_cap && (rc = dev_alloc(reinterpret_cast<void **>(&R.dev_arena[i]), R.dev_cap))) return rc;
        if (R.host_cap) {
            if ((rc = host_alloc(reinterpret_cast<void **>(&R.host_arena[i]), R.host_cap))) return rc;
            cudaError_t ce = cudaHostGetDevicePointer(reinterpret_cast<void **>(&R.host_arena_dev[i]), R.host_arena[i], 0);
            if (ce != cudaSuccess) return set_error(QSIM_E_CUDA, "cudaHostGetDevicePointer failed");
        }
    }
    if ((rc = R.bumps.alloc(4)) || (rc = R.tables.alloc(2 * R.nblocks)) || (rc = R.accs.alloc(R.nst + 1)) ||
        (rc = R.init_ids.alloc(2)) || (rc = R.tmpl.alloc(2)) ||
        (R.collect && (rc = R.log_rows.alloc(R.nst * R.nblocks * (kMlpIn + 1)))))
        return rc;
    CUDA_TRY(cudaMemsetAsync(R.bumps.p, 0, 4 * sizeof(uint64_t), main));
    CUDA_TRY(cudaMemsetAsync(R.accs.p, 0, (R.nst + 1) * sizeof(StageAccum), main));
    CUDA_TRY(cudaMemsetAsync(R.tables.p, 0, 2 * R.nblocks * sizeof(BlockSlot), main));
    return QSIM_OK;
}

// Initial store (Sec. 4.2): encode the basis block and one zero block once, every
// other block gets a copy of the zero stream. Runs on w.s; w.wv holds two blocks.
static int init_store(RunCtx &R, StreamWork &w, int *status) {
    const qsim_config &cfg = R.p->cfg;
    const uint32_t m = R.m;
    const uint32_t b0 = uint32_t(cfg.init_basis >> m);
    const uint64_t loc = cfg.init_basis & ((1ull << m) - 1);
    k_init_blocks<<<256, 256, 0, w.s>>>(w.wv.p, m, loc);
    count_launch();
    static const uint32_t h_ids[2] = {0, 1};
    CUDA_TRY(cudaMemcpyAsync(R.init_ids.p, h_ids, sizeof(h_ids), cudaMemcpyHostToDevice, w.s));
    // encode both blocks into slots of arena 0; tmpl[0] is the basis block, tmpl[1] the zero template
    if (R.raw) {
        launch_reserve(2, nullptr, R.worst, nullptr, 0, R.worst, R.arena_dev(0), R.arena_host(0), w.tgt.p, w.res.p, 0,
                       status, w.s);
        launch_copy_out(w.wv.p, 2, m, w.tgt.p, R.init_ids.p, R.tmpl.p, nullptr, status, w.s);
    } else if (R.rel) {
        // the in-place encoder and its frame copy (relative-bound streams)
        launch_encode_ip(w.wv.p, w.imsc.p, 2, int(m), R.e, w.lb_ctr.p + 3, R.arena_dev(0), R.arena_host(0), w.tgt.p,
                         w.res.p, nullptr, w.wrec.p, w.flen.p, w.fwords.p, w.foff.p, w.part.p, status, w.s, true,
                         w.fmixed.p);
        launch_frame_copy(w.wv.p, w.imsc.p, 2, int(m), R.e, w.tgt.p, w.res.p, R.init_ids.p, R.tmpl.p, nullptr, w.wrec.p,
                          w.flen.p, w.fwords.p, w.foff.p, w.s, true, w.fmixed.p);
    } else {
        launch_size_reserve(w.wv.p, 2, m, R.e, w.sizes.p, w.lb_ctr.p + 3, R.arena_dev(0), R.arena_host(0), w.tgt.p,
                            w.res.p, status, w.s);
        LookbackScratch scr = make_scratch(w.lb_state.p, w.lb_ctr.p);
        launch_encode(w.wv.p, 2, m, R.e, w.tgt.p, w.res.p, 0, R.init_ids.p, R.tmpl.p, nullptr, scr, status, w.s);
    }
    BlockSlot *tab0 = R.tables.p;
    k_copy_slot<<<1, 1, 0, w.s>>>(tab0 + b0, R.tmpl.p + 0);
    count_launch();
    // the zero template slot stays allocated in arena 0 until stage 0 has read its copies
    k_replicate_zero<<<unsigned(std::min<uint64_t>(R.nblocks, 152 * 8)), 128, 0, w.s>>>(
        tab0, uint32_t(R.nblocks), b0, R.tmpl.p + 1, R.arena_dev(0), R.arena_host(0), status);
    count_launch();
    k_sum_table<<<64, 256, 0, w.s>>>(tab0, R.nblocks, R.accs.p + R.nst);
    count_launch();
    return QSIM_OK;
}

// Mode B: the persistent stage kernel over a queue of segments (one stage of
// one circuit each). One circuit: one launch per stage (optionally the stage
// loop captured in one CUDA graph). Several circuits: one launch for all of
// them, stages dealt round-robin over the circuits so that one circuit's stage
// boundary overlaps the other circuits' work.
struct PBlockBufs {
    DevBuf<EncTarget> tgt;
    DevBuf<EncResult> res;
    DevBuf<uint64_t> sizes;
    DevBuf<uint32_t> hist;
};

static int run_persistent(const std::vector<RunCtx *> &rs, bool one_launch, cudaStream_t main, int *status,
                          Profiler &prof, const DeviceCtx &dctx, uint64_t slot_budget_amps) {
    const qsim_config &cfg0 = rs[0]->p->cfg;
    const int prec = int(cfg0.prec);
    // ---- segments in queue order ----
    struct SegRef {
        uint32_t c, si;
    };
    std::vector<SegRef> order;
    size_t max_nst = 0;
    for (const RunCtx *R : rs) max_nst = std::max(max_nst, R->nst);
    for (size_t r = 0; r < max_nst; ++r)
        for (uint32_t c = 0; c < rs.size(); ++c)
            if (r < rs[c]->nst) order.push_back({c, uint32_t(r)});
    const size_t nseg = order.size();
    if (!nseg) return QSIM_OK;
    std::vector<std::vector<uint32_t>> seg_of(rs.size());
    for (uint32_t c = 0; c < rs.size(); ++c) seg_of[c].assign(rs[c]->nst, 0);
    for (size_t k = 0; k < nseg; ++k) seg_of[order[k].c][order[k].si] = uint32_t(k);

    uint64_t total_groups = 0;
    size_t max_pass_bytes = 0;
    bool um_any = false;  // tcgen05 passes in the launch: the kernel holds TMEM and an MMA mbarrier
    for (const SegRef &sr : order) {
        const RunCtx &R = *rs[sr.c];
        const StageDev &sd = R.pd->stages[sr.si];
        total_groups += sd.ngroups;
        for (const PassDev &ps : sd.passes_host) {
            max_pass_bytes = std::max(max_pass_bytes, (size_t(1) << ps.T) * sizeof(float2) + size_t(ps.blob_words) * 16 +
                                                          size_t(ps.mat_elems) * sizeof(float2) +
                                                          umma_pass_smem(ps.umma));
            um_any |= (ps.umma & 1u) != 0;
            if (ps.kmax > 5 && !(ps.umma & 8u))
                return set_error(QSIM_E_INVALID, "persistent mode fuses k = 6 only as TF32 on tcgen05");
        }
    }
    if (um_any && prec == QSIM_PREC_FP32)
        return set_error(QSIM_E_INVALID, "internal: tcgen05 passes in an FP32 plan");
    std::vector<std::unique_ptr<PBlockBufs>> bb(rs.size());
    int rc;
    for (size_t c = 0; c < rs.size(); ++c) {
        const RunCtx &R = *rs[c];
        bb[c].reset(new PBlockBufs());
        PBlockBufs &b = *bb[c];
        if ((rc = b.tgt.alloc(R.nblocks)) || (rc = b.res.alloc(R.nblocks)) || (rc = b.sizes.alloc(R.nblocks)) ||
            (R.predict && (rc = b.hist.alloc(R.nblocks * 32))))
            return rc;
        CUDA_TRY(cudaMemsetAsync(b.sizes.p, 0, R.nblocks * sizeof(uint64_t), main));
        if (R.predict) CUDA_TRY(cudaMemsetAsync(b.hist.p, 0, R.nblocks * 32 * sizeof(uint32_t), main));
    }
    // Working-vector slots, planned per launch: one ring of slots per working-vector size (2^W amplitudes),
    // each ring about slot_budget_amps large (at least 2 slots, at most the launch's groups of that size);
    // a group takes the next slot of its ring and waits for the slot's previous group.
    std::vector<uint64_t> g_wv(total_groups);
    std::vector<uint32_t> g_frame(total_groups), g_prev(total_groups, kNoGroup);
    uint64_t wv_total = 0, frames_total = 0;
    {
        const size_t nlaunch_plan = one_launch ? 1 : nseg;
        uint64_t q_global = 0;
        for (size_t l = 0; l < nlaunch_plan; ++l) {
            const size_t k0 = one_launch ? 0 : l, k1 = one_launch ? nseg : l + 1;
            struct Ring {
                uint64_t amps = 0, frames = 0, groups = 0, slots = 0, used = 0, wv_base = 0, fr_base = 0;
                std::vector<uint32_t> last;  // per slot: launch group that used it last
            };
            std::map<uint32_t, Ring> rings;  // by W
            for (size_t k = k0; k < k1; ++k) {
                const RunCtx &R = *rs[order[k].c];
                const StageDev &sd = R.pd->stages[order[k].si];
                Ring &rg = rings[sd.W];
                rg.amps = 1ull << sd.W;
                rg.frames = std::max<uint64_t>(rg.frames, uint64_t(sd.G) * R.nframes);
                rg.groups += sd.ngroups;
            }
            uint64_t wv_l = 0, fr_l = 0;
            for (auto &kv : rings) {
                Ring &rg = kv.second;
                rg.slots = std::max<uint64_t>(2, std::min<uint64_t>(rg.groups, slot_budget_amps / rg.amps));
                rg.slots = std::min<uint64_t>(rg.slots, rg.groups);
                rg.last.assign(rg.slots, kNoGroup);
                rg.wv_base = wv_l;
                rg.fr_base = fr_l;
                wv_l += rg.slots * rg.amps;
                fr_l += rg.slots * rg.frames;
            }
            wv_total = std::max(wv_total, wv_l);
            frames_total = std::max(frames_total, fr_l);
            uint32_t q_local = 0;
            for (size_t k = k0; k < k1; ++k) {
                const StageDev &sd = rs[order[k].c]->pd->stages[order[k].si];
                Ring &rg = rings[sd.W];
                for (uint32_t gi = 0; gi < sd.ngroups; ++gi, ++q_local, ++q_global) {
                    const uint64_t slot = rg.used++ % rg.slots;
                    g_wv[q_global] = rg.wv_base + slot * rg.amps;
                    g_frame[q_global] = uint32_t(rg.fr_base + slot * rg.frames);
                    g_prev[q_global] = rg.last[slot];
                    rg.last[slot] = q_local;
                }
            }
        }
        if (frames_total >= (1ull << 32)) return set_error(QSIM_E_UNSUPPORTED, "working-vector slot plan too large");
    }
    const bool rel = rs[0]->rel;  // one codec per launch (the batch entry points check it)
    DevBuf<float2> wv, part;
    DevBuf<uint8_t> wrec;
    DevBuf<uint32_t> flen, foff, fwords, fmixed, im;
    DevBuf<uint64_t> lb, dg_wv;
    DevBuf<uint32_t> sync, fin, ctr, dg_frame, dg_prev;
    DevBuf<PSeg> dsegs;
    if ((rc = wv.alloc(wv_total)) || (rc = lb.alloc(frames_total)) || (rc = part.alloc(frames_total)) ||
        (rc = sync.alloc(2 * total_groups * kMaxPhases)) || (rc = fin.alloc(2 * nseg)) || (rc = ctr.alloc(4)) ||
        (rc = dsegs.alloc(nseg)) || (rc = dg_wv.alloc(total_groups)) || (rc = dg_frame.alloc(total_groups)) ||
        (rc = dg_prev.alloc(total_groups)) || (rc = wrec.alloc(frames_total * (rel ? kQszrSideBytes : 256))) ||
        (rc = flen.alloc(frames_total)) || (rc = foff.alloc(frames_total)) ||
        (rel && ((rc = fwords.alloc(frames_total)) || (rc = fmixed.alloc(frames_total)) || (rc = im.alloc(wv_total)))))
        return rc;
    CUDA_TRY(cudaMemcpyAsync(dg_wv.p, g_wv.data(), total_groups * sizeof(uint64_t), cudaMemcpyHostToDevice, main));
    CUDA_TRY(cudaMemcpyAsync(dg_frame.p, g_frame.data(), total_groups * sizeof(uint32_t), cudaMemcpyHostToDevice,
                             main));
    CUDA_TRY(cudaMemcpyAsync(dg_prev.p, g_prev.data(), total_groups * sizeof(uint32_t), cudaMemcpyHostToDevice, main));
    CUDA_TRY(cudaMemsetAsync(lb.p, 0, lb.n * sizeof(uint64_t), main));
    CUDA_TRY(cudaMemsetAsync(sync.p, 0, sync.n * sizeof(uint32_t), main));
    CUDA_TRY(cudaMemsetAsync(fin.p, 0, fin.n * sizeof(uint32_t), main));
    CUDA_TRY(cudaMemsetAsync(ctr.p, 0, 4 * sizeof(uint32_t), main));

    // ---- segment descriptors ----
    std::vector<PSeg> segs(nseg);
    std::vector<uint64_t> seg_items(nseg), seg_group_off(nseg);  // group offset into the done/arrive arrays
    uint64_t group_off = 0;
    bool stall = false;
    for (size_t k = 0; k < nseg; ++k) {
        const RunCtx &R = *rs[order[k].c];
        const size_t si = order[k].si;
        const qsim_config &cfg = R.p->cfg;
        const StageDev &sd = R.pd->stages[si];
        const int in_par = si & 1, out_par = (si + 1) & 1;
        PSeg &a = segs[k];
        memset(&a, 0, sizeof(a));
        a.W = sd.W;
        a.G = sd.G;
        a.ngroups = sd.ngroups;
        a.m = R.m;
        a.e = R.e;
        a.npre = sd.npre;
        a.pre_begin = sd.pre_begin;
        a.pbf16 = uint32_t(dctx.pred_bf16);
        uint32_t nph = 0;
        const uint32_t gframes = sd.G * uint32_t(R.nframes);
        const uint32_t fpi = persistent_frames_per_item(um_any);
        auto add = [&](uint32_t type, uint32_t count, uint32_t arg) {
            if (nph < uint32_t(kMaxPhases)) {
                a.ph[nph].type = type;
                a.ph[nph].count = count;
                a.ph[nph].arg = arg;
            }
            ++nph;
        };
        add(PH_DECODE, (gframes + fpi - 1) / fpi, 0);
        if (R.predict) add(PH_PREDICT, 1, 0);
        for (uint32_t pi = 0; pi < sd.npasses; ++pi) add(PH_PASS, 1u << sd.passes_host[pi].nout, pi);
        if (R.rel) {
            // relative-bound codec: in-place encoder (exact slots, or predicted slots kept when they fit), copy
            add(PH_ENCODE_IP, (gframes + fpi - 1) / fpi, 0);
            add(PH_COPY, (gframes + fpi - 1) / fpi, 0);
        } else if (R.predict) {
            add(PH_ENCODE, (gframes + fpi - 1) / fpi, 0);
            add(PH_FIX, 1, 0);
            add(PH_REENCODE, (gframes + fpi - 1) / fpi, 0);
        } else {
            add(PH_SIZE_W, (gframes + fpi - 1) / fpi, 0);
            add(PH_ENCODE_W, (gframes + fpi - 1) / fpi, 0);
        }
        // the last phase index is the group's finished flag
        if (nph > uint32_t(kMaxPhases) - 1)
            return set_error(QSIM_E_UNSUPPORTED, "stage has too many passes for the persistent kernel");
        a.nphases = nph;
        uint32_t acc_items = 0;
        for (uint32_t t = 0; t < nph; ++t) {
            a.ph_start[t] = acc_items;
            acc_items += a.ph[t].count;
        }
        a.per_group = acc_items;
        seg_items[k] = uint64_t(sd.ngroups) * acc_items;
        a.passes = R.pd->passes.p + sd.pass_begin;
        a.ops = R.pd->ops.p;
        a.mats = R.pd->mats.p;
        a.blob = R.pd->blob.p;
        a.bfr = R.pd->bfr.p;
        a.ids = R.pd->ids.p + R.pd->ids_off[si];
        a.gbase = R.pd->gbase.p + R.pd->gbase_off[si];
        a.tab_in = R.tables.p + in_par * R.nblocks;
        a.tab_out = R.tables.p + out_par * R.nblocks;
        a.acc = R.accs.p + si;
        a.dev = R.arena_dev(out_par);
        a.host = R.arena_host(out_par);
        a.data_start = qsz_data_start(int(R.m));
        a.worst = R.worst;
        PBlockBufs &b = *bb[order[k].c];
        a.tgt = b.tgt.p;
        a.res = b.res.p;
        a.sizes = b.sizes.p;
        a.hist = R.predict ? b.hist.p : nullptr;
        a.pparams = R.predict ? dctx.pred_params : nullptr;
        a.sf = stage_features(R.p, si, R.e);
        a.margin = cfg.predictor_margin;
        a.stall_test = (si == 0 && (cfg.reserved[0] & 1)) ? 1u : 0u;
        stall = stall || a.stall_test;
        a.prev_flag = (one_launch && si > 0) ? fin.p + 2 * seg_of[order[k].c][si - 1] + 1 : nullptr;
        a.fin_count = fin.p + 2 * k;
        a.fin_flag = fin.p + 2 * k + 1;
        a.reset_bumps = R.bumps.p + 2 * in_par;  // the next stage writes where this one read
        seg_group_off[k] = group_off;
        group_off += sd.ngroups;
    }
    // queue positions: one launch for everything, or one launch per segment
    {
        uint64_t item = 0;
        uint32_t group = 0;
        for (size_t k = 0; k < nseg; ++k) {
            if (!one_launch) item = 0, group = 0;
            segs[k].item_begin = item;
            segs[k].group_begin = group;
            item += seg_items[k];
            group += segs[k].ngroups;
            if (item >= (1ull << 32)) return set_error(QSIM_E_UNSUPPORTED, "work queue longer than 2^32 items");
        }
    }
    CUDA_TRY(cudaMemcpyAsync(dsegs.p, segs.data(), nseg * sizeof(PSeg), cudaMemcpyHostToDevice, main));
    const size_t smem = persistent_smem_bytes(max_pass_bytes);
    if ((rc = prepare_stage_persistent(prec, smem, rel, um_any))) return set_error(rc, "persistent kernel set-up failed");

    PLaunch L{};
    L.wv = wv.p;
    L.wrec = wrec.p;
    L.flen = flen.p;
    L.foff = foff.p;
    L.im = im.p;
    L.fwords = fwords.p;
    L.fmixed = fmixed.p;
    L.lb = lb.p;
    L.part = part.p;
    L.ctr = ctr.p;
    L.status = status;
    L.wait_ns = stall ? 200000000ull : 2000000000ull;  // 0.2 s in the bounded-wait test, else 2 s

    const bool graph = cfg0.graph != 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the caller's stream may be the legacy default stream, which cannot be captured: capture on our own
    cudaStream_t cs = main;
    cudaEvent_t ev_join = nullptr;
    if (graph) {
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(ev_join, main));
        CUDA_TRY(cudaStreamWaitEvent(cs, ev_join, 0));
        CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    }
    auto end_capture_on_error = [&]() {
        if (graph) {
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaEventDestroy(ev_join);
            cudaStreamDestroy(cs);
        }
    };
    const size_t nlaunch = one_launch ? 1 : nseg;
    for (size_t l = 0; l < nlaunch; ++l) {
        NvtxRange launch_range(one_launch ? "persistent launch: %zu segments" : "persistent stage %zu",
                               one_launch ? nseg : l);
        const size_t k0 = one_launch ? 0 : l, k1 = one_launch ? nseg : l + 1;
        L.segs = dsegs.p + k0;
        L.nseg = uint32_t(k1 - k0);
        L.total_items = segs[k1 - 1].item_begin + seg_items[k1 - 1];
        L.total_groups = segs[k1 - 1].group_begin + segs[k1 - 1].ngroups;
        L.g_wv = dg_wv.p + seg_group_off[k0];
        L.g_frame = dg_frame.p + seg_group_off[k0];
        L.g_prev = dg_prev.p + seg_group_off[k0];
        L.done = sync.p + seg_group_off[k0] * kMaxPhases;
        L.arrive = sync.p + (total_groups + seg_group_off[k0]) * kMaxPhases;
        prof.begin(P_STAGE, cs);
        rc = launch_stage_persistent(L, prec, smem, cs, nullptr, rel, um_any);
        prof.end(cs);
        if (rc) {
            end_capture_on_error();
            return set_error(rc, "persistent stage launch failed");
        }
    }
    if (graph) {
        cudaError_t ge = cudaStreamEndCapture(cs, &g);
        if (ge == cudaSuccess) ge = cudaGraphInstantiate(&exec, g, 0);
        if (ge == cudaSuccess) ge = cudaGraphLaunch(exec, cs);
        if (ge == cudaSuccess) ge = cudaEventRecord(ev_join, cs);
        if (ge == cudaSuccess) ge = cudaStreamWaitEvent(main, ev_join, 0);
        if (ge == cudaSuccess) ge = cudaStreamSynchronize(cs);
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        cudaEventDestroy(ev_join);
        cudaStreamDestroy(cs);
        if (ge != cudaSuccess) return set_error(QSIM_E_CUDA, "graph: %s", cudaGetErrorString(ge));
    } else {
        CUDA_TRY(cudaStreamSynchronize(main));  // the local buffers are released on return
    }
    return QSIM_OK;
}

// The run's state handle and statistics (after the stream has been synchronised).
static int finish_run(RunCtx &R, int dev, double ms, Profiler *prof, qsim_stats *stats, qsim_state **out) {
    const qsim_plan *p = R.p;
    PlanDev *pd = R.pd;
    const size_t nst = R.nst;
    const bool raw = R.raw, predict = R.predict;
    const uint64_t nblocks = R.nblocks;
    int rc;
    qsim_state *S = new qsim_state();
    S->device = dev;
    S->n = R.n;
    S->m = R.m;
    S->codec = p->cfg.codec;
    S->e = R.e;
    S->stage_acc.resize(nst + 1);
    CUDA_TRY(cudaMemcpy(S->stage_acc.data(), R.accs.p, (nst + 1) * sizeof(StageAccum), cudaMemcpyDeviceToHost));
    if (R.collect && R.log_next) {
        S->train_rows.resize(R.log_next * (kMlpIn + 1));
        CUDA_TRY(cudaMemcpy(S->train_rows.data(), R.log_rows.p, S->train_rows.size() * sizeof(float),
                            cudaMemcpyDeviceToHost));
    }
    const int fin = nst & 1;
    S->dev_arena = R.dev_arena[fin];
    S->host_arena = R.host_arena[fin];
    R.dev_arena[fin] = nullptr;
    R.host_arena[fin] = nullptr;
    R.free_arenas();
    if ((rc = dev_alloc(reinterpret_cast<void **>(&S->table), nblocks * sizeof(BlockSlot)))) {
        qsim_state_free(S);
        return rc;
    }
    CUDA_TRY(cudaMemcpy(S->table, R.tables.p + fin * nblocks, nblocks * sizeof(BlockSlot), cudaMemcpyDeviceToDevice));

    if (prof && prof->on) {
        double secs[P_NCAT];
        uint64_t launches[P_NCAT];
        prof->collect(secs, launches);
        double bytes[P_NCAT] = {0}, flops[P_NCAT] = {0};
        const double amps = std::ldexp(1.0, int(R.n));
        for (size_t i = 0; i < nst; ++i) {
            const double in_store = double(i == 0 ? S->stage_acc[nst].store_bytes : S->stage_acc[i - 1].store_bytes);
            const double out_store = double(S->stage_acc[i].store_bytes);
            const StageDev &sd = pd->stages[i];
            bytes[raw ? P_COPY_IN : P_DECODE] += in_store + 8 * amps;
            bytes[P_PASS] += 16 * amps * sd.npasses;
            bytes[P_STAGE] += in_store + out_store + 8 * amps * (2 + (predict ? 0 : 1)) + 16 * amps * sd.npasses;
            for (const Op &op : p->stages[i].ops) {
                const double fl = (op.type == OP_DENSE ? 8.0 * double(1u << op.k)
                                   : op.type == OP_DIAG ? 6.0 : op.type == OP_CSEP ? 12.0 : 0.0) * amps;
                flops[P_PASS] += fl;
                flops[P_STAGE] += fl;
            }
            if (raw) {
                bytes[P_COPY_OUT] += 8 * amps + out_store;
            } else {
                bytes[P_ENCODE] += 8 * amps + out_store;  // frames written in place
                bytes[P_FRAME_COPY] += 2 * out_store;
            }
        }
        for (int c = 0; c < P_NCAT; ++c) {
            if (!launches[c]) continue;
            qsim_kernel_stat ks;
            memset(&ks, 0, sizeof(ks));
            snprintf(ks.name, sizeof(ks.name), "%s", kProfNames[c]);
            ks.launches = launches[c];
            ks.seconds = secs[c];
            ks.alg_bytes = bytes[c];
            ks.alg_flops = flops[c];
            S->kstats.push_back(ks);
        }
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->seconds = ms * 1e-3;
        stats->nstages = nst;
        double E = 0, E2 = 0;
        for (size_t i = 0; i < nst; ++i) {
            const StageAccum &a = S->stage_acc[i];
            E += std::sqrt(a.err_sq);
            E2 += a.err_sq;
            stats->peak_store_bytes = std::max<uint64_t>(stats->peak_store_bytes, a.store_bytes);
            stats->peak_reserved_bytes = std::max<uint64_t>(stats->peak_reserved_bytes, a.reserved_bytes);
            stats->host_tier_peak_bytes = std::max<uint64_t>(stats->host_tier_peak_bytes, a.host_bytes);
            stats->overflow_blocks += a.overflow_blocks;
            stats->blocks_encoded += a.blocks;
            stats->groups += pd->stages[i].ngroups;
        }
        stats->err_norm_sum = E;
        stats->err_sq_total = E2;
        if (nst) {
            stats->final_store_bytes = S->stage_acc[nst - 1].store_bytes;
            stats->norm_sq = raw ? 0.0 : S->stage_acc[nst - 1].norm_sq;
        }
        if (raw) {
            double ns = 0;
            qsim_state_norm(S, &ns);
            stats->norm_sq = ns;
        }
        const double b = std::sqrt(stats->norm_sq);
        stats->fidelity_lower_bound = b > 0 ? std::min(1.0, (1.0 + stats->norm_sq - E * E) / (2.0 * b)) : 0.0;
        stats->kernel_launches = g_launches.load();
        stats->h2d_bytes = pd->counted ? 0 : pd->upload_bytes;
        stats->d2h_bytes = (nst + 1) * sizeof(StageAccum) + sizeof(int);
    }
    pd->counted = true;
    *out = S;
    return QSIM_OK;
}

// A streams-mode run between its stages: the compressed store (RunCtx), the per-stream work buffers and the
// run's events. run_plan drives one through every stage; a sharded run (qsim_shard_*) drives one stage at a
// time over the SV groups its rank holds and moves blocks between the stages.
struct StreamsRun {
    RunCtx RC;
    DeviceCtx *dctx = nullptr;
    int dev = 0;
    cudaStream_t main = nullptr;
    std::vector<StreamWork> sw;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr, ev_fork = nullptr;
    Profiler prof;
    int *status = nullptr;
    uint64_t batch_amps = 0;
    uint64_t groups_run = 0;  // SV groups processed (all stages)
    ~StreamsRun() {
        for (auto &x : sw) {
            if (x.s) cudaStreamDestroy(x.s);
            if (x.done) cudaEventDestroy(x.done);
        }
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_stop) cudaEventDestroy(ev_stop);
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
};

// Validation, the compressed store's tiers, the per-stream buffers and the initial store (Sec. 4.2); the start
// event is recorded on `main` before the initial store.
static int streams_begin(StreamsRun &S, const qsim_plan *p, cudaStream_t main) {
    const qsim_config &cfg = p->cfg;
    CUDA_TRY(cudaGetDevice(&S.dev));
    S.dctx = &device_ctx(S.dev);
    DeviceCtx &dctx = *S.dctx;
    {
        std::lock_guard<std::mutex> lk(dctx.mu);
        int rc = ensure_device_ctx(dctx);
        if (rc) return rc;
    }
    S.main = main;
    RunCtx &RC = S.RC;
    int rc = prepare_run(RC, p, dctx);
    if (rc) return rc;
    PlanDev *pd = RC.pd;
    const bool persistent = RC.persistent, raw = RC.raw;
    const uint32_t m = RC.m;
    const uint64_t nframes = RC.nframes;

    // ---- pool sizing: device arenas first, pinned host for the rest ----
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    free_b += cached_dev_bytes();  // an earlier run's cached arenas are reused or released
    uint32_t maxW = m;
    for (const StageDev &sd : pd->stages) maxW = std::max(maxW, sd.W);
    const uint32_t nstreams = persistent ? 1 : cfg.streams;
    const uint64_t batch_amps = std::max<uint64_t>(1ull << maxW, 1ull << 22);
    S.batch_amps = batch_amps;
    const uint64_t work_bytes = nstreams * batch_amps * 8 * 2;
    const uint64_t dev_budget = free_b > work_bytes ? uint64_t(0.85 * double(free_b - work_bytes)) : 0;
    // the pinned-host level holds at most 30 % of the host's memory per stage parity
    if ((rc = alloc_run(RC, dev_budget, uint64_t(0.3 * double(host_phys_bytes())), main))) return rc;

    // ---- per-stream work buffers ----
    std::vector<StreamWork> &sw = S.sw;
    sw.resize(nstreams);
    uint64_t max_batch_blocks = 0;
    for (const StageDev &sd : pd->stages) {
        uint64_t gpb = std::min<uint64_t>(std::max<uint64_t>(1, batch_amps >> sd.W), 32768);
        gpb = std::min<uint64_t>(gpb, sd.ngroups);
        max_batch_blocks = std::max<uint64_t>(max_batch_blocks, gpb * sd.G);
    }
    max_batch_blocks = std::max<uint64_t>(max_batch_blocks, 2);
    if (persistent) max_batch_blocks = 2;  // the stream buffers only serve the initial store
    for (uint32_t i = 0; i < nstreams; ++i) {
        StreamWork &w = sw[i];
        CUDA_TRY(cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
        if ((rc = w.wv.alloc(max_batch_blocks << m)) || (rc = w.refs.alloc(max_batch_blocks)) ||
            (rc = w.tgt.alloc(max_batch_blocks)) || (rc = w.res.alloc(max_batch_blocks)) ||
            (rc = w.sizes.alloc(max_batch_blocks)) || (rc = w.lb_state.alloc(max_batch_blocks * nframes)) ||
            (rc = w.part.alloc(max_batch_blocks * nframes)) || (rc = w.hist.alloc(max_batch_blocks * 32)) ||
            (rc = w.pred.alloc(max_batch_blocks)) ||
            ((!persistent || RC.rel) && (rc = w.wrec.alloc(max_batch_blocks * nframes * (RC.rel ? kQszrSideBytes : 256)))) ||
            ((!persistent || RC.rel) && !raw && (rc = w.imsc.alloc(max_batch_blocks << m))) ||
            ((!persistent || RC.rel) && (rc = w.fwords.alloc(max_batch_blocks * nframes))) ||
            (RC.rel && (rc = w.fmixed.alloc(max_batch_blocks * nframes))) ||
            (rc = w.flen.alloc(max_batch_blocks * nframes)) || (rc = w.foff.alloc(max_batch_blocks * nframes)) ||
            (rc = w.lb_ctr.alloc(16)))
            return rc;
        CUDA_TRY(cudaMemsetAsync(w.lb_state.p, 0, max_batch_blocks * nframes * sizeof(uint64_t), main));
        CUDA_TRY(cudaMemsetAsync(w.lb_ctr.p, 0, 16 * sizeof(uint32_t), main));  // [8], [9]: gate-pass tile counter
        CUDA_TRY(cudaMemsetAsync(w.sizes.p, 0, max_batch_blocks * sizeof(uint64_t), main));
    }
    CUDA_TRY(cudaEventCreate(&S.ev_start));
    CUDA_TRY(cudaEventCreate(&S.ev_stop));
    CUDA_TRY(cudaEventCreateWithFlags(&S.ev_fork, cudaEventDisableTiming));
    S.status = dctx.status;
    S.prof.on = g_profile.load() != 0 && !(persistent && cfg.graph);
    CUDA_TRY(cudaEventRecord(S.ev_start, main));

    // ---- initial store ----
    {
        StreamWork &w = sw[0];
        CUDA_TRY(cudaEventRecord(S.ev_fork, main));
        CUDA_TRY(cudaStreamWaitEvent(w.s, S.ev_fork, 0));
        if ((rc = init_store(RC, w, S.status))) return rc;
        CUDA_TRY(cudaEventRecord(w.done, w.s));
        CUDA_TRY(cudaStreamWaitEvent(main, w.done, 0));
    }
    return QSIM_OK;
}

// Stage si over `ngroups` SV groups: ids_stage holds their block ids (group-major, G per group), gb_stage their
// outer bits (device arrays). Work runs on the run's streams, joined back to S.main.
static int streams_stage(StreamsRun &S, size_t si, const uint32_t *ids_stage, const uint64_t *gb_stage,
                         uint64_t ngroups) {
    RunCtx &RC = S.RC;
    const qsim_plan *p = RC.p;
    const qsim_config &cfg = p->cfg;
    PlanDev *pd = RC.pd;
    DeviceCtx &dctx = *S.dctx;
    const bool raw = RC.raw, predict = RC.predict, collect = RC.collect;
    const uint32_t m = RC.m;
    const uint64_t nblocks = RC.nblocks, worst = RC.worst;
    const int e = RC.e;
    const uint32_t nstreams = uint32_t(S.sw.size());
    std::vector<StreamWork> &sw = S.sw;
    const uint64_t batch_amps = S.batch_amps;
    cudaStream_t main = S.main;
    cudaEvent_t ev_fork = S.ev_fork;
    Profiler &prof = S.prof;
    int *status = S.status;
    auto arena_dev = [&](int parity) { return RC.arena_dev(parity); };
    auto arena_host = [&](int parity) { return RC.arena_host(parity); };
    BlockSlot *const tables_p = RC.tables.p;
    StageAccum *const accs_p = RC.accs.p;
    uint64_t *const bumps_p = RC.bumps.p;
    {
        NvtxRange stage_range("stage %zu", si);
        const StageDev &sd = pd->stages[si];
        const int in_par = si & 1, out_par = (si + 1) & 1;
        BlockSlot *tab_in = tables_p + in_par * nblocks;
        BlockSlot *tab_out = tables_p + out_par * nblocks;
        CUDA_TRY(cudaMemsetAsync(bumps_p + 2 * out_par, 0, 2 * sizeof(uint64_t), main));
        CUDA_TRY(cudaEventRecord(ev_fork, main));
        for (auto &w : sw) CUDA_TRY(cudaStreamWaitEvent(w.s, ev_fork, 0));
        const uint64_t gpb = std::min<uint64_t>(std::min<uint64_t>(std::max<uint64_t>(1, batch_amps >> sd.W), 32768),
                                                std::max<uint64_t>(1, ngroups));
        const uint64_t nbatches = (ngroups + gpb - 1) / gpb;
        S.groups_run += ngroups;
        StageAccum *acc = accs_p + si;
        StageFeatures sf{};
        {
            const Stage &st = p->stages[si];
            uint32_t dense = 0, diag = 0, kmax = 0, nondiag = 0;
            for (const Op &op : st.ops) {
                if (op.type == OP_DENSE) { ++dense; kmax = std::max(kmax, op.k); }
                else ++diag;
            }
            for (size_t gi = st.first_gate; gi < st.first_gate + st.ngates; ++gi) nondiag += p->gates[gi].diag ? 0 : 1;
            sf.v[0] = float(m) / 32.f;
            sf.v[1] = float(st.inner.size()) / 8.f;
            sf.v[2] = float(dense) / 16.f;
            sf.v[3] = float(diag) / 16.f;
            sf.v[4] = float(kmax) / 6.f;
            sf.v[5] = float(-e) / 64.f;
            sf.v[6] = float(st.ngates) / 64.f;
            sf.v[7] = st.ngates ? float(nondiag) / float(st.ngates) : 0.f;
        }
        for (uint64_t b = 0; b < nbatches; ++b) {
            NvtxRange group_range("groups %llu..", (unsigned long long)(b * gpb));
            StreamWork &w = sw[b % nstreams];
            const uint64_t g0 = b * gpb;
            const uint32_t ng = uint32_t(std::min<uint64_t>(gpb, ngroups - g0));
            const uint32_t nb = ng * sd.G;
            const uint32_t *ids = ids_stage + g0 * sd.G;
            if (raw) {
                prof.begin(P_GATHER, w.s);
                launch_gather_refs(tab_in, ids, nb, w.refs.p, w.s);
                prof.end(w.s);
                prof.begin(P_COPY_IN, w.s);
                launch_copy_in(w.refs.p, nb, m, w.wv.p, status, w.s);
            } else {
                prof.begin(P_DECODE, w.s);
                PreOps pre;
                pre.ops = pd->ops.p + sd.pre_begin;
                pre.count = sd.npre;
                pre.G = sd.G;
                pre.mats = pd->mats.p;
                pre.gbase = gb_stage + g0;
                uint32_t *hist = (predict || collect) ? w.hist.p : nullptr;
                if (hist) CUDA_TRY(cudaMemsetAsync(hist, 0, size_t(nb) * 32 * sizeof(uint32_t), w.s));
                launch_decode_table(tab_in, ids, nb, m, w.wv.p, hist, status, pre, w.s, RC.rel);
            }
            prof.end(w.s);
            float *log_ptr = collect ? RC.log_rows.p + RC.log_next * (kMlpIn + 1) : nullptr;
            if (predict || collect) {
                prof.begin(P_PREDICT, w.s);
                launch_predict_sizes(w.hist.p, nb, sd.G, m, sf, predict ? dctx.pred_params : nullptr,
                                     dctx.pred_bf16, w.pred.p, log_ptr, w.s);
                prof.end(w.s);
            }
            for (uint32_t pi = 0; pi < sd.npasses; ++pi) {
                prof.begin(P_PASS, w.s);
                launch_pass(w.wv.p, sd.W, ng, &sd.passes_host[pi], pd->blob.p, pd->mats.p, pd->bfr.p, gb_stage + g0,
                            cfg.prec, w.s, w.lb_ctr.p + 8, status);
                prof.end(w.s);
            }
            if (raw) {
                prof.begin(P_RESERVE, w.s);
                launch_reserve(nb, nullptr, worst, nullptr, 0, worst, arena_dev(out_par), arena_host(out_par),
                               w.tgt.p, w.res.p, 0, status, w.s);
                prof.end(w.s);
                prof.begin(P_COPY_OUT, w.s);
                launch_copy_out(w.wv.p, nb, m, w.tgt.p, ids, tab_out, acc, status, w.s);
                prof.end(w.s);
            } else {
                if (predict) {
                    // reserve 2^pred (1 + margin) bytes per block ahead of the encoder; the in-place encoder keeps
                    // every slot its block fits and reserves exact slots for under-estimated blocks; copy
                    prof.begin(P_RESERVE, w.s);
                    launch_reserve(nb, nullptr, 0, w.pred.p, cfg.predictor_margin, worst, arena_dev(out_par),
                                   arena_host(out_par), w.tgt.p, w.res.p, 0, status, w.s);
                    prof.end(w.s);
                    prof.begin(P_ENCODE, w.s);
                    launch_encode_ip(w.wv.p, w.imsc.p, nb, m, e, w.lb_ctr.p + 3, arena_dev(out_par),
                                     arena_host(out_par), w.tgt.p, w.res.p, acc, w.wrec.p, w.flen.p, w.fwords.p,
                                     w.foff.p, w.part.p, status, w.s, RC.rel, w.fmixed.p, true);
                    prof.end(w.s);
                    prof.begin(P_FRAME_COPY, w.s);
                    launch_frame_copy(w.wv.p, w.imsc.p, nb, m, e, w.tgt.p, w.res.p, ids, tab_out, acc, w.wrec.p,
                                      w.flen.p, w.fwords.p, w.foff.p, w.s, RC.rel, w.fmixed.p);
                    prof.end(w.s);
                } else {
                    // exact sizing: encode every frame in place, reserve exact slots, copy the frames over
                    prof.begin(P_ENCODE, w.s);
                    launch_encode_ip(w.wv.p, w.imsc.p, nb, m, e, w.lb_ctr.p + 3, arena_dev(out_par),
                                     arena_host(out_par), w.tgt.p, w.res.p, acc, w.wrec.p, w.flen.p, w.fwords.p,
                                     w.foff.p, w.part.p, status, w.s, RC.rel, w.fmixed.p);
                    prof.end(w.s);
                    prof.begin(P_FRAME_COPY, w.s);
                    launch_frame_copy(w.wv.p, w.imsc.p, nb, m, e, w.tgt.p, w.res.p, ids, tab_out, acc, w.wrec.p,
                                      w.flen.p, w.fwords.p, w.foff.p, w.s, RC.rel, w.fmixed.p);
                    prof.end(w.s);
                }
                if (collect) {
                    launch_log_targets(w.res.p, nb, m, log_ptr, w.s);
                    RC.log_next += nb;
                }
            }
        }
        for (auto &w : sw) {
            CUDA_TRY(cudaEventRecord(w.done, w.s));
            CUDA_TRY(cudaStreamWaitEvent(main, w.done, 0));
        }
        }
    return QSIM_OK;
}

// The run's end: stop event, status, and the state handle with the statistics.
static int streams_finish(StreamsRun &S, qsim_state **out, qsim_stats *stats) {
    CUDA_TRY(cudaEventRecord(S.ev_stop, S.main));
    CUDA_TRY(cudaEventSynchronize(S.ev_stop));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, S.ev_start, S.ev_stop));
    int st_code = read_status(S.status, S.main);
    if (st_code) return set_error(st_code, "qsim_run: %s", status_text(st_code));
    return finish_run(S.RC, S.dev, ms, &S.prof, stats, out);
}

static int run_plan(const qsim_plan *p, cudaStream_t main, qsim_state **out, qsim_stats *stats) {
    NvtxRange run_range("qsim_run n=%u", p->n);
    StreamsRun S;
    int rc = streams_begin(S, p, main);
    if (rc) return rc;
    PlanDev *pd = S.RC.pd;
    if (S.RC.persistent) {
        std::vector<RunCtx *> one{&S.RC};
        if ((rc = run_persistent(one, false, main, S.status, S.prof, *S.dctx, 1ull << 25))) return rc;
    } else {
        for (size_t si = 0; si < S.RC.nst; ++si) {
            const StageDev &sd = pd->stages[si];
            if ((rc = streams_stage(S, si, pd->ids.p + pd->ids_off[si], pd->gbase.p + pd->gbase_off[si], sd.ngroups)))
                return rc;
        }
    }
    return streams_finish(S, out, stats);
}

// A batch of circuits: initial stores, then one persistent launch over every
// stage of every circuit.
static int run_batch(const qsim_plan *const *plans, size_t count, cudaStream_t main, qsim_state **out,
                     qsim_stats *stats, qsim_kernel_stat *launch_stat) {
    NvtxRange batch_range("qsim_run_batch %zu circuits", count);
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    DeviceCtx &dctx = device_ctx(dev);
    {
        std::lock_guard<std::mutex> lk(dctx.mu);
        int rc = ensure_device_ctx(dctx);
        if (rc) return rc;
    }
    std::vector<std::unique_ptr<RunCtx>> rs(count);
    std::vector<RunCtx *> rp(count);
    int rc;
    uint64_t sum_need = 0;
    std::map<uint32_t, uint64_t> w_groups;  // working-vector sizes of the batch and their group counts
    uint32_t mmax = 0;
    for (size_t c = 0; c < count; ++c) {
        const qsim_plan *p = plans[c];
        if (!p) return set_error(QSIM_E_INVALID, "batch entry %zu is null", c);
        const qsim_config &cfg = p->cfg;
        if (cfg.codec == QSIM_CODEC_NONE || cfg.collect)
            return set_error(QSIM_E_INVALID, "batch entry %zu: a batch runs the compressed store without row collection",
                             c);
        if (cfg.codec != plans[0]->cfg.codec)
            return set_error(QSIM_E_INVALID, "batch entry %zu: every circuit of a batch uses the same codec", c);
        if (cfg.prec != plans[0]->cfg.prec)
            return set_error(QSIM_E_INVALID, "batch entry %zu: every circuit of a batch uses the same precision", c);
        rs[c].reset(new RunCtx());
        rp[c] = rs[c].get();
        if ((rc = prepare_run(*rs[c], p, dctx))) return rc;
        for (const StageDev &sd : rs[c]->pd->stages) w_groups[sd.W] += sd.ngroups;
        sum_need += rs[c]->need_per_parity;
        mmax = std::max(mmax, rs[c]->m);
    }
    const uint64_t slot_budget = 1ull << 27;  // working-vector slots of the launch: about 1 GiB
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    free_b += cached_dev_bytes();
    // working-vector slot rings (one per size) with their frame scratch, and the initial-store buffers
    uint64_t ring_amps = 0;
    for (const auto &kv : w_groups)
        ring_amps += std::min<uint64_t>(kv.second, std::max<uint64_t>(2, slot_budget >> kv.first)) << kv.first;
    const bool rel = plans[0]->cfg.codec == QSIM_CODEC_QSZR;
    // 8 B per amplitude and a quarter for the frame scratch; the relative codec adds its 4 B imaginary words
    const uint64_t work_bytes = ring_amps * (rel ? 12 : 10) + (16ull << (mmax + 1)) * (rel ? 2 : 1);
    const double dev_budget = free_b > work_bytes ? 0.85 * double(free_b - work_bytes) : 0.0;
    const double host_budget = 0.3 * double(host_phys_bytes());
    // each circuit's share of both levels follows its worst-case need
    for (size_t c = 0; c < count; ++c) {
        const double f = double(rs[c]->need_per_parity) / double(sum_need);
        if ((rc = alloc_run(*rs[c], uint64_t(dev_budget * f), uint64_t(host_budget * f), main))) return rc;
    }
    StreamWork w;
    const uint64_t nframes_max = qsz_nframes(int(mmax));
    if ((rc = w.wv.alloc(2ull << mmax)) || (rc = w.tgt.alloc(2)) || (rc = w.res.alloc(2)) || (rc = w.sizes.alloc(2)) ||
        (rc = w.lb_state.alloc(2 * nframes_max)) || (rc = w.lb_ctr.alloc(4)) ||
        (rel && ((rc = w.imsc.alloc(2ull << mmax)) || (rc = w.wrec.alloc(2 * nframes_max * kQszrSideBytes)) ||
                 (rc = w.fwords.alloc(2 * nframes_max)) || (rc = w.fmixed.alloc(2 * nframes_max)) ||
                 (rc = w.flen.alloc(2 * nframes_max)) || (rc = w.foff.alloc(2 * nframes_max)) ||
                 (rc = w.part.alloc(2 * nframes_max)))))
        return rc;
    CUDA_TRY(cudaMemsetAsync(w.lb_state.p, 0, 2 * nframes_max * sizeof(uint64_t), main));
    CUDA_TRY(cudaMemsetAsync(w.lb_ctr.p, 0, 4 * sizeof(uint32_t), main));
    CUDA_TRY(cudaMemsetAsync(w.sizes.p, 0, 2 * sizeof(uint64_t), main));
    w.s = main;  // the initial stores run on the caller's stream, one after another
    cudaEvent_t ev_start, ev_stop;
    CUDA_TRY(cudaEventCreate(&ev_start));
    CUDA_TRY(cudaEventCreate(&ev_stop));
    int *status = dctx.status;
    Profiler prof;
    prof.on = (g_profile.load() != 0 || launch_stat) && !plans[0]->cfg.graph;
    CUDA_TRY(cudaEventRecord(ev_start, main));
    for (size_t c = 0; c < count && !rc; ++c) rc = init_store(*rs[c], w, status);
    w.s = nullptr;  // not ours to destroy
    if (rc) return rc;
    if ((rc = run_persistent(rp, true, main, status, prof, dctx, slot_budget))) return rc;
    CUDA_TRY(cudaEventRecord(ev_stop, main));
    CUDA_TRY(cudaEventSynchronize(ev_stop));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev_start, ev_stop));
    cudaEventDestroy(ev_start);
    cudaEventDestroy(ev_stop);
    int st_code = read_status(status, main);
    if (st_code) return set_error(st_code, "qsim_run_batch: %s", status_text(st_code));
    double alg_bytes = 0, alg_flops = 0;
    for (size_t c = 0; c < count; ++c) {
        if ((rc = finish_run(*rs[c], dev, ms, nullptr, stats ? stats + c : nullptr, out + c))) {
            for (size_t d = 0; d < c; ++d) {
                qsim_state_free(out[d]);
                out[d] = nullptr;
            }
            return rc;
        }
        const RunCtx &R = *rs[c];
        const qsim_state *S = out[c];
        const double amps = std::ldexp(1.0, int(R.n));
        for (size_t i = 0; i < R.nst; ++i) {
            const double in_store = double(i == 0 ? S->stage_acc[R.nst].store_bytes : S->stage_acc[i - 1].store_bytes);
            const double out_store = double(S->stage_acc[i].store_bytes);
            alg_bytes += in_store + out_store + 8 * amps * (2 + (R.predict ? 0 : 1)) +
                         16 * amps * R.pd->stages[i].npasses;
            for (const Op &op : R.p->stages[i].ops)
                alg_flops += (op.type == OP_DENSE ? 8.0 * double(1u << op.k)
                              : op.type == OP_DIAG ? 6.0 : op.type == OP_CSEP ? 12.0 : 0.0) * amps;
        }
    }
    if (launch_stat) {
        memset(launch_stat, 0, sizeof(*launch_stat));
        snprintf(launch_stat->name, sizeof(launch_stat->name), "%s", kProfNames[P_STAGE]);
        double secs[P_NCAT];
        uint64_t launches[P_NCAT];
        prof.collect(secs, launches);
        launch_stat->launches = launches[P_STAGE];
        launch_stat->seconds = secs[P_STAGE];
        launch_stat->alg_bytes = alg_bytes;
        launch_stat->alg_flops = alg_flops;
    }
    return QSIM_OK;
}

// decode blocks [b0, b0 + count) of a state (block order) into dst
static int decode_state_blocks(const qsim_state *st, uint64_t b0, uint32_t count, float2 *dst, BlockRef *refs,
                               uint32_t *ids_dev, int *status, cudaStream_t s) {
    std::vector<uint32_t> ids(count);
    for (uint32_t i = 0; i < count; ++i) ids[i] = uint32_t(b0 + i);
    CUDA_TRY(cudaMemcpyAsync(ids_dev, ids.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    launch_gather_refs(st->table, ids_dev, count, refs, s);
    if (st->codec == QSIM_CODEC_NONE) launch_copy_in(refs, count, st->m, dst, status, s);
    else launch_decode(refs, count, st->m, dst, nullptr, status, s, st->codec == QSIM_CODEC_QSZR);
    CUDA_TRY(cudaStreamSynchronize(s));
    return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void qsim_config_default(qsim_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->m = 20;
    cfg->inner = 2;
    cfg->k = 4;
    cfg->prec = QSIM_PREC_FP32;
    cfg->mode = QSIM_MODE_STREAMS;
    cfg->streams = 2;
    cfg->sizing = QSIM_SIZING_EXACT;
    cfg->codec = QSIM_CODEC_QSZ1;
    cfg->eps = 1e-3;
    cfg->predictor_margin = 0.05;
}

const char *qsim_last_error(void) { return g_err; }

uint64_t qsim_alloc_count(void) { return g_allocs.load(); }
uint64_t qsim_kernel_launch_count(void) { return g_launches.load(); }

void qsim_release_cached_memory(void) {
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto &kv : c.dev_free) cudaFree(kv.second);
    for (auto &kv : c.host_free) cudaFreeHost(kv.second);
    c.dev_free.clear();
    c.host_free.clear();
}

size_t qsim_worst_case_bytes(uint32_t m) {
    if (m < uint32_t(kQszMinM) || m > uint32_t(kQszMaxM)) return 0;
    return size_t(qsz_worst_case(int(m)));
}

size_t qsim_worst_case_bytes_rel(uint32_t m) {
    if (m < uint32_t(kQszMinM) || m > uint32_t(kQszMaxM)) return 0;
    return size_t(qszr_worst_case(int(m)));
}

int qsim_plan_stages(uint32_t n, const qsim_gate *gates, size_t ngates, const qsim_config *cfg, qsim_plan **out) {
    try {
        return build_plan(n, gates, ngates, cfg, out);
    } catch (const std::bad_alloc &) {
        return set_error(QSIM_E_NOMEM, "host allocation failed while planning");
    } catch (...) {
        return set_error(QSIM_E_INVALID, "planning failed");
    }
}

int qsim_plan_info(const qsim_plan *plan, size_t *nstages, uint32_t *stage_inner_masks) {
    if (!plan || !nstages) return set_error(QSIM_E_INVALID, "null argument");
    *nstages = plan->stages.size();
    if (stage_inner_masks)
        for (size_t i = 0; i < plan->stages.size(); ++i) {
            uint32_t mk = 0;
            for (uint32_t q : plan->stages[i].inner) mk |= 1u << (q - plan->cfg.m);
            stage_inner_masks[i] = mk;
        }
    return QSIM_OK;
}

int qsim_plan_shards(const qsim_plan *plan, uint32_t log2_ranks, uint32_t *rank_qubits) {
    return plan_shards(plan, log2_ranks, rank_qubits);
}

int qsim_plan_stage_gates(const qsim_plan *plan, size_t stage, size_t *first, size_t *count) {
    if (!plan || !first || !count) return set_error(QSIM_E_INVALID, "null argument");
    if (stage >= plan->stages.size()) return set_error(QSIM_E_INVALID, "stage index out of range");
    *first = plan->stages[stage].first_gate;
    *count = plan->stages[stage].ngates;
    return QSIM_OK;
}

int qsim_plan_get_stats(const qsim_plan *plan, qsim_plan_stats *out) {
    if (!plan || !out) return set_error(QSIM_E_INVALID, "null argument");
    *out = plan->stats;
    return QSIM_OK;
}

int qsim_plan_stage_ops(const qsim_plan *plan, size_t stage, size_t *count, qsim_op_info *ops) {
    if (!plan || !count) return set_error(QSIM_E_INVALID, "null argument");
    if (stage >= plan->stages.size()) return set_error(QSIM_E_INVALID, "stage index out of range");
    const Stage &st = plan->stages[stage];
    const size_t cap = *count;
    *count = st.ops.size();
    if (!ops) return QSIM_OK;
    if (cap < st.ops.size()) return set_error(QSIM_E_CAPACITY, "ops capacity %zu < %zu", cap, st.ops.size());
    const uint32_t m = plan->cfg.m;
    for (size_t i = 0; i < st.ops.size(); ++i) {
        const Op &op = st.ops[i];
        qsim_op_info &o = ops[i];
        memset(&o, 0, sizeof(o));
        o.type = op.type;
        o.ngates = op.ngates;
        o.basis = op.basis;
        if (op.type == OP_DENSE) {
            o.nq = op.k;
            for (uint32_t j = 0; j < op.k; ++j) o.qubits[j] = op.wq[j] < m ? op.wq[j] : st.inner[op.wq[j] - m];
        } else if (op.type == OP_DIAG) {
            o.nq = op.k;
            for (uint32_t j = 0; j < op.k; ++j) o.qubits[j] = op.fq[j];
            o.quadratic = op.quad ? 1u : 0u;
        } else if (op.type == OP_CSEP) {
            o.nq = uint32_t(op.csep_q.size());
            for (uint32_t j = 0; j < o.nq && j < 8; ++j) o.qubits[j] = op.csep_q[j];
            o.qlist = op.csep_q.data();
        }
        o.u = op.u.empty() ? nullptr : reinterpret_cast<const double *>(op.u.data());
        o.pass = 0xFFFFFFFFu;  // applied by the decoder
        for (size_t pi = 0; pi < st.passes.size(); ++pi)
            for (uint32_t oi : st.passes[pi].ops)
                if (oi == i) o.pass = uint32_t(pi);
    }
    return QSIM_OK;
}

void qsim_plan_free(qsim_plan *plan) {
    if (!plan) return;
    drop_plan_dev(plan);
    delete plan;
}

int qsim_run(const qsim_plan *plan, void *cuda_stream, qsim_state **out, qsim_stats *stats) {
    if (!plan || !out) return set_error(QSIM_E_INVALID, "null argument");
    *out = nullptr;
    try {
        return run_plan(plan, static_cast<cudaStream_t>(cuda_stream), out, stats);
    } catch (const std::bad_alloc &) {
        return set_error(QSIM_E_NOMEM, "host allocation failed");
    } catch (...) {
        return set_error(QSIM_E_CUDA, "run failed");
    }
}

// ---------------------------------------------------------------------------
// sharded runs: one rank's SV groups, stage by stage, blocks moved between stages by the caller
// ---------------------------------------------------------------------------
}  // extern "C"

namespace qsim {

// the streams of `count` blocks (table entries of `tab`) packed at byte offsets dst_off of dst, 16-byte words;
// each copied entry is then cleared (the block has left this rank)
__global__ void k_export_streams(BlockSlot *tab, const uint64_t *__restrict__ ids, const uint64_t *__restrict__ dst_off,
                                 uint32_t count, uint8_t *__restrict__ dst) {
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const BlockSlot sl = tab[ids[i]];
        const uint4 *src = reinterpret_cast<const uint4 *>(sl.ptr);
        uint4 *d = reinterpret_cast<uint4 *>(dst + dst_off[i]);
        for (uint64_t k = threadIdx.x; k < sl.bytes / 16; k += blockDim.x) d[k] = src[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            tab[ids[i]].ptr = nullptr;
            tab[ids[i]].bytes = 0;
        }
    }
}

// received streams (at byte offsets src_off of src, sizes bytes[i]) placed in slots of the current arena
// (device tier, then pinned host), their table entries set
__global__ void k_import_streams(BlockSlot *tab, const uint64_t *__restrict__ ids, const uint64_t *__restrict__ src_off,
                                 const uint64_t *__restrict__ bytes, uint32_t count, const uint8_t *__restrict__ src,
                                 ArenaDev dev, ArenaDev host, int *status) {
    __shared__ uint8_t *dst;
    __shared__ uint32_t tier;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const uint64_t nb = bytes[i];
        if (threadIdx.x == 0) {
            const uint64_t sz = (nb + 255) & ~255ull;
            uint64_t off = atomicAdd(reinterpret_cast<unsigned long long *>(dev.bump), sz);
            dst = nullptr;
            tier = 0;
            if (off + sz <= dev.cap) {
                dst = dev.base + off;
            } else if (host.base) {
                off = atomicAdd(reinterpret_cast<unsigned long long *>(host.bump), sz);
                if (off + sz <= host.cap) {
                    dst = host.base + off;
                    tier = 1;
                }
            }
            if (!dst) raise_status(status, QSIM_E_NOMEM);
            tab[ids[i]].ptr = dst;
            tab[ids[i]].bytes = dst ? nb : 0;
            tab[ids[i]].tier = tier;
        }
        __syncthreads();
        if (dst) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src + src_off[i]);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (uint64_t k = threadIdx.x; k < nb / 16; k += blockDim.x) d4[k] = s4[k];
        }
        __syncthreads();
    }
}

__global__ void k_clear_slots(BlockSlot *tab, const uint8_t *__restrict__ held, uint64_t nblocks) {
    for (uint64_t b = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; b < nblocks; b += uint64_t(gridDim.x) * blockDim.x)
        if (!held[b]) {
            tab[b].ptr = nullptr;
            tab[b].bytes = 0;
        }
}

}  // namespace qsim

struct qsim_shard_run {
    qsim::StreamsRun S;
    uint32_t r = 0, rank = 0;
    std::vector<uint32_t> rq;         // nstages x r rank qubits
    std::vector<uint8_t> held;        // blocks this rank holds now
    qsim::DevBuf<uint32_t> ids;       // per stage: the rank's groups' block ids, group-major
    qsim::DevBuf<uint64_t> gb;        // per stage: their outer bits
    std::vector<size_t> ids_off, gb_off;
    std::vector<uint64_t> ngroups;
    size_t next = 0;                  // the next stage to run
    qsim::DevBuf<uint64_t> xbuf;      // export/import lists
    bool failed = false;
};

using namespace qsim;

static uint32_t shard_owner(const qsim_shard_run *R, size_t stage, uint64_t block) {
    const uint32_t m = R->S.RC.m;
    uint32_t o = 0;
    for (uint32_t j = 0; j < R->r; ++j) o |= uint32_t((block >> (R->rq[stage * R->r + j] - m)) & 1ull) << j;
    return o;
}

extern "C" {

int qsim_shard_begin(const qsim_plan *plan, const uint32_t *rank_qubits, uint32_t log2_ranks, uint32_t rank,
                     void *cuda_stream, qsim_shard_run **out) {
    if (!plan || !out || (log2_ranks && !rank_qubits)) return set_error(QSIM_E_INVALID, "null argument");
    *out = nullptr;
    if (plan->cfg.mode != QSIM_MODE_STREAMS) return set_error(QSIM_E_INVALID, "sharded runs use streams mode");
    if (log2_ranks > 16 || rank >= (1u << log2_ranks)) return set_error(QSIM_E_INVALID, "rank out of range");
    const size_t nst = plan->stages.size();
    const uint32_t n = plan->n, m = plan->cfg.m;
    for (size_t s = 0; s < nst; ++s)
        for (uint32_t j = 0; j < log2_ranks; ++j) {
            const uint32_t q = rank_qubits[s * log2_ranks + j];
            const auto &in = plan->stages[s].inner;
            if (q < m || q >= n || std::find(in.begin(), in.end(), q) != in.end())
                return set_error(QSIM_E_INVALID, "stage %zu: rank qubit %u is not an outer qubit", s, q);
            for (uint32_t k = 0; k < j; ++k)
                if (rank_qubits[s * log2_ranks + k] == q)
                    return set_error(QSIM_E_INVALID, "stage %zu: rank qubit %u repeated", s, q);
        }
    try {
        std::unique_ptr<qsim_shard_run> R(new qsim_shard_run());
        R->r = log2_ranks;
        R->rank = rank;
        R->rq.assign(rank_qubits, rank_qubits + nst * log2_ranks);
        int rc = streams_begin(R->S, plan, static_cast<cudaStream_t>(cuda_stream));
        if (rc) return rc;
        const uint64_t nblocks = R->S.RC.nblocks;
        R->held.assign(nblocks, 0);
        if (nst)
            for (uint64_t b = 0; b < nblocks; ++b) R->held[b] = shard_owner(R.get(), 0, b) == rank;
        else
            for (uint64_t b = 0; b < nblocks; ++b) R->held[b] = rank == 0;
        // the rank's groups of every stage, in the plan's group order
        PlanDev *pd = R->S.RC.pd;
        std::vector<uint32_t> hid, sub_ids;
        std::vector<uint64_t> hgb, sub_gb;
        for (size_t s = 0; s < nst; ++s) {
            const StageDev &sd = pd->stages[s];
            hid.resize(size_t(sd.ngroups) * sd.G);
            hgb.resize(sd.ngroups);
            CUDA_TRY(cudaMemcpy(hid.data(), pd->ids.p + pd->ids_off[s], hid.size() * 4, cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(hgb.data(), pd->gbase.p + pd->gbase_off[s], hgb.size() * 8, cudaMemcpyDeviceToHost));
            R->ids_off.push_back(sub_ids.size());
            R->gb_off.push_back(sub_gb.size());
            uint64_t ng = 0;
            for (uint32_t g = 0; g < sd.ngroups; ++g) {
                if (shard_owner(R.get(), s, hid[size_t(g) * sd.G]) != rank) continue;
                sub_ids.insert(sub_ids.end(), hid.begin() + size_t(g) * sd.G, hid.begin() + size_t(g + 1) * sd.G);
                sub_gb.push_back(hgb[g]);
                ++ng;
            }
            R->ngroups.push_back(ng);
        }
        if ((rc = R->ids.alloc(std::max<size_t>(1, sub_ids.size()))) || (rc = R->gb.alloc(std::max<size_t>(1, sub_gb.size()))))
            return rc;
        if (!sub_ids.empty())
            CUDA_TRY(cudaMemcpy(R->ids.p, sub_ids.data(), sub_ids.size() * 4, cudaMemcpyHostToDevice));
        if (!sub_gb.empty())
            CUDA_TRY(cudaMemcpy(R->gb.p, sub_gb.data(), sub_gb.size() * 8, cudaMemcpyHostToDevice));
        *out = R.release();
        return QSIM_OK;
    } catch (const std::bad_alloc &) {
        return set_error(QSIM_E_NOMEM, "host allocation failed");
    }
}

int qsim_shard_stage(qsim_shard_run *R, size_t stage) {
    if (!R) return set_error(QSIM_E_INVALID, "null argument");
    if (R->failed) return set_error(QSIM_E_INVALID, "the sharded run failed earlier");
    if (stage != R->next || stage >= R->S.RC.nst)
        return set_error(QSIM_E_INVALID, "stage %zu: the next stage to run is %zu", stage, R->next);
    for (uint64_t b = 0; b < R->S.RC.nblocks; ++b)
        if (bool(R->held[b]) != (shard_owner(R, stage, b) == R->rank))
            return set_error(QSIM_E_INVALID, "stage %zu: block %llu is %s this rank, the rank qubits say otherwise",
                             stage, (unsigned long long)b, R->held[b] ? "on" : "not on");
    int rc = streams_stage(R->S, stage, R->ids.p + R->ids_off[stage], R->gb.p + R->gb_off[stage], R->ngroups[stage]);
    if (rc) {
        R->failed = true;
        return rc;
    }
    ++R->next;
    return QSIM_OK;
}

int qsim_shard_block_bytes(qsim_shard_run *R, const uint64_t *blocks, size_t count, uint64_t *bytes) {
    if (!R || (count && (!blocks || !bytes))) return set_error(QSIM_E_INVALID, "null argument");
    const uint64_t nblocks = R->S.RC.nblocks;
    for (size_t i = 0; i < count; ++i)
        if (blocks[i] >= nblocks || !R->held[blocks[i]])
            return set_error(QSIM_E_INVALID, "block %llu is not on this rank", (unsigned long long)blocks[i]);
    CUDA_TRY(cudaStreamSynchronize(R->S.main));
    std::vector<BlockSlot> tab(nblocks);
    const BlockSlot *cur = R->S.RC.tables.p + (R->next & 1) * nblocks;
    CUDA_TRY(cudaMemcpy(tab.data(), cur, nblocks * sizeof(BlockSlot), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < count; ++i) bytes[i] = tab[blocks[i]].bytes;
    return QSIM_OK;
}

int qsim_shard_export(qsim_shard_run *R, const uint64_t *blocks, size_t count, void *d_packed, size_t cap) {
    if (!R || (count && (!blocks || !d_packed))) return set_error(QSIM_E_INVALID, "null argument");
    if (reinterpret_cast<uintptr_t>(d_packed) & 15) return set_error(QSIM_E_INVALID, "d_packed must be 16-byte aligned");
    if (!count) return QSIM_OK;
    std::vector<uint64_t> bytes(count);
    int rc = qsim_shard_block_bytes(R, blocks, count, bytes.data());
    if (rc) return rc;
    std::vector<uint64_t> lists(2 * count);
    uint64_t off = 0;
    for (size_t i = 0; i < count; ++i) {
        lists[i] = blocks[i];
        lists[count + i] = off;
        off += bytes[i];
    }
    if (off > cap) return set_error(QSIM_E_CAPACITY, "the blocks need %llu bytes, cap is %zu", (unsigned long long)off, cap);
    if ((rc = R->xbuf.alloc(3 * count))) return rc;
    cudaStream_t s = R->S.main;
    CUDA_TRY(cudaMemcpyAsync(R->xbuf.p, lists.data(), 2 * count * 8, cudaMemcpyHostToDevice, s));
    BlockSlot *cur = R->S.RC.tables.p + (R->next & 1) * R->S.RC.nblocks;
    k_export_streams<<<unsigned(std::min<size_t>(count, 152 * 8)), 256, 0, s>>>(cur, R->xbuf.p, R->xbuf.p + count,
                                                                               uint32_t(count), static_cast<uint8_t *>(d_packed));
    count_launch();
    CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t i = 0; i < count; ++i) R->held[blocks[i]] = 0;
    return QSIM_OK;
}

int qsim_shard_import(qsim_shard_run *R, const uint64_t *blocks, const uint64_t *bytes, size_t count,
                      const void *d_packed) {
    if (!R || (count && (!blocks || !bytes || !d_packed))) return set_error(QSIM_E_INVALID, "null argument");
    if (reinterpret_cast<uintptr_t>(d_packed) & 15) return set_error(QSIM_E_INVALID, "d_packed must be 16-byte aligned");
    if (!count) return QSIM_OK;
    const uint64_t nblocks = R->S.RC.nblocks;
    std::vector<uint64_t> lists(3 * count);
    uint64_t off = 0;
    for (size_t i = 0; i < count; ++i) {
        if (blocks[i] >= nblocks || R->held[blocks[i]])
            return set_error(QSIM_E_INVALID, "block %llu: out of range or already on this rank", (unsigned long long)blocks[i]);
        if (bytes[i] & 15) return set_error(QSIM_E_CORRUPT, "block %llu: stream size not a multiple of 16", (unsigned long long)blocks[i]);
        lists[i] = blocks[i];
        lists[count + i] = off;
        lists[2 * count + i] = bytes[i];
        off += bytes[i];
    }
    int rc;
    if ((rc = R->xbuf.alloc(3 * count))) return rc;
    cudaStream_t s = R->S.main;
    CUDA_TRY(cudaMemcpyAsync(R->xbuf.p, lists.data(), 3 * count * 8, cudaMemcpyHostToDevice, s));
    const int par = int(R->next & 1);
    BlockSlot *cur = R->S.RC.tables.p + par * nblocks;
    k_import_streams<<<unsigned(std::min<size_t>(count, 152 * 8)), 256, 0, s>>>(
        cur, R->xbuf.p, R->xbuf.p + count, R->xbuf.p + 2 * count, uint32_t(count),
        static_cast<const uint8_t *>(d_packed), R->S.RC.arena_dev(par), R->S.RC.arena_host(par), R->S.status);
    count_launch();
    CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t i = 0; i < count; ++i) R->held[blocks[i]] = 1;
    return QSIM_OK;
}

int qsim_shard_finish(qsim_shard_run *R, qsim_state **out, qsim_stats *stats) {
    if (!R || !out) return set_error(QSIM_E_INVALID, "null argument");
    *out = nullptr;
    if (R->failed) return set_error(QSIM_E_INVALID, "the sharded run failed earlier");
    if (R->next != R->S.RC.nst) return set_error(QSIM_E_INVALID, "%zu of %zu stages run", R->next, R->S.RC.nst);
    // blocks not on this rank: clear their final table entries (readout of them reports a corrupt block)
    const uint64_t nblocks = R->S.RC.nblocks;
    DevBuf<uint8_t> held;
    int rc = held.alloc(nblocks);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(held.p, R->held.data(), nblocks, cudaMemcpyHostToDevice, R->S.main));
    k_clear_slots<<<64, 256, 0, R->S.main>>>(R->S.RC.tables.p + (R->next & 1) * nblocks, held.p, nblocks);
    count_launch();
    CUDA_TRY(cudaStreamSynchronize(R->S.main));
    try {
        return streams_finish(R->S, out, stats);
    } catch (const std::bad_alloc &) {
        return set_error(QSIM_E_NOMEM, "host allocation failed");
    }
}

void qsim_shard_free(qsim_shard_run *R) { delete R; }

int qsim_run_batch(const qsim_plan *const *plans, size_t count, void *cuda_stream, qsim_state **states,
                   qsim_stats *stats, qsim_kernel_stat *launch) {
    if (!plans || !states || count == 0) return set_error(QSIM_E_INVALID, "empty batch or null argument");
    for (size_t c = 0; c < count; ++c) states[c] = nullptr;
    try {
        return run_batch(plans, count, static_cast<cudaStream_t>(cuda_stream), states, stats, launch);
    } catch (const std::bad_alloc &) {
        return set_error(QSIM_E_NOMEM, "host allocation failed");
    } catch (...) {
        return set_error(QSIM_E_CUDA, "batch run failed");
    }
}

int qsim_state_stage_stats(const qsim_state *st, size_t stage, uint64_t *store_bytes, uint64_t *reserved_bytes,
                           double *err_sq) {
    if (!st) return set_error(QSIM_E_INVALID, "null state");
    if (stage + 1 >= st->stage_acc.size()) return set_error(QSIM_E_INVALID, "stage index out of range");
    const StageAccum &a = st->stage_acc[stage];
    if (store_bytes) *store_bytes = a.store_bytes;
    if (reserved_bytes) *reserved_bytes = a.reserved_bytes;
    if (err_sq) *err_sq = a.err_sq;
    return QSIM_OK;
}

int qsim_mlp_forward(const float *d_params, const float *d_x, size_t batch, float *d_y, int bf16_weights,
                     void *cuda_stream) {
    if (!d_params || (batch && (!d_x || !d_y))) return set_error(QSIM_E_INVALID, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    launch_mlp_forward(d_params, d_x, uint32_t(batch), d_y, bf16_weights, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    return QSIM_OK;
}

int qsim_mlp_loss_grad(const float *d_params, const float *d_x, const float *d_t, size_t batch, float *d_grad,
                       float *loss, void *cuda_stream) {
    if (!d_params || !d_x || !d_t || !d_grad || !batch) return set_error(QSIM_E_INVALID, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    DevBuf<float> dl;
    int rc = dl.alloc(1);
    if (rc) return rc;
    rc = launch_mlp_loss_grad(d_params, d_x, kMlpIn, d_t, 1, nullptr, 0, uint32_t(batch), d_grad, dl.p, s);
    if (rc) return set_error(rc, "loss/grad launch failed");
    float h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, dl.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (loss) *loss = h;
    return QSIM_OK;
}

int qsim_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, size_t n, int t, float lr,
                   float beta1, float beta2, float eps, void *cuda_stream) {
    if (!d_params || !d_grad || !d_m || !d_v || t < 1) return set_error(QSIM_E_INVALID, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    launch_adam(d_params, d_grad, d_m, d_v, uint32_t(n), t, lr, beta1, beta2, eps, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    return QSIM_OK;
}

static int predictor_ctx(DeviceCtx **out) {
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    DeviceCtx &c = device_ctx(dev);
    int rc = ensure_device_ctx(c);
    if (rc) return rc;
    *out = &c;
    return QSIM_OK;
}

int qsim_predictor_set(const float *params, size_t n, int bf16_inference) {
    if (!params || n != size_t(kMlpParams)) return set_error(QSIM_E_INVALID, "need %d parameters", kMlpParams);
    DeviceCtx *c;
    int rc = predictor_ctx(&c);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpy(c->pred_params, params, n * sizeof(float), cudaMemcpyHostToDevice));
    c->pred_bf16 = bf16_inference;
    c->pred_ready = true;
    return QSIM_OK;
}

int qsim_predictor_get(float *params, size_t n) {
    if (!params || n != size_t(kMlpParams)) return set_error(QSIM_E_INVALID, "need %d parameters", kMlpParams);
    DeviceCtx *c;
    int rc = predictor_ctx(&c);
    if (rc) return rc;
    if (!c->pred_ready) return set_error(QSIM_E_INVALID, "predictor has no weights");
    CUDA_TRY(cudaMemcpy(params, c->pred_params, n * sizeof(float), cudaMemcpyDeviceToHost));
    return QSIM_OK;
}

static uint64_t splitmix_next(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int qsim_predictor_train(const float *rows, size_t count, const qsim_train_config *tc, double *final_loss) {
    if (!rows || !count || !tc || !tc->epochs || !tc->batch) return set_error(QSIM_E_INVALID, "bad argument");
    DeviceCtx *c;
    int rc = predictor_ctx(&c);
    if (rc) return rc;
    const size_t rowf = kMlpIn + 1;
    DevBuf<float> d_rows, p, g, m1, m2, loss;
    DevBuf<uint32_t> perm;
    if ((rc = d_rows.alloc(count * rowf)) || (rc = p.alloc(kMlpParams)) || (rc = g.alloc(kMlpParams)) ||
        (rc = m1.alloc(kMlpParams)) || (rc = m2.alloc(kMlpParams)) || (rc = loss.alloc(1)) || (rc = perm.alloc(count)))
        return rc;
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CUDA_TRY(cudaMemcpyAsync(d_rows.p, rows, count * rowf * sizeof(float), cudaMemcpyHostToDevice, s));
    // He-uniform initialisation from splitmix64; zero biases
    uint64_t st = tc->seed;
    std::vector<float> hp(kMlpParams, 0.f);
    auto fill = [&](size_t off, int fan_out, int fan_in) {
        const double lim = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < fan_out * fan_in; ++i) {
            const double u = double(splitmix_next(st) >> 11) * (1.0 / 9007199254740992.0);
            hp[off + i] = float((2 * u - 1) * lim);
        }
    };
    fill(0, kMlpHidden, kMlpIn);
    fill(kMlpHidden * kMlpIn + kMlpHidden, kMlpHidden, kMlpHidden);
    fill(kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden, 1, kMlpHidden);
    CUDA_TRY(cudaMemcpyAsync(p.p, hp.data(), kMlpParams * sizeof(float), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(m1.p, 0, kMlpParams * sizeof(float), s));
    CUDA_TRY(cudaMemsetAsync(m2.p, 0, kMlpParams * sizeof(float), s));
    std::vector<uint32_t> hperm(count);
    int t = 0;
    for (uint32_t ep = 0; ep < tc->epochs; ++ep) {
        for (size_t i = 0; i < count; ++i) hperm[i] = uint32_t(i);
        for (size_t i = count - 1; i > 0; --i) std::swap(hperm[i], hperm[splitmix_next(st) % (i + 1)]);
        CUDA_TRY(cudaStreamSynchronize(s));  // hperm is reused: the previous upload must have landed
        CUDA_TRY(cudaMemcpyAsync(perm.p, hperm.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        for (size_t b0 = 0; b0 < count; b0 += tc->batch) {
            const uint32_t nb = uint32_t(std::min<size_t>(tc->batch, count - b0));
            rc = launch_mlp_loss_grad(p.p, d_rows.p, rowf, d_rows.p + kMlpIn, rowf, perm.p, uint32_t(b0), nb, g.p,
                                      nullptr, s);
            if (rc) { cudaStreamDestroy(s); return set_error(rc, "loss/grad launch failed"); }
            launch_adam(p.p, g.p, m1.p, m2.p, kMlpParams, ++t, tc->lr, 0.9f, 0.999f, 1e-8f, s);
        }
    }
    rc = launch_mlp_loss_grad(p.p, d_rows.p, rowf, d_rows.p + kMlpIn, rowf, nullptr, 0, uint32_t(count), g.p, loss.p, s);
    float hl = 0;
    CUDA_TRY(cudaMemcpyAsync(&hl, loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(c->pred_params, p.p, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    cudaStreamDestroy(s);
    c->pred_bf16 = int(tc->bf16_inference);
    c->pred_ready = true;
    if (final_loss) *final_loss = hl;
    return QSIM_OK;
}

int qsim_state_training_data(const qsim_state *st, float *rows_out, size_t cap_rows, size_t *rows) {
    if (!st || !rows) return set_error(QSIM_E_INVALID, "null argument");
    const size_t rowf = kMlpIn + 1;
    const size_t have = st->train_rows.size() / rowf;
    *rows = have;
    if (!rows_out) return QSIM_OK;
    if (cap_rows < have) return set_error(QSIM_E_CAPACITY, "capacity %zu < %zu rows", cap_rows, have);
    memcpy(rows_out, st->train_rows.data(), have * rowf * sizeof(float));
    return QSIM_OK;
}

void qsim_profile_enable(int on) { g_profile.store(on ? 1 : 0); }

int qsim_state_kernel_stats(const qsim_state *st, qsim_kernel_stat *out, size_t cap, size_t *count) {
    if (!st || !count) return set_error(QSIM_E_INVALID, "null argument");
    *count = st->kstats.size();
    if (!out) return QSIM_OK;
    if (cap < st->kstats.size()) return set_error(QSIM_E_CAPACITY, "capacity %zu < %zu", cap, st->kstats.size());
    for (size_t i = 0; i < st->kstats.size(); ++i) out[i] = st->kstats[i];
    return QSIM_OK;
}

void qsim_state_free(qsim_state *st) {
    if (!st) return;
    dev_free(st->dev_arena);
    host_free(st->host_arena);
    dev_free(st->table);
    delete st;
}

int qsim_state_decompress(const qsim_state *st, float *d_out, void *cuda_stream) {
    if (!st || !d_out) return set_error(QSIM_E_INVALID, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const uint64_t nblocks = 1ull << (st->n - st->m);
    DevBuf<BlockRef> refs;
    DevBuf<uint32_t> ids;
    int rc;
    const uint32_t chunk = uint32_t(std::min<uint64_t>(nblocks, 4096));
    if ((rc = refs.alloc(chunk)) || (rc = ids.alloc(chunk))) return rc;
    int *status = device_ctx(st->device).status;
    for (uint64_t b = 0; b < nblocks; b += chunk) {
        uint32_t cnt = uint32_t(std::min<uint64_t>(chunk, nblocks - b));
        rc = decode_state_blocks(st, b, cnt, reinterpret_cast<float2 *>(d_out) + (b << st->m), refs.p, ids.p, status, s);
        if (rc) return rc;
    }
    int code = read_status(status, s);
    if (code) return set_error(code, "decompress: %s", status_text(code));
    return QSIM_OK;
}

// Compressed states: only the frames (4096 amplitudes, or the whole block below 2^12) holding the requested
// amplitudes are decoded, through the streams' frame offsets.
static int amplitudes_by_frame(const qsim_state *st, const uint64_t *idx, size_t count, float *out) {
    const uint32_t m = st->m, fl = m < 12 ? m : 12;
    std::map<uint64_t, uint32_t> item;  // global frame number -> position in the decode list
    for (size_t i = 0; i < count; ++i) item.emplace(idx[i] >> fl, 0);
    std::vector<uint2> frames;
    frames.reserve(item.size());
    for (auto &kv : item) {
        kv.second = uint32_t(frames.size());
        frames.push_back(make_uint2(uint32_t(kv.first >> (m - fl)), uint32_t(kv.first & ((1ull << (m - fl)) - 1))));
    }
    const uint32_t chunk = uint32_t(std::min<size_t>(frames.size(), size_t(1) << (24 - fl)));  // 2^24 amplitudes
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    DevBuf<uint2> d_frames;
    DevBuf<uint32_t> d_slot, d_local;
    DevBuf<float2> buf, d_out;
    int rc;
    if ((rc = d_frames.alloc(frames.size())) || (rc = buf.alloc(uint64_t(chunk) << fl)) ||
        (rc = d_slot.alloc(count)) || (rc = d_local.alloc(count)) || (rc = d_out.alloc(count))) {
        cudaStreamDestroy(s);
        return rc;
    }
    int *status = device_ctx(st->device).status;
    CUDA_TRY(cudaMemcpyAsync(d_frames.p, frames.data(), frames.size() * sizeof(uint2), cudaMemcpyHostToDevice, s));
    std::vector<float2> host(count);
    for (size_t f0 = 0; f0 < frames.size(); f0 += chunk) {
        const uint32_t cnt = uint32_t(std::min<size_t>(chunk, frames.size() - f0));
        launch_decode_frames(st->table, d_frames.p + f0, cnt, int(m), buf.p, status, s,
                             st->codec == QSIM_CODEC_QSZR);
        std::vector<uint32_t> sel_slot, sel_local;
        std::vector<size_t> sel_pos;
        for (size_t i = 0; i < count; ++i) {
            const uint32_t it = item[idx[i] >> fl];
            if (it >= f0 && it < f0 + cnt) {
                sel_slot.push_back(uint32_t(it - f0));
                sel_local.push_back(uint32_t(idx[i] & ((1ull << fl) - 1)));
                sel_pos.push_back(i);
            }
        }
        CUDA_TRY(cudaMemcpyAsync(d_slot.p, sel_slot.data(), sel_slot.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_local.p, sel_local.data(), sel_local.size() * 4, cudaMemcpyHostToDevice, s));
        k_gather_amps<<<unsigned((sel_pos.size() + 255) / 256), 256, 0, s>>>(buf.p, d_slot.p, d_local.p,
                                                                            sel_pos.size(), int(fl), d_out.p);
        count_launch();
        std::vector<float2> tmp(sel_pos.size());
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), d_out.p, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t t = 0; t < sel_pos.size(); ++t) host[sel_pos[t]] = tmp[t];
    }
    int code = read_status(status, s);
    cudaStreamDestroy(s);
    if (code) return set_error(code, "amplitudes: %s", status_text(code));
    memcpy(out, host.data(), count * sizeof(float2));
    return QSIM_OK;
}

int qsim_amplitudes(const qsim_state *st, const uint64_t *idx, size_t count, float *out) {
    if (!st || (count && (!idx || !out))) return set_error(QSIM_E_INVALID, "null argument");
    if (!count) return QSIM_OK;
    const uint32_t m = st->m;
    const uint64_t N = 1ull << st->n;
    for (size_t i = 0; i < count; ++i)
        if (idx[i] >= N) return set_error(QSIM_E_INVALID, "amplitude index out of range");
    if (st->codec != QSIM_CODEC_NONE) return amplitudes_by_frame(st, idx, count, out);
    std::map<uint64_t, uint32_t> slot;
    for (size_t i = 0; i < count; ++i) {
        if (idx[i] >= N) return set_error(QSIM_E_INVALID, "amplitude index out of range");
        slot.emplace(idx[i] >> m, 0);
    }
    uint32_t k = 0;
    std::vector<uint32_t> bids;
    for (auto &kv : slot) {
        kv.second = k++;
        bids.push_back(uint32_t(kv.first));
    }
    std::vector<uint32_t> h_slot(count), h_local(count);
    for (size_t i = 0; i < count; ++i) {
        h_slot[i] = slot[idx[i] >> m];
        h_local[i] = uint32_t(idx[i] & ((1ull << m) - 1));
    }
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    DevBuf<BlockRef> refs;
    DevBuf<uint32_t> ids, d_slot, d_local;
    DevBuf<float2> blocks, d_out;
    const uint32_t chunk = uint32_t(std::min<size_t>(bids.size(), std::max<uint64_t>(1, (1ull << 26) >> m)));
    int rc;
    if ((rc = refs.alloc(chunk)) || (rc = ids.alloc(chunk)) || (rc = blocks.alloc(uint64_t(chunk) << m)) ||
        (rc = d_slot.alloc(count)) || (rc = d_local.alloc(count)) || (rc = d_out.alloc(count))) {
        cudaStreamDestroy(s);
        return rc;
    }
    int *status = device_ctx(st->device).status;
    std::vector<float2> host(count);
    // process the touched blocks chunk by chunk
    for (size_t b0 = 0; b0 < bids.size(); b0 += chunk) {
        const uint32_t cnt = uint32_t(std::min<size_t>(chunk, bids.size() - b0));
        CUDA_TRY(cudaMemcpyAsync(ids.p, bids.data() + b0, cnt * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        launch_gather_refs(st->table, ids.p, cnt, refs.p, s);
        if (st->codec == QSIM_CODEC_NONE) launch_copy_in(refs.p, cnt, m, blocks.p, status, s);
        else launch_decode(refs.p, cnt, m, blocks.p, nullptr, status, s, st->codec == QSIM_CODEC_QSZR);
        std::vector<uint32_t> sel_slot, sel_local;
        std::vector<size_t> sel_pos;
        for (size_t i = 0; i < count; ++i)
            if (h_slot[i] >= b0 && h_slot[i] < b0 + cnt) {
                sel_slot.push_back(uint32_t(h_slot[i] - b0));
                sel_local.push_back(h_local[i]);
                sel_pos.push_back(i);
            }
        if (sel_pos.empty()) continue;
        CUDA_TRY(cudaMemcpyAsync(d_slot.p, sel_slot.data(), sel_slot.size() * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_local.p, sel_local.data(), sel_local.size() * 4, cudaMemcpyHostToDevice, s));
        k_gather_amps<<<unsigned((sel_pos.size() + 255) / 256), 256, 0, s>>>(blocks.p, d_slot.p, d_local.p,
                                                                            sel_pos.size(), int(m), d_out.p);
        count_launch();
        std::vector<float2> tmp(sel_pos.size());
        CUDA_TRY(cudaMemcpyAsync(tmp.data(), d_out.p, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t t = 0; t < sel_pos.size(); ++t) host[sel_pos[t]] = tmp[t];
    }
    int code = read_status(status, s);
    cudaStreamDestroy(s);
    if (code) return set_error(code, "amplitudes: %s", status_text(code));
    memcpy(out, host.data(), count * sizeof(float2));
    return QSIM_OK;
}

static int reduce_state(const qsim_state *st, const double *ref, double acc_out[4]) {
    const uint32_t m = st->m;
    const uint64_t nblocks = 1ull << (st->n - st->m);
    cudaPointerAttributes attr{};
    bool ref_dev = false;
    if (ref) {
        if (cudaPointerGetAttributes(&attr, ref) == cudaSuccess && attr.type == cudaMemoryTypeDevice) ref_dev = true;
        cudaGetLastError();
    }
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const uint32_t chunk = uint32_t(std::min<uint64_t>(nblocks, std::max<uint64_t>(1, (1ull << 24) >> m)));
    DevBuf<BlockRef> refs;
    DevBuf<uint32_t> ids;
    DevBuf<float2> blocks;
    DevBuf<double2> rbuf;
    DevBuf<double> acc;
    int rc;
    if ((rc = refs.alloc(chunk)) || (rc = ids.alloc(chunk)) || (rc = blocks.alloc(uint64_t(chunk) << m)) ||
        (rc = acc.alloc(4)) || (ref && !ref_dev && (rc = rbuf.alloc(uint64_t(chunk) << m)))) {
        cudaStreamDestroy(s);
        return rc;
    }
    CUDA_TRY(cudaMemsetAsync(acc.p, 0, 4 * sizeof(double), s));
    int *status = device_ctx(st->device).status;
    for (uint64_t b = 0; b < nblocks; b += chunk) {
        const uint32_t cnt = uint32_t(std::min<uint64_t>(chunk, nblocks - b));
        rc = decode_state_blocks(st, b, cnt, blocks.p, refs.p, ids.p, status, s);
        if (rc) { cudaStreamDestroy(s); return rc; }
        const uint64_t amps = uint64_t(cnt) << m;
        const double2 *r = nullptr;
        if (ref) {
            if (ref_dev) {
                r = reinterpret_cast<const double2 *>(ref) + (b << m);
            } else {
                CUDA_TRY(cudaMemcpyAsync(rbuf.p, ref + 2 * (b << m), amps * sizeof(double2), cudaMemcpyHostToDevice, s));
                r = rbuf.p;
            }
        }
        k_reduce_fid<<<unsigned(std::min<uint64_t>(152 * 4, (amps + 255) / 256)), 256, 0, s>>>(r, blocks.p, amps, acc.p);
        count_launch();
    }
    CUDA_TRY(cudaMemcpyAsync(acc_out, acc.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int code = read_status(status, s);
    cudaStreamDestroy(s);
    if (code) return set_error(code, "readout: %s", status_text(code));
    return QSIM_OK;
}

int qsim_fidelity(const qsim_state *st, const double *ref, double *f) {
    if (!st || !ref || !f) return set_error(QSIM_E_INVALID, "null argument");
    double a[4];
    int rc = reduce_state(st, ref, a);
    if (rc) return rc;
    const double den = std::sqrt(a[2] * a[3]);
    *f = den > 0 ? std::sqrt(a[0] * a[0] + a[1] * a[1]) / den : 0.0;
    return QSIM_OK;
}

int qsim_state_norm(const qsim_state *st, double *norm_sq) {
    if (!st || !norm_sq) return set_error(QSIM_E_INVALID, "null argument");
    double a[4];
    int rc = reduce_state(st, nullptr, a);
    if (rc) return rc;
    *norm_sq = a[3];
    return QSIM_OK;
}

int qsim_state_block_stream(const qsim_state *st, uint64_t block, void *host_out, size_t cap, size_t *bytes) {
    if (!st || !bytes) return set_error(QSIM_E_INVALID, "null argument");
    const uint64_t nblocks = 1ull << (st->n - st->m);
    if (block >= nblocks) return set_error(QSIM_E_INVALID, "block index out of range");
    BlockSlot slot;
    CUDA_TRY(cudaMemcpy(&slot, st->table + block, sizeof(slot), cudaMemcpyDeviceToHost));
    *bytes = slot.bytes;
    if (cap < slot.bytes) return set_error(QSIM_E_CAPACITY, "buffer of %zu bytes < stream of %llu", cap,
                                           (unsigned long long)slot.bytes);
    if (!slot.bytes) return QSIM_OK;  // a block this state does not hold (a sharded rank's)
    if (!host_out) return set_error(QSIM_E_INVALID, "null output");
    CUDA_TRY(cudaMemcpy(host_out, slot.ptr, slot.bytes, cudaMemcpyDefault));
    return QSIM_OK;
}

int qsim_compress_block(const float *d_amps, uint32_t m, double eb, void *d_out, size_t cap, size_t *out_bytes,
                        void *cuda_stream) {
    if (!d_amps || !d_out || !out_bytes) return set_error(QSIM_E_INVALID, "null argument");
    if (m < uint32_t(kQszMinM) || m > uint32_t(kQszMaxM)) return set_error(QSIM_E_INVALID, "m=%u not in 5..26", m);
    if ((reinterpret_cast<uintptr_t>(d_amps) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
        return set_error(QSIM_E_INVALID, "device buffers must be 16-byte aligned");
    int e;
    if (!qsz_step_exponent(eb, &e)) return set_error(QSIM_E_INVALID, "error bound out of range");
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    DeviceCtx &c = device_ctx(dev);
    std::lock_guard<std::mutex> lk(c.mu);
    int rc = ensure_device_ctx(c);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    EncTarget t{};
    t.ptr = static_cast<uint8_t *>(d_out);
    t.cap = cap;
    EncResult r{};
    CUDA_TRY(cudaMemcpyAsync(c.tgt, &t, sizeof(t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c.res, &r, sizeof(r), cudaMemcpyHostToDevice, s));
    launch_encode(reinterpret_cast<const float2 *>(d_amps), 1, int(m), e, c.tgt, c.res, 0, nullptr, nullptr, nullptr,
                  make_scratch(c.lb_state, c.lb_ctr), c.status, s);
    CUDA_TRY(cudaMemcpyAsync(&r, c.res, sizeof(r), cudaMemcpyDeviceToHost, s));
    int code = read_status(c.status, s);
    if (code) return set_error(code, "compress: %s", status_text(code));
    *out_bytes = r.total;
    if (r.overflow) return set_error(QSIM_E_CAPACITY, "stream needs %llu bytes, cap is %zu",
                                     (unsigned long long)r.total, cap);
    return QSIM_OK;
}

int qsim_compress_block_rel(const float *d_amps, uint32_t m, double rel, void *d_out, size_t cap,
                            size_t *out_bytes, void *cuda_stream) {
    if (!d_amps || !d_out || !out_bytes) return set_error(QSIM_E_INVALID, "null argument");
    if (m < uint32_t(kQszMinM) || m > uint32_t(kQszMaxM)) return set_error(QSIM_E_INVALID, "m=%u not in 5..26", m);
    if ((reinterpret_cast<uintptr_t>(d_amps) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
        return set_error(QSIM_E_INVALID, "device buffers must be 16-byte aligned");
    int k;
    if (!qszr_shift(rel, &k)) return set_error(QSIM_E_INVALID, "relative bound out of range");
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    DeviceCtx &c = device_ctx(dev);
    std::lock_guard<std::mutex> lk(c.mu);
    int rc = ensure_device_ctx(c);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // scratch layout: block copy (8 B / amplitude), Im words (4 B), side records, then five per-frame arrays
    const uint64_t N = 1ull << m, nf = qsz_nframes(int(m));
    const size_t need = size_t(12 * N + nf * (kQszrSideBytes + 4 * 4 + 8));
    if (need > c.rel_cap) {
        if (c.rel_buf) CUDA_TRY(cudaFree(c.rel_buf));
        c.rel_buf = nullptr;
        c.rel_cap = 0;
        if (cudaMalloc(&c.rel_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QSIM_E_NOMEM, "relative-codec scratch of %zu bytes", need);
        }
        g_allocs.fetch_add(1, std::memory_order_relaxed);
        c.rel_cap = need;
    }
    float2 *wv = reinterpret_cast<float2 *>(c.rel_buf);
    uint32_t *im = reinterpret_cast<uint32_t *>(c.rel_buf + 8 * N);
    uint8_t *side = c.rel_buf + 12 * N;
    uint32_t *flen = reinterpret_cast<uint32_t *>(side + nf * kQszrSideBytes);
    uint32_t *fwords = flen + nf, *fmixed = fwords + nf, *foff = fmixed + nf;
    float2 *part = reinterpret_cast<float2 *>(foff + nf);
    CUDA_TRY(cudaMemcpyAsync(wv, d_amps, 8 * N, cudaMemcpyDeviceToDevice, s));
    EncTarget t{};
    t.ptr = static_cast<uint8_t *>(d_out);
    t.cap = cap;
    EncResult r{};
    CUDA_TRY(cudaMemcpyAsync(c.tgt, &t, sizeof(t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c.res, &r, sizeof(r), cudaMemcpyHostToDevice, s));
    const ArenaDev none{};
    launch_encode_ip(wv, im, 1, int(m), k, c.lb_ctr + 3, none, none, c.tgt, c.res, nullptr, side, flen, fwords, foff,
                     part, c.status, s, true, fmixed);
    launch_frame_copy(wv, im, 1, int(m), k, c.tgt, c.res, nullptr, nullptr, nullptr, side, flen, fwords, foff, s, true,
                      fmixed);
    CUDA_TRY(cudaMemcpyAsync(&r, c.res, sizeof(r), cudaMemcpyDeviceToHost, s));
    int code = read_status(c.status, s);
    if (code) return set_error(code, "compress_rel: %s", status_text(code));
    *out_bytes = r.total;
    if (r.overflow) return set_error(QSIM_E_CAPACITY, "stream needs %llu bytes, cap is %zu",
                                     (unsigned long long)r.total, cap);
    return QSIM_OK;
}

int qsim_decompress_block(const void *d_in, size_t in_bytes, float *d_amps, uint32_t m, void *cuda_stream) {
    if (!d_in || !d_amps) return set_error(QSIM_E_INVALID, "null argument");
    if (m < uint32_t(kQszMinM) || m > uint32_t(kQszMaxM)) return set_error(QSIM_E_INVALID, "m=%u not in 5..26", m);
    if ((reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_amps) & 15))
        return set_error(QSIM_E_INVALID, "device buffers must be 16-byte aligned");
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    DeviceCtx &c = device_ctx(dev);
    std::lock_guard<std::mutex> lk(c.mu);
    int rc = ensure_device_ctx(c);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    BlockRef r{static_cast<const uint8_t *>(d_in), in_bytes};
    uint32_t magic = 0;  // the format: QSZ1 or QSZR (any other value fails the kernel's header check)
    if (in_bytes >= 4) {
        CUDA_TRY(cudaMemcpyAsync(&magic, d_in, 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
    }
    CUDA_TRY(cudaMemcpyAsync(c.ref, &r, sizeof(r), cudaMemcpyHostToDevice, s));
    launch_decode(c.ref, 1, int(m), reinterpret_cast<float2 *>(d_amps), nullptr, c.status, s, magic == kQszrMagic);
    int code = read_status(c.status, s);
    if (code) return set_error(code, "decompress: %s", status_text(code));
    return QSIM_OK;
}

}  // extern "C"
