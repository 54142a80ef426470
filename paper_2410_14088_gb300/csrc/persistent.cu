// Persistent stage kernel (sm_103a): one launch runs a whole stage.
//
// The paper overlaps the SV groups of a stage by dealing them round-robin to
// CUDA streams (Sec. 4.2). Here the same overlap happens inside one launch:
// every CTA repeatedly takes the next work item from a global queue, whose
// order is, group after group, the group's phases
//     decode frames -> [predict + reserve] -> gate-pass tiles (pass by pass)
//     -> [sizing frames] -> encode frames -> [exact re-reserve -> re-encode]
// and waits (bounded spin) until the group's previous phase is complete
// before running its item. Groups are independent (Sec. 4.1), so different
// CTAs work on different phases of different groups at the same time, and a
// group's work item only waits on items that come earlier in the queue, which
// were taken by CTAs that are already running: the schedule cannot deadlock
// even when not every CTA is resident. Working vectors live in slots planned
// on the host: one ring of slots per working-vector size, so that many small
// groups can be in flight next to a few large ones; the first item of a group
// also waits for the slot's previous group (earlier in the queue) to finish.
//
// Data produced by other CTAs of the same launch is read through L2 (ld.cg),
// since the per-SM L1 caches are not coherent within a launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "codec_dev.cuh"
#include "device_common.cuh"
#include "gates.cuh"
#include "gates_dev.cuh"
#include "mlp.cuh"
#include "persistent.cuh"

namespace qsim {

namespace {

using cdev::FrameGeom;
using cdev::geom;

// threads per CTA: one warp per frame of a frame-parallel item
template <bool UM>
constexpr int kPT = 32 * int(persistent_frames_per_item(UM));

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ EncTarget load_target(const EncTarget *t) {
    EncTarget r;
    r.ptr = reinterpret_cast<uint8_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&t->ptr)));
    r.cap = __ldcg(reinterpret_cast<const unsigned long long *>(&t->cap));
    r.tier = __ldcg(&t->tier);
    r.pad = 0;
    return r;
}

// REL: the relative-bound codec (QSZR) in the decode phase and the in-place exact phases. UM: the plan's dense ops
// of width 3 to 5 (TF32 or split BF16) and 6 (TF32) run on tcgen05 (TMEM accumulator and MMA mbarrier held by each
// CTA for the launch).
template <int PREC, bool REL, bool UM>
__global__ void __launch_bounds__(kPT<UM>, 512 / kPT<UM>) k_stage_persistent(PLaunch L) {
    constexpr int PT = kPT<UM>;
    extern __shared__ float4 dsm[];
    __shared__ gdev::PassSmem PS;
    __shared__ uint32_t s_wb[PT / 32][64];
    __shared__ OpDev s_pre[kMaxPreOps];
    __shared__ uint2 s_pre_ab[kMaxPreOps];
    __shared__ __align__(16) PSeg S;
    __shared__ uint32_t s_hist[PT / 32][32];
    __shared__ uint32_t s_item, s_epoch, s_seg, s_next;
    __shared__ uint32_t s_pcache[2];  // key (segment x 256 + pass) of the pass staged in dsm; its B resident
    __shared__ int s_flag, s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        s_epoch = ld_relaxed_u32(L.ctr + 2) & cdev::kEpochMask;
        s_seg = ~0u;
        s_pcache[0] = ~0u;
        s_pcache[1] = 0;
    }
    uint32_t mphase = 0;     // parity of the MMA mbarrier's next phase (UM)
    bool mma_ok = true;      // false after an MMA wait ran out (then a last bounded wait before TMEM is freed)
    if constexpr (UM) {
        if (warp == 0) umma::tmem_alloc(umma::smem_addr(&PS.tmem), gdev::umma_pass_tmem_cols(0));
        if (tid == 0) umma::mbar_init(umma::smem_addr(&PS.mbar), 1);
        umma::fence_before_sync();
    }
    __syncthreads();
    if constexpr (UM) umma::fence_after_sync();

    // thread 0: the next item, claimed one item ahead so that the claim's latency hides under the current item
    // (every dependency points to an earlier item, and the grid is one wave of resident CTAs, so the smallest
    // unfinished item is always some CTA's current item and the queue keeps moving)
    uint32_t nx_item = 0;
    // thread 0: the (launch group, phase) whose dependencies this CTA last saw met; later items of the same
    // phase of the same group skip the wait (the counters only grow within a launch)
    uint64_t dep_key = ~0ull;
    if (tid == 0) nx_item = atomicAdd(L.ctr, 1u);
    // thread 0: a done counter of a per-item phase whose increments this CTA holds back, and their number; they are
    // added (after a fence) when the CTA completes an item of another phase, before it waits on any dependency and
    // when it leaves, so a CTA that waits never holds counts another CTA waits for
    uint32_t *pend_done = nullptr;
    uint32_t pend_cnt = 0;
    auto flush = [&]() {
        if (pend_cnt) {
            __threadfence();
            atomicAdd(pend_done, pend_cnt);
            pend_cnt = 0;
        }
    };
    // thread 0: wait for the item's dependencies (the group's previous phase; for its first phase the slot's
    // previous group and the circuit's previous stage); returns 1 when the item must skip its work (a device
    // error, or a wait that ran out)
    auto deps = [&](uint32_t it) -> int {
        const uint32_t rel = uint32_t(it - S.item_begin);
        const uint32_t grp = rel / S.per_group, r = rel % S.per_group;
        const uint32_t q = S.group_begin + grp;
        uint32_t p = 0;
        while (p + 1 < S.nphases && r >= S.ph_start[p + 1]) ++p;
        const uint64_t key = uint64_t(q) * kMaxPhases + p;
        if (key == dep_key) return ld_relaxed_u32(reinterpret_cast<const uint32_t *>(L.status)) != 0;
        flush();
        const uint32_t *flag = nullptr, *flag2 = nullptr;
        uint32_t need = 0;
        if (p > 0) {
            flag = L.done + uint64_t(q) * kMaxPhases + p - 1;
            need = S.ph[p - 1].count;
        } else {
            const uint32_t prev = L.g_prev[q];
            if (prev != kNoGroup) {  // the slot's previous group must have finished
                flag = L.done + uint64_t(prev) * kMaxPhases + kMaxPhases - 1;
                need = 1;
            }
            flag2 = S.prev_flag;
        }
        if (S.stall_test && grp == 0 && p == 1) ++need;  // never reached: exercises the time limit
        bool met = true;
        if (flag || flag2) {
            const uint64_t t0 = global_ns();
            while ((flag && ld_acquire_u32(flag) < need) || (flag2 && ld_acquire_u32(flag2) == 0)) {
                if (global_ns() - t0 > L.wait_ns) {
                    raise_status(L.status, QSIM_E_TIMEOUT);
                    met = false;
                    break;
                }
                __nanosleep(256);
            }
        }
        if (met) dep_key = key;
        // after any device error the remaining items only keep the schedule going
        return (!met || ld_relaxed_u32(reinterpret_cast<const uint32_t *>(L.status)) != 0) ? 1 : 0;
    };

    while (true) {
        if (tid == 0) {
            const uint32_t it = nx_item;
            s_item = it;
            // the segment holding the item: last one with item_begin <= item
            uint32_t lo = 0;
            if (it < L.total_items) {
                nx_item = atomicAdd(L.ctr, 1u);
                uint32_t hi = L.nseg - 1;
                if (s_seg != ~0u && it >= S.item_begin && it - S.item_begin < uint64_t(S.ngroups) * S.per_group)
                    lo = hi = s_seg;  // still in the segment whose descriptor is staged
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(reinterpret_cast<const unsigned long long *>(&L.segs[mid].item_begin)) <= it)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
            }
            s_next = lo;
            // the current segment's descriptor is in S: check the dependencies before the barrier
            if (it < L.total_items && lo == s_seg) s_abort = deps(it);
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= L.total_items) break;
        const uint32_t want = s_next;
        if (want != s_seg) {  // uniform: a new segment, load its descriptor and leading phase ops
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(L.segs + want);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&S);
            for (int t = tid; t < int(sizeof(PSeg) / 8); t += PT) dst[t] = __ldg(src + t);
            __syncthreads();
            if (tid < int(S.npre)) {
                s_pre[tid] = S.ops[S.pre_begin + tid];
                s_pre_ab[tid] = cdev::pre_setup(S.ops[S.pre_begin + tid]);
            }
            if (tid == 0) {
                s_seg = want;
                s_abort = deps(item);
            }
            __syncthreads();
        }
        const FrameGeom g = geom(int(S.m));
        const uint32_t nph = S.nphases;
        const uint32_t gframes = S.G * g.nframes;
        const uint32_t rel = uint32_t(item - S.item_begin);
        const uint32_t grp = rel / S.per_group, r = rel % S.per_group;
        const uint32_t q = S.group_begin + grp;  // the group's number in this launch
        uint32_t p = 0;
        while (p + 1 < nph && r >= S.ph_start[p + 1]) ++p;
        const uint32_t i = r - S.ph_start[p];
        const uint32_t type = S.ph[p].type;
        const bool abort_item = s_abort != 0;
        float2 *wv = L.wv + L.g_wv[q];
        float2 *part = L.part + L.g_frame[q];
        const uint32_t *ids = S.ids + uint64_t(grp) * S.G;
        const uint64_t gb = S.gbase[grp];
        const uint64_t bbase = uint64_t(grp) * S.G;  // per-group block arrays
        const uint32_t sf0 = L.g_frame[q];  // the slot's first frame in wrec / flen / foff / part / lb
        bool by_arrival = type == PH_ENCODE || type == PH_REENCODE || type == PH_SIZE_W ||
                          type == PH_ENCODE_W || type == PH_ENCODE_IP || type == PH_COPY;
        if (abort_item) {
            // skip the work, keep the counts
        } else if (type == PH_DECODE) {
            const uint32_t fi = i * (PT / 32) + warp;
            if (fi < gframes) {
                const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                const BlockSlot sl = S.tab_in[ids[jj]];
                cdev::decode_frame_warp<kMaxPreOps, false, REL>(sl.ptr, sl.bytes, g, int(S.m), f,
                                                    wv + (uint64_t(jj) << S.m) + uint64_t(f) * g.F,
                                                    S.hist ? S.hist + (bbase + jj) * 32 : nullptr, s_hist[warp],
                                                    L.status, s_pre, s_pre_ab, S.npre, S.mats,
                                                    uint64_t(jj) << S.m, gb);
            }
        } else if (type == PH_PASS) {
            if constexpr (UM) {
                // tile loads by cp.async (L1-cached): the item's dependencies were acquired by thread 0 (for this
                // group and phase, in this item or an earlier one of this CTA) before the CTA barrier above, so the
                // memory model orders them after the previous phase's writes; L1 starts empty at the launch
                mma_ok &= gdev::pass_tile<PT, 5, PREC, false, true>(wv, S.passes[S.ph[p].arg], S.blob, S.mats, S.bfr,
                                                                   i, gb, PS, reinterpret_cast<float2 *>(dsm),
                                                                   L.status, &mphase, s_pcache,
                                                                   s_seg * 256u + S.ph[p].arg);
            } else {
                gdev::pass_tile<PT, 5, PREC, false>(wv, S.passes[S.ph[p].arg], S.blob, S.mats, S.bfr, i, gb, PS,
                                                   reinterpret_cast<float2 *>(dsm), L.status, nullptr, s_pcache,
                                                   s_seg * 256u + S.ph[p].arg);
            }
        } else if (REL && type == PH_ENCODE_IP) {
            if constexpr (REL) {
                const uint32_t fi = i * (PT / 32) + warp;
                if (fi < gframes) {
                    const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                    const uint64_t a0 = (uint64_t(jj) << S.m) + uint64_t(f) * g.F;
                    uint32_t words, mixed;
                    const uint32_t len = cdev::encode_frame_warp_ip<true, true>(
                        wv + a0, L.im + L.g_wv[q] + a0, g, S.e, L.wrec + uint64_t(sf0 + fi) * kQszrSideBytes, words,
                        mixed, part + fi, L.status);
                    if ((tid & 31) == 0) {
                        L.flen[sf0 + fi] = len;
                        L.fwords[sf0 + fi] = words;
                        L.fmixed[sf0 + fi] = mixed;
                        __threadfence();  // read by the phase's last item and the copy phase on other CTAs
                    }
                }
            }
        } else if (REL && type == PH_COPY) {
            if constexpr (REL) {
                const uint32_t fi = i * (PT / 32) + warp;
                if (fi < gframes) {
                    const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                    const uint64_t a0 = (uint64_t(jj) << S.m) + uint64_t(f) * g.F;
                    cdev::copy_frame_warp<true>(reinterpret_cast<const uint32_t *>(wv + a0), L.im + L.g_wv[q] + a0,
                                                L.wrec + uint64_t(sf0 + fi) * kQszrSideBytes,
                                                __ldcg(L.fwords + sf0 + fi), __ldcg(L.fmixed + sf0 + fi),
                                                __ldcg(L.flen + sf0 + fi), __ldcg(L.foff + sf0 + fi), g, int(S.m),
                                                S.e, f, load_target(&S.tgt[bbase + jj]), &S.res[bbase + jj],
                                                S.tab_out + ids[jj], S.acc);
                }
            }
        } else if (type == PH_SIZE_W) {
            const uint32_t fi = i * (PT / 32) + warp;
            if (fi < gframes) {
                const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                const uint32_t len = cdev::size_frame_warp<true>(wv + (uint64_t(jj) << S.m) + uint64_t(f) * g.F, g,
                                                                 S.e, L.wrec + uint64_t(sf0 + fi) * 256, L.status);
                if ((tid & 31) == 0) {
                    L.flen[sf0 + fi] = len;
                    __threadfence();  // read by the phase's last item on another CTA
                }
            }
        } else if (type == PH_ENCODE_W) {
            const uint32_t fi = i * (PT / 32) + warp;
            if (fi < gframes) {
                const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                cdev::encode_frame_warp_known<true>(wv + (uint64_t(jj) << S.m) + uint64_t(f) * g.F, g, int(S.m), S.e,
                                                    f, L.wrec + uint64_t(sf0 + fi) * 256, __ldcg(L.foff + sf0 + fi),
                                                    __ldcg(L.flen + sf0 + fi), load_target(&S.tgt[bbase + jj]),
                                                    &S.res[bbase + jj], S.tab_out + ids[jj], S.acc, part + fi,
                                                    L.status);
            }
        } else if (type == PH_PREDICT) {
            float *w = reinterpret_cast<float *>(dsm);
            if (tid == 0) s_pcache[0] = ~0u;  // dsm is overwritten: no pass stays staged
            for (int t = tid; t < kMlpParams; t += PT) {
                const float v = S.pparams[t];
                w[t] = S.pbf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
            }
            __syncthreads();
            for (uint32_t jj = tid; jj < S.G; jj += PT) {
                float x[kMlpIn];
                mlp_features(S.hist + bbase * 32, jj, S.G, int(S.m), S.sf, x);
                double pr = double(mlp_forward_one(w, x)) + double(S.m + 3);
                pr = pr < 0 ? 0 : (pr > 40 ? 40 : pr);
                const double want_b = exp2(pr) * (1.0 + S.margin);
                EncResult &rs = S.res[bbase + jj];
                rs.total = 0;
                rs.overflow = 0;
                rs.err_sq = 0;
                rs.norm_sq = 0;
                cdev::reserve_slot(want_b >= double(S.worst) ? S.worst : uint64_t(want_b), S.dev, S.host,
                                   &S.tgt[bbase + jj], L.status);
            }
            __syncthreads();
            // the group's histograms are consumed: leave them zero for the next stage
            for (uint32_t t = tid; t < S.G * 32; t += PT) S.hist[bbase * 32 + t] = 0;
        } else if (type == PH_ENCODE || type == PH_REENCODE) {
            // learned sizing: one frame per warp, offsets by warp look-back
            const uint32_t fi = i * (PT / 32) + warp;
            const bool retry = type == PH_REENCODE;
            if (fi < gframes) {
                const uint32_t jj = fi / g.nframes, f = fi % g.nframes;
                if (!retry || __ldcg(&S.res[bbase + jj].overflow) != 0) {
                    const uint32_t epoch = (s_epoch + 2 * q + (retry ? 1 : 0)) & cdev::kEpochMask;
                    cdev::encode_frame_warp_lb<true>(wv + (uint64_t(jj) << S.m) + uint64_t(f) * g.F, g, int(S.m), S.e,
                                                     f, L.lb + L.g_frame[q] + uint64_t(jj) * g.nframes, epoch,
                                                     load_target(&S.tgt[bbase + jj]), &S.res[bbase + jj],
                                                     S.tab_out + ids[jj], S.acc, retry ? nullptr : part + fi,
                                                     s_wb[warp], L.status);
                }
            }
        } else if (type == PH_FIX) {
            for (uint32_t jj = tid; jj < S.G; jj += PT) {
                EncResult &rs = S.res[bbase + jj];
                if (__ldcg(&rs.overflow))
                    cdev::reserve_slot(__ldcg(reinterpret_cast<const unsigned long long *>(&rs.total)), S.dev, S.host,
                                       &S.tgt[bbase + jj], L.status);
            }
        }
        // ---- completion ----
        __syncthreads();
        uint32_t *done = L.done + uint64_t(q) * kMaxPhases + p;
        if (!by_arrival) {
            if (tid == 0) {
                if (done != pend_done) {
                    flush();
                    pend_done = done;
                }
                ++pend_cnt;
            }
            continue;
        }
        if (tid == 0) {
            __threadfence();
            s_flag = atomicAdd(L.arrive + uint64_t(q) * kMaxPhases + p, 1u) == S.ph[p].count - 1;
        }
        __syncthreads();
        if (!s_flag) continue;
        __threadfence();
        if (abort_item) {
            // no reservation or statistics after an error
        } else if (type == PH_SIZE_W || type == PH_ENCODE_IP) {
            // the group's frame lengths are complete: frame offsets (warp per block) and the group's slots (the
            // in-place phase with learned sizing keeps every predicted slot its block fits)
            const int lane = tid & 31;
            for (uint32_t jj = warp; jj < S.G; jj += PT / 32) {
                uint32_t run = uint32_t(S.data_start);
                for (uint32_t f0 = 0; f0 < g.nframes; f0 += 32) {
                    const uint32_t fi = sf0 + jj * g.nframes + f0 + lane;
                    const uint32_t v = f0 + lane < g.nframes ? __ldcg(L.flen + fi) : 0u;
                    uint32_t incl = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += t;
                    }
                    if (f0 + lane < g.nframes) L.foff[fi] = run + incl - v;
                    run += __shfl_sync(kFull, incl, 31);
                }
                if (lane == 0) {
                    EncResult &rs = S.res[bbase + jj];
                    rs.total = 0;
                    rs.overflow = 0;
                    rs.err_sq = 0;
                    rs.norm_sq = 0;
                    EncTarget &t = S.tgt[bbase + jj];
                    if (type == PH_ENCODE_IP && S.pparams) {
                        if (t.ptr == nullptr || run > t.cap) {
                            atomicAdd(reinterpret_cast<unsigned long long *>(&S.acc->overflow_blocks), 1ull);
                            cdev::reserve_slot(run, S.dev, S.host, &t, L.status);
                        }
                    } else {
                        cdev::reserve_slot(run, S.dev, S.host, &t, L.status);
                    }
                }
            }
        }
        if (!abort_item && (type == PH_ENCODE || type == PH_ENCODE_W || type == PH_ENCODE_IP)) {
            // the group's frames are encoded: fold their error partials into the stage totals
            double a = 0, b = 0;
            for (uint32_t t = tid; t < gframes; t += PT) {
                const float2 v = __ldcg(part + t);
                a += double(v.x);
                b += double(v.y);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                a += __shfl_xor_sync(kFull, a, o);
                b += __shfl_xor_sync(kFull, b, o);
            }
            if ((tid & 31) == 0) {
                atomicAdd(&S.acc->err_sq, a);
                atomicAdd(&S.acc->norm_sq, b);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicExch(done, S.ph[p].count);
            if (p == nph - 1) {
                // the group is finished: its slot may be reused; the stage may be complete
                atomicExch(L.done + uint64_t(q) * kMaxPhases + kMaxPhases - 1, 1u);
                if (atomicAdd(S.fin_count, 1u) == S.ngroups - 1) {
                    if (S.reset_bumps) {
                        // every group of the stage has read its input arena: the next stage writes there
                        S.reset_bumps[0] = 0;
                        S.reset_bumps[1] = 0;
                    }
                    __threadfence();
                    atomicExch(S.fin_flag, 1u);
                }
            }
        }
    }
    if (tid == 0) flush();
    if constexpr (UM) {
        // after an MMA wait that ran out, wait (bounded) once more for that op's MMAs before TMEM is freed
        if (!mma_ok) umma::mbar_wait(umma::smem_addr(&PS.mbar), mphase ^ 1u, gdev::kUmmaWaitNs);
        umma::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            umma::fence_after_sync();
            umma::tmem_dealloc(PS.tmem, gdev::umma_pass_tmem_cols(0));
        }
    }
    // the last CTA out resets the queue and advances the look-back epoch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(L.ctr + 1, 1u) == gridDim.x - 1) {
            L.ctr[0] = 0;
            L.ctr[1] = 0;
            __threadfence();
            atomicExch(L.ctr + 2, (s_epoch + 2 * L.total_groups) & cdev::kEpochMask);
        }
    }
}

template <int PREC, bool REL, bool UM>
struct LaunchShape {
    static int grid;
    static size_t attr_smem;
};
template <int PREC, bool REL, bool UM> int LaunchShape<PREC, REL, UM>::grid = 0;
template <int PREC, bool REL, bool UM> size_t LaunchShape<PREC, REL, UM>::attr_smem = 0;

// kernel attributes and the grid (one wave of resident CTAs); done outside any stream capture
template <int PREC, bool REL, bool UM>
int prepare_prec(size_t smem) {
    using Shape = LaunchShape<PREC, REL, UM>;
    if (Shape::attr_smem < smem) {
        if (cudaFuncSetAttribute(k_stage_persistent<PREC, REL, UM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem)) != cudaSuccess)
            return QSIM_E_CUDA;
        Shape::attr_smem = smem;
        Shape::grid = 0;
    }
    if (!Shape::grid) {
        // resident CTAs per SM from the kernel's registers and shared memory and the SM's limits (65536 registers,
        // 2048 threads, 228 KB of shared memory with 1 KB reserved per CTA); the runtime's occupancy query was
        // seen to answer 1 where more CTAs were resident
        int dev = 0, sms = 0, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, k_stage_persistent<PREC, REL, UM>) == cudaSuccess) {
            const int regs = ((fa.numRegs > 0 ? fa.numRegs : 255) + 7) & ~7;
            constexpr int PT = kPT<UM>;
            const int by_regs = 65536 / (regs * PT);
            const int by_smem = int((228u * 1024u) / (smem + fa.sharedSizeBytes + 1024u));
            per_sm = by_regs < by_smem ? by_regs : by_smem;
            if (per_sm > 2048 / PT) per_sm = 2048 / PT;
            // each CTA of a tcgen05 launch holds its TMEM columns for the launch: no more than the SM's 512
            if (UM && per_sm > int(512u / gdev::umma_pass_tmem_cols(0))) per_sm = int(512u / gdev::umma_pass_tmem_cols(0));
            if (per_sm < 1) per_sm = 1;
        }
        Shape::grid = (sms > 0 ? sms : 1) * per_sm;
    }
    return QSIM_OK;
}

template <int PREC, bool REL, bool UM>
int launch_stage_prec(const PLaunch &a, size_t smem, cudaStream_t s, int *grid_out) {
    using Shape = LaunchShape<PREC, REL, UM>;
    if (Shape::attr_smem < smem || !Shape::grid) return QSIM_E_INVALID;
    const int grid = Shape::grid;
    k_stage_persistent<PREC, REL, UM><<<grid, kPT<UM>, smem, s>>>(a);
    if (grid_out) *grid_out = grid;
    count_launch();
    return QSIM_OK;
}

// tcgen05 (um) only for TF32: the split-BF16 form keeps 128-thread CTAs, which this kernel does not have
template <bool REL>
int prepare_codec(int prec, size_t smem, bool um) {
    if (prec == QSIM_PREC_TF32)
        return um ? prepare_prec<QSIM_PREC_TF32, REL, true>(smem) : prepare_prec<QSIM_PREC_TF32, REL, false>(smem);
    if (prec == QSIM_PREC_BF16X3)
        return um ? prepare_prec<QSIM_PREC_BF16X3, REL, true>(smem) : prepare_prec<QSIM_PREC_BF16X3, REL, false>(smem);
    return prepare_prec<QSIM_PREC_FP32, REL, false>(smem);
}

template <bool REL>
int launch_codec(const PLaunch &a, int prec, size_t smem, cudaStream_t s, int *grid, bool um) {
    if (prec == QSIM_PREC_TF32)
        return um ? launch_stage_prec<QSIM_PREC_TF32, REL, true>(a, smem, s, grid)
                  : launch_stage_prec<QSIM_PREC_TF32, REL, false>(a, smem, s, grid);
    if (prec == QSIM_PREC_BF16X3)
        return um ? launch_stage_prec<QSIM_PREC_BF16X3, REL, true>(a, smem, s, grid)
                  : launch_stage_prec<QSIM_PREC_BF16X3, REL, false>(a, smem, s, grid);
    return launch_stage_prec<QSIM_PREC_FP32, REL, false>(a, smem, s, grid);
}

}  // namespace

size_t persistent_smem_bytes(size_t pass_bytes) {
    const size_t mlp = size_t(kMlpParams) * sizeof(float);
    return pass_bytes > mlp ? pass_bytes : mlp;
}

int prepare_stage_persistent(int prec, size_t smem, bool rel, bool um) {
    return rel ? prepare_codec<true>(prec, smem, um) : prepare_codec<false>(prec, smem, um);
}

int launch_stage_persistent(const PLaunch &a, int prec, size_t smem, cudaStream_t s, int *grid, bool rel, bool um) {
    return rel ? launch_codec<true>(a, prec, smem, s, grid, um) : launch_codec<false>(a, prec, smem, s, grid, um);
}

}  // namespace qsim
