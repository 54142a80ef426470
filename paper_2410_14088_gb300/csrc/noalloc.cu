// Allocation-free single-block compressor.
//
// qsim_compress_block obtains its device scratch (the look-back words that
// let each frame find its byte offset, the ticket counters, a status word and
// the result record) with cudaMalloc the first time it runs on a device.
// Some callers cannot allow that: a host application whose framework already
// owns the device memory through its own pool, a service that must keep a
// fixed memory footprint after start-up, or a latency-critical loop in which
// cudaMalloc/cudaFree would synchronise the device. For them this file keeps
// the same scratch in one fixed array of device memory that is part of the
// loaded library image, so the entry point below never allocates.
//
// The array holds look-back words for up to 2^(QSIM_NOALLOC_MAX_M - 12)
// frames (blocks of up to 2^24 amplitudes: 32 KiB) plus 256 bytes of
// counters, status and result. Every GPU that loads the library keeps it until
// the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "codec.cuh"
#include "qsim_internal.h"

namespace qsim {

namespace {

constexpr uint32_t kNoAllocMaxFrames = 1u << (QSIM_NOALLOC_MAX_M - kQszMaxFrameLog);
constexpr size_t kLookbackBytes = size_t(kNoAllocMaxFrames) * sizeof(uint64_t);
// layout of the tail: counters [0,16), status [16,20), target [32,56), result [64,96)
constexpr size_t kTailBytes = 256;
constexpr size_t kScratchBytes = kLookbackBytes + kTailBytes;

// the fixed scratch; host code must not use this name as an address
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch on that device
};

std::mutex g_noalloc_mu;
DeviceScratch g_noalloc_dev[64];

// Once per device, with that device current: look up the array's device
// address. The first call on a device does this.
int scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(QSIM_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return set_error(QSIM_E_INVALID, "device index %d out of range", dev);
    DeviceScratch &d = g_noalloc_dev[dev];
    if (!d.base) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(QSIM_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        d.base = static_cast<unsigned char *>(p);
    }
    *out = d.base;
    return QSIM_OK;
}

}  // namespace

}  // namespace qsim

using namespace qsim;

extern "C" int qsim_compress_block_noalloc(const float *d_amps, uint32_t m, double eb, void *d_out, size_t cap,
                                           size_t *out_bytes, void *cuda_stream) {
    if (!d_amps || !d_out || !out_bytes) return set_error(QSIM_E_INVALID, "null argument");
    if (m < uint32_t(kQszMinM)) return set_error(QSIM_E_INVALID, "m=%u below 5", m);
    if (m > uint32_t(QSIM_NOALLOC_MAX_M))
        return set_error(QSIM_E_INVALID,
                         "qsim_compress_block_noalloc: m=%u exceeds %d (its fixed scratch covers %u frames); "
                         "use qsim_compress_block for larger blocks",
                         m, QSIM_NOALLOC_MAX_M, kNoAllocMaxFrames);
    if ((reinterpret_cast<uintptr_t>(d_amps) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
        return set_error(QSIM_E_INVALID, "device buffers must be 16-byte aligned");
    int e;
    if (!qsz_step_exponent(eb, &e)) return set_error(QSIM_E_INVALID, "error bound out of range");

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned char *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint64_t *lookback = reinterpret_cast<uint64_t *>(base);
    unsigned char *tail = base + kLookbackBytes;
    uint32_t *counters = reinterpret_cast<uint32_t *>(tail);
    int *status = reinterpret_cast<int *>(tail + 16);
    EncTarget *tgt = reinterpret_cast<EncTarget *>(tail + 32);
    EncResult *res = reinterpret_cast<EncResult *>(tail + 64);

    // The array keeps the previous call's contents: clear the look-back words
    // of the frames this block uses and the whole tail (counters, status,
    // result) so the encoder starts from zero.
    const size_t nframes = size_t(qsz_nframes(int(m)));
    cudaError_t ce = cudaMemsetAsync(lookback, 0, nframes * sizeof(uint64_t), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(tail, 0, kTailBytes, s);
    EncTarget t;
    memset(&t, 0, sizeof(t));
    t.ptr = static_cast<uint8_t *>(d_out);
    t.cap = cap;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(tgt, &t, sizeof(t), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return set_error(QSIM_E_CUDA, "scratch set-up: %s", cudaGetErrorString(ce));

    LookbackScratch scr{};
    scr.state = lookback;
    scr.ticket = counters;
    scr.done = counters + 1;
    scr.epoch = counters + 2;
    launch_encode(reinterpret_cast<const float2 *>(d_amps), 1, int(m), e, tgt, res, 0, nullptr, nullptr, nullptr, scr,
                  status, s);

    EncResult r;
    int h_status = 0;
    ce = cudaMemcpyAsync(&r, res, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    // Once the encoder is queued, wait for the stream on every path, failed copies included: the next call
    // (possibly on another stream) clears the shared array and must not do so under a running encoder.
    const cudaError_t se = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) return set_error(QSIM_E_CUDA, "compress (no-alloc): %s", cudaGetErrorString(ce));
    if (h_status) return set_error(h_status, "compress (no-alloc): device status %d", h_status);
    *out_bytes = size_t(r.total);
    if (r.overflow)
        return set_error(QSIM_E_CAPACITY, "stream needs %llu bytes, cap is %zu", (unsigned long long)r.total, cap);
    return QSIM_OK;
}
