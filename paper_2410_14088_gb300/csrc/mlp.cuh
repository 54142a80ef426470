// Learned block-size predictor (device side): constants and launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"

namespace qsim {

constexpr int kMlpIn = 41, kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;

// eight per-stage inputs of the predictor
struct StageFeatures {
    float v[8];
};

// forward of one sample with the weights in shared memory (layout of qsim.h)
__device__ __forceinline__ float mlp_forward_one(const float *w, const float *x) {
    constexpr int IN = kMlpIn, HID = kMlpHidden;
    constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
                  OB3 = OW3 + HID;
    float h1[HID];
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float a = w[OB1 + i];
        for (int j = 0; j < IN; ++j) a = fmaf(w[OW1 + i * IN + j], x[j], a);
        h1[i] = fmaxf(a, 0.f);
    }
    float y = w[OB3];
    for (int i = 0; i < HID; ++i) {
        float a = w[OB2 + i];
#pragma unroll
        for (int j = 0; j < HID; ++j) a = fmaf(w[OW2 + i * HID + j], h1[j], a);
        y = fmaf(w[OW3 + i], fmaxf(a, 0.f), y);
    }
    return y;
}

// the 41 inputs of block j of a batch: its SV group's code-width histogram (each 32-value chunk of the decoded
// input counts 32 in the bin of its width; G blocks of 2^(m+1) values each, hist read through L2), the largest
// populated bin / 32 and the stage features
__device__ __forceinline__ void mlp_features(const uint32_t *hist, uint32_t j, uint32_t G, int m,
                                             const StageFeatures &sf, float *x) {
    const float inv = 1.0f / (float(G) * float(2ull << m));
    const uint64_t g0 = uint64_t(j / G) * G;
    int maxb = 0;
    for (int b = 0; b < 32; ++b) {
        uint32_t c = 0;
        for (uint32_t jj = 0; jj < G; ++jj) c += __ldcg(hist + (g0 + jj) * 32 + b);
        x[b] = float(c) * inv;
        if (c) maxb = b;
    }
    x[32] = float(maxb) / 32.f;
    for (int t = 0; t < 8; ++t) x[33 + t] = sf.v[t];
}

void launch_mlp_forward(const float *params, const float *x, uint32_t batch, float *y, int bf16, cudaStream_t s);
// features from the decoder's histogram (+ stage features) -> predicted log2 bytes; feat_out (nullable) receives
// rows of kMlpIn features followed by one target slot
void launch_predict_sizes(const uint32_t *hist, uint32_t nblocks, uint32_t G, int m, const StageFeatures &sf,
                          const float *params, int bf16, float *pred, float *feat_out, cudaStream_t s);
void launch_log_targets(const EncResult *res, uint32_t nblocks, int m, float *rows, cudaStream_t s);
int launch_mlp_loss_grad(const float *params, const float *x, uint32_t xstride, const float *t, uint32_t tstride,
                         const uint32_t *perm, uint32_t start, uint32_t count, float *grad, float *loss,
                         cudaStream_t s);
void launch_adam(float *p, const float *g, float *m1, float *m2, uint32_t n, int t, float lr, float beta1, float beta2,
                 float eps, cudaStream_t s);

}  // namespace qsim
