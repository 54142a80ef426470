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
