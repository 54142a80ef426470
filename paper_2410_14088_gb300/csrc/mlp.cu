// Learned block-size predictor: a 41 -> 64 -> 64 -> 1 ReLU MLP, with its own
// forward, loss/gradient and Adam kernels (sm_103a).
//
// The paper handles the unpredictable size of compressed blocks with a second
// memory level (Sec. 4.4). Here the size of each block's next stream is
// predicted from cheap statistics so that a slot can be reserved before the
// block is encoded, without a sizing pass; an under-estimate falls back to an
// exact re-encode.
//
// Inputs (x, 41 floats): the 32-bin histogram of code bit lengths
// (bit length of |q|, as fractions of the 2^(m+1) values of each block of the
// block's SV group, which the stage mixes), the largest bit length / 32, and
// 8 stage features. Output: log2(stream bytes) - (m + 3),
// i.e. minus the log2 of the block's compression ratio.
// Parameter layout (6913 floats): W1[64][41], b1[64], W2[64][64], b2[64],
// W3[64], b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "codec.cuh"
#include "device_common.cuh"
#include "mlp.cuh"

namespace qsim {

namespace {

constexpr int IN = kMlpIn, HID = kMlpHidden, NP = kMlpParams;
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + HID;

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void load_weights(float *w, const float *params, bool bf16) {
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = bf16 ? round_bf16(params[i]) : params[i];
}

__global__ void k_mlp_forward(const float *__restrict__ params, const float *__restrict__ x, uint32_t batch,
                              float *__restrict__ y, int bf16) {
    __shared__ float w[NP];
    load_weights(w, params, bf16 != 0);
    __syncthreads();
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
        float xs[IN];
        for (int j = 0; j < IN; ++j) xs[j] = x[uint64_t(b) * IN + j];
        y[b] = mlp_forward_one(w, xs);
    }
}

// Features of each block of a batch from the decoder's bit-length histogram,
// then the prediction; optionally the features are also written out (for
// the training log, completed by the target once the exact size is known).
// One warp per block: the features (the SV group's width histogram, the largest
// populated bin, the stage features), then the forward pass with the hidden
// units spread over the lanes (two per lane per layer).
__global__ void __launch_bounds__(128) k_predict_sizes(const uint32_t *__restrict__ hist, uint32_t nblocks,
                                                       uint32_t G, int m, StageFeatures sf,
                                                       const float *__restrict__ params, int bf16,
                                                       float *__restrict__ pred, float *__restrict__ feat_out) {
    __shared__ float w[NP];
    __shared__ float xs[4][IN + 1];
    __shared__ float hs[4][HID];
    if (params) load_weights(w, params, bf16 != 0);
    __syncthreads();
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const float inv = 1.0f / (float(G) * float(2ull << m));
    for (uint32_t j = blockIdx.x * 4 + wi; j < nblocks; j += gridDim.x * 4) {
        // a stage mixes the G blocks of an SV group, so the histogram is the group's
        const uint64_t g0 = uint64_t(j / G) * G;
        uint32_t c = 0;
        for (uint32_t jj = 0; jj < G; ++jj) c += __ldcg(hist + (g0 + jj) * 32 + lane);
        const uint32_t nz = __ballot_sync(0xffffffffu, c != 0);
        xs[wi][lane] = float(c) * inv;
        if (lane == 0) xs[wi][32] = float(nz ? 31 - __clz(nz) : 0) / 32.f;
        if (lane < 8) xs[wi][33 + lane] = sf.v[lane];
        __syncwarp();
        if (feat_out)
            for (int t = lane; t < IN; t += 32) feat_out[uint64_t(j) * (IN + 1) + t] = xs[wi][t];
        if (params && pred) {
            float a0 = w[OB1 + lane], a1 = w[OB1 + lane + 32];
            for (int t = 0; t < IN; ++t) {
                const float x = xs[wi][t];
                a0 = fmaf(w[OW1 + lane * IN + t], x, a0);
                a1 = fmaf(w[OW1 + (lane + 32) * IN + t], x, a1);
            }
            hs[wi][lane] = fmaxf(a0, 0.f);
            hs[wi][lane + 32] = fmaxf(a1, 0.f);
            __syncwarp();
            float b0 = w[OB2 + lane], b1 = w[OB2 + lane + 32];
            for (int t = 0; t < HID; ++t) {
                const float h = hs[wi][t];
                b0 = fmaf(w[OW2 + lane * HID + t], h, b0);
                b1 = fmaf(w[OW2 + (lane + 32) * HID + t], h, b1);
            }
            float y = w[OW3 + lane] * fmaxf(b0, 0.f) + w[OW3 + lane + 32] * fmaxf(b1, 0.f);
#pragma unroll
            for (int o = 16; o; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if (lane == 0) pred[j] = y + w[OB3] + float(m + 3);
        }
        __syncwarp();
    }
}

// Writes the training target log2(bytes) - (m + 3) beside each logged feature row.
__global__ void k_log_targets(const EncResult *__restrict__ res, uint32_t nblocks, int m, float *__restrict__ rows) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nblocks) rows[uint64_t(j) * (IN + 1) + IN] = log2f(float(res[j].total)) - float(m + 3);
}

// Mean-squared-error loss 0.5/B sum (y - t)^2 and its gradient over a batch
// of samples (perm selects them; null = 0..count-1), one CTA, deterministic:
// every gradient entry is one thread's dot product over the batch.
constexpr int CH = 64;  // samples per chunk
__global__ void __launch_bounds__(256) k_mlp_loss_grad(const float *__restrict__ params, const float *__restrict__ x,
                                                      uint32_t xstride, const float *__restrict__ t,
                                                      uint32_t tstride, const uint32_t *__restrict__ perm,
                                                      uint32_t start, uint32_t count, float *__restrict__ grad,
                                                      float *__restrict__ loss_out) {
    extern __shared__ float sm[];
    float *w = sm;                  // NP
    float *g = w + NP;              // NP
    float *X = g + NP;              // CH x IN
    float *A1 = X + CH * IN;        // CH x HID (pre-activation), then dH1
    float *A2 = A1 + CH * HID;      // CH x HID (pre-activation), then dH2
    float *H1 = A2 + CH * HID;      // CH x HID
    float *dY = H1 + CH * HID;      // CH
    __shared__ float s_loss;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < NP; i += nt) {
        w[i] = params[i];
        g[i] = 0.f;
    }
    if (tid == 0) s_loss = 0.f;
    __syncthreads();
    const float invB = 1.0f / float(count);
    for (uint32_t c0 = 0; c0 < count; c0 += CH) {
        const uint32_t nb = min(uint32_t(CH), count - c0);
        for (uint32_t i = tid; i < nb * IN; i += nt) {
            const uint32_t b = i / IN, jx = i % IN;
            const uint32_t s = perm ? perm[start + c0 + b] : start + c0 + b;
            X[b * IN + jx] = x[uint64_t(s) * xstride + jx];
        }
        __syncthreads();
        for (uint32_t i = tid; i < nb * HID; i += nt) {  // layer 1
            const uint32_t b = i / HID, h = i % HID;
            float a = w[OB1 + h];
            for (int jx = 0; jx < IN; ++jx) a = fmaf(w[OW1 + h * IN + jx], X[b * IN + jx], a);
            A1[b * HID + h] = a;
            H1[b * HID + h] = fmaxf(a, 0.f);
        }
        __syncthreads();
        for (uint32_t i = tid; i < nb * HID; i += nt) {  // layer 2
            const uint32_t b = i / HID, h = i % HID;
            float a = w[OB2 + h];
            for (int jx = 0; jx < HID; ++jx) a = fmaf(w[OW2 + h * HID + jx], H1[b * HID + jx], a);
            A2[b * HID + h] = a;
        }
        __syncthreads();
        for (uint32_t b = tid; b < nb; b += nt) {  // output and dL/dy
            float y = w[OB3];
            for (int h = 0; h < HID; ++h) y = fmaf(w[OW3 + h], fmaxf(A2[b * HID + h], 0.f), y);
            const uint32_t s = perm ? perm[start + c0 + b] : start + c0 + b;
            const float r = y - t[uint64_t(s) * tstride];
            dY[b] = r * invB;
            atomicAdd(&s_loss, 0.5f * r * r * invB);
        }
        __syncthreads();
        // output layer gradients, and dH2 (overwrites A2 after use: keep the ReLU mask)
        for (int h = tid; h < HID; h += nt) {
            float gw = 0.f;
            for (uint32_t b = 0; b < nb; ++b) gw = fmaf(dY[b], fmaxf(A2[b * HID + h], 0.f), gw);
            g[OW3 + h] += gw;
        }
        if (tid == 0) {
            float gb = 0.f;
            for (uint32_t b = 0; b < nb; ++b) gb += dY[b];
            g[OB3] += gb;
        }
        __syncthreads();
        for (uint32_t i = tid; i < nb * HID; i += nt) {
            const uint32_t b = i / HID, h = i % HID;
            A2[b * HID + h] = A2[b * HID + h] > 0.f ? dY[b] * w[OW3 + h] : 0.f;  // dA2
        }
        __syncthreads();
        for (int i = tid; i < HID * HID; i += nt) {  // gW2 = dA2^T H1
            const int h = i / HID, jx = i % HID;
            float a = 0.f;
            for (uint32_t b = 0; b < nb; ++b) a = fmaf(A2[b * HID + h], H1[b * HID + jx], a);
            g[OW2 + i] += a;
        }
        for (int h = tid; h < HID; h += nt) {
            float a = 0.f;
            for (uint32_t b = 0; b < nb; ++b) a += A2[b * HID + h];
            g[OB2 + h] += a;
        }
        __syncthreads();
        for (uint32_t i = tid; i < nb * HID; i += nt) {  // dA1 = (dA2 W2) * relu'(A1)
            const uint32_t b = i / HID, jx = i % HID;
            float a = 0.f;
            for (int h = 0; h < HID; ++h) a = fmaf(A2[b * HID + h], w[OW2 + h * HID + jx], a);
            A1[b * HID + jx] = A1[b * HID + jx] > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < HID * IN; i += nt) {  // gW1 = dA1^T X
            const int h = i / IN, jx = i % IN;
            float a = 0.f;
            for (uint32_t b = 0; b < nb; ++b) a = fmaf(A1[b * HID + h], X[b * IN + jx], a);
            g[OW1 + i] += a;
        }
        for (int h = tid; h < HID; h += nt) {
            float a = 0.f;
            for (uint32_t b = 0; b < nb; ++b) a += A1[b * HID + h];
            g[OB1 + h] += a;
        }
        __syncthreads();
    }
    for (int i = tid; i < NP; i += nt) grad[i] = g[i];
    if (tid == 0 && loss_out) *loss_out = s_loss;
}

// Adam (Kingma & Ba 2015) with bias correction; t is 1-based.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, uint32_t n, int t, float lr, float beta1, float beta2, float eps) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c1 = 1.f - powf(beta1, float(t)), c2 = 1.f - powf(beta2, float(t));
    const float gi = g[i];
    const float a = beta1 * m1[i] + (1.f - beta1) * gi;
    const float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

size_t grad_smem_bytes() { return sizeof(float) * (2 * NP + CH * IN + 3 * CH * HID + CH); }

}  // namespace

void launch_mlp_forward(const float *params, const float *x, uint32_t batch, float *y, int bf16, cudaStream_t s) {
    const unsigned grid = (batch + 127) / 128;
    k_mlp_forward<<<grid ? grid : 1, 128, 0, s>>>(params, x, batch, y, bf16);
    count_launch();
}

void launch_predict_sizes(const uint32_t *hist, uint32_t nblocks, uint32_t G, int m, const StageFeatures &sf,
                          const float *params, int bf16, float *pred, float *feat_out, cudaStream_t s) {
    const unsigned grid = (nblocks + 3) / 4;
    k_predict_sizes<<<grid ? grid : 1, 128, 0, s>>>(hist, nblocks, G, m, sf, params, bf16, pred, feat_out);
    count_launch();
}

void launch_log_targets(const EncResult *res, uint32_t nblocks, int m, float *rows, cudaStream_t s) {
    k_log_targets<<<(nblocks + 127) / 128, 128, 0, s>>>(res, nblocks, m, rows);
    count_launch();
}

int launch_mlp_loss_grad(const float *params, const float *x, uint32_t xstride, const float *t, uint32_t tstride,
                         const uint32_t *perm, uint32_t start, uint32_t count, float *grad, float *loss,
                         cudaStream_t s) {
    static bool attr = false;
    const size_t smem = grad_smem_bytes();
    if (!attr) {
        if (cudaFuncSetAttribute(k_mlp_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
            return QSIM_E_CUDA;
        attr = true;
    }
    k_mlp_loss_grad<<<1, 256, smem, s>>>(params, x, xstride, t, tstride, perm, start, count, grad, loss);
    count_launch();
    return QSIM_OK;
}

void launch_adam(float *p, const float *g, float *m1, float *m2, uint32_t n, int t, float lr, float beta1, float beta2,
                 float eps, cudaStream_t s) {
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m1, m2, n, t, lr, beta1, beta2, eps);
    count_launch();
}

}  // namespace qsim
