// Rank predictor kernels: a three-layer perceptron of width 64 on 8 block
// features (FP32), its forward pass over many samples, the loss gradient of
// one minibatch (forward + backpropagation in one CTA, sums over the batch in
// a fixed order, so results are deterministic) and the Adam update.
//
// Parameter layout (kMlpParams floats): W1 (64 x 8, row-major), b1 (64),
// W2 (64 x 64, row-major), b2 (64), w3 (64), b3 (1).
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3;
// loss (1/B) sum (y - t)^2; ReLU'(0) = 0.  Adam: Kingma and Ba (2015).
#include <cstdint>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kIn = kMlpIn, kH = kMlpHidden;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
static_assert(oB3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ float relu(float a) { return a > 0.f ? a : 0.f; }

// y[i] = network(x[i]) for i < n; the weights are staged in shared memory.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ theta, const float* __restrict__ x,
                                                      int64_t n, float* __restrict__ y) {
    __shared__ float th[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xi[kIn], h1[kH];
#pragma unroll
    for (int i = 0; i < kIn; i++) xi[i] = x[s * kIn + i];
#pragma unroll
    for (int j = 0; j < kH; j++) {
        float a = th[oB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; i++) a += th[oW1 + j * kIn + i] * xi[i];
        h1[j] = relu(a);
    }
    float out = th[oB3];
    for (int j = 0; j < kH; j++) {
        float a = th[oB2 + j];
#pragma unroll
        for (int k = 0; k < kH; k++) a += th[oW2 + j * kH + k] * h1[k];
        out += th[oW3 + j] * relu(a);
    }
    y[s] = out;
}

// Loss and gradient of one minibatch (B <= kMlpMaxBatch samples, rows
// idx[b] of x / t, or rows 0..B-1 when idx is null), one CTA.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ x,
                                                        const float* __restrict__ t, const int32_t* __restrict__ idx,
                                                        int B, float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* th = sm;                      // kMlpParams
    float* xs = th + kMlpParams;         // B x 8
    float* a1 = xs + kMlpMaxBatch * kIn; // B x 64: pre-activations, later dL/da1
    float* a2 = a1 + kMlpMaxBatch * kH;  // B x 64: pre-activations, later dL/da2
    float* gy = a2 + kMlpMaxBatch * kH;  // B
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int i = tid; i < kMlpParams; i += NT) th[i] = theta[i];
    for (int i = tid; i < B * kIn; i += NT) {
        const int b = i / kIn;
        const int64_t row = idx ? idx[b] : b;
        xs[i] = x[row * kIn + i % kIn];
    }
    __syncthreads();
    for (int i = tid; i < B * kH; i += NT) {
        const int b = i / kH, j = i % kH;
        float a = th[oB1 + j];
        for (int k = 0; k < kIn; k++) a += th[oW1 + j * kIn + k] * xs[b * kIn + k];
        a1[i] = a;
    }
    __syncthreads();
    for (int i = tid; i < B * kH; i += NT) {
        const int b = i / kH, j = i % kH;
        float a = th[oB2 + j];
        for (int k = 0; k < kH; k++) a += th[oW2 + j * kH + k] * relu(a1[b * kH + k]);
        a2[i] = a;
    }
    __syncthreads();
    for (int b = tid; b < B; b += NT) {
        float y = th[oB3];
        for (int j = 0; j < kH; j++) y += th[oW3 + j] * relu(a2[b * kH + j]);
        const int64_t row = idx ? idx[b] : b;
        gy[b] = y - t[row];  // residual; scaled below
    }
    __syncthreads();
    if (tid == 0) {
        float L = 0.f;
        for (int b = 0; b < B; b++) L += gy[b] * gy[b];
        *loss = L / (float)B;
    }
    __syncthreads();  // the loss reads every residual before they are scaled
    for (int b = tid; b < B; b += NT) gy[b] *= 2.f / (float)B;  // dL/dy
    __syncthreads();
    // output layer, then dL/da2 in place
    for (int j = tid; j <= kH; j += NT) {
        float g = 0.f;
        if (j < kH) {
            for (int b = 0; b < B; b++) g += gy[b] * relu(a2[b * kH + j]);
            grad[oW3 + j] = g;
        } else {
            for (int b = 0; b < B; b++) g += gy[b];
            grad[oB3] = g;
        }
    }
    __syncthreads();
    for (int i = tid; i < B * kH; i += NT) {
        const int b = i / kH, j = i % kH;
        a2[i] = a2[i] > 0.f ? gy[b] * th[oW3 + j] : 0.f;
    }
    __syncthreads();
    // hidden layer 2: dW2 = sum_b da2 h1^T, db2 = sum_b da2
    for (int i = tid; i < kH * kH + kH; i += NT) {
        float g = 0.f;
        if (i < kH * kH) {
            const int j = i / kH, k = i % kH;
            for (int b = 0; b < B; b++) g += a2[b * kH + j] * relu(a1[b * kH + k]);
            grad[oW2 + i] = g;
        } else {
            const int j = i - kH * kH;
            for (int b = 0; b < B; b++) g += a2[b * kH + j];
            grad[oB2 + j] = g;
        }
    }
    __syncthreads();
    // dL/da1 = (W2^T da2) * [a1 > 0], in place
    for (int i = tid; i < B * kH; i += NT) {
        const int b = i / kH, k = i % kH;
        float g = 0.f;
        for (int j = 0; j < kH; j++) g += a2[b * kH + j] * th[oW2 + j * kH + k];
        a1[i] = a1[i] > 0.f ? g : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kH * kIn + kH; i += NT) {
        float g = 0.f;
        if (i < kH * kIn) {
            const int j = i / kIn, k = i % kIn;
            for (int b = 0; b < B; b++) g += a1[b * kH + j] * xs[b * kIn + k];
            grad[oW1 + i] = g;
        } else {
            const int j = i - kH * kIn;
            for (int b = 0; b < B; b++) g += a1[b * kH + j];
            grad[oB1 + j] = g;
        }
    }
}

__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float g = grad[i];
    const float mi = kAdamBeta1 * m[i] + (1.f - kAdamBeta1) * g;
    const float vi = kAdamBeta2 * v[i] + (1.f - kAdamBeta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + kAdamEps);
}

}  // namespace

size_t mlp_grad_smem_bytes() {
    return sizeof(float) * ((size_t)kMlpParams + (size_t)kMlpMaxBatch * (kIn + 2 * kH + 1));
}

cudaError_t launch_mlp_forward(cudaStream_t st, const float* theta, const float* x, int64_t n, float* y) {
    if (n <= 0) return cudaSuccess;
    launch_count_add(1);
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(theta, x, n, y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t st, const float* theta, const float* x, const float* t, const int32_t* idx,
                            int B, float* grad, float* loss) {
    if (B <= 0 || B > kMlpMaxBatch) return cudaErrorInvalidValue;
    const size_t smem = mlp_grad_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    launch_count_add(1);
    k_mlp_grad<<<1, kMlpThreads, smem, st>>>(theta, x, t, idx, B, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(cudaStream_t st, float* theta, const float* grad, float* m, float* v, int step,
                            float lr) {
    if (step < 1) return cudaErrorInvalidValue;
    launch_count_add(1);
    const float c1 = 1.f - powf(kAdamBeta1, (float)step), c2 = 1.f - powf(kAdamBeta2, (float)step);
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(theta, grad, m, v, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace hs
