// k_cost.cu -- learned cost model of a tick: a multilayer perceptron
// 5 -> 64 -> 64 -> 1 (ReLU hidden layers) mapping tick features to the
// logarithm of the tick's time, trained by full-batch Adam on logged ticks.
// The paper models the cost of its phases analytically (Sec. 5.4 filtering
// complexity, the subquery-count estimate of Sec. 6); this learns it from
// measurements instead, to choose the index configuration of the next tick.
// Choices never change results (every index configuration answers exactly).
//
// Parameter layout (P floats): W1[64][5], b1[64], W2[64][64], b2[64],
// W3[64], b3.  The training kernel is one block: parameters, gradients,
// Adam moments and the activations of a chunk of samples live in shared
// memory; every gradient entry is owned by one thread (no atomics).
#include "mqr_internal.cuh"

namespace mqr {

constexpr int kCostIn = 5, kCostH = 64, kCostChunk = 32, kCostThreads = 256;
constexpr int kOW1 = 0, kOB1 = kOW1 + kCostH * kCostIn, kOW2 = kOB1 + kCostH, kOB2 = kOW2 + kCostH * kCostH,
              kOW3 = kOB2 + kCostH, kOB3 = kOW3 + kCostH, kCostP = kOB3 + 1;

size_t cost_param_count() { return kCostP; }

// smem: p[P], g[P], h1[H][C], h2[H][C], d2[H][C], d1[H][C], x[C][5], dout[C]
constexpr size_t kCostSmem = sizeof(float) * (2 * kCostP + 4 * kCostH * kCostChunk + kCostChunk * kCostIn +
                                              kCostChunk + 8);
size_t cost_train_smem() { return kCostSmem; }

__global__ void __launch_bounds__(kCostThreads)
cost_train_kernel(float *__restrict__ params, float *__restrict__ adam_m, float *__restrict__ adam_v,
                  uint32_t step0, const float *__restrict__ X, const float *__restrict__ y, uint32_t n,
                  uint32_t epochs, float lr, float *__restrict__ loss_out, float *__restrict__ grad_out) {
    extern __shared__ float sm[];
    float *p = sm, *g = p + kCostP;
    float *h1 = g + kCostP, *h2 = h1 + kCostH * kCostChunk, *d2 = h2 + kCostH * kCostChunk,
          *d1 = d2 + kCostH * kCostChunk, *xs = d1 + kCostH * kCostChunk, *dout = xs + kCostChunk * kCostIn;
    float *red = dout + kCostChunk;
    const int tid = threadIdx.x;
    for (int i = tid; i < kCostP; i += kCostThreads) p[i] = params[i];
    __syncthreads();
    const float b1m = 0.9f, b2m = 0.999f, eps = 1e-8f;
    float loss = 0.f;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        for (int i = tid; i < kCostP; i += kCostThreads) g[i] = 0.f;
        if (tid == 0) red[0] = 0.f;
        __syncthreads();
        for (uint32_t c0 = 0; c0 < n; c0 += kCostChunk) {
            const int cn = (int)min((uint32_t)kCostChunk, n - c0);
            for (int i = tid; i < kCostChunk * kCostIn; i += kCostThreads) {
                const int s = i / kCostIn;
                xs[i] = s < cn ? X[(size_t)(c0 + s) * kCostIn + (i % kCostIn)] : 0.f;
            }
            __syncthreads();
            // forward: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), out = W3 h2 + b3
            for (int i = tid; i < kCostH * kCostChunk; i += kCostThreads) {
                const int j = i / kCostChunk, s = i % kCostChunk;
                float a = p[kOB1 + j];
                for (int k = 0; k < kCostIn; ++k) a += p[kOW1 + j * kCostIn + k] * xs[s * kCostIn + k];
                h1[i] = a > 0.f ? a : 0.f;
            }
            __syncthreads();
            for (int i = tid; i < kCostH * kCostChunk; i += kCostThreads) {
                const int j = i / kCostChunk, s = i % kCostChunk;
                float a = p[kOB2 + j];
                for (int k = 0; k < kCostH; ++k) a += p[kOW2 + j * kCostH + k] * h1[k * kCostChunk + s];
                h2[i] = a > 0.f ? a : 0.f;
            }
            __syncthreads();
            if (tid < kCostChunk) {
                const int s = tid;
                float o = p[kOB3];
                for (int j = 0; j < kCostH; ++j) o += p[kOW3 + j] * h2[j * kCostChunk + s];
                const float e = s < cn ? o - y[c0 + s] : 0.f;
                dout[s] = 2.f * e / (float)n;                         // d(mean squared error)/d(out)
                atomicAdd(&red[0], e * e);
            }
            __syncthreads();
            // backward
            for (int i = tid; i < kCostH * kCostChunk; i += kCostThreads) {
                const int j = i / kCostChunk, s = i % kCostChunk;
                d2[i] = h2[i] > 0.f ? dout[s] * p[kOW3 + j] : 0.f;
            }
            if (tid < kCostH) {
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += dout[s] * h2[tid * kCostChunk + s];
                g[kOW3 + tid] += a;
            }
            if (tid == kCostH) {
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += dout[s];
                g[kOB3] += a;
            }
            __syncthreads();
            for (int i = tid; i < kCostH * kCostH; i += kCostThreads) {
                const int j = i / kCostH, k = i % kCostH;
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += d2[j * kCostChunk + s] * h1[k * kCostChunk + s];
                g[kOW2 + i] += a;
            }
            if (tid < kCostH) {
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += d2[tid * kCostChunk + s];
                g[kOB2 + tid] += a;
            }
            for (int i = tid; i < kCostH * kCostChunk; i += kCostThreads) {
                const int k = i / kCostChunk, s = i % kCostChunk;
                float a = 0.f;
                for (int j = 0; j < kCostH; ++j) a += p[kOW2 + j * kCostH + k] * d2[j * kCostChunk + s];
                d1[i] = h1[i] > 0.f ? a : 0.f;
            }
            __syncthreads();
            for (int i = tid; i < kCostH * kCostIn; i += kCostThreads) {
                const int j = i / kCostIn, k = i % kCostIn;
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += d1[j * kCostChunk + s] * xs[s * kCostIn + k];
                g[kOW1 + i] += a;
            }
            if (tid < kCostH) {
                float a = 0.f;
                for (int s = 0; s < kCostChunk; ++s) a += d1[tid * kCostChunk + s];
                g[kOB1 + tid] += a;
            }
            __syncthreads();
        }
        loss = red[0] / (float)n;
        if (grad_out) {                 // gradient only: report it, leave the parameters
            for (int i = tid; i < kCostP; i += kCostThreads) grad_out[i] = g[i];
            if (tid == 0) *loss_out = loss;
            return;
        }
        // Adam (Kingma & Ba), bias-corrected
        const float t = (float)(step0 + ep + 1);
        const float c1 = 1.f - powf(b1m, t), c2 = 1.f - powf(b2m, t);
        for (int i = tid; i < kCostP; i += kCostThreads) {
            const float gi = g[i];
            const float m = b1m * adam_m[i] + (1.f - b1m) * gi;
            const float v = b2m * adam_v[i] + (1.f - b2m) * gi * gi;
            adam_m[i] = m;
            adam_v[i] = v;
            p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
        __syncthreads();
    }
    for (int i = tid; i < kCostP; i += kCostThreads) params[i] = p[i];
    if (tid == 0) *loss_out = loss;
}

__global__ void cost_predict_kernel(const float *__restrict__ p, const float *__restrict__ X, uint32_t n,
                                    float *__restrict__ out) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        float x[kCostIn];
        for (int k = 0; k < kCostIn; ++k) x[k] = X[(size_t)s * kCostIn + k];
        float h1[kCostH];
        for (int j = 0; j < kCostH; ++j) {
            float a = p[kOB1 + j];
            for (int k = 0; k < kCostIn; ++k) a += p[kOW1 + j * kCostIn + k] * x[k];
            h1[j] = a > 0.f ? a : 0.f;
        }
        float o = p[kOB3];
        for (int j = 0; j < kCostH; ++j) {
            float a = p[kOB2 + j];
            for (int k = 0; k < kCostH; ++k) a += p[kOW2 + j * kCostH + k] * h1[k];
            o += p[kOW3 + j] * (a > 0.f ? a : 0.f);
        }
        out[s] = o;
    }
}

cudaError_t launch_cost_train(cudaStream_t st, float *params, float *m, float *v, uint32_t step0, const float *X,
                              const float *y, uint32_t n, uint32_t epochs, float lr, float *loss, float *grad) {
    cudaError_t e = cudaFuncSetAttribute(cost_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCostSmem);
    if (e != cudaSuccess) return e;
    cost_train_kernel<<<1, kCostThreads, kCostSmem, st>>>(params, m, v, step0, X, y, n, epochs, lr, loss, grad);
    return cudaGetLastError();
}

cudaError_t launch_cost_predict(cudaStream_t st, const float *params, const float *X, uint32_t n, float *out) {
    if (n == 0) return cudaSuccess;
    cost_predict_kernel<<<(n + 127) / 128, 128, 0, st>>>(params, X, n, out);
    return cudaGetLastError();
}

}  // namespace mqr
