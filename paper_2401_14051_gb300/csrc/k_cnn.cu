// Per-layer 3D-CNN over the transmittance stencil (Sec. III.B.1, Fig. 3), FP32 SIMT path:
// conv 3x3x3 1->16 + ReLU (5x5x9 -> 3x3x7), conv 3x3x3 16->16 + ReLU (-> 1x1x5), output
// flattened position-major [5][16].  One CTA per (group of kPts points, layer); the
// layer's 7376 weights are staged once in shared memory.
#include "nis_internal.h"

namespace nis {

namespace {
constexpr int kPts = 8;
constexpr int kW1 = kCnnCh * 27, kW2 = kCnnCh * kCnnCh * 27;
constexpr int kY1 = kCnnCh * 63;           // 16 channels x 3 x 3 x 7
constexpr int kSmemFloats = kW1 + kCnnCh + kW2 + kCnnCh + kPts * kLat + kPts * kY1;
}

__global__ void __launch_bounds__(256) cnn_f32_kernel(const float *__restrict__ H_T, int count,
                                                      const float *__restrict__ wbase,
                                                      WeightOffsets o, float *__restrict__ X_T) {
    extern __shared__ float sm[];
    float *w1 = sm, *b1 = w1 + kW1, *w2 = b1 + kCnnCh, *b2 = w2 + kW2;
    float *xin = b2 + kCnnCh, *y1 = xin + kPts * kLat;
    const int k = blockIdx.y;
    const int p0 = blockIdx.x * kPts;
    const int np = min(kPts, count - p0);
    for (int i = threadIdx.x; i < kW1; i += blockDim.x) w1[i] = wbase[o.cnn_w1[k] + i];
    for (int i = threadIdx.x; i < kW2; i += blockDim.x) w2[i] = wbase[o.cnn_w2[k] + i];
    if (threadIdx.x < kCnnCh) {
        b1[threadIdx.x] = wbase[o.cnn_b1[k] + threadIdx.x];
        b2[threadIdx.x] = wbase[o.cnn_b2[k] + threadIdx.x];
    }
    for (int i = threadIdx.x; i < kPts * kLat; i += blockDim.x) {
        int q = i / kLat, t = i % kLat;
        xin[i] = q < np ? H_T[((size_t)(p0 + q) * kLayers + k) * kLat + t] : 0.f;
    }
    __syncthreads();
    // conv1: y1[q][c][d][h][w], d, h < 3, w < 7
    for (int i = threadIdx.x; i < kPts * kY1; i += blockDim.x) {
        int q = i / kY1, r = i % kY1;
        int c = r / 63, pos = r % 63, d = pos / 21, h = (pos / 7) % 3, w = pos % 7;
        const float *x = xin + q * kLat;
        const float *wk = w1 + c * 27;
        float acc = b1[c];
#pragma unroll
        for (int kd = 0; kd < 3; ++kd)
#pragma unroll
            for (int kh = 0; kh < 3; ++kh)
#pragma unroll
                for (int kw = 0; kw < 3; ++kw)
                    acc += wk[(kd * 3 + kh) * 3 + kw] * x[((d + kd) * 5 + (h + kh)) * 9 + (w + kw)];
        y1[i] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    // conv2: out[q][w][c], w < 5
    for (int i = threadIdx.x; i < kPts * 80; i += blockDim.x) {
        int q = i / 80, r = i % 80, w = r / kCnnCh, c = r % kCnnCh;
        if (q >= np) continue;
        const float *y = y1 + q * kY1;
        float acc = b2[c];
        for (int ci = 0; ci < kCnnCh; ++ci) {
            const float *wk = w2 + (c * kCnnCh + ci) * 27;
            const float *yc = y + ci * 63;
#pragma unroll
            for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                for (int kh = 0; kh < 3; ++kh)
#pragma unroll
                    for (int kw = 0; kw < 3; ++kw)
                        acc += wk[(kd * 3 + kh) * 3 + kw] * yc[(kd * 3 + kh) * 7 + w + kw];
        }
        X_T[((size_t)(p0 + q) * kLayers + k) * kDT + r] = fmaxf(acc, 0.f);
    }
}

void launch_cnn_f32(const float *H_T, int count, const float *wbase, const WeightOffsets &o,
                    float *X_T, cudaStream_t s) {
    if (count <= 0) return;
    size_t smem = kSmemFloats * sizeof(float);
    static bool attr_set = false;   // per process; the attribute is per function
    if (!attr_set) {
        cudaFuncSetAttribute(cnn_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    dim3 grid((count + kPts - 1) / kPts, kLayers);
    note_launch();
    cnn_f32_kernel<<<grid, 256, smem, s>>>(H_T, count, wbase, o, X_T);
}

}  // namespace nis
