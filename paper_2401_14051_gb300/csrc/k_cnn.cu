// Per-layer 3D-CNN over the transmittance stencil (Sec. III.B.1, Fig. 3), FP32 SIMT path:
// conv 3x3x3 1->16 + ReLU (5x5x9 -> 3x3x7), conv 3x3x3 16->16 + ReLU (-> 1x1x5), output
// flattened position-major [5][16].
//
// One CTA of 160 threads per (layer, run of groups of kPts points).  The layer's weights are
// staged once in shared memory transposed to channel-fastest order, so a thread that owns
// one output position keeps its input window in registers and reads the weights of 8 or 16
// output channels with warp-broadcast float4 loads (several FMAs per shared-memory load).
#include "nis_internal.h"

namespace nis {

namespace {
constexpr int kPts = 16;                         // points per group
constexpr int kThreads = 160;
constexpr int kGroupsPerCta = 4;
constexpr int kPos1 = 63;                        // conv1 output positions (3 x 3 x 7)
constexpr int kY1 = 1016;                        // per-point stride of y1 (16 x 63 = 1008,
                                                 // padded so conv2's 4 points hit distinct banks)
// shared memory (floats): w1t [27][16], b1 [16], w2t [16 ci][27 tap][16 co], b2 [16],
// x [kPts][225], y1 [kPts][16][63]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 27 * kCnnCh, kOffW2 = kOffB1 + kCnnCh,
              kOffB2 = kOffW2 + kCnnCh * 27 * kCnnCh, kOffX = kOffB2 + kCnnCh,
              kOffY1 = kOffX + kPts * kLat, kSmemFloats = kOffY1 + kPts * kY1;
}  // namespace

__global__ void __launch_bounds__(kThreads) cnn_f32_kernel(const float *__restrict__ H_T,
                                                           int count,
                                                           const float *__restrict__ wbase,
                                                           const __grid_constant__ WeightOffsets o,
                                                           float *__restrict__ X_T,
                                                           __nv_bfloat16 *__restrict__ X_T_bf,
                                                           size_t split_part) {
    extern __shared__ __align__(16) float sm[];
    float *w1t = sm + kOffW1, *b1 = sm + kOffB1, *w2t = sm + kOffW2, *b2 = sm + kOffB2;
    float *xin = sm + kOffX, *y1 = sm + kOffY1;
    const int k = blockIdx.y;
    const int tid = threadIdx.x;
    {
        const float *g1 = wbase + o.cnn_w1[k];          // [co][tap]
        for (int i = tid; i < 27 * kCnnCh; i += kThreads) {
            int co = i / 27, tap = i % 27;
            w1t[tap * kCnnCh + co] = g1[i];
        }
        const float *g2 = wbase + o.cnn_w2[k];          // [co][ci][tap]
        for (int i = tid; i < kCnnCh * kCnnCh * 27; i += kThreads) {
            int co = i / (kCnnCh * 27), r = i % (kCnnCh * 27), ci = r / 27, tap = r % 27;
            w2t[(ci * 27 + tap) * kCnnCh + co] = g2[i];
        }
        if (tid < kCnnCh) {
            b1[tid] = wbase[o.cnn_b1[k] + tid];
            b2[tid] = wbase[o.cnn_b2[k] + tid];
        }
    }
    const int n_groups = (count + kPts - 1) / kPts;
    for (int grp = blockIdx.x * kGroupsPerCta;
         grp < n_groups && grp < (blockIdx.x + 1) * kGroupsPerCta; ++grp) {
        const int p0 = grp * kPts;
        const int np = min(kPts, count - p0);
        __syncthreads();                                  // weights ready / previous group done
        for (int i = tid; i < kPts * kLat; i += kThreads) {
            int q = i / kLat, t = i % kLat;
            xin[i] = q < np ? H_T[((size_t)(p0 + q) * kLayers + k) * kLat + t] : 0.f;
        }
        __syncthreads();
        // conv1: task = (point, position); 16 output channels per task
        for (int task = tid; task < kPts * kPos1; task += kThreads) {
            int q = task / kPos1, pos = task % kPos1;
            int d = pos / 21, h = (pos / 7) % 3, w = pos % 7;
            const float *x = xin + q * kLat + (d * 5 + h) * 9 + w;
            float win[27];
#pragma unroll
            for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                for (int kh = 0; kh < 3; ++kh)
#pragma unroll
                    for (int kw = 0; kw < 3; ++kw) win[(kd * 3 + kh) * 3 + kw] = x[(kd * 5 + kh) * 9 + kw];
            float acc[kCnnCh];
#pragma unroll
            for (int c = 0; c < kCnnCh; ++c) acc[c] = b1[c];
            // keep the weight loads inside the task loop: hoisted, all 432 would spill
            int zero = 0;
            asm volatile("" : "+r"(zero));
            const float *w1p = w1t + zero;
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const float4 *wv = reinterpret_cast<const float4 *>(w1p + tap * kCnnCh);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    float4 ww = wv[c4];
                    acc[4 * c4 + 0] += ww.x * win[tap];
                    acc[4 * c4 + 1] += ww.y * win[tap];
                    acc[4 * c4 + 2] += ww.z * win[tap];
                    acc[4 * c4 + 3] += ww.w * win[tap];
                }
            }
            float *yo = y1 + q * kY1 + pos;
#pragma unroll
            for (int c = 0; c < kCnnCh; ++c) yo[c * kPos1] = fmaxf(acc[c], 0.f);
        }
        __syncthreads();
        // conv2: thread = (point, output position w, half of the output channels)
        {
            const int half = tid & 1, pw = tid >> 1;          // 80 (point, w) pairs
            const int q = pw / 5, w = pw % 5;
            const float *y = y1 + q * kY1 + w;
            float acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = b2[half * 8 + c];
            for (int ci = 0; ci < kCnnCh; ++ci) {
                const float *yc = y + ci * kPos1;
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int kd = tap / 9, kh = (tap / 3) % 3, kw = tap % 3;
                    float v = yc[(kd * 3 + kh) * 7 + kw];
                    const float4 *wv =
                        reinterpret_cast<const float4 *>(w2t + (ci * 27 + tap) * kCnnCh + half * 8);
                    float4 wa = wv[0], wb = wv[1];
                    acc[0] += wa.x * v; acc[1] += wa.y * v; acc[2] += wa.z * v; acc[3] += wa.w * v;
                    acc[4] += wb.x * v; acc[5] += wb.y * v; acc[6] += wb.z * v; acc[7] += wb.w * v;
                }
            }
            if (q < np) {
                const size_t o = ((size_t)(p0 + q) * kLayers + k) * kDT + w * kCnnCh + half * 8;
                if (X_T_bf) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float r = fmaxf(acc[c], 0.f);
                        const int parts = split_part ? 3 : 1;
                        for (int q = 0; q < parts; ++q) {
                            __nv_bfloat16 b = __float2bfloat16_rn(r);
                            X_T_bf[o + c + q * split_part] = b;
                            r -= __bfloat162float(b);
                        }
                    }
                }
                if (X_T) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) X_T[o + c] = fmaxf(acc[c], 0.f);
                }
            }
        }
    }
}

void launch_cnn_f32(const float *H_T, int count, const float *wbase, const WeightOffsets &o,
                    float *X_T, __nv_bfloat16 *X_T_bf, cudaStream_t s, size_t split_part) {
    if (count <= 0) return;
    size_t smem = kSmemFloats * sizeof(float);
    static bool attr_set = false;   // per process; the attribute is per function
    if (!attr_set) {
        cudaFuncSetAttribute(cnn_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    int n_groups = (count + kPts - 1) / kPts;
    dim3 grid((n_groups + kGroupsPerCta - 1) / kGroupsPerCta, kLayers);
    note_launch();
    cnn_f32_kernel<<<grid, kThreads, smem, s>>>(H_T, count, wbase, o, X_T, X_T_bf, split_part);
}

}  // namespace nis
