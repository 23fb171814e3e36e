// Per-layer 3D-CNN over the transmittance stencil (Sec. III.B.1, Fig. 3), FP32 math:
// conv 3x3x3 1->16 + ReLU (5x5x9 -> 3x3x7), conv 3x3x3 16->16 + ReLU (-> 1x1x5), output
// flattened position-major [5][16].
//
// One CTA of 288 threads per (layer, run of groups of kPts points); the layer's weights are
// staged once in shared memory, channel-fastest.  Both convolutions use sliding-window
// register tiles along the 9-long c axis:
//   conv1: a thread owns (point, d, h, half of the 16 output channels): for each (kd, kh) it
//          loads one 9-value input row and updates 7 outputs x 8 channels (168 FMAs for 9
//          input loads and 6 broadcast float4 weight loads);
//   conv2: warp g (of 8) owns input channels g and g + 8, a lane owns (point, half of the
//          output channels) and all 5 outputs: for each (ci, kd, kh) one 7-value row of
//          conv1 output and 6 float4 weight loads feed 120 FMAs.  Every lane of a warp reads
//          the same weights (broadcast) and its own point's row (the per-point stride of the
//          conv1 output, 1071 floats, puts the 16 points in 16 banks).  The eight partial
//          sums of each output go through shared memory and are added in a fixed order.
#include <cuda_fp8.h>

#include "nis_internal.h"
#include "tc_common.h"

namespace nis {

namespace {
constexpr int kPts = 16;                         // points per group
constexpr int kThreads = 288;
constexpr int kGroupsPerCta = 16;                // the layer's weights are staged once per 16 groups
                                                 // (4 per CTA: 3 % slower, from the staging traffic)
constexpr int kCiGroups = 8;                     // conv2: warps, input channels g and g + 8
// conv1 output y1[q][ci][d][h][w]: 63 values per channel at a stride of 66, 1071 per point.
// With these strides the conv1 stores of a warp (16 (point, d, h) rows x 2 channel halves)
// and the conv2 loads (16 points, one channel) each fall in 32 different banks.
constexpr int kY1Ci = 66;
constexpr int kY1 = 1071;
constexpr int kPartLd = 41;                      // conv2 partial sums: stride per (group, lane)
static_assert(kCiGroups * 32 * kPartLd <= kPts * kY1, "partial sums alias the conv1 output");
constexpr int kW2Ci = 436;                       // per-input-channel stride of w2t (27 x 16, padded)
// shared memory (floats): w1t [27 taps][16 co], b1 [16], w2t [16 ci][kW2Ci: 27 taps x 16 co],
// b2 [16], x [kPts][kLatT] (one TMA box), y1 [kPts][16 ci][kY1Ci], an mbarrier
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 27 * kCnnCh, kOffW2 = kOffB1 + kCnnCh,
              kOffB2 = kOffW2 + kCnnCh * kW2Ci, kOffX = (kOffB2 + kCnnCh + 31) & ~31,
              kOffY1 = kOffX + kPts * kLatT, kOffBar = (kOffY1 + kPts * kY1 + 1) & ~1,
              kSmemFloats = kOffBar + 4;
static_assert(kOffX % 32 == 0, "a TMA box lands at a 128-byte aligned shared-memory address");
static_assert(kOffW2 % 4 == 0 && kW2Ci % 4 == 0, "float4 weight loads need 16-byte alignment");

// Packed FP32 pairs (two output channels): acc += w * (v, v) with fma.rn.f32x2, the same
// rounding per lane as two scalar fmaf.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_dup(float v) {
    f2_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ f2_t f2_make(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_fma(f2_t &acc, f2_t w, f2_t v) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(w), "l"(v));
}
__device__ __forceinline__ float f2_lo(f2_t a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float f2_hi(f2_t a) { return __uint_as_float((unsigned)(a >> 32)); }
}  // namespace

// kTma: a group's inputs arrive as one TMA box ([16 points][kLatT] of one layer), issued once
// the previous group's conv1 has read its own, so that the load overlaps conv2; otherwise
// they are plain loads.
template <bool kTma>
__global__ void __launch_bounds__(kThreads, 2) cnn_f32_kernel(const __grid_constant__ CUtensorMap map_ht,
                                                           const float *__restrict__ H_T,
                                                           int count,
                                                           const float *__restrict__ wbase,
                                                           const __grid_constant__ WeightOffsets o,
                                                           float *__restrict__ X_T,
                                                           __nv_bfloat16 *__restrict__ X_T_bf,
                                                           size_t split_part, unsigned *err) {
    extern __shared__ __align__(128) float sm[];
    float *w1t = sm + kOffW1, *b1 = sm + kOffB1, *w2t = sm + kOffW2, *b2 = sm + kOffB2;
    float *xin = sm + kOffX, *y1 = sm + kOffY1;
    uint64_t *xbar = reinterpret_cast<uint64_t *>(sm + kOffBar);
    int *abort_flag = reinterpret_cast<int *>(sm + kOffBar + 2);
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
            w2t[ci * kW2Ci + tap * kCnnCh + co] = g2[i];
        }
        if (tid < kCnnCh) {
            b1[tid] = wbase[o.cnn_b1[k] + tid];
            b2[tid] = wbase[o.cnn_b2[k] + tid];
        }
    }
    const int n_groups = (count + kPts - 1) / kPts;
    const int g_end = min(n_groups, (int)(blockIdx.x + 1) * kGroupsPerCta);
    uint32_t xphase = 0, x_issued = 0;
    if (kTma && tid == 0) {
        tc::mbar_init(xbar, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
        if ((int)blockIdx.x * kGroupsPerCta < g_end) {
            tc::mbar_expect_tx(xbar, kPts * kLatT * 4);
            tc::tma_load_3d(xin, &map_ht, 0, k, blockIdx.x * kGroupsPerCta * kPts, xbar);
            x_issued = 1;
        }
    }
    for (int grp = blockIdx.x * kGroupsPerCta; grp < g_end; ++grp) {
        const int p0 = grp * kPts;
        const int np = min(kPts, count - p0);
        if constexpr (kTma) {
            __syncthreads();                              // weights ready / previous group done
            const bool got = tc::mbar_wait(xbar, xphase & 1);
            ++xphase;
            if (!got) {
                *abort_flag = 1;
                if (err) atomicOr(err, kErrTimeout);
            }
            __syncthreads();
            if (*(volatile int *)abort_flag) break;
        } else {
            // the group's input: all of this thread's loads issued before any store, so that
            // their latencies overlap (a load-store loop waits for each load in turn)
            constexpr int kXPer = (kPts * kLat + kThreads - 1) / kThreads;
            float xr[kXPer];
#pragma unroll
            for (int i = 0; i < kXPer; ++i) {
                const int idx = tid + i * kThreads, q = idx / kLat, t = idx % kLat;
                xr[i] = (idx < kPts * kLat && q < np) ? H_T[((size_t)(p0 + q) * kLayers + k) * kLatT + t] : 0.f;
            }
            __syncthreads();                              // weights ready / previous group done
#pragma unroll
            for (int i = 0; i < kXPer; ++i) {
                const int idx = tid + i * kThreads, q = idx / kLat, t = idx % kLat;
                if (idx < kPts * kLat) xin[q * kLatT + t] = xr[i];
            }
            __syncthreads();
        }
        // conv1: thread = (point q, row d, row h, channel half); 7 outputs x 8 channels
        {
            const int half = tid & 1, r = tid >> 1;            // 144 (q, d, h) rows
            const int q = r / 9, dh = r % 9, d = dh / 3, h = dh % 3;
            f2_t acc[7][4];                                    // channel pairs
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const f2_t b = f2_make(b1[half * 8 + 2 * c], b1[half * 8 + 2 * c + 1]);
#pragma unroll
                for (int w = 0; w < 7; ++w) acc[w][c] = b;
            }
#pragma unroll
            for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                for (int kh = 0; kh < 3; ++kh) {
                    const float *xr = xin + q * kLatT + ((d + kd) * 5 + (h + kh)) * 9;
                    f2_t row[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) row[i] = f2_dup(xr[i]);
#pragma unroll
                    for (int kw = 0; kw < 3; ++kw) {
                        const ulonglong2 *wv = reinterpret_cast<const ulonglong2 *>(
                            w1t + ((kd * 3 + kh) * 3 + kw) * kCnnCh + half * 8);
                        const ulonglong2 wa = wv[0], wb = wv[1];
#pragma unroll
                        for (int w = 0; w < 7; ++w) {
                            const f2_t v = row[w + kw];
                            f2_fma(acc[w][0], wa.x, v); f2_fma(acc[w][1], wa.y, v);
                            f2_fma(acc[w][2], wb.x, v); f2_fma(acc[w][3], wb.y, v);
                        }
                    }
                }
            float *yo = y1 + q * kY1 + (d * 3 + h) * 7;        // y1[q][ci][d][h][w]
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int w = 0; w < 7; ++w) {
                    yo[(half * 8 + 2 * c) * kY1Ci + w] = fmaxf(f2_lo(acc[w][c]), 0.f);
                    yo[(half * 8 + 2 * c + 1) * kY1Ci + w] = fmaxf(f2_hi(acc[w][c]), 0.f);
                }
        }
        __syncthreads();
        if (kTma && tid == 0 && grp + 1 < g_end) {        // conv1 is done with x: the next group
            tc::fence_async_smem();
            tc::mbar_expect_tx(xbar, kPts * kLatT * 4);
            tc::tma_load_3d(xin, &map_ht, 0, k, (grp + 1) * kPts, xbar);
            ++x_issued;
        }
        // conv2: warp g = input channels g and g + 8, lane = (channel half, point q);
        // 5 outputs x 8 channels, partial sums over 2 input channels
        const int warp = tid >> 5, lane = tid & 31;
        float *part = y1;                                 // [g][lane][kPartLd] partial sums
        if (warp < kCiGroups) {
            const int half = lane >> 4, q = lane & 15;
            f2_t acc[5][4];                                    // channel pairs
#pragma unroll
            for (int w = 0; w < 5; ++w)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[w][c] = 0ull;
            for (int cc = 0; cc < kCnnCh / kCiGroups; ++cc) {
                const int ci = warp + kCiGroups * cc;
#pragma unroll
                for (int kd = 0; kd < 3; ++kd)
#pragma unroll
                    for (int kh = 0; kh < 3; ++kh) {
                        const float *yr = y1 + q * kY1 + ci * kY1Ci + (kd * 3 + kh) * 7;
                        f2_t row[7];
#pragma unroll
                        for (int i = 0; i < 7; ++i) row[i] = f2_dup(yr[i]);
#pragma unroll
                        for (int kw = 0; kw < 3; ++kw) {
                            const ulonglong2 *wv = reinterpret_cast<const ulonglong2 *>(
                                w2t + ci * kW2Ci + ((kd * 3 + kh) * 3 + kw) * kCnnCh + half * 8);
                            const ulonglong2 wa = wv[0], wb = wv[1];
#pragma unroll
                            for (int w = 0; w < 5; ++w) {
                                const f2_t v = row[w + kw];
                                f2_fma(acc[w][0], wa.x, v); f2_fma(acc[w][1], wa.y, v);
                                f2_fma(acc[w][2], wb.x, v); f2_fma(acc[w][3], wb.y, v);
                            }
                        }
                    }
            }
            // the conv2 warps (named barrier 1, 256 threads) are done reading the conv1
            // output, which the partial sums overwrite
            asm volatile("bar.sync 1, %0;" ::"r"(kCiGroups * 32) : "memory");
#pragma unroll
            for (int w = 0; w < 5; ++w)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    part[(warp * 32 + lane) * kPartLd + w * 8 + 2 * c] = f2_lo(acc[w][c]);
                    part[(warp * 32 + lane) * kPartLd + w * 8 + 2 * c + 1] = f2_hi(acc[w][c]);
                }
        }
        __syncthreads();
        // output (point q, entry r = position w x 16 + channel co): the eight groups' partial
        // sums in order g = 0..7, + bias, ReLU; consecutive threads take consecutive entries
        for (int e = tid; e < kPts * kDT; e += kThreads) {
            const int q = e / kDT, r = e % kDT;
            if (q >= np) continue;
            const int w = r / kCnnCh, co = r % kCnnCh;
            const int slot = ((co >> 3) * 16 + q) * kPartLd + w * 8 + (co & 7);
            float sum = 0.f;
#pragma unroll
            for (int g = 0; g < kCiGroups; ++g) sum += part[g * 32 * kPartLd + slot];
            const float v = fmaxf(sum + b2[co], 0.f);
            const size_t o = ((size_t)(p0 + q) * kLayers + k) * kDT + r;
            if (X_T_bf) {
                float rr = v;
                const int parts = split_part ? 3 : 1;
                for (int s2 = 0; s2 < parts; ++s2) {
                    __nv_bfloat16 b = __float2bfloat16_rn(rr);
                    X_T_bf[o + s2 * split_part] = b;
                    rr -= __bfloat162float(b);
                }
            }
            if (X_T) X_T[o] = v;
        }
    }
    // an input load still in flight (after a time-out) lands before the CTA exits
    if (kTma && tid == 0 && x_issued > xphase) tc::mbar_wait(xbar, xphase & 1, 1u << 20);
}

void launch_cnn_f32(const float *H_T, int count, const float *wbase, const WeightOffsets &o,
                    float *X_T, __nv_bfloat16 *X_T_bf, cudaStream_t s, size_t split_part,
                    const CUtensorMap *map_ht, unsigned *err) {
    if (count <= 0) return;
    size_t smem = kSmemFloats * sizeof(float);
    static bool attr_set = false;   // per process; the attribute is per function
    if (!attr_set) {
        cudaFuncSetAttribute(cnn_f32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(cnn_f32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    static const CUtensorMap unused{};
    int n_groups = (count + kPts - 1) / kPts;
    dim3 grid((n_groups + kGroupsPerCta - 1) / kGroupsPerCta, kLayers);
    note_launch();
    if (map_ht)
        cnn_f32_kernel<true><<<grid, kThreads, smem, s>>>(*map_ht, H_T, count, wbase, o, X_T, X_T_bf,
                                                          split_part, err);
    else
        cnn_f32_kernel<false><<<grid, kThreads, smem, s>>>(unused, H_T, count, wbase, o, X_T, X_T_bf,
                                                           split_part, err);
}

}  // namespace nis
