// Per-layer 3D-CNN (Sec. III.B.1, Fig. 3) with BF16 operands on the tensor cores and FP32
// accumulation in tensor memory: the CNN of the BF16 and FP8 precision modes.  Both
// convolutions are implicit GEMMs with N = 16 output channels and M = 128-row tiles, for a
// group of 16 points of one template layer:
//   conv1  rows (point, output position of the 3x3x7 grid), 1008 of them in 8 tiles; K = the
//          27 taps, padded to 32.  Its operand is gathered from the points' 5x5x9 inputs into
//          shared memory (im2col), four tiles at a time.
//   conv2  rows (point, w) with w padded to 8 (5 used): one tile; K = 27 taps x 16 input
//          channels, one K = 16 MMA per tap.  Its operand is read in place from conv1's
//          output, stored as [point][channel half][position][8 channels] so that the rows of
//          tap (kd, kh, kw) are the 16-byte rows at positions (3 kd + kh) 7 + kw + w: each tap's
//          MMA takes a descriptor on that output, nothing is copied.
// Operands use the no-swizzle K-major layout (8-row x 16-byte core matrices).  ReLU and the
// biases are applied in FP32 on the accumulators; conv1's output is rounded to BF16 (the
// operand of conv2), the result is written as BF16 (and e4m3 / FP32 when asked).
// Every mbarrier wait is bounded: on a time-out the kernel records kErrTimeout and stops.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "nis_internal.h"
#include "tc_common.h"

namespace nis {

namespace {
constexpr int kGP = 16;                       // points per group
constexpr int kThreadsTC = 256;               // 8 warps
constexpr int kRows1 = kGP * 63;              // conv1 rows (1008)
constexpr uint32_t kTileA1 = 128 * 32 * 2;    // one conv1 operand tile: 128 rows x 32 K BF16
constexpr uint32_t kY1Point = 2 * 63 * 16;    // conv1 output per point: 2 channel halves x 63 x 16 B
// shared memory (bytes)
constexpr uint32_t kB1 = 0;                   // [2 co groups][4 k groups][8][8] BF16
constexpr uint32_t kB2 = kB1 + 1024;          // [27 taps][2 co groups][2 ci groups][8][8] BF16
constexpr uint32_t kBias = kB2 + 27 * 512;    // b1[16], b2[16] FP32
constexpr uint32_t kX = kBias + 128;          // [16 points][kLatT] FP32, one TMA box
constexpr uint32_t kXBytes = kGP * kLatT * 4;
constexpr uint32_t kA1 = 30720;               // 4 conv1 tiles
constexpr uint32_t kY1 = kA1 + 4 * kTileA1;   // [16 points][2][63][16 B] + read-past pad
constexpr uint32_t kBar = kY1 + kGP * kY1Point + 256;
constexpr uint32_t kSmemTC = kBar + 64;
static_assert(kX + kXBytes <= kA1, "conv1 input overlaps the operand tiles");
static_assert(kX % 128 == 0, "a TMA box lands at a 128-byte aligned shared-memory address");
static_assert(kA1 % 1024 == 0 && kY1 % 16 == 0 && kBar % 8 == 0, "alignment");

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
}  // namespace

__global__ void __launch_bounds__(kThreadsTC, 2)
    cnn_tc_kernel(const __grid_constant__ CUtensorMap map_ht, int count, const float *__restrict__ wbase,
                  const __grid_constant__ WeightOffsets o, float *__restrict__ X_T,
                  __nv_bfloat16 *__restrict__ X_T_bf, uint8_t *__restrict__ X_T_f8, unsigned *err, int xt_ld) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int k = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *x = reinterpret_cast<float *>(sm + kX);
    const float *bias = reinterpret_cast<const float *>(sm + kBias);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kBar);      // [0] MMA done, [1] drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kBar + 16);
    int *abort_flag = reinterpret_cast<int *>(sm + kBar + 20);
    uint64_t *xbar = reinterpret_cast<uint64_t *>(sm + kBar + 24);  // a group's inputs landed
    const uint32_t sbase = tc::smem_u32(sm);

    // this layer's weights as BF16 core matrices, and the biases
    {
        __nv_bfloat16 *b1 = reinterpret_cast<__nv_bfloat16 *>(sm + kB1);
        const float *g1 = wbase + o.cnn_w1[k];                  // [co][27]
        for (int i = tid; i < 16 * 32; i += kThreadsTC) {
            const int co = i >> 5, kk = i & 31;
            const float v = kk < 27 ? g1[co * 27 + kk] : 0.f;
            b1[((co >> 3) * 512 + (kk >> 3) * 128 + (co & 7) * 16 + (kk & 7) * 2) / 2] = __float2bfloat16_rn(v);
        }
        __nv_bfloat16 *b2 = reinterpret_cast<__nv_bfloat16 *>(sm + kB2);
        const float *g2 = wbase + o.cnn_w2[k];                  // [co][ci][27]
        for (int i = tid; i < 27 * 256; i += kThreadsTC) {
            const int t = i >> 8, co = (i >> 4) & 15, ci = i & 15;
            b2[(t * 512 + (co >> 3) * 256 + (ci >> 3) * 128 + (co & 7) * 16 + (ci & 7) * 2) / 2] =
                __float2bfloat16_rn(g2[(co * 16 + ci) * 27 + t]);
        }
        float *bw = reinterpret_cast<float *>(sm + kBias);
        if (tid < 16) bw[tid] = wbase[o.cnn_b1[k] + tid];
        else if (tid < 32) bw[tid] = wbase[o.cnn_b2[k] + tid - 16];
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_init(xbar, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, 256);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::idesc_bf16_f32(128, 16);
    uint32_t phase = 0;
    bool ok = true;
    // all threads wait for the MMAs committed to bar[0]; the outcome is made uniform over
    // the CTA (a time-out anywhere stops every thread at the same point)
    auto wait_mma = [&]() -> bool {
        const bool got = tc::mbar_wait(&bar[0], phase & 1);
        ++phase;
        if (!got) {
            atomicOr(err, kErrTimeout);
            *abort_flag = 1;
        }
        __syncthreads();
        tc::fence_after_sync();
        return !*(volatile int *)abort_flag;
    };

    const int n_groups = (count + kGP - 1) / kGP;
    // a group's inputs: rows (p0 .. p0 + 15, layer k) of H_T as one TMA box [16][kLatT], issued
    // as soon as the previous group's conv1 operands are built, so that it lands while that
    // group's MMAs and epilogues run (rows past the points are read but never written out)
    uint32_t xphase = 0, x_issued = 0;
    if (tid == 0 && (int)blockIdx.x < n_groups) {
        tc::mbar_expect_tx(xbar, kXBytes);
        tc::tma_load_3d(x, &map_ht, 0, k, blockIdx.x * kGP, xbar);
        x_issued = 1;
    }
    for (int grp = blockIdx.x; grp < n_groups && ok; grp += gridDim.x) {
        const int p0 = grp * kGP, np = min(kGP, count - p0);
        __syncthreads();                           // previous group done with y1 and TMEM
        {
            const bool got = tc::mbar_wait(xbar, xphase & 1);
            ++xphase;
            if (!got) {
                atomicOr(err, kErrTimeout);
                *abort_flag = 1;
            }
            __syncthreads();
            if (*(volatile int *)abort_flag) break;
        }
        // conv1, in two halves of four tiles
        for (int half = 0; half < 2 && ok; ++half) {
            for (int rl = tid; rl < 512; rl += kThreadsTC) {
                const int r = half * 512 + rl;
                uint32_t pk[16];
                if (r < kRows1) {
                    const int p = r / 63, pos = r % 63;
                    const int d = pos / 21, h = (pos / 7) % 3, w = pos % 7;
                    const float *xp = x + p * kLatT + d * 45 + h * 9 + w;
                    float v[32];
#pragma unroll
                    for (int kk = 0; kk < 32; ++kk) {
                        const int kd = kk / 9, kh = (kk / 3) % 3, kw = kk % 3;
                        v[kk] = kk < 27 ? xp[kd * 45 + kh * 9 + kw] : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) pk[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) pk[j] = 0u;
                }
                const int tt = rl >> 7, rr = rl & 127;
                uint8_t *row = sm + kA1 + tt * kTileA1 + (rr >> 3) * 512 + (rr & 7) * 16;
#pragma unroll
                for (int kg = 0; kg < 4; ++kg)
                    *reinterpret_cast<uint4 *>(row + kg * 128) =
                        make_uint4(pk[4 * kg], pk[4 * kg + 1], pk[4 * kg + 2], pk[4 * kg + 3]);
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                if (half == 1 && grp + (int)gridDim.x < n_groups) {   // x is free: the next group
                    tc::fence_async_smem();
                    tc::mbar_expect_tx(xbar, kXBytes);
                    tc::tma_load_3d(x, &map_ht, 0, k, (grp + gridDim.x) * kGP, xbar);
                    ++x_issued;
                }
                for (int tt = 0; tt < 4; ++tt)
#pragma unroll
                    for (int s = 0; s < 2; ++s)
                        tc::mma_f16(tmem + (half * 4 + tt) * 16,
                                    tc::smem_desc_noswz(sbase + kA1 + tt * kTileA1 + s * 256, 128, 512),
                                    tc::smem_desc_noswz(sbase + kB1 + s * 256, 128, 512), idesc, s);
                tc::mma_commit(&bar[0]);
            }
            ok = wait_mma();
        }
        if (!ok) break;
        // conv1 epilogue: ReLU(acc + b1) -> BF16 -> y1[p][channel half][pos][8]
        {
            const int q = warp & 3;
            for (int t = (warp >> 2) * 4; t < (warp >> 2) * 4 + 4; ++t) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + t * 16, v);
                tc::tmem_ld_wait();
                const int r = t * 128 + q * 32 + lane;
                if (r < kRows1) {
                    const int p = r / 63, pos = r % 63;
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        pk[j] = pack_bf16x2(fmaxf(v[2 * j] + bias[2 * j], 0.f),
                                            fmaxf(v[2 * j + 1] + bias[2 * j + 1], 0.f));
                    uint8_t *dst = sm + kY1 + p * kY1Point + pos * 16;
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4 *>(dst + 1008) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
        tc::fence_before_sync();
        tc::fence_async_smem();
        __syncthreads();
        // conv2: one K = 16 MMA per tap, the operand read in place from y1
        if (tid == 0) {
            tc::fence_after_sync();
            for (int t = 0; t < 27; ++t) {
                const int kd = t / 9, kh = (t / 3) % 3, kw = t % 3;
                const uint32_t a = sbase + kY1 + ((kd * 3 + kh) * 7 + kw) * 16;
                tc::mma_f16(tmem + 128, tc::smem_desc_noswz(a, 1008, 2016),
                            tc::smem_desc_noswz(sbase + kB2 + t * 512, 128, 256), idesc, t);
            }
            tc::mma_commit(&bar[0]);
        }
        ok = wait_mma();
        if (!ok) break;
        // conv2 epilogue: ReLU(acc + b2), rows (p, w < 5) -> X_T[p][k][w 16 + co]
        if (warp < 4) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 128, v);
            tc::tmem_ld_wait();
            const int r = warp * 32 + lane, p = r >> 3, w = r & 7;
            if (w < 5 && p < np) {
                float z[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) z[c] = fmaxf(v[c] + bias[16 + c], 0.f);
                const size_t off = ((size_t)(p0 + p) * kLayers + k) * kDT + w * 16;
                if (X_T_bf) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) pk[j] = pack_bf16x2(z[2 * j], z[2 * j + 1]);
                    uint4 *dst = reinterpret_cast<uint4 *>(X_T_bf + ((size_t)(p0 + p) * kLayers + k) * xt_ld + w * 16);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
                if (X_T) {
                    float4 *dst = reinterpret_cast<float4 *>(X_T + off);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
                }
                if (X_T_f8) {
                    uint32_t b[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        b[c >> 2] |= (uint32_t)__nv_cvt_float_to_fp8(z[c], __NV_SATFINITE, __NV_E4M3) << (8 * (c & 3));
                    *reinterpret_cast<uint4 *>(X_T_f8 + off) = make_uint4(b[0], b[1], b[2], b[3]);
                }
            }
        }
        tc::fence_before_sync();
    }
    // MMAs issued before a time-out complete before TMEM is released, and an input load in
    // flight lands before the CTA's shared memory goes away
    __syncthreads();
    if (tid == 0) {
        tc::mma_commit(&bar[1]);
        tc::mbar_wait(&bar[1], 0, 1u << 20);
        if (x_issued > xphase) tc::mbar_wait(xbar, xphase & 1, 1u << 20);
    }
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

void launch_cnn_tc(const CUtensorMap &map_ht, int count, const float *wbase, const WeightOffsets &o,
                   float *X_T, __nv_bfloat16 *X_T_bf, uint8_t *X_T_f8, unsigned *err, int num_sms,
                   cudaStream_t s, int xt_ld) {
    if (count <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(cnn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC);
        attr_set = true;
    }
    // two CTAs per SM, persistent over the point groups of each layer
    const int n_groups = (count + kGP - 1) / kGP;
    int per_layer = (2 * num_sms) / kLayers;
    if (per_layer < 1) per_layer = 1;
    if (per_layer > n_groups) per_layer = n_groups;
    note_launch();
    cnn_tc_kernel<<<dim3(per_layer, kLayers), kThreadsTC, kSmemTC, s>>>(map_ht, count, wbase, o, X_T,
                                                                        X_T_bf, X_T_f8, err, xt_ld);
}

}  // namespace nis
