// Dense layers of the backbone (Sec. III.C.2, Fig. 6) on the 5th-generation tensor cores:
// out = epilogue(A B^T) with A = activations [rows][K] and B = weights [N][K], both K-major,
// FP32 accumulation in tensor memory.
//
// Persistent kernel, one CTA per SM, 6 or 10 warps:
//   warp 0     TMA producer: fills a ring of shared-memory stages, one K slab per stage
//   warp 1     TMEM owner and MMA issuer: 128 x N_mma tcgen05.mma per 32-byte K slice,
//              two accumulator buffers (columns 0 and 256) so the epilogue of one tile
//              overlaps the MMAs of the next
//   warps 2-   epilogue: one (FP32 split) or two (BF16, FP8) warps per TMEM lane quarter,
//              each thread one row of the tile.  A warp takes 32 columns at a time: its
//              32 x 32 residual chunk arrives by TMA two chunks ahead, it applies the
//              layer's fused epilogue and stages the result in shared memory, from where
//              one lane writes it with a TMA store (rows of 128 contiguous bytes instead of
//              one row per lane)
// Stage layouts:
//   one part (BF16, FP8)   3 stages of {A 128 x 128 B, B N_mma x 128 B}, 128-byte swizzle
//   three parts (FP32 as   2 stages of {A0 A1 A2 128 x 64 B, B0 B1 B2 N_mma x 64 B}, 64-byte
//   three BF16 parts)      swizzle.  A first sweep over K brings each 32-wide slab with all
//                          its parts and sums the five smaller products of the split; a
//                          second sweep brings A0 B0 (three slabs per stage) and adds the
//                          leading product, so the small terms are summed while the
//                          accumulator is still small (all six products per slab in one
//                          sweep measured about 7x the end-to-end error of this order).  A0
//                          and B0 are the only operands fetched twice.
// Consecutive layers are programmatic dependent launches: the prologue (barriers, TMEM,
// per-column constants) overlaps the previous layer's tail.
// Every mbarrier wait is bounded: on a time-out the kernel records kErrTimeout in the
// context's error word and winds down (draining its MMAs before releasing TMEM).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "nis_internal.h"
#include "tc_common.h"

namespace nis {

namespace {
constexpr int TM = 128, TK = 64, TN_MAX = 208, STAGES = 4;
constexpr uint32_t A_STAGE = TM * TK * 2;                 // 16 KB
constexpr uint32_t B_STAGE = TN_MAX * TK * 2;             // 26 KB (208 rows)
// three-part stages: rows of kSplitSlabK BF16 of K (64 bytes: 64-byte swizzle)
constexpr uint32_t ROW3 = kSplitSlabK * 2;
constexpr int STAGES3 = kSplitSlabK == 16 ? 4 : 2;
constexpr uint32_t A_PART3 = TM * ROW3;                   // 8 KB
constexpr uint32_t B_PART3 = TN_MAX * ROW3;               // 13 KB
constexpr uint32_t STAGE3 = 3 * A_PART3 + 3 * B_PART3;    // 63 KB
// Epilogue warps (the kernel's template argument EPI): 8 (two per TMEM lane quarter,
// alternate 32-column chunks) for BF16 and FP8, whose epilogue is the bottleneck; 4 (one per
// quarter) for the FP32 split, where they measured faster (more registers per thread, less
// L1 contention with the operand loads).
// Per epilogue warp, staging for the TMA stores of a 32 x 32 chunk: FP32 o1 (4 KB) + three
// BF16 parts of o2 (6 KB) with the split, o1 + o2 as BF16 (2 + 2 KB) without.  With eight
// epilogue warps each has two such buffers, so a chunk is staged while the previous chunk's
// stores still read theirs (measured: 9 % faster BF16 and 21 % faster FP8 dense layers);
// with the split one (shared memory; storing 16-column halves from two 5 KB buffers instead
// measured 10 % slower).
constexpr uint32_t STG_SPLIT = 10240, STG_ONE = 4096;
template <int EPI>
__host__ __device__ constexpr int stg_bufs() { return EPI == 8 ? 2 : 1; }
constexpr uint32_t SMEM_CONST = 7 * TN_MAX * 4;          // per-column epilogue constants
// per epilogue warp, two 32 x 32 residual chunks loaded by TMA: FP32 with the split, BF16
// otherwise
constexpr uint32_t PRE_SPLIT = 2 * 32 * 32 * 4, PRE_ONE = 2 * 32 * 32 * 2;
// one-part stages: four with four epilogue warps, two with eight (shared memory; their
// epilogue, not the operand pipeline, sets the pace)
template <int EPI>
__host__ __device__ constexpr int stages_one() { return EPI == 8 ? 2 : STAGES; }
template <int EPI>
__host__ __device__ constexpr uint32_t smem_tiles() {
    // the FP32 split runs with four epilogue warps only
    const uint32_t split = EPI == 4 ? STAGES3 * STAGE3 + EPI * (STG_SPLIT + PRE_SPLIT) : 0;
    const uint32_t one = stages_one<EPI>() * (A_STAGE + B_STAGE) + EPI * (stg_bufs<EPI>() * STG_ONE + PRE_ONE);
    return split > one ? split : one;
}
template <int EPI>
__host__ __device__ constexpr uint32_t smem_bytes() { return smem_tiles<EPI>() + 256 + SMEM_CONST + 1024; }  // + alignment slack
static_assert(smem_bytes<8>() <= 227 * 1024 && smem_bytes<4>() <= 227 * 1024,
              "shared memory of tc_gemm_kernel");
static_assert((A_STAGE + B_STAGE) % 1024 == 0 && STAGE3 % 256 == 0 && B_PART3 % 256 == 0 &&
                  (STAGES3 * STAGE3) % 1024 == 0 && STG_SPLIT % 1024 == 0 && STG_ONE % 1024 == 0,
              "stages, parts and staging buffers must keep the 1024-byte swizzle-atom alignment");

__device__ __forceinline__ void record_timeout(unsigned *err, int *abort_flag) {
    *abort_flag = 1;
    if (err) atomicOr(err, kErrTimeout);
}

// Shared-memory descriptor of a split stage's operand rows.
__device__ __forceinline__ uint64_t split_desc(uint32_t saddr) {
    return kSplitSlabK == 16 ? tc::smem_desc_sw32(saddr) : tc::smem_desc_sw64(saddr);
}

// Six products of the three-way split, small to large: (A part, B part).
__device__ constexpr int kPassA[6] = {2, 1, 0, 1, 0, 0};
__device__ constexpr int kPassB[6] = {0, 1, 2, 0, 1, 0};

__device__ __forceinline__ void store_bf16x8(__nv_bfloat16 *dst, const float *v) {
    __align__(16) __nv_bfloat162 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(p);
}
// 8 values as BF16, or as the three BF16 parts of their split (part stride `part`).
__device__ __forceinline__ void store_out8(__nv_bfloat16 *dst, const float *v, int split, size_t part) {
    if (!split) { store_bf16x8(dst, v); return; }
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = v[i];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        store_bf16x8(dst + q * part, r);
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = r[i] - __bfloat162float(__float2bfloat16_rn(r[i]));
    }
}
// 8 values as e4m3 (saturating), one 8-byte store.
__device__ __forceinline__ void store_f8x8(uint8_t *dst, const float *v) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        lo |= (uint32_t)__nv_cvt_float_to_fp8(v[i], __NV_SATFINITE, __NV_E4M3) << (8 * i);
        hi |= (uint32_t)__nv_cvt_float_to_fp8(v[4 + i], __NV_SATFINITE, __NV_E4M3) << (8 * i);
    }
    *reinterpret_cast<uint2 *>(dst) = make_uint2(lo, hi);
}
__device__ __forceinline__ void store_f32x8(float *dst, const float *v) {
    reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// Staging of one 32 x 32 chunk for a TMA store, thread `lane` holding row `lane`, in the
// layouts the tensor maps' swizzle modes read: FP32 rows of 128 bytes with 128-byte swizzle
// (16-byte unit j of row r at unit j ^ (r mod 8)); BF16 rows of 64 bytes with 64-byte swizzle
// (unit j at j ^ ((r / 2) mod 4)), one 2 KB block per part of a split.  Both write eight
// different 16-byte bank groups per eight lanes, so the stores are free of bank conflicts.
__device__ __forceinline__ void stage_f32(uint8_t *buf, int lane, const float (&v)[32]) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4 *>(buf + lane * 128 + ((j ^ (lane & 7)) << 4)) =
            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}
__device__ __forceinline__ void stage_bf16(uint8_t *buf, int lane, const float (&v)[32], int parts) {
    float r[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = v[i];
    for (int q = 0; q < parts; ++q) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __align__(16) __nv_bfloat162 p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(r[8 * j + 2 * i], r[8 * j + 2 * i + 1]);
            *reinterpret_cast<uint4 *>(buf + q * 2048 + lane * 64 + ((j ^ ((lane >> 1) & 3)) << 4)) =
                *reinterpret_cast<const uint4 *>(p);
        }
        if (q + 1 < parts) {
#pragma unroll
            for (int i = 0; i < 32; ++i) r[i] = r[i] - __bfloat162float(__float2bfloat16_rn(r[i]));
        }
    }
}
__device__ __forceinline__ void stage_out(uint8_t *buf, int lane, const float (&v)[32], int kind, int parts) {
    if (kind == kOutF32) stage_f32(buf, lane, v);
    else stage_bf16(buf, lane, v, parts);
}

__device__ __forceinline__ void load_bf16x8(const __nv_bfloat16 *src, float *v) {
    uint4 raw = *reinterpret_cast<const uint4 *>(src);
    const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __bfloat1622float2(p[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// Fused epilogue math of 32 consecutive columns [c0, c0 + 32) of one row (FP32 accumulators
// in v): v becomes the layer's output o1 (FC-1: e), sv FC-1's s = h_prev + e.  s_bias / s_wa:
// per-column constants in shared memory (bias with the material's part of the configuration
// vector folded in; weight of alpha).  sc, alpha: this row's SE weight and view angle.
// pre: the residual / running-state values of this chunk.
__device__ __forceinline__ void epilogue_math(const TcGemmArgs &a, int c0, float (&v)[32], float (&sv)[32],
                                              const float *s_bias, const float *s_wa, float sc,
                                              float alpha, const float (&pre)[32],
                                              const float *s_wm, const float (&rc)[4],
                                              const float *s_ws) {
    if (a.col_scale) {                                   // FP8: per-output-channel weight scale
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= s_ws[c0 + j];
    }
    switch (a.epi) {
    case kEpiFc1: {
        // e = ReLU(w_se * acc + W_cfg c + b); s = h_prev + e
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float b = fmaf(s_wa[c0 + j], alpha, s_bias[c0 + j]);
            if (a.cfg_per_row) {                 // mixed batch: this row's g and albedo
                const float *wm = s_wm + 4 * (c0 + j);
                b = fmaf(wm[0], rc[0], fmaf(wm[1], rc[1], fmaf(wm[2], rc[2], fmaf(wm[3], rc[3], b))));
            }
            float e = fmaxf(fmaf(v[j], sc, b), 0.f);
            v[j] = e;
            sv[j] = (a.h_prev || a.pre_f32) ? pre[j] + e : e;
        }
        break;
    }
    case kEpiFc2:        // h = ReLU(acc + b) + e
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + s_bias[c0 + j], 0.f) + pre[j];
        break;
    case kEpiRelu:
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + s_bias[c0 + j], 0.f);
        break;
    default:             // kEpiPlain: the accumulators; kEpiDecode: in epilogue_emit
        break;
    }
}

// Output of one chunk.  With TMA outputs (a.o1_kind != kOutDirect) every lane stages its row
// into `stg` (o1 at 0, o2 at o2_off) and the caller issues the stores; otherwise live rows
// store through the pointers.
__device__ __forceinline__ void epilogue_emit(const TcGemmArgs &a, int r, int c0, const float (&v)[32],
                                              const float (&sv)[32], const float *s_bias,
                                              uint8_t *stg, uint32_t o2_off, int lane, bool live) {
    const int N = a.N;
    if (a.o1_kind != kOutDirect) {
        stage_out(stg, lane, v, a.o1_kind, a.o1_parts);
        if (a.o2_kind != kOutDirect) stage_out(stg + o2_off, lane, sv, a.o2_kind, a.o2_parts);
        return;
    }
    if (!live) return;
    switch (a.epi) {
    case kEpiPlain: {
        float *o = a.out_f32 + (size_t)r * a.ldo;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < N) o[c0 + j] = v[j];
        break;
    }
    case kEpiFc1:
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (c0 + 8 * g < N) {
                if (a.out_e_f32) store_f32x8(a.out_e_f32 + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g);
                else store_bf16x8(a.out_e + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g);
                if (a.out_s8) store_f8x8(a.out_s8 + (size_t)r * kWidth8 + c0 + 8 * g, sv + 8 * g);
                else store_out8(a.out_s + (size_t)r * a.ldo + c0 + 8 * g, sv + 8 * g, a.out_split, a.out_part);
            }
        break;
    case kEpiFc2:
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (c0 + 8 * g < N) {
                if (a.out_h_f32) store_f32x8(a.out_h_f32 + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g);
                else if (a.out_f8) store_f8x8(a.out_f8 + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g);
                else store_out8(a.out_bf + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g, a.out_split, a.out_part);
            }
        break;
    case kEpiRelu:
#pragma unroll
        for (int g = 0; g < 4; ++g)
            if (c0 + 8 * g < N) {
                if (a.out_f8) store_f8x8(a.out_f8 + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g);
                else store_out8(a.out_bf + (size_t)r * a.ldo + c0 + 8 * g, v + 8 * g, a.out_split, a.out_part);
            }
        break;
    default:  // kEpiDecode: rgb = I albedo^4 expm1(acc + b), N = 3
        if (c0 == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float y = v[j] + s_bias[j];
                if (a.y_out) a.y_out[(size_t)r * 3 + j] = y;
                const float ds = a.dec_rows ? a.dec_rows[(size_t)r * 3 + j] : a.dec_scale[j];
                a.out_f32[(size_t)r * 3 + j] = ds * expm1f(y);
            }
        }
        break;
    }
}

// Residual (FC-2) or running state (FC-1) of one chunk, BF16 -> FP32; zeros if absent.
__device__ __forceinline__ void load_pre(const TcGemmArgs &a, int r, int c0, float (&pre)[32]) {
    if (a.pre_f32 && (a.epi == kEpiFc1 || a.epi == kEpiFc2)) {
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            if (c0 + 4 * g < a.N) {
                float4 f = *reinterpret_cast<const float4 *>(a.pre_f32 + (size_t)r * a.ld_pre + c0 + 4 * g);
                pre[4 * g] = f.x; pre[4 * g + 1] = f.y; pre[4 * g + 2] = f.z; pre[4 * g + 3] = f.w;
            } else {
                pre[4 * g] = pre[4 * g + 1] = pre[4 * g + 2] = pre[4 * g + 3] = 0.f;
            }
        }
        return;
    }
    const __nv_bfloat16 *src = a.epi == kEpiFc1 ? a.h_prev : (a.epi == kEpiFc2 ? a.resid : nullptr);
    const int ld = a.epi == kEpiFc1 ? a.ld_h : a.ld_resid;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (src && c0 + 8 * g < a.N) load_bf16x8(src + (size_t)r * ld + c0 + 8 * g, pre + 8 * g);
        else {
#pragma unroll
            for (int i = 0; i < 8; ++i) pre[8 * g + i] = 0.f;
        }
    }
}
}  // namespace

// Threads per CTA: producer, MMA and EPI epilogue warps, plus (FP32 split) two more producer
// warps, so that each of a stage's three parts is issued by its own thread: loads issued by
// one thread complete one after another, and a split stage has six of them.
template <int EPI>
__host__ __device__ constexpr int tc_threads() { return 64 + 32 * EPI + (EPI == 4 ? 64 : 0); }

template <int EPI>
__global__ void __launch_bounds__(tc_threads<EPI>(), 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                   const __grid_constant__ CUtensorMap map_o1, const __grid_constant__ CUtensorMap map_o2,
                   const __grid_constant__ CUtensorMap map_pre, const __grid_constant__ TcGemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const bool split3 = a.n_pass > 1;              // three-part stages (FP32 split)
    const int n_stages = split3 ? STAGES3 : stages_one<EPI>();
    const uint32_t stage_bytes = split3 ? STAGE3 : A_STAGE + B_STAGE;
    const uint32_t b_off = split3 ? 3 * A_PART3 : A_STAGE;   // B's offset inside a stage
    uint8_t *staging = smem + n_stages * stage_bytes;          // epilogue warps' TMA staging
    const uint32_t stg_stride = split3 ? STG_SPLIT : stg_bufs<EPI>() * STG_ONE;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + smem_tiles<EPI>());
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *drain = acc_empty + 2;
    uint64_t *pre_full = drain + 1;           // [EPI][2] residual-chunk barriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(pre_full + 2 * EPI);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
    float *s_bias = reinterpret_cast<float *>(smem + smem_tiles<EPI>() + 256);
    float *s_wa = s_bias + TN_MAX;
    float *s_wm = s_wa + TN_MAX;              // [TN_MAX][4] weights of g and albedo (mixed)
    float *s_ws = s_wm + 4 * TN_MAX;          // FP8 weight scales

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (a.M + TM - 1) / TM;
    const int n_mma = a.n_mma;
    const uint32_t slab_tx = A_PART3 + (uint32_t)n_mma * ROW3;      // one part of A and of B
    const uint32_t stage_tx = split3 ? 3 * slab_tx : A_STAGE + (uint32_t)n_mma * TK * 2;
    // stages per tile: one per K slab; the split adds a second sweep of A0 B0, three slabs
    // per stage
    const int n_sweep1 = a.k_tiles;
    const int n_steps = split3 ? n_sweep1 + (a.k_tiles + 2) / 3 : a.k_tiles;
    const uint32_t idesc = a.fp8 ? tc::idesc_e4m3_f32(TM, n_mma) : tc::idesc_bf16_f32(TM, n_mma);
    const int tk = split3 ? kSplitSlabK : (a.fp8 ? 128 : TK);   // K elements per stage row
    const int kslice = a.fp8 ? 32 : 16;                // K elements per MMA (32 bytes)

    if (threadIdx.x == 0) {
        for (int s = 0; s < n_stages; ++s) {
            tc::mbar_init(&full[s], split3 ? 3 : 1);      // one arrival per producer thread
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) { tc::mbar_init(&acc_full[b], 1); tc::mbar_init(&acc_empty[b], EPI); }
        tc::mbar_init(drain, 1);
        for (int i = 0; i < 2 * EPI; ++i) tc::mbar_init(&pre_full[i], 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) { tc::prefetch_tmap(&map_a); tc::prefetch_tmap(&map_b); }
    if (warp == 3 && lane == 0 && a.pre_tma) tc::prefetch_tmap(&map_pre);
    if (warp == 2 && lane == 0 && a.o1_kind != kOutDirect) {
        tc::prefetch_tmap(&map_o1);
        if (a.o2_kind != kOutDirect) tc::prefetch_tmap(&map_o2);
    }
    // per-column epilogue constants (columns >= N read as zero)
    for (int c = threadIdx.x; c < TN_MAX; c += blockDim.x) {
        float b = 0.f, wa = 0.f, wm[4] = {0.f, 0.f, 0.f, 0.f};
        if (c < a.N && a.bias) {
            b = a.bias[c];
            if (a.epi == kEpiFc1) {
                const float *wc = a.w_cfg + (size_t)c * a.w_cfg_ld;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (a.cfg_per_row) wm[q] = wc[q];
                    else b += wc[q] * a.mat_cfg[q];
                }
                wa = wc[4];
            }
        }
        s_bias[c] = b;
        s_wa[c] = wa;
        s_ws[c] = (a.col_scale && c < a.N) ? a.col_scale[c] : 1.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) s_wm[4 * c + q] = wm[q];
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;
    // Programmatic dependent launch: everything above reads only the weights, so it overlaps
    // the previous layer's tail; the activations it wrote are read only after it completes.
    // This kernel's own dependents may launch now: they wait for its completion the same way,
    // and every CTA of this grid is already resident.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // producer threads: warp 0, and with the split warps 2 + EPI and 3 + EPI; producer pi
    // loads part pi of each first-sweep slab and slab pi of each second-sweep stage
    const bool producer = warp == 0 || (split3 && EPI == 4 && warp >= 2 + EPI);
    if (producer) {
        const int pi = warp == 0 ? 0 : warp - (1 + EPI);
        if (lane == 0) {
            int it = 0;
            for (int tile = blockIdx.x; tile < n_tiles && !*(volatile int *)abort_flag; tile += gridDim.x) {
                for (int step = 0; step < n_steps; ++step, ++it) {
                    const int s = it % n_stages;
                    const uint32_t ph = (it / n_stages) & 1;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1)) { record_timeout(a.err, abort_flag); break; }
                    uint8_t *st = smem + s * stage_bytes;
                    if (!split3) {
                        tc::mbar_expect_tx(&full[s], stage_tx);
                        tc::tma_load_2d(st, &map_a, a.a_col0 + step * tk, tile * TM, &full[s]);
                        tc::tma_load_2d(st + b_off, &map_b, step * tk, 0, &full[s]);
                    } else if (step < n_sweep1) {              // slab `step`, part pi
                        tc::mbar_expect_tx(&full[s], slab_tx);
                        tc::tma_load_2d(st + pi * A_PART3, &map_a, a.a_col0 + step * tk,
                                        pi * a.a_part_rows + tile * TM, &full[s]);
                        tc::tma_load_2d(st + b_off + pi * B_PART3, &map_b, step * tk,
                                        pi * a.b_part_rows, &full[s]);
                    } else {                                   // slab j0 + pi of A0 B0, if any
                        const int j0 = 3 * (step - n_sweep1);
                        const int nb = a.k_tiles - j0 < 3 ? a.k_tiles - j0 : 3;
                        if (pi < nb) {
                            tc::mbar_expect_tx(&full[s], slab_tx);
                            tc::tma_load_2d(st + pi * A_PART3, &map_a, a.a_col0 + (j0 + pi) * tk,
                                            tile * TM, &full[s]);
                            tc::tma_load_2d(st + b_off + pi * B_PART3, &map_b, (j0 + pi) * tk, 0,
                                            &full[s]);
                        } else {
                            tc::mbar_arrive(&full[s]);
                        }
                    }
                }
            }
            // wait until every stage issued has landed (the consumer may have stopped early)
            for (int j = 0; j < n_stages && j < it; ++j) {
                const int i2 = it - 1 - j;
                tc::mbar_wait(&full[i2 % n_stages], (i2 / n_stages) & 1, 1u << 16);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, t = 0;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
                if (*(volatile int *)abort_flag) break;
                const int buf = t & 1;
                if (!tc::mbar_wait(&acc_empty[buf], ((t >> 1) & 1) ^ 1)) { record_timeout(a.err, abort_flag); break; }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem_base + buf * 256;
                bool ok = true;
                auto slices = [&](int kt) {                    // MMAs of K slab kt
                    const int k_left = a.K - kt * tk;
                    return k_left >= tk ? tk / kslice : (k_left + kslice - 1) / kslice;
                };
                for (int step = 0; step < n_steps; ++step, ++it) {
                    const int s = it % n_stages;
                    if (!tc::mbar_wait(&full[s], (it / n_stages) & 1)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t a_addr = tc::smem_u32(smem + s * stage_bytes);
                    const uint32_t b_addr = a_addr + b_off;
                    if (!split3) {
                        const int n_sl = slices(step);
                        for (int k = 0; k < n_sl; ++k) {
                            const uint64_t ad = tc::smem_desc_sw128(a_addr + k * 32);
                            const uint64_t bd = tc::smem_desc_sw128(b_addr + k * 32);
                            if (a.fp8) tc::mma_f8(d_tmem, ad, bd, idesc, (step | k) != 0);
                            else tc::mma_f16(d_tmem, ad, bd, idesc, (step | k) != 0);
                        }
                    } else if (step < n_sweep1) {
                        // first sweep: the five products below the leading one, smallest
                        // first, so that the accumulator holds only small terms while they
                        // are summed
                        const int n_sl = slices(step);
                        for (int p = 0; p < 5; ++p) {
                            const uint32_t pa = a_addr + kPassA[p] * A_PART3;
                            const uint32_t pb = b_addr + kPassB[p] * B_PART3;
                            for (int k = 0; k < n_sl; ++k)
                                tc::mma_f16(d_tmem, split_desc(pa + k * 32), split_desc(pb + k * 32), idesc,
                                            (step | p | k) != 0);
                        }
                    } else {
                        // second sweep: the leading product A0 B0 on top
                        const int j0 = 3 * (step - n_sweep1);
                        const int nb = a.k_tiles - j0 < 3 ? a.k_tiles - j0 : 3;
                        for (int j = 0; j < nb; ++j) {
                            const int n_sl = slices(j0 + j);
                            for (int k = 0; k < n_sl; ++k)
                                tc::mma_f16(d_tmem, split_desc(a_addr + j * A_PART3 + k * 32),
                                            split_desc(b_addr + j * B_PART3 + k * 32), idesc, 1);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) { record_timeout(a.err, abort_flag); break; }
                tc::mma_commit(&acc_full[buf]);
            }
            // all MMAs issued by this thread complete before TMEM is released
            tc::mma_commit(drain);
            tc::mbar_wait(drain, 0, 1u << 20);
        }
    } else if (warp < 2 + EPI) {
        const int q = warp & 3;                        // TMEM lane quarter of this warp
        // which 32-column chunks this warp takes: every one (EPI 4) or every other (EPI 8)
        const int half = EPI == 8 ? (warp - 2) >> 2 : 0;
        constexpr int kStride = EPI == 8 ? 64 : 32;
        const bool staged = a.o1_kind != kOutDirect;
        uint8_t *stg = staging + (warp - 2) * stg_stride;
        const uint32_t o2_off = a.o1_kind == kOutF32 ? 4096u : 2048u * (uint32_t)a.o1_parts;
        // each 32 x 32 residual chunk of this warp arrives by TMA, two chunks ahead, in one of
        // its two buffers: FP32 rows of 128 bytes (128-byte swizzle: unit j of row r at
        // j ^ (r mod 8)) with the split, BF16 rows of 64 bytes (64-byte swizzle: unit j at
        // j ^ ((r / 2) mod 4)) otherwise
        const bool pre_tma = a.pre_tma != 0;
        const bool pre_f32 = a.pre_tma == 1;
        const uint32_t pre_chunk = pre_f32 ? 4096u : 2048u;
        uint8_t *pbuf = staging + EPI * stg_stride + (warp - 2) * 2 * pre_chunk;
        uint64_t *pbar = pre_full + 2 * (warp - 2);
        uint32_t pre_issued = 0, pre_used = 0;
        uint32_t n_staged = 0;                         // chunks staged by this warp
        auto issue_pre = [&](int c0, int row0) {
            const int b = pre_issued & 1;
            if (lane == 0) {
                tc::mbar_expect_tx(&pbar[b], pre_chunk);
                tc::tma_load_3d(pbuf + b * pre_chunk, &map_pre, c0, row0, 0, &pbar[b]);
            }
            ++pre_issued;
        };
        int t = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
            const int buf = t & 1;
            const int r = tile * TM + q * 32 + lane;
            const bool live = r < a.M;
            float sc = 0.f, alpha = 0.f, rc[4] = {0.f, 0.f, 0.f, 0.f};
            if (live && a.epi == kEpiFc1) {
                sc = a.row_scale[(size_t)r * a.row_scale_ld];
                if (a.row_scale2) sc *= a.row_scale2[(size_t)r * a.row_scale2_ld];
                alpha = a.cfg[(size_t)r * kCfg + 4];
                if (a.cfg_per_row)
                    for (int q = 0; q < 4; ++q) rc[q] = a.cfg[(size_t)r * kCfg + q];
            }
            float pre[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) pre[i] = 0.f;
            const int row0 = tile * TM + q * 32;
            if (pre_tma) {
                if (half * 32 < a.N) issue_pre(half * 32, row0);
                if (half * 32 + kStride < a.N) issue_pre(half * 32 + kStride, row0);
            } else if (live && half * 32 < a.N) {
                load_pre(a, r, half * 32, pre);
            }
            bool ok = tc::mbar_wait(&acc_full[buf], (t >> 1) & 1);
            if (!ok || *(volatile int *)abort_flag) {
                if (!ok && lane == 0) record_timeout(a.err, abort_flag);
                break;
            }
            tc::fence_after_sync();
            const uint32_t lane_addr = tmem_base + buf * 256 + ((uint32_t)(q * 32) << 16);
            for (int c0 = half * 32; c0 < a.N; c0 += kStride) {
                float v[32];
                tc::tmem_ld32(lane_addr + c0, v);
                float cur[32];
                if (pre_tma) {
                    const int b = pre_used & 1;
                    const uint32_t ph = (pre_used >> 1) & 1;
                    ++pre_used;
                    if (!tc::mbar_wait(&pbar[b], ph)) {
                        if (lane == 0) record_timeout(a.err, abort_flag);
                        ok = false;
                        break;
                    }
                    if (pre_f32) {
                        const uint8_t *src = pbuf + b * pre_chunk + lane * 128;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 f = *reinterpret_cast<const float4 *>(src + ((j ^ (lane & 7)) << 4));
                            cur[4 * j] = f.x; cur[4 * j + 1] = f.y; cur[4 * j + 2] = f.z; cur[4 * j + 3] = f.w;
                        }
                    } else {
                        const uint8_t *src = pbuf + b * pre_chunk + lane * 64;
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            load_bf16x8(reinterpret_cast<const __nv_bfloat16 *>(src + ((j ^ ((lane >> 1) & 3)) << 4)),
                                        cur + 8 * j);
                    }
                    __syncwarp();                      // every lane has read buffer b
                    if (c0 + 2 * kStride < a.N) issue_pre(c0 + 2 * kStride, row0);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) cur[i] = pre[i];
                    // next chunk's residual loads overlap this chunk's TMEM load and math
                    if (live && c0 + kStride < a.N) load_pre(a, r, c0 + kStride, pre);
                }
                tc::tmem_ld_wait();
                float sv[32];
                epilogue_math(a, c0, v, sv, s_bias, s_wa, sc, alpha, cur, s_wm, rc, s_ws);
                // this chunk's staging buffer: the stores that last read it (one chunk ago
                // with one buffer, two with two) are done reading
                uint8_t *sb = stg + (stg_bufs<EPI>() == 2 ? (n_staged & 1) * STG_ONE : 0);
                if (staged) {
                    if (lane == 0) {
                        if (stg_bufs<EPI>() == 2) tc::bulk_wait_read1();
                        else tc::bulk_wait_read();
                    }
                    __syncwarp();
                }
                epilogue_emit(a, r, c0, v, sv, s_bias, sb, o2_off, lane, live);
                if (staged) {
                    tc::fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tc::tma_store_3d(&map_o1, sb, c0, row0, 0);
                        if (a.o2_kind != kOutDirect) tc::tma_store_3d(&map_o2, sb + o2_off, c0, row0, 0);
                        tc::bulk_commit();
                    }
                    ++n_staged;
                }
            }
            if (!ok) break;
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
        }
        // residual loads still in flight (after a time-out) land before the CTA exits
        for (; pre_used < pre_issued; ++pre_used)
            tc::mbar_wait(&pbar[pre_used & 1], (pre_used >> 1) & 1, 1u << 16);
        if (staged && lane == 0) tc::bulk_wait();     // every store of this warp has landed
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, 512);
    }
}

__global__ void pack_bf16_kernel(const float *__restrict__ src, int N, int K, int ld_src,
                                 __nv_bfloat16 *__restrict__ dst, int Np, int Kp, int part) {
    size_t total = (size_t)Np * Kp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        int n = (int)(i / Kp), k = (int)(i % Kp);
        float x = n < N && k < K ? src[(size_t)n * ld_src + k] : 0.f;
        dst[i] = __float2bfloat16_rn(part > 0 ? split_residual(x, part) : x);
    }
}

void launch_pack_bf16(const float *src, int N, int K, int ld_src, __nv_bfloat16 *dst, int Np,
                      int Kp, cudaStream_t s, int split_part) {
    size_t total = (size_t)Np * Kp;
    int blocks = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
    note_launch();
    pack_bf16_kernel<<<blocks, 256, 0, s>>>(src, N, K, ld_src, dst, Np, Kp, split_part);
}

// FP8 weights: one warp per output row n finds max |W[n][:K]| and writes the row scale and
// the e4m3 values W / scale (zero padding beyond N and K).
__global__ void pack_fp8_kernel(const float *__restrict__ src, int N, int K, int ld_src,
                                uint8_t *__restrict__ dst, float *__restrict__ scale, int Np, int Kp) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= Np) return;
    float mx = 0.f;
    if (n < N)
        for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(src[(size_t)n * ld_src + k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(~0u, mx, o));
    const float sc = mx > 0.f ? mx / 448.f : 1.f;
    if (lane == 0) scale[n] = sc;
    for (int k = lane; k < Kp; k += 32) {
        float x = (n < N && k < K) ? src[(size_t)n * ld_src + k] / sc : 0.f;
        dst[(size_t)n * Kp + k] = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
    }
}

void launch_pack_fp8(const float *src, int N, int K, int ld_src, uint8_t *dst, float *scale,
                     int Np, int Kp, cudaStream_t s) {
    note_launch();
    pack_fp8_kernel<<<(Np + 7) / 8, 256, 0, s>>>(src, N, K, ld_src, dst, scale, Np, Kp);
}

void launch_tc_gemm(const TcGemmArgs &a, const CUtensorMap &map_a, const CUtensorMap &map_b,
                    int num_sms, cudaStream_t s, const CUtensorMap *map_o1, const CUtensorMap *map_o2,
                    const CUtensorMap *map_pre) {
    static const CUtensorMap unused{};            // stands in for outputs written directly
    if (a.M <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<4>());
        cudaFuncSetAttribute(tc_gemm_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<8>());
        attr_set = true;
    }
    int tiles = (a.M + TM - 1) / TM;
    int grid = tiles < num_sms ? tiles : num_sms;
    note_launch();
    const CUtensorMap &o1 = map_o1 ? *map_o1 : unused, &o2 = map_o2 ? *map_o2 : unused;
    const CUtensorMap &pr = map_pre ? *map_pre : unused;
    // launched as a programmatic dependent of the previous kernel in the stream (see the
    // griddepcontrol instructions in the kernel)
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (a.n_pass > 1) {
        cfg.blockDim = dim3(tc_threads<4>());
        cfg.dynamicSmemBytes = smem_bytes<4>();
        cudaLaunchKernelEx(&cfg, tc_gemm_kernel<4>, map_a, map_b, o1, o2, pr, a);
    } else {
        cfg.blockDim = dim3(tc_threads<8>());
        cfg.dynamicSmemBytes = smem_bytes<8>();
        cudaLaunchKernelEx(&cfg, tc_gemm_kernel<8>, map_a, map_b, o1, o2, pr, a);
    }
}

}  // namespace nis
