// The network after the features, fused (Sec. III.C.2, Fig. 6; Eq. 21): per type the
// diffuse and highlight chains of blocks
//   e = ReLU(W1 [w_se x_k; c] + b1),  h_k = ReLU(W2 (h_{k-1} + e) + b2) + e,
// the merge of each type's two chain ends, the head 600 -> 200 -> 200 -> 3 and the decode
// F = I albedo^4 expm1(y), for 128-point tiles in one persistent tcgen05 kernel: BF16
// operands, FP32 accumulation in tensor memory, the running state on chip.
//
// One CTA per SM, 12 warps:
//   warps 0, 11 producers of ring G: per 64-column K block of an op whose operand is in
//               global memory (FC-1, merge, head 1), its weight block (pre-swizzled in global
//               memory, L2-resident) by a 1-D bulk copy (warp 0) and the 128 x 64 operand box
//               by TMA (warp 11) into one slot, completing on the slot's barrier
//   warp 1      TMEM owner and MMA issuer: per block one barrier wait, up to four
//               128 x N x 16 tcgen05.mma (N = 208, or 16 for the last head layer), one commit
//               per slot; two accumulator regions X (columns 0-207) and Y (256-463) used by
//               alternate ops, so one op's epilogue overlaps the next op's MMAs
//   warp 2      producer of ring S: the weight blocks of the ops whose operand is the s buffer
//               (FC-2, head 2 and 3), so that they do not queue behind ring G's; prefetches
//               feature boxes a few ops ahead into L2
//   warps 3-10  epilogue, two warps per TMEM lane quarter, each thread one row; the two
//               warps of a quarter take alternate 32-column chunks
// Per tile the ops run in the order of fused_program: for each type, FC-1 / FC-2 of the
// diffuse layers 0-7, then of the highlight layers 8-11, then the merge; then the head.
//   FC-1  A = the layer's features followed by 13 configuration columns holding c / w_se and
//         1 / w_se (two BF16 parts each) against W_c and the bias:
//         acc = W1 x + (W_c c + b) / w_se, and e = w_se ReLU(acc) (w_se > 0, so this is
//         Eq. 26's scaling inside the block).  s = h_{k-1} + e goes to the on-chip s buffer
//         (BF16, FC-2's operand), e to the state.
//   FC-2  A = s (64-column blocks consumed as the epilogue finishes them); h = ReLU(acc) + e
//         to the state, or, at a chain end, to global memory (BF16) for the merge.
//   merge, head: A from global memory (chain ends, merge outputs) or the s buffer; biases
//         ride in two operand columns of ones against the bias's two BF16 parts.
// State of a row: the 200 values e or h (they replace each other in place), BF16 pairs in the
// 96 TMEM columns left over by X and Y for columns 0-191, FP32 in shared memory for 192-199.
// Every mbarrier wait is bounded: on a time-out the kernel records kErrTimeout in the
// context's error word and winds down (draining its MMAs and copies before releasing TMEM).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "nis_internal.h"
#include "tc_common.h"

namespace nis {

namespace {
constexpr int FM = 128;                                // rows per tile
// Two rings of shared-memory slots, each with its own producer thread, so that the weights of
// an op whose operand is in global memory (FC-1, merge, head 1: ring G, slots of a weight
// block and an operand box) are fetched while an FC-2 still waits for its s blocks (ring S,
// weight blocks only).
constexpr int NG = 2, NS = 3;
constexpr uint32_t B_SLOT = 208 * 128;                 // [208][64] BF16, 128-byte rows
constexpr uint32_t A_SLOT = FM * 128;                  // [128][64] BF16
constexpr uint32_t G_SLOT = B_SLOT + A_SLOT;           // weight block, then operand box
constexpr uint32_t S_BLK = FM * 128;                   // s buffer: 3 blocks of 64 columns ...
constexpr uint32_t S_BYTES = 3 * S_BLK + FM * 32;      // ... and a 16-column tail (32-byte rows)
constexpr uint32_t OFF_SR = NG * G_SLOT;              // ring S
constexpr uint32_t OFF_S = OFF_SR + NS * B_SLOT;
constexpr uint32_t OFF_ST6 = OFF_S + S_BYTES;          // state of chunk 6: [128][16] FP32
constexpr uint32_t OFF_BAR = OFF_ST6 + FM * 64;
constexpr uint32_t OFF_OPS = OFF_BAR + 512;
constexpr uint32_t SMEM_FUSED = OFF_OPS + kFuseMaxOps * sizeof(FusedOp) + 1024;   // + alignment
static_assert(SMEM_FUSED <= 227 * 1024, "shared memory of mlp_fused_kernel");
static_assert(B_SLOT % 1024 == 0 && G_SLOT % 1024 == 0 && OFF_SR % 1024 == 0 && OFF_S % 1024 == 0 && S_BLK % 1024 == 0,
              "slots keep the 1024-byte swizzle-atom alignment");
constexpr int kPrefetchOps = 5;                        // L2 prefetch distance of the features
constexpr int kWarps = 12, kThreads = kWarps * 32;
constexpr int kEpiWarps = 8;
// barriers (uint64 each) at OFF_BAR
constexpr int GF = 0, GE = GF + NG, SF = GE + NG, SE = SF + NS;    // slots: full / empty
constexpr int XF = SE + NS, XE = XF + 1, YF = XE + 1, YE = YF + 1; // accumulators: full / free
constexpr int SR = YE + 1;                                         // s blocks 0-2 and tail
constexpr int MR = SR + 4, HR = MR + 1, DR = HR + 1, NBAR = DR + 1; // chain ends, merges, drain
static_assert(NBAR * 8 <= 384, "barrier area");

__device__ __forceinline__ void record_timeout(unsigned *err, int *abort_flag) {
    *(volatile int *)abort_flag = 1;
    if (err) atomicOr(err, kErrTimeout);
}
__device__ __forceinline__ bool aborted(const int *abort_flag) { return *(const volatile int *)abort_flag != 0; }

// An op's weight/operand blocks: 64-column blocks of its K, or, for an e4m3 FC-1, two
// 128-column e4m3 blocks and the 16-column configuration block.
// column of an e4m3 FC-1's configuration operand in the [rows][12 x 2 x 16] source
__device__ __forceinline__ int cfg8_col(const FusedOp &op) { return (op.layer * 2 + op.type) * 16; }

// 8 floats as BF16, one 16-byte word
__device__ __forceinline__ uint4 pack8(const float *v) {
    __align__(16) __nv_bfloat162 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return *reinterpret_cast<const uint4 *>(p);
}

// The running state of chunk c (0..5, 32 columns) of a row: 16 TMEM columns of packed BF16
// pairs (column j holds output columns 32 c + 2 j, + 1), in the columns left over by X and Y
__device__ __forceinline__ uint32_t state_col(int c) { return c < 3 ? 208u + 16u * c : 464u + 16u * (c - 3); }
__device__ __forceinline__ float pack2(float x, float y) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    return __uint_as_float(*reinterpret_cast<uint32_t *>(&h));
}
__device__ __forceinline__ float2 unpack2(float p) {
    uint32_t u = __float_as_uint(p);
    return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u));
}
// chunk 6 (the 16-column tail, 8 outputs used) of the state in shared memory, FP32 rows of
// 64 bytes, 16-byte unit j at j ^ ((row / 2) mod 4): eight lanes cover eight bank groups
__device__ __forceinline__ void tail_state_load(const uint8_t *smem, int rl, float (&h)[16]) {
    const uint8_t *row = smem + OFF_ST6 + rl * 64;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 f = *reinterpret_cast<const float4 *>(row + ((j ^ ((rl >> 1) & 3)) << 4));
        h[4 * j] = f.x; h[4 * j + 1] = f.y; h[4 * j + 2] = f.z; h[4 * j + 3] = f.w;
    }
}
__device__ __forceinline__ void tail_state_store(uint8_t *smem, int rl, const float (&h)[16]) {
    uint8_t *row = smem + OFF_ST6 + rl * 64;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4 *>(row + ((j ^ ((rl >> 1) & 3)) << 4)) =
            make_float4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
}

// Chunk c of the s buffer (the A operand of the next op) for this thread's row, in the
// layouts the MMA descriptors read: 64-column blocks with 128-byte swizzle (16-byte unit u of
// row r at u ^ (r mod 8); chunk c is units 4 (c mod 2) .. +3 of block c / 2), the 16-column
// tail (chunk 6) with 32-byte swizzle (unit u at u ^ ((r / 4) mod 2)).
template <int W>
__device__ __forceinline__ void write_s(uint8_t *smem, int c, int rl, const float (&s)[W]) {
    if constexpr (W == 32) {
        uint8_t *row = smem + OFF_S + (c >> 1) * S_BLK + rl * 128;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint4 *>(row + (((4 * (c & 1) + j) ^ (rl & 7)) << 4)) = pack8(s + 8 * j);
    } else {
        uint8_t *row = smem + OFF_S + 3 * S_BLK + rl * 32;
#pragma unroll
        for (int j = 0; j < 2; ++j) *reinterpret_cast<uint4 *>(row + ((j ^ ((rl >> 2) & 1)) << 4)) = pack8(s + 8 * j);
    }
}

// W columns of a row to global memory as BF16; for the tail chunk (W = 16) only the 8 real
// columns of a 208-column output
template <int W>
__device__ __forceinline__ void write_row(__nv_bfloat16 *dst, const float (&v)[W]) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int j = 0; j < (W == 32 ? 4 : 1); ++j) d[j] = pack8(v + 8 * j);
}
// the tail after a 200-wide operand: [1, 1, 0 ...] (words of 8 columns)
__device__ __forceinline__ void write_ones_tail(__nv_bfloat16 *dst, int words) {
    const float t[8] = {1.f, 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = pack8(t);
    for (int j = 1; j < words; ++j) d[j] = pack8(z);
}

// s chunk c is written: publish it to the MMA (async proxy) and count it on its block
__device__ __forceinline__ void s_done(uint64_t *bar, int c, int lane) {
    tc::fence_async_smem();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&bar[SR + (c >> 1)]);
}

// One 32-column chunk c (0..5) of an op's epilogue, thread = row rl.  The accumulator chunk and
// the state chunk are loaded together (one wait).
__device__ __forceinline__ void epi_chunk32(const FusedOp &op, int c, uint32_t acc_tm, uint32_t lane_tm,
                                            uint8_t *smem, uint64_t *bar, int rl, int r, bool live, float sc,
                                            const FusedArgs &a, int lane) {
    float v[32], st[16];
    tc::tmem_ld32(acc_tm + 32 * c, v);
    const bool first = op.flags & 1;
    if ((op.kind == kFuseFc1 && !first) || op.kind == kFuseFc2) tc::tmem_ld16(lane_tm + state_col(c), st);
    tc::tmem_ld_wait();
    switch (op.kind) {
    case kFuseFc1: {
        // e = w_se ReLU(acc) to the state; s = h + e (e at a chain's first layer) to the s buffer
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float e0 = fmaxf(v[2 * j], 0.f) * sc, e1 = fmaxf(v[2 * j + 1], 0.f) * sc;
            const float2 h = first ? make_float2(0.f, 0.f) : unpack2(st[j]);
            v[2 * j] = h.x + e0;
            v[2 * j + 1] = h.y + e1;
            st[j] = pack2(e0, e1);
        }
        tc::tmem_st16(lane_tm + state_col(c), st);
        write_s<32>(smem, c, rl, v);
        s_done(bar, c, lane);
        break;
    }
    case kFuseFc2: {
        // h = ReLU(acc) + e to the state, or at a chain end to the merge operand
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float2 e = unpack2(st[j]);
            v[2 * j] = fmaxf(v[2 * j], 0.f) + e.x;
            v[2 * j + 1] = fmaxf(v[2 * j + 1], 0.f) + e.y;
            st[j] = pack2(v[2 * j], v[2 * j + 1]);
        }
        if (op.flags & 2) {
            if (live)
                write_row<32>(a.mrg + (size_t)r * (3 * kFuseMrgLd) + op.type * kFuseMrgLd + op.chain * kWidth + 32 * c, v);
        } else {
            tc::tmem_st16(lane_tm + state_col(c), st);
        }
        break;
    }
    case kFuseMerge: {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
        if (live) write_row<32>(a.head + (size_t)r * kFuseHeadLd + op.type * kWidth + 32 * c, v);
        break;
    }
    default: {                                        // kFuseHead1, kFuseHead2
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
        write_s<32>(smem, c, rl, v);
        s_done(bar, c, lane);
        break;
    }
    }
}

// The 16-column tail of an op's epilogue: chunk 6 of a 208-column op (8 real outputs; state
// in shared memory), or the 16 columns of the last head layer (chunk 0: the decode, Eq. 21).
__device__ __forceinline__ void epi_tail(const FusedOp &op, int c, uint32_t acc_tm, uint8_t *smem, uint64_t *bar,
                                         int rl, int r, bool live, float sc, const FusedArgs &a, int lane) {
    float v[16], h[16];
    tc::tmem_ld16(acc_tm + 32 * c, v);
    tc::tmem_ld_wait();
    switch (op.kind) {
    case kFuseFc1: {
        const bool first = op.flags & 1;
        if (!first) tail_state_load(smem, rl, h);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = fmaxf(v[j], 0.f) * sc;
            h[j] = first ? v[j] : h[j] + v[j];
        }
        tail_state_store(smem, rl, v);
        h[8] = 1.f; h[9] = 1.f;                        // FC-2's bias columns 200, 201
        write_s<16>(smem, c, rl, h);
        s_done(bar, c, lane);
        break;
    }
    case kFuseFc2: {
        tail_state_load(smem, rl, h);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f) + h[j];
        if (op.flags & 2) {
            if (live) {
                __nv_bfloat16 *row = a.mrg + (size_t)r * (3 * kFuseMrgLd) + op.type * kFuseMrgLd;
                write_row<16>(row + op.chain * kWidth + 32 * c, v);
                if (op.chain == 1) write_ones_tail(row + 2 * kWidth, 2);
            }
        } else {
            tail_state_store(smem, rl, v);
        }
        break;
    }
    case kFuseMerge: {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        if (live) {
            __nv_bfloat16 *row = a.head + (size_t)r * kFuseHeadLd;
            write_row<16>(row + op.type * kWidth + 32 * c, v);
            if (op.type == 2) write_ones_tail(row + 3 * kWidth, 1);
        }
        break;
    }
    case kFuseHead1:
    case kFuseHead2: {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        v[8] = 1.f; v[9] = 1.f;                        // the next layer's bias columns
        write_s<16>(smem, c, rl, v);
        s_done(bar, c, lane);
        break;
    }
    default: {                                        // kFuseHead3: the decode (Eq. 21)
        if (live) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float y = v[j];
                const float ds = a.dec_rows ? a.dec_rows[(size_t)r * 3 + j] : a.dec_scale[j];
                if (a.y_out) a.y_out[(size_t)r * 3 + j] = y;
                a.rgb[(size_t)r * 3 + j] = ds * expm1f(y);
            }
        }
        break;
    }
    }
}
}  // namespace

// kF8: the e4m3 mode (a separate instantiation, so that the BF16 kernel's issue loops carry
// none of its branches)
template <bool kF8>
__global__ void __launch_bounds__(kThreads, 1)
    mlp_fused_kernel(const __grid_constant__ FusedMaps maps, const __grid_constant__ FusedArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + 384);
    int *abort_flag = reinterpret_cast<int *>(smem + OFF_BAR + 388);
    FusedOp *ops = reinterpret_cast<FusedOp *>(smem + OFF_OPS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (a.M + FM - 1) / FM;
    const int n_ops = a.n_ops;

    for (int i = threadIdx.x; i < n_ops * 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(ops)[i] = reinterpret_cast<const uint32_t *>(a.ops)[i];
    if (threadIdx.x == 0) {
        // a G slot fills from two lanes (weight block, operand box): two arrivals per phase
        for (int s = 0; s < NG; ++s) { tc::mbar_init(&bar[GF + s], 2); tc::mbar_init(&bar[GE + s], 1); }
        for (int s = 0; s < NS; ++s) { tc::mbar_init(&bar[SF + s], 1); tc::mbar_init(&bar[SE + s], 1); }
        tc::mbar_init(&bar[XF], 1); tc::mbar_init(&bar[YF], 1);
        tc::mbar_init(&bar[XE], kEpiWarps); tc::mbar_init(&bar[YE], kEpiWarps);
        for (int b = 0; b < 3; ++b) tc::mbar_init(&bar[SR + b], 8);   // both warps of each quarter
        tc::mbar_init(&bar[SR + 3], 4);                               // the tail: half 0 only
        tc::mbar_init(&bar[MR], kEpiWarps); tc::mbar_init(&bar[HR], kEpiWarps);
        tc::mbar_init(&bar[DR], 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        for (int i = 0; i < kFuseSrcs; ++i) tc::prefetch_tmap(&maps.m64[i]);
        if (kF8) tc::prefetch_tmap(&maps.cfg8);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 || warp == 2 || warp == 11) {
        // ---- producers.  Bulk copies issued by one thread complete one after another, and
        // lanes of one warp that wait hold each other up, so each copy stream has a warp of its
        // own: ring G's weight blocks (warp 0) and operand boxes (warp 11) of the ops whose
        // operand is in global memory fill a slot together; ring S's weight blocks of the
        // s-buffer ops (warp 2), which also prefetches the feature boxes kPrefetchOps ops ahead
        // into L2 as it goes.
        const bool ring_g = warp != 2;
        const bool is_a = warp == 11;
        if (lane == 0) {
            const int ns = ring_g ? NG : NS;
            const int full = ring_g ? GF : SF, empty = ring_g ? GE : SE;
            const uint32_t slot = ring_g ? G_SLOT : B_SLOT, base = ring_g ? 0u : OFF_SR;
            uint32_t it = 0, mr = 0, hr = 0;
            bool ok = true;
            const uint64_t keep = tc::policy_evict_last();   // every CTA re-reads the weights
            const uint64_t once = tc::policy_evict_first();  // operands: read once
            // L2 prefetch of block j (all blocks if j < 0) of the feature op i of the tile at row y
            auto prefetch = [&](int i, int y, int j) {
                const FusedOp &op = ops[i];
                if (op.src > kSrcT) return;
                const bool f8 = kF8 && (op.flags & kFuseF8Flag) != 0;
                for (int b = 0; b < (f8 ? 3 : (op.k + 63) / 64); ++b)
                    if (j < 0 || b == j) {
                        if (f8 && b == 2) tc::tma_prefetch_2d(&maps.cfg8, cfg8_col(op), y);
                        else tc::tma_prefetch_2d(&maps.m64[op.src], op.a_col0 + (f8 ? 128 : 64) * b, y);
                    }
            };
            if (!ring_g && blockIdx.x < n_tiles)
                for (int i = 0; i < kPrefetchOps && i < n_ops; ++i) prefetch(i, blockIdx.x * FM, -1);
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
                for (int i = 0; i < n_ops && ok; ++i) {
                    const FusedOp op = ops[i];
                    const int y = tile * FM;
                    const bool a_glob = op.src != kSrcS;
                    if (a_glob != ring_g) continue;
                    // operands written by this CTA's epilogue (chain ends, merge outputs): wait
                    // until they are out before loading any block of the op
                    if (is_a && (op.src == kSrcMrg || op.src == kSrcHead)) {
                        uint32_t &cnt = op.src == kSrcMrg ? mr : hr;
                        if (!tc::mbar_wait(&bar[op.src == kSrcMrg ? MR : HR], cnt & 1)) {
                            record_timeout(a.err, abort_flag);
                            ok = false;
                            break;
                        }
                        ++cnt;
                    }
                    const uint8_t *src = a.wpack + op.b_off;
                    const bool f8 = kF8 && (op.flags & kFuseF8Flag) != 0;
                    const int nblk = f8 ? 3 : (op.k + 63) / 64;
                    for (int j = 0; j < nblk; ++j, ++it) {
                        // 32-byte rows: the s buffer's 16-column tail, or an e4m3 op's
                        // configuration block
                        const bool tail = f8 ? j == 2 : (!a_glob && op.k - 64 * j == 16);
                        const uint32_t bbytes = (uint32_t)op.n_mma * (tail ? 32u : 128u);
                        const int ss = it % ns;
                        if (aborted(abort_flag)) { ok = false; break; }
                        if (!tc::mbar_wait(&bar[empty + ss], ((it / ns) & 1) ^ 1)) {
                            record_timeout(a.err, abort_flag);
                            ok = false;
                            break;
                        }
                        uint8_t *dst = smem + base + ss * slot;
                        if (!is_a) {
                            tc::mbar_expect_tx(&bar[full + ss], bbytes);
                            tc::bulk_load_hint(dst, src, bbytes, &bar[full + ss], keep);
                            if (!ring_g) {
                                if (i + kPrefetchOps < n_ops) prefetch(i + kPrefetchOps, y, j);
                                else if (tile + (int)gridDim.x < n_tiles)
                                    prefetch(i + kPrefetchOps - n_ops, y + gridDim.x * FM, j);
                            }
                        } else if (f8 && j == 2) {
                            tc::mbar_expect_tx(&bar[full + ss], FM * 32);
                            tc::tma_load_2d_hint(dst + B_SLOT, &maps.cfg8, cfg8_col(op), y, &bar[full + ss], once);
                        } else {
                            tc::mbar_expect_tx(&bar[full + ss], A_SLOT);
                            tc::tma_load_2d_hint(dst + B_SLOT, &maps.m64[op.src], op.a_col0 + (f8 ? 128 : 64) * j, y,
                                                 &bar[full + ss], once);
                        }
                        src += bbytes;
                    }
                }
            // every copy issued lands before the CTA exits (the consumer may have stopped)
            for (uint32_t j = 0; j < (uint32_t)ns && j < it; ++j) {
                const uint32_t i2 = it - 1 - j;
                tc::mbar_wait(&bar[full + i2 % ns], (i2 / ns) & 1, 1u << 16);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            uint32_t g_it = 0, s_it = 0, xu = 0, yu = 0, sg = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
                for (int i = 0; i < n_ops && ok; ++i) {
                    const FusedOp op = ops[i];
                    const bool on_y = (op.flags & 4) != 0;
                    const uint32_t u = on_y ? yu++ : xu++;
                    if (aborted(abort_flag) || !tc::mbar_wait(&bar[on_y ? YE : XE], (u & 1) ^ 1)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t d = tmem_base + (on_y ? 256u : 0u);
                    const uint32_t idesc = tc::idesc_bf16_f32(FM, op.n_mma);
                    const bool a_glob = op.src != kSrcS;
                    const bool f8 = kF8 && (op.flags & kFuseF8Flag) != 0;
                    const int nblk = f8 ? 3 : (op.k + 63) / 64;
                    for (int j = 0; j < nblk; ++j) {
                        const int w = op.k - 64 * j < 64 ? op.k - 64 * j : 64;
                        const bool tail = f8 ? j == 2 : (!a_glob && w == 16);
                        uint32_t a_addr, b_addr;
                        uint64_t *freed;
                        if (a_glob) {
                            const int gs = g_it % NG;
                            if (!tc::mbar_wait(&bar[GF + gs], (g_it / NG) & 1)) { ok = false; break; }
                            b_addr = tc::smem_u32(smem + gs * G_SLOT);
                            a_addr = b_addr + B_SLOT;
                            freed = &bar[GE + gs];
                            ++g_it;
                        } else {
                            const int ss = s_it % NS;
                            if (!tc::mbar_wait(&bar[SF + ss], (s_it / NS) & 1) ||
                                !tc::mbar_wait(&bar[SR + (tail ? 3 : j)], sg & 1)) {
                                ok = false;
                                break;
                            }
                            b_addr = tc::smem_u32(smem + OFF_SR + ss * B_SLOT);
                            a_addr = tc::smem_u32(smem + OFF_S + j * S_BLK);
                            freed = &bar[SE + ss];
                            ++s_it;
                        }
                        if (tail) {
                            tc::mma_f16(d, tc::smem_desc_sw32(a_addr), tc::smem_desc_sw32(b_addr), idesc, j != 0);
                        } else if (f8) {
                            // e4m3 x e4m3, K = 32 per MMA: four MMAs per 128-byte row block
                            const uint32_t idesc8 = tc::idesc_e4m3_f32(FM, op.n_mma);
                            const uint64_t ad = tc::smem_desc_sw128(a_addr), bd = tc::smem_desc_sw128(b_addr);
                            for (int k = 0; k < 4; ++k) tc::mma_f8(d, ad + 2 * k, bd + 2 * k, idesc8, (j | k) != 0);
                        } else {
                            const uint64_t ad = tc::smem_desc_sw128(a_addr), bd = tc::smem_desc_sw128(b_addr);
                            tc::mma_f16(d, ad, bd, idesc, j != 0);
                            // the K advance of 32 bytes inside the 128-byte rows: +2 in the
                            // descriptor's start-address field (16-byte units)
                            for (int k = 1; k < (w >> 4); ++k) tc::mma_f16(d, ad + 2 * k, bd + 2 * k, idesc, 1);
                        }
                        tc::mma_commit(freed);
                    }
                    if (!ok) break;
                    tc::mma_commit(&bar[on_y ? YF : XF]);
                    if (!a_glob) ++sg;
                }
            if (!ok && !aborted(abort_flag)) record_timeout(a.err, abort_flag);
            // every MMA issued completes before TMEM is released
            tc::mma_commit(&bar[DR]);
            tc::mbar_wait(&bar[DR], 0, 1u << 20);
        }
    } else if (warp >= 3 && warp <= 10) {
        // ---- epilogue ----
        const int q = warp & 3;                 // TMEM lane quarter
        const int hf = (warp - 3) >> 2;         // chunks hf, hf + 2, ...
        const int rl = q * 32 + lane;
        const uint32_t lane_tm = tmem_base + ((uint32_t)(q * 32) << 16);
        uint32_t xu = 0, yu = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            const int r = tile * FM + rl;
            const bool live = r < a.M;
            for (int i = 0; i < n_ops; ++i) {
                const FusedOp op = ops[i];
                const bool on_y = (op.flags & 4) != 0;
                const uint32_t u = on_y ? yu++ : xu++;
                // warp-uniform outcome: the tcgen05.ld below is issued by the whole warp
                const bool got = __all_sync(~0u, tc::mbar_wait(&bar[on_y ? YF : XF], u & 1));
                if (!got) {
                    if (lane == 0) record_timeout(a.err, abort_flag);
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                if (__any_sync(~0u, aborted(abort_flag))) { ok = false; break; }
                const uint32_t acc_tm = lane_tm + (on_y ? 256u : 0u);
                float sc = 1.f;
                if (op.kind == kFuseFc1 && live)
                    sc = fmaxf((kF8 ? a.fc1_scale : a.w_se)[(size_t)r * (kLayers * 3) + op.layer * 3 + op.type],
                               kSeFloor);
                for (int c = hf; 32 * c < op.n_mma; c += 2) {
                    if (32 * c + 32 <= op.n_mma) epi_chunk32(op, c, acc_tm, lane_tm, smem, bar, rl, r, live, sc, a, lane);
                    else epi_tail(op, c, acc_tm, smem, bar, rl, r, live, sc, a, lane);
                }
                tc::tmem_st_wait();                    // state writes to TMEM are done
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar[on_y ? YE : XE]);
                // global operands of a later op (the merge, the head) are out
                if (op.flags & (8 | 16)) {
                    tc::fence_async_global();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bar[(op.flags & 8) ? MR : HR]);
                }
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, 512);
    }
}

// Weight blocks of one op (blockIdx.y): per 64-column K block [n_mma][64] BF16 with 128-byte
// swizzle (16-byte unit u of row n at u ^ (n mod 8)), or, for the 16-column tail of an s-buffer
// operand, [n_mma][16] with 32-byte swizzle (unit u at u ^ ((n / 4) mod 2)): the byte layout
// the MMA descriptors read, so the producer copies each block as one contiguous piece.
// Column kk of the main operand is weight column kk (zero past k_main, with the bias's two
// BF16 parts at k_main and k_main + 1 when bias_main); FC-1's configuration columns k_main +
// 0..12 are [W_c (5), W_c (5), b_hi, b_lo, b_hi] against the operand [c/w hi (5), c/w lo (5),
// 1/w hi, 1/w hi, 1/w lo].
// An e4m3 op (fp8): two [n_mma][128] e4m3 blocks of W / S_w (128-byte swizzle, 16 values per
// unit) and the [n_mma][16] BF16 configuration block (32-byte swizzle).
__device__ void fused_pack_f8(const FusedPackOp &p, uint8_t *__restrict__ dst) {
    const int u8 = 2 * p.n_mma * 8;
    const int units = u8 + p.n_mma * 2;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < units; u += gridDim.x * blockDim.x) {
        if (u < u8) {
            const int j = u / (p.n_mma * 8), rem = u - j * p.n_mma * 8;
            const int n = rem >> 3, pu = rem & 7, lu = pu ^ (n & 7);
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (int e = 0; e < 16; e += 2) {
                const int kk = 128 * j + 16 * lu + e;
                float x0 = 0.f, x1 = 0.f;
                if (n < p.n_out) {
                    const float *wr = p.W + (size_t)n * p.ld;
                    if (kk < p.k_main) x0 = wr[kk] * p.f8_inv;
                    if (kk + 1 < p.k_main) x1 = wr[kk + 1] * p.f8_inv;
                }
                const uint32_t q = __nv_cvt_float2_to_fp8x2(make_float2(x0, x1), __NV_SATFINITE, __NV_E4M3);
                w[e >> 2] |= q << (8 * (e & 3));        // bytes e, e + 1 of the unit
            }
            *reinterpret_cast<uint4 *>(dst + p.b_off + (size_t)j * p.n_mma * 128 + n * 128 + pu * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            const int rem = u - u8, n = rem >> 1, pu = rem & 1, lu = pu ^ ((n >> 2) & 1);
            float v[8];
            float bh = 0.f, bl = 0.f;
            if (n < p.n_out) {
                const float b = p.bias[n];
                bh = __bfloat162float(__float2bfloat16_rn(b));
                bl = b - bh;
            }
            for (int e = 0; e < 8; ++e) {
                const int kc = 8 * lu + e;
                float x = 0.f;
                if (n < p.n_out) {
                    const float *wr = p.W + (size_t)n * p.ld;
                    if (kc < 5) x = wr[p.k_main + kc];
                    else if (kc < 10) x = wr[p.k_main + kc - 5];
                    else if (kc == 10 || kc == 12) x = bh;
                    else if (kc == 11) x = bl;
                }
                v[e] = x;
            }
            *reinterpret_cast<uint4 *>(dst + p.b_off + (size_t)2 * p.n_mma * 128 + n * 32 + pu * 16) = pack8(v);
        }
    }
}

__global__ void fused_pack_kernel(const FusedPackOp *__restrict__ pk, uint8_t *__restrict__ dst) {
    const FusedPackOp p = pk[blockIdx.y];
    if (p.fp8) {
        fused_pack_f8(p, dst);
        return;
    }
    const int nblk = (p.k + 63) / 64;
    const int full = p.s_tail ? nblk - 1 : nblk;            // 128-byte-row blocks
    const int u128 = full * p.n_mma * 8;                     // their 16-byte units
    const int units = u128 + (p.s_tail ? p.n_mma * 2 : 0);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < units; u += gridDim.x * blockDim.x) {
        int j, n, lu;
        size_t off = p.b_off;
        if (u < u128) {
            j = u / (p.n_mma * 8);
            const int rem = u - j * p.n_mma * 8;
            n = rem >> 3;
            const int pu = rem & 7;
            lu = pu ^ (n & 7);
            off += (size_t)j * p.n_mma * 128 + n * 128 + pu * 16;
        } else {
            j = full;
            const int rem = u - u128;
            n = rem >> 1;
            const int pu = rem & 1;
            lu = pu ^ ((n >> 2) & 1);
            off += (size_t)full * p.n_mma * 128 + n * 32 + pu * 16;
        }
        float v[8];
        float bh = 0.f, bl = 0.f;
        if (n < p.n_out) {
            const float b = p.bias[n];
            bh = __bfloat162float(__float2bfloat16_rn(b));
            bl = b - bh;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float x = 0.f;
            const int kk = 64 * j + 8 * lu + e;
            if (n < p.n_out) {
                const float *wr = p.W + (size_t)n * p.ld;
                if (kk < p.k_main) x = wr[kk];
                else if (p.cfg) {
                    const int kc = kk - p.k_main;
                    if (kc < 5) x = wr[p.k_main + kc];
                    else if (kc < 10) x = wr[p.k_main + kc - 5];
                    else if (kc == 10 || kc == 12) x = bh;
                    else if (kc == 11) x = bl;
                } else if (p.bias_main && kk == p.k_main) x = bh;
                else if (p.bias_main && kk == p.k_main + 1) x = bl;
            }
            v[e] = x;
        }
        *reinterpret_cast<uint4 *>(dst + off) = pack8(v);
    }
}

void fused_program(const WeightOffsets &o, const float *W, FusedOp *ops, FusedPackOp *pack, int *n_ops,
                   size_t *bytes, const float (*sw)[2]) {
    int n = 0;
    uint32_t off = 0;
    auto add = [&](int kind, int src, int type, int layer, int chain, int flags, int col0, int k, int n_mma,
                   const float *w, int ld, int n_out, int k_main, const float *b, float f8_inv = 0.f) {
        FusedOp f{};
        f.kind = (uint8_t)kind; f.src = (uint8_t)src; f.type = (uint8_t)type; f.layer = (uint8_t)layer;
        f.chain = (uint8_t)chain; f.flags = (uint8_t)(flags | ((n & 1) ? 4 : 0));   // X, Y alternate
        f.a_col0 = (uint16_t)col0; f.n_mma = (uint16_t)n_mma; f.k = (uint16_t)k;
        FusedPackOp p{};
        p.W = w; p.ld = ld; p.n_out = n_out; p.k_main = k_main; p.bias = b;
        p.cfg = kind == kFuseFc1 ? 1 : 0;
        p.bias_main = kind == kFuseFc1 ? 0 : 1;
        p.k = k; p.n_mma = n_mma; p.s_tail = src == kSrcS ? 1 : 0;
        f.b_off = p.b_off = off;
        if (flags & kFuseF8Flag) {
            p.fp8 = 1;
            p.f8_inv = f8_inv;
            off += (uint32_t)n_mma * (2u * 128u + 32u);
        } else {
            const int nblk = (k + 63) / 64;
            off += (uint32_t)n_mma * (p.s_tail ? 128u * (nblk - 1) + 32u : 128u * nblk);
        }
        ops[n] = f;
        pack[n] = p;
        ++n;
    };
    for (int t = 0; t < 3; ++t) {
        for (int chain = 0; chain < 2; ++chain) {
            const int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
            for (int k = k0; k < k1; ++k) {
                const int d = feat_dim(t);
                const int ld = t == 2 ? kFuseXtLd : kFuseLatLd;
                if (sw && t < 2)        // e4m3 features: columns k * kF8LatLd of their source
                    add(kFuseFc1, t, t, k, chain, (k == k0 ? 1 : 0) | kFuseF8Flag, k * kF8LatLd, kF8LatLd + 16,
                        208, W + o.blk_w1[t][k], d + kCfg, kWidth, d, W + o.blk_b1[t][k], 1.0f / sw[k][t]);
                else
                    add(kFuseFc1, t, t, k, chain, k == k0 ? 1 : 0, k * ld, ld, 208, W + o.blk_w1[t][k], d + kCfg,
                        kWidth, d, W + o.blk_b1[t][k]);
                const int fl = (k == k1 - 1 ? 2 : 0) | (k == k1 - 1 && chain == 1 ? 8 : 0);
                add(kFuseFc2, kSrcS, t, k, chain, fl, 0, 208, 208, W + o.blk_w2[t][k], kWidth, kWidth, kWidth,
                    W + o.blk_b2[t][k]);
            }
        }
        add(kFuseMerge, kSrcMrg, t, 0, 0, t == 2 ? 16 : 0, t * kFuseMrgLd, kFuseMrgLd, 208, W + o.mrg_w[t],
            2 * kWidth, kWidth, 2 * kWidth, W + o.mrg_b[t]);
    }
    add(kFuseHead1, kSrcHead, 0, 0, 0, 0, 0, kFuseHeadLd, 208, W + o.head_w[0], 3 * kWidth, kWidth, 3 * kWidth,
        W + o.head_b[0]);
    add(kFuseHead2, kSrcS, 0, 0, 0, 0, 0, 208, 208, W + o.head_w[1], kWidth, kWidth, kWidth, W + o.head_b[1]);
    add(kFuseHead3, kSrcS, 0, 0, 0, 0, 0, 208, 16, W + o.head_w[2], kWidth, 3, kWidth, W + o.head_b[2]);
    *n_ops = n;
    *bytes = off;
}

void launch_fused_pack(const FusedPackOp *pack_dev, int n_ops, uint8_t *dst, cudaStream_t s) {
    if (n_ops <= 0) return;
    note_launch();
    fused_pack_kernel<<<dim3(32, n_ops), 256, 0, s>>>(pack_dev, dst);
}

void launch_mlp_fused(const FusedArgs &a, const FusedMaps &maps, int num_sms, cudaStream_t s) {
    if (a.M <= 0 || a.n_ops <= 0 || a.n_ops > kFuseMaxOps) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(mlp_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_FUSED);
        cudaFuncSetAttribute(mlp_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_FUSED);
        attr_set = true;
    }
    const int tiles = (a.M + FM - 1) / FM;
    const int grid = tiles < num_sms ? tiles : num_sms;
    note_launch();
    if (a.fc1_scale) mlp_fused_kernel<true><<<grid, kThreads, SMEM_FUSED, s>>>(maps, a);
    else mlp_fused_kernel<false><<<grid, kThreads, SMEM_FUSED, s>>>(maps, a);
}

}  // namespace nis
