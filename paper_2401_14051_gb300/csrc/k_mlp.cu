// Dense layers of the backbone (Sec. III.C.2, Fig. 6), FP32 SIMT path: a 64x64-tile GEMM
// out = epilogue(A W^T + b) whose A operand is assembled on the fly -- the SE-scaled
// template features concatenated with the configuration vector (FC-1), the running
// state plus the block input (FC-2), or a concatenation of chain outputs (merge, head).
#include "nis_internal.h"

namespace nis {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

template <int MODE>
__device__ __forceinline__ float load_a(const FcArgs &a, int r, int kk) {
    if (r >= a.count || kk >= a.K) return 0.f;
    if (MODE == kFcFeat) {
        if (kk < a.d)
            return a.w_se[(size_t)r * (kLayers * 3) + a.layer * 3 + a.type] *
                   a.X[(size_t)r * a.ldx + kk];
        return a.cfg[(size_t)r * kCfg + (kk - a.d)];
    } else if (MODE == kFcSum) {
        float v = a.a1[(size_t)r * a.seg + kk];
        if (a.a0) v += a.a0[(size_t)r * a.seg + kk];
        return v;
    } else {
        int s = kk / a.seg, c = kk - s * a.seg;
        const float *src = s == 0 ? a.a0 : (s == 1 ? a.a1 : a.a2);
        return src[(size_t)r * a.seg + c];
    }
}
}  // namespace

template <int MODE>
__global__ void __launch_bounds__(256) fc_f32_kernel(const __grid_constant__ FcArgs a) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < a.K; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int r = e / BK, kk = e % BK;
            As[kk][r] = load_a<MODE>(a, row0 + r, k0 + kk);
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            int c = e / BK, kk = e % BK;
            int gc = col0 + c, gk = k0 + kk;
            Bs[kk][c] = (gc < a.N && gk < a.K) ? __ldg(a.W + (size_t)gc * a.K + gk) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = row0 + ty * 4 + i;
        if (r >= a.count) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = col0 + tx * 4 + j;
            if (c >= a.N) continue;
            float v = acc[i][j] + a.b[c];
            if (a.relu) v = fmaxf(v, 0.f);
            if (a.resid) v += a.resid[(size_t)r * a.ldo + c];
            if (a.decode) {
                if (a.y_out) a.y_out[(size_t)r * 3 + c] = v;
                const float ds = a.dec_rows ? a.dec_rows[(size_t)r * 3 + c] : a.dec_scale[c];
                a.out[(size_t)r * 3 + c] = ds * expm1f(v);
            } else {
                a.out[(size_t)r * a.ldo + c] = v;
            }
        }
    }
}

// Wide layers (N <= 208): 128 x 208 output tile per CTA, 256 threads as 16 x 16, each
// thread owns rows ty + 16 i (i < 8) and columns tx + 16 j (j < 13): per k step it reads 8 A
// and 13 B values from shared memory for 104 FMAs.  The next K slice is fetched into
// registers while the current one is consumed (two shared-memory buffers).
namespace {
constexpr int WM = 128, WN = 208, WK = 16, WI = 8, WJ = 13;
}

template <int MODE>
__global__ void __launch_bounds__(256, 1) fc_f32_wide_kernel(const __grid_constant__ FcArgs a) {
    __shared__ __align__(16) float As[2][WK][WM];
    __shared__ __align__(16) float Bs[2][WK][WN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.x * WM;
    float acc[WI][WJ];
#pragma unroll
    for (int i = 0; i < WI; ++i)
#pragma unroll
        for (int j = 0; j < WJ; ++j) acc[i][j] = 0.f;
    float ra[WM * WK / 256], rb[WN * WK / 256];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < WM * WK / 256; ++u) {
            int e = tid + 256 * u, r = e / WK, kk = e % WK;
            ra[u] = load_a<MODE>(a, row0 + r, k0 + kk);
        }
#pragma unroll
        for (int u = 0; u < WN * WK / 256; ++u) {
            int e = tid + 256 * u, c = e / WK, kk = e % WK, gk = k0 + kk;
            rb[u] = (c < a.N && gk < a.K) ? __ldg(a.W + (size_t)c * a.K + gk) : 0.f;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int u = 0; u < WM * WK / 256; ++u) {
            int e = tid + 256 * u;
            As[buf][e % WK][e / WK] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < WN * WK / 256; ++u) {
            int e = tid + 256 * u;
            Bs[buf][e % WK][e / WK] = rb[u];
        }
    };
    const int nk = (a.K + WK - 1) / WK;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int s = 0; s < nk; ++s) {
        const int buf = s & 1;
        if (s + 1 < nk) fetch((s + 1) * WK);
#pragma unroll
        for (int kk = 0; kk < WK; ++kk) {
            float av[WI], bv[WJ];
#pragma unroll
            for (int i = 0; i < WI; ++i) av[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < WJ; ++j) bv[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < WI; ++i)
#pragma unroll
                for (int j = 0; j < WJ; ++j) acc[i][j] += av[i] * bv[j];
        }
        if (s + 1 < nk) stash(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < WI; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= a.count) continue;
#pragma unroll
        for (int j = 0; j < WJ; ++j) {
            const int c = tx + 16 * j;
            if (c >= a.N) continue;
            float v = acc[i][j] + a.b[c];
            if (a.relu) v = fmaxf(v, 0.f);
            if (a.resid) v += a.resid[(size_t)r * a.ldo + c];
            a.out[(size_t)r * a.ldo + c] = v;
        }
    }
}

void launch_fc_f32(const FcArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    if (!a.decode && a.N > 64 && a.N <= WN) {
        dim3 grid((a.count + WM - 1) / WM);
        if (a.mode == kFcFeat) { note_launch(); fc_f32_wide_kernel<kFcFeat><<<grid, 256, 0, s>>>(a); }
        else if (a.mode == kFcSum) { note_launch(); fc_f32_wide_kernel<kFcSum><<<grid, 256, 0, s>>>(a); }
        else { note_launch(); fc_f32_wide_kernel<kFcCat><<<grid, 256, 0, s>>>(a); }
        return;
    }
    dim3 grid((a.count + BM - 1) / BM, (a.N + BN - 1) / BN);
    if (a.mode == kFcFeat) { note_launch(); fc_f32_kernel<kFcFeat><<<grid, 256, 0, s>>>(a); }
    else if (a.mode == kFcSum) { note_launch(); fc_f32_kernel<kFcSum><<<grid, 256, 0, s>>>(a); }
    else { note_launch(); fc_f32_kernel<kFcCat><<<grid, 256, 0, s>>>(a); }
}

}  // namespace nis
