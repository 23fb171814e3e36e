// Density upload (conversion + checks) and the mip pyramid (Sec. III.B.1).
#include <cuda_fp16.h>

#include "nis_internal.h"

namespace nis {

// Converts the caller's density to float32 times `scale`, flags NaN/inf/negative values in
// the error word and tracks the maximum (non-negative floats order like their bit patterns).
template <typename T>
__global__ void convert_density_kernel(const T *__restrict__ src, float scale, size_t count,
                                       float *__restrict__ dst, unsigned *err,
                                       float *sigma_max) {
    float local_max = 0.f;
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        float v = (float)src[i] * scale;
        if (!(v >= 0.f) || isinf(v)) { bad = true; v = 0.f; }
        dst[i] = v;
        local_max = fmaxf(local_max, v);
    }
    for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(~0u, local_max, o));
    unsigned any_bad = __any_sync(~0u, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned *>(sigma_max), __float_as_uint(local_max));
        if (any_bad) atomicOr(err, kErrBadDensity);
    }
}

void launch_convert_density(const void *src, int dtype, float scale, size_t count,
                            float *dst, unsigned *err, float *sigma_max, cudaStream_t s) {
    cudaMemsetAsync(sigma_max, 0, sizeof(float), s);
    const int threads = 256;
    size_t want = (count + threads - 1) / threads;
    int blocks = (int)(want < 152 * 16 ? (want ? want : 1) : 152 * 16);
    note_launch();
    if (dtype == NIS_DTYPE_F16)
        convert_density_kernel<<<blocks, threads, 0, s>>>(static_cast<const __half *>(src), scale,
                                                          count, dst, err, sigma_max);
    else
        convert_density_kernel<<<blocks, threads, 0, s>>>(static_cast<const float *>(src), scale,
                                                          count, dst, err, sigma_max);
}

// downsample and occupancy take one grid row per block, (j, k) = (blockIdx.x, blockIdx.y),
// its threads striding over i: no index division (the cell-entry packing's rows of n + 1
// entries measured faster as a flat grid-stride loop).

// One level coarser: parent (i, j, k) of an m^3 grid averages its in-range children
// (2i + a, 2j + b, 2k + c) < n of the n^3 grid (reading: box mean, ceil(n/2) for odd n).
__global__ void downsample_kernel(const float *__restrict__ src, int n, float *__restrict__ dst,
                                  int m) {
    const int j = blockIdx.x, k = blockIdx.y;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const size_t idx = ((size_t)k * m + j) * m + i;
        float sum = 0.f;
        int cnt = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            int x = 2 * i + (c & 1), y = 2 * j + ((c >> 1) & 1), z = 2 * k + (c >> 2);
            if (x < n && y < n && z < n) {
                sum += __ldg(src + ((size_t)z * n + y) * n + x);
                ++cnt;
            }
        }
        dst[idx] = sum / (float)cnt;
    }
}

// threads per row block: the row length rounded up to a warp, at most 256
static int row_threads(int len) { return len >= 256 ? 256 : ((len + 31) / 32) * 32; }

void launch_downsample(const float *src, int n, float *dst, int m, cudaStream_t s) {
    note_launch();
    downsample_kernel<<<dim3(m, m), row_threads(m), 0, s>>>(src, n, dst, m);
}

__global__ void occupancy_kernel(const float *__restrict__ level, int n, unsigned char *occ) {
    const size_t nn = (size_t)n * n;
    const int j = blockIdx.x, k = blockIdx.y;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t idx = (size_t)k * nn + (size_t)j * n + i;
        const size_t dx = i + 1 < n ? 1 : 0, dy = j + 1 < n ? (size_t)n : 0, dz = k + 1 < n ? nn : 0;
        const float *p = level + idx;
        const bool any = __ldg(p) != 0.f || __ldg(p + dx) != 0.f || __ldg(p + dy) != 0.f ||
                         __ldg(p + dy + dx) != 0.f || __ldg(p + dz) != 0.f ||
                         __ldg(p + dz + dx) != 0.f || __ldg(p + dz + dy) != 0.f ||
                         __ldg(p + dz + dy + dx) != 0.f;
        occ[idx] = any ? 1 : 0;
    }
}

void launch_occupancy(const float *level, int n, unsigned char *occ, cudaStream_t s) {
    note_launch();
    occupancy_kernel<<<dim3(n, n), row_threads(n), 0, s>>>(level, n, occ);
}

// out[c][r] = in[r][c] for an R x C row-major matrix, through 32 x 32 shared-memory tiles
// (one tile per block, 32 x 8 threads, both sides coalesced)
__global__ void __launch_bounds__(256) transpose_kernel(const float *__restrict__ in, size_t R,
                                                        size_t C, size_t tiles_c,
                                                        float *__restrict__ out) {
    __shared__ float tile[32][33];
    const size_t r0 = (blockIdx.x / tiles_c) * 32, c0 = (blockIdx.x % tiles_c) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8)
        if (r0 + i < R && c0 + tx < C) tile[i][tx] = __ldg(in + (r0 + i) * C + c0 + tx);
    __syncthreads();
    for (int i = ty; i < 32; i += 8)
        if (c0 + i < C && r0 + tx < R) out[(c0 + i) * R + r0 + tx] = tile[tx][i];
}

void launch_transpose(const float *in, size_t R, size_t C, float *out, cudaStream_t s) {
    const size_t tiles_r = (R + 31) / 32, tiles_c = (C + 31) / 32;
    note_launch();
    transpose_kernel<<<(unsigned)(tiles_r * tiles_c), 256, 0, s>>>(in, R, C, tiles_c, out);
}

// PairView level: entry (z, j, i) = {rho, T} at (y, x) in {j - 1, j} x {i - 1, i} (borders 0
// and 1), as two float4 (row y = j - 1, then y = j).
__global__ void pack_pairs_kernel(const float *__restrict__ rho, const float *__restrict__ T, int n,
                                  float4 *__restrict__ out) {
    const size_t m = (size_t)n + 1, total = (size_t)n * m * m;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)((e / m) % m);
        const size_t z = e / (m * m);
        const int x0 = i - 1, x1 = i;
        float4 q[2];
        for (int r = 0; r < 2; ++r) {
            const int y = j - 1 + r;
            const bool yin = y >= 0 && y < n;
            const float *rr = rho + (z * n + (size_t)(yin ? y : 0)) * n, *tt = T + (z * n + (size_t)(yin ? y : 0)) * n;
            q[r].x = yin && x0 >= 0 ? rr[x0] : 0.0f;
            q[r].y = yin && x0 >= 0 ? tt[x0] : 1.0f;
            q[r].z = yin && x1 < n ? rr[x1] : 0.0f;
            q[r].w = yin && x1 < n ? tt[x1] : 1.0f;
        }
        out[2 * e] = q[0];
        out[2 * e + 1] = q[1];
    }
}

void launch_pack_pairs(const float *rho, const float *T, int n, float4 *out, cudaStream_t s) {
    const size_t total = (size_t)n * ((size_t)n + 1) * ((size_t)n + 1);
    const int blocks = (int)((total + 255) / 256 < 16384 ? (total + 255) / 256 : 16384);
    note_launch();
    pack_pairs_kernel<<<blocks, 256, 0, s>>>(rho, T, n, out);
}

}  // namespace nis
