// Camera rays and first-hit search (the shading point of each pixel), plus the scatter of
// shaded radiance back to pixels.
#include "nis_internal.h"

namespace nis {

// Per pixel: ray from the camera, clipped to the unit cube; samples at t_in + (j + 1/2) *
// 0.5/n; the first whose zero-border trilinear level-0 density reaches kHitFraction *
// sigma_max is the shading point x; d is the ray direction.  With the level's cell
// occupancy (occ0, built with the pyramid; null otherwise) a sample in an interior cell
// whose eight corners are all zero reads one byte instead of eight corners: its density is
// exactly zero, so the test gives the same answer.
__device__ __forceinline__ bool first_hit(const float *__restrict__ rho0,
                                          const unsigned char *__restrict__ occ0, int n,
                                          const float *__restrict__ sigma_max,
                                          const CameraArgs &c, int idx, float (&x)[3],
                                          float (&d)[3]) {
    int px = idx % c.width, py = idx / c.width;
    float sx = ((px + 0.5f) / c.width) * 2.0f - 1.0f;
    float sy = 1.0f - ((py + 0.5f) / c.height) * 2.0f;
    float o[3];
    if (c.type == NIS_CAMERA_PERSP) {
        float a = sx * c.tan_half * c.aspect, b = sy * c.tan_half;
        for (int q = 0; q < 3; ++q) { o[q] = c.eye[q]; d[q] = c.fwd[q] + a * c.right[q] + b * c.up[q]; }
        float inv = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int q = 0; q < 3; ++q) d[q] *= inv;
    } else {
        float a = sx * c.half_h * c.aspect, b = sy * c.half_h;
        for (int q = 0; q < 3; ++q) { o[q] = c.eye[q] + a * c.right[q] + b * c.up[q]; d[q] = c.fwd[q]; }
    }
    float t0 = 0.f, t1 = 3.0e38f;
    for (int q = 0; q < 3; ++q) {
        float lo, hi;
        if (d[q] != 0.f) {
            float ta = (0.f - o[q]) / d[q], tb = (1.f - o[q]) / d[q];
            lo = fminf(ta, tb); hi = fmaxf(ta, tb);
        } else if (o[q] >= 0.f && o[q] <= 1.f) {
            lo = -3.0e38f; hi = 3.0e38f;
        } else {
            lo = 3.0e38f; hi = -3.0e38f;
        }
        t0 = fmaxf(t0, lo); t1 = fminf(t1, hi);
    }
    bool hit = false;
    x[0] = x[1] = x[2] = 0.f;
    if (t1 > t0) {
        const float thr = kHitFraction * __ldg(sigma_max);
        const float step = 0.5f / n;
        // at most ceil((t1 - t0) / step) samples; the cube's diagonal bounds that by 4n + 4
        int steps = (int)fminf(ceilf((t1 - t0) / step), (float)(4 * n + 4));
        for (int j = 0; j < steps; ++j) {
            float t = t0 + (j + 0.5f) * step;
            if (!(t < t1)) break;
            for (int q = 0; q < 3; ++q) x[q] = o[q] + t * d[q];
            if (sample_border(rho0, n, x[0], x[1], x[2], 0.0f, occ0) >= thr) { hit = true; break; }
        }
    }
    return hit;
}

// Compacted output (pix_index != null): slot from an atomic counter; otherwise one entry per
// pixel, and with block_count != null the number of hits among the block's 256 pixels goes to
// block_count[blockIdx.x].
__global__ void __launch_bounds__(256) find_hits_kernel(const float *__restrict__ rho0,
                                 const unsigned char *__restrict__ occ0, int n,
                                 const float *__restrict__ sigma_max,
                                 const __grid_constant__ CameraArgs c,
                                 int *hit_flag, float *points, float *omega, int *pix_index,
                                 int *counter, int *block_count) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool hit = false;
    if (idx < c.width * c.height) {
        float x[3], d[3];
        hit = first_hit(rho0, occ0, n, sigma_max, c, idx, x, d);
        if (pix_index) {
            if (hit) {
                int slot = atomicAdd(counter, 1);
                for (int q = 0; q < 3; ++q) { points[3 * slot + q] = x[q]; omega[3 * slot + q] = -d[q]; }
                pix_index[slot] = idx;
            }
        } else {
            hit_flag[idx] = hit ? 1 : 0;
            for (int q = 0; q < 3; ++q) {
                points[3 * (size_t)idx + q] = hit ? x[q] : 0.f;
                omega[3 * (size_t)idx + q] = -d[q];
            }
        }
    }
    if (block_count) {                      // uniform over the block: every thread gets here
        const int k = __syncthreads_count(hit);
        if (threadIdx.x == 0) block_count[blockIdx.x] = k;
    }
}

void launch_find_hits(const float *rho0, const unsigned char *occ0, int n, const float *sigma_max,
                      const CameraArgs &c, int *hit_flag, float *points, float *omega,
                      int *pix_index, int *counter, cudaStream_t s) {
    int total = c.width * c.height;
    note_launch();
    find_hits_kernel<<<(total + 255) / 256, 256, 0, s>>>(rho0, occ0, n, sigma_max, c, hit_flag, points,
                                                         omega, pix_index, counter, nullptr);
}

// ---- hits in pixel order -------------------------------------------------------------------
// The atomic compaction above lists a frame's hits in whatever order the threads reach the
// counter.  Splitting one frame's shading points into ranges (one per process) needs an order
// that every process computes alike, so the ordered variant lists them by pixel index: per-pixel
// hits with a count per 256-pixel block, one exclusive scan of the block counts, then a pass
// that writes hit k of the frame to slot k - first when first <= k < first + count.

// Exclusive prefix sum of the nb block counts by one block of 1024 threads (each thread sums a
// run of consecutive blocks, then the runs are scanned by warp shuffles):
// offsets[b] = hits in the blocks before b, offsets[nb] = *total = the frame's hits.
__global__ void __launch_bounds__(1024) hit_block_scan_kernel(const int *__restrict__ count,
                                                              int nb, int *offsets, int *total) {
    __shared__ int warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (nb + 1023) / 1024;
    const int b0 = min(t * per, nb), b1 = min(b0 + per, nb);
    int mine = 0;
    for (int b = b0; b < b1; ++b) mine += count[b];
    int v = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sum[w] = v;
    __syncthreads();
    if (w == 0) {
        int u = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        warp_sum[lane] = u;
    }
    __syncthreads();
    int run = v - mine + (w ? warp_sum[w - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        offsets[b] = run;
        run += count[b];
    }
    if (t == 1023) {
        offsets[nb] = run;
        *total = run;
    }
}

// One block per 256-pixel block of find_hits_kernel: a hit's rank in the frame is its block's
// offset plus the hits before it in the block (warp ballots).  Blocks whose hits all fall
// outside [first, first + count) leave at once.
__global__ void __launch_bounds__(256) hits_range_kernel(const int *__restrict__ flag,
                                                         const float *__restrict__ pts_px,
                                                         const float *__restrict__ om_px,
                                                         const int *__restrict__ offsets,
                                                         int pixels, long long first, int count,
                                                         float *pts, float *om, int *pix) {
    const long long lo = offsets[blockIdx.x], hi = offsets[blockIdx.x + 1];
    if (hi <= first || lo >= first + count) return;    // uniform over the block
    __shared__ int warp_n[8];
    const int idx = blockIdx.x * 256 + threadIdx.x;
    const bool hit = idx < pixels && flag[idx] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_n[w] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int j = 0; j < w; ++j) before += warp_n[j];
    const long long k = lo + before + __popc(m & ((1u << lane) - 1u));
    if (hit && k >= first && k < first + count) {
        const size_t o = (size_t)(k - first);
        for (int q = 0; q < 3; ++q) {
            pts[3 * o + q] = pts_px[3 * (size_t)idx + q];
            om[3 * o + q] = om_px[3 * (size_t)idx + q];
        }
        pix[o] = idx;
    }
}

void launch_find_hits_ordered(const float *rho0, const unsigned char *occ0, int n,
                              const float *sigma_max, const CameraArgs &c, int *flag,
                              float *pts_px, float *om_px, int *block_count, int *offsets,
                              int *total, cudaStream_t s) {
    const int pixels = c.width * c.height, nb = (pixels + 255) / 256;
    note_launch();
    find_hits_kernel<<<nb, 256, 0, s>>>(rho0, occ0, n, sigma_max, c, flag, pts_px, om_px, nullptr,
                                        nullptr, block_count);
    note_launch();
    hit_block_scan_kernel<<<1, 1024, 0, s>>>(block_count, nb, offsets, total);
}

void launch_hits_range(const int *flag, const float *pts_px, const float *om_px,
                       const int *offsets, int pixels, long long first, int count, float *pts,
                       float *om, int *pix, cudaStream_t s) {
    if (count <= 0) return;
    note_launch();
    hits_range_kernel<<<(pixels + 255) / 256, 256, 0, s>>>(flag, pts_px, om_px, offsets, pixels,
                                                           first, count, pts, om, pix);
}

// Writes (or, with accumulate, adds) each shading point's radiance to its pixel; a pixel
// has at most one shading point, so the additions do not race.  Pixel indices outside
// [0, n_pixels) are skipped (they can come from another process's buffer).
__global__ void scatter_rgb_kernel(const float *__restrict__ rgb, const int *__restrict__ pix,
                                   int count, float *image, int n_pixels, int accumulate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int p = pix[i];
    if (p < 0 || p >= n_pixels) return;
    for (int c = 0; c < 3; ++c) {
        const float v = rgb[3 * (size_t)i + c];
        image[3 * (size_t)p + c] = accumulate ? image[3 * (size_t)p + c] + v : v;
    }
}

void launch_scatter_rgb(const float *rgb, const int *pix_index, int count, float *image,
                        int n_pixels, cudaStream_t s, bool accumulate) {
    if (count <= 0) return;
    note_launch();
    scatter_rgb_kernel<<<(count + 255) / 256, 256, 0, s>>>(rgb, pix_index, count, image,
                                                           n_pixels, accumulate ? 1 : 0);
}

}  // namespace nis
