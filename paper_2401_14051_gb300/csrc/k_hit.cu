// Camera rays and first-hit search (the shading point of each pixel), plus the scatter of
// shaded radiance back to pixels.
#include "nis_internal.h"

namespace nis {

// Per pixel: ray from the camera, clipped to the unit cube; samples at t_in + (j + 1/2) *
// 0.5/n; the first whose zero-border trilinear level-0 density reaches kHitFraction *
// sigma_max is the shading point.  Compacted output (pix_index != null): slot from an
// atomic counter; otherwise one entry per pixel.
__global__ void find_hits_kernel(const float *__restrict__ rho0, int n,
                                 const float *__restrict__ sigma_max,
                                 const __grid_constant__ CameraArgs c,
                                 int *hit_flag, float *points, float *omega, int *pix_index,
                                 int *counter) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= c.width * c.height) return;
    int px = idx % c.width, py = idx / c.width;
    float sx = ((px + 0.5f) / c.width) * 2.0f - 1.0f;
    float sy = 1.0f - ((py + 0.5f) / c.height) * 2.0f;
    float o[3], d[3];
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
    float x[3] = {0.f, 0.f, 0.f};
    if (t1 > t0) {
        const float thr = kHitFraction * __ldg(sigma_max);
        const float step = 0.5f / n;
        // at most ceil((t1 - t0) / step) samples; the cube's diagonal bounds that by 4n + 4
        int steps = (int)fminf(ceilf((t1 - t0) / step), (float)(4 * n + 4));
        for (int j = 0; j < steps; ++j) {
            float t = t0 + (j + 0.5f) * step;
            if (!(t < t1)) break;
            for (int q = 0; q < 3; ++q) x[q] = o[q] + t * d[q];
            if (sample_border(rho0, n, x[0], x[1], x[2], 0.0f) >= thr) { hit = true; break; }
        }
    }
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

void launch_find_hits(const float *rho0, int n, const float *sigma_max, const CameraArgs &c,
                      int *hit_flag, float *points, float *omega, int *pix_index, int *counter,
                      cudaStream_t s) {
    int total = c.width * c.height;
    note_launch();
    find_hits_kernel<<<(total + 255) / 256, 256, 0, s>>>(rho0, n, sigma_max, c, hit_flag, points,
                                                         omega, pix_index, counter);
}

// Writes (or, with accumulate, adds) each shading point's radiance to its pixel; a pixel
// has at most one shading point, so the additions do not race.
__global__ void scatter_rgb_kernel(const float *__restrict__ rgb, const int *__restrict__ pix,
                                   int count, float *image, int accumulate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int p = pix[i];
    for (int c = 0; c < 3; ++c) {
        const float v = rgb[3 * (size_t)i + c];
        image[3 * (size_t)p + c] = accumulate ? image[3 * (size_t)p + c] + v : v;
    }
}

void launch_scatter_rgb(const float *rgb, const int *pix_index, int count, float *image,
                        cudaStream_t s, bool accumulate) {
    if (count <= 0) return;
    note_launch();
    scatter_rgb_kernel<<<(count + 255) / 256, 256, 0, s>>>(rgb, pix_index, count, image,
                                                           accumulate ? 1 : 0);
}

}  // namespace nis
