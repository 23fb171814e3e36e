// Graded transmittance fields (Eq. 1, Eq. 15): one thread per voxel centre of a level,
// marching toward the light through the same level's density.
#include "nis_internal.h"

namespace nis {

// T_m(x) = exp(-lam^(m+1) * sum of midpoint samples), step 1/n from x to the cube exit,
// the last step partial; the march stops once the scaled optical depth passes kTauMax.
// Neighbouring threads own x-neighbouring voxels, so their rays run parallel one voxel
// apart and their trilinear loads hit the same cache lines.  The march is bound by its
// instruction count, so a sample is computed in grid units: sample s of the ray from voxel
// (i, j, k) sits at g = (i, j, k) + u (s + 1/2) (g = x n - 1/2), clamped to the grid; a cell
// flagged empty in the occupancy (all eight corners zero) costs one byte load instead of
// eight.  The positions, the sums and the stop rule are those of the midpoint rule.
template <typename Index>
__device__ __forceinline__ float sample_cell(const float *__restrict__ g,
                                             const unsigned char *__restrict__ occ, Index n,
                                             float hi, float top, Index d1, Index dn, Index dnn,
                                             float gx, float gy, float gz) {
    gx = fminf(fmaxf(gx, 0.0f), hi);
    gy = fminf(fmaxf(gy, 0.0f), hi);
    gz = fminf(fmaxf(gz, 0.0f), hi);
    const float flx = fminf(floorf(gx), top), fly = fminf(floorf(gy), top), flz = fminf(floorf(gz), top);
    const Index idx = ((Index)flz * n + (Index)fly) * n + (Index)flx;
    if (!__ldg(occ + idx)) return 0.f;
    const float fx = gx - flx, fy = gy - fly, fz = gz - flz;
    const float *p = g + idx;
    const float v0 = __ldg(p), v1 = __ldg(p + d1), v2 = __ldg(p + dn), v3 = __ldg(p + dn + d1);
    const float v4 = __ldg(p + dnn), v5 = __ldg(p + dnn + d1), v6 = __ldg(p + dnn + dn),
                v7 = __ldg(p + dnn + dn + d1);
    const float c00 = v0 + fx * (v1 - v0), c01 = v2 + fx * (v3 - v2);
    const float c10 = v4 + fx * (v5 - v4), c11 = v6 + fx * (v7 - v6);
    const float c0 = c00 + fy * (c01 - c00), c1 = c10 + fy * (c11 - c10);
    return c0 + fz * (c1 - c0);
}

// Index: 32-bit for levels up to 1024^3 (2^30 voxels), 64-bit beyond.
template <typename Index>
__global__ void __launch_bounds__(256) march_kernel(const float *__restrict__ level,
                                                    const unsigned char *__restrict__ occ, int n,
                                                    float ux, float uy, float uz, float scale,
                                                    float *__restrict__ out) {
    size_t total = (size_t)n * n * n;
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int i = (int)(idx % n), j = (int)((idx / n) % n), k = (int)(idx / ((size_t)n * n));
    const float inv_n = 1.0f / (float)n;
    float x = (i + 0.5f) * inv_n, y = (j + 0.5f) * inv_n, z = (k + 0.5f) * inv_n;
    float d = exit_distance(x, y, z, ux, uy, uz);
    float nfull = floorf(d * n);
    int steps = (int)nfull;
    float sum = 0.f;
    const float limit = kTauMax / scale;     // stop rule on the unscaled sum
    bool stopped = false;
    // corner offsets of a cell (a 1^3 level has one voxel: all corners are that voxel)
    const Index N = (Index)n, d1 = n > 1 ? 1 : 0, dn = n > 1 ? N : 0, dnn = n > 1 ? N * N : 0;
    const float hi = (float)(n - 1), top = (float)(n > 1 ? n - 2 : 0);
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    for (int s = 0; s < steps; ++s) {
        const float a = s + 0.5f;
        sum += sample_cell<Index>(level, occ, N, hi, top, d1, dn, dnn, fmaf(ux, a, fi), fmaf(uy, a, fj),
                                  fmaf(uz, a, fk)) * inv_n;
        if (sum > limit) { stopped = true; break; }
    }
    if (!stopped) {
        float rest = d - nfull * inv_n;
        if (rest > 0.f) {
            const float a = nfull + 0.5f * rest * n;
            sum += sample_cell<Index>(level, occ, N, hi, top, d1, dn, dnn, fmaf(ux, a, fi),
                                      fmaf(uy, a, fj), fmaf(uz, a, fk)) * rest;
        }
    }
    out[idx] = expf(-scale * sum);
}

void launch_march(const float *level, const unsigned char *occ, int n, int m, float ux,
                  float uy, float uz, float lam, float *out, cudaStream_t s) {
    float scale = powf(lam, (float)(m + 1));
    size_t total = (size_t)n * n * n;
    const int threads = 256;
    unsigned blocks = (unsigned)((total + threads - 1) / threads);
    note_launch();
    if (n <= 1024)
        march_kernel<unsigned><<<blocks, threads, 0, s>>>(level, occ, n, ux, uy, uz, scale, out);
    else
        march_kernel<size_t><<<blocks, threads, 0, s>>>(level, occ, n, ux, uy, uz, scale, out);
}

}  // namespace nis
