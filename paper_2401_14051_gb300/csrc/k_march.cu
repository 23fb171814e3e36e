// Graded transmittance fields (Eq. 1, Eq. 15): one thread per voxel centre of a level,
// marching toward the light through the same level's density.
#include "nis_internal.h"

namespace nis {

// T_m(x) = exp(-lam^(m+1) * sum of midpoint samples), step 1/n from x to the cube exit,
// the last step partial; the march stops once the scaled optical depth passes kTauMax.
// Neighbouring threads own x-neighbouring voxels, so their rays run parallel one voxel
// apart and their trilinear loads hit the same cache lines.  Samples in empty bricks cost
// one byte load instead of eight (exact empty-space skipping: the positions, the sums and
// the stop rule are unchanged).
// Trilinear clamp-to-edge sample that skips the eight loads when the cell's brick is empty
// (exact: all eight corners are zero there).
__device__ __forceinline__ float sample_clamped_occ(const float *__restrict__ g,
                                                    const unsigned char *__restrict__ occ, int nb,
                                                    int n, float x, float y, float z) {
    const float hi = (float)(n - 1);
    float gx = fminf(fmaxf(x * n - 0.5f, 0.0f), hi);
    float gy = fminf(fmaxf(y * n - 0.5f, 0.0f), hi);
    float gz = fminf(fmaxf(z * n - 0.5f, 0.0f), hi);
    const int top = n > 1 ? n - 2 : 0;
    int ix = min((int)floorf(gx), top), iy = min((int)floorf(gy), top), iz = min((int)floorf(gz), top);
    if (!__ldg(occ + ((size_t)(iz / kBrick) * nb + iy / kBrick) * nb + ix / kBrick)) return 0.f;
    float fx = gx - ix, fy = gy - iy, fz = gz - iz;
    int dx = (ix + 1 < n) ? 1 : 0;
    int dy = (iy + 1 < n) ? n : 0;
    int dz = (iz + 1 < n) ? n * n : 0;
    const float *p = g + ((size_t)iz * n + iy) * n + ix;
    float c00 = __ldg(p) + fx * (__ldg(p + dx) - __ldg(p));
    float c01 = __ldg(p + dy) + fx * (__ldg(p + dy + dx) - __ldg(p + dy));
    float c10 = __ldg(p + dz) + fx * (__ldg(p + dz + dx) - __ldg(p + dz));
    float c11 = __ldg(p + dz + dy) + fx * (__ldg(p + dz + dy + dx) - __ldg(p + dz + dy));
    float c0 = c00 + fy * (c01 - c00);
    float c1 = c10 + fy * (c11 - c10);
    return c0 + fz * (c1 - c0);
}

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
    const int nb = bricks_of(n);
    for (int s = 0; s < steps; ++s) {
        float t = (s + 0.5f) * inv_n;
        sum += sample_clamped_occ(level, occ, nb, n, x + ux * t, y + uy * t, z + uz * t) * inv_n;
        if (sum > limit) { stopped = true; break; }
    }
    if (!stopped) {
        float rest = d - nfull * inv_n;
        if (rest > 0.f) {
            float t = nfull * inv_n + 0.5f * rest;
            sum += sample_clamped_occ(level, occ, nb, n, x + ux * t, y + uy * t, z + uz * t) * rest;
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
    march_kernel<<<blocks, threads, 0, s>>>(level, occ, n, ux, uy, uz, scale, out);
}

}  // namespace nis
