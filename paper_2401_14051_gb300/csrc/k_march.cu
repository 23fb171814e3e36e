// Graded transmittance fields (Eq. 1, Eq. 15): one thread per voxel centre of a level,
// marching toward the light through the same level's density.
#include "nis_internal.h"

namespace nis {

// T_m(x) = exp(-lam^(m+1) * sum of midpoint samples), step 1/n from x to the cube exit,
// the last step partial; the march stops once the scaled optical depth passes kTauMax.
// Neighbouring threads own x-neighbouring voxels, so their rays run parallel one voxel
// apart and their trilinear loads hit the same cache lines.
__global__ void __launch_bounds__(256) march_kernel(const float *__restrict__ level, int n,
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
    for (int s = 0; s < steps; ++s) {
        float t = (s + 0.5f) * inv_n;
        sum += sample_clamped(level, n, x + ux * t, y + uy * t, z + uz * t) * inv_n;
        if (sum > limit) { stopped = true; break; }
    }
    if (!stopped) {
        float rest = d - nfull * inv_n;
        if (rest > 0.f) {
            float t = nfull * inv_n + 0.5f * rest;
            sum += sample_clamped(level, n, x + ux * t, y + uy * t, z + uz * t) * rest;
        }
    }
    out[idx] = expf(-scale * sum);
}

void launch_march(const float *level, int n, int m, float ux, float uy, float uz, float lam,
                  float *out, cudaStream_t s) {
    float scale = powf(lam, (float)(m + 1));
    size_t total = (size_t)n * n * n;
    const int threads = 256;
    unsigned blocks = (unsigned)((total + threads - 1) / threads);
    note_launch();
    march_kernel<<<blocks, threads, 0, s>>>(level, n, ux, uy, uz, scale, out);
}

}  // namespace nis
