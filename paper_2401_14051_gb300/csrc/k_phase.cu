// Precomputed phase features over all light-view angles (Sec. III.B.5; Eq. 5, 8, 9).
#include "nis_internal.h"

namespace nis {

__device__ __forceinline__ float hg(float c, float g, float k_g) {
    float base = 1.0f + g * g - 2.0f * g * c;         // >= (1 - |g|)^2 > 0
    return k_g / (base * sqrtf(base));
}

// Mean of HG(phi . b) over the cap of half-angle beta around an axis a with
// a . b = cos_g: rings at psi_i = beta (i + 1/2) / kRings weighted by sin(psi_i), kAzim
// azimuths measured from b (the cap stands for the solid angle the template point's
// ball subtends from p, Eq. 9).
__device__ float cap_mean(float cos_g, float beta, float g, float k_g,
                          const float *__restrict__ az_cos) {
    float sin_g = sqrtf(fmaxf(0.f, 1.f - cos_g * cos_g));
    float acc = 0.f, wsum = 0.f;
    for (int i = 0; i < kRings; ++i) {
        float psi = beta * ((i + 0.5f) / kRings);
        float s, mu;
        sincosf(psi, &s, &mu);
        float ring = 0.f;
#pragma unroll 8
        for (int j = 0; j < kAzim; ++j) ring += hg(mu * cos_g + s * sin_g * az_cos[j], g, k_g);
        acc += s * ring;
        wsum += s * kAzim;
    }
    return acc / wsum;
}

// table[a][set][t]: feature of lattice point t of point set `set` at alpha_a = a pi/1023.
// Offsets q = (a, b, c) spacings from p in the light frame (e_z toward the light); the
// highlight set j is shifted 9 (j + 1/2) spacings toward the light.  In that frame
// l = (0, 0, -1) and omega = (sin alpha, 0, -cos alpha); the direction from the template
// point toward p is n = -q/|q|, and f = capmean(n . l) * capmean(n . omega) (Eq. 8).
__global__ void phase_table_kernel(float g, float *__restrict__ table) {
    __shared__ float az_cos[kAzim];
    if (threadIdx.x < kAzim) az_cos[threadIdx.x] = cospif((2.0f * threadIdx.x + 1.0f) / kAzim);
    __syncthreads();
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kAlpha * kPhaseSets * kLat) return;
    int t = idx % kLat, set = (idx / kLat) % kPhaseSets, a = idx / (kLat * kPhaseSets);
    float qa = (float)(t / 45 - 2), qb = (float)((t / 9) % 5 - 2), qc = (float)(t % 9 - 4);
    if (set > 0) qc += 9.0f * ((set - 1) + 0.5f);
    float r2 = qa * qa + qb * qb + qc * qc;
    float val;
    if (r2 == 0.f) {
        val = 1.0f / (16.0f * 3.14159265358979f * 3.14159265358979f);
    } else {
        float r = sqrtf(r2);
        float nx = -qa / r, nz = -qc / r;
        float beta = atanf(0.5f / r);
        float alpha = (float)a * (3.14159265358979f / (kAlpha - 1));
        float sa, ca;
        sincosf(alpha, &sa, &ca);
        float k_g = (1.0f - g * g) / (4.0f * 3.14159265358979f);
        float f_l = cap_mean(-nz, beta, g, k_g, az_cos);
        float f_w = cap_mean(nx * sa - nz * ca, beta, g, k_g, az_cos);
        val = f_l * f_w;
    }
    table[idx] = val;
}

void launch_phase_table(float g, float *table, cudaStream_t s) {
    const int threads = 256;
    int total = kAlpha * kPhaseSets * kLat;
    note_launch();
    phase_table_kernel<<<(total + threads - 1) / threads, threads, 0, s>>>(g, table);
}

}  // namespace nis
