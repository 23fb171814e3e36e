// Precomputed phase features over all light-view angles (Sec. III.B.5; Eq. 5, 8, 9).
#include "nis_internal.h"

namespace nis {

// Mean of the phase function (Eq. 5/6) of the angle theta between b and the directions phi
// of the cap of half-angle beta around an axis a, where gamma = angle(a, b): rings at
// psi_i = beta (i + 1/2) / kRings weighted by sin(psi_i), kAzim azimuths phi_j measured
// from b (the cap stands for the solid angle the template point's ball subtends from p,
// Eq. 9).  1 -/+ cos(theta) come from the haversine form of the spherical law of cosines,
//   1 - cos(theta) = 2 [sin^2((psi - gamma)/2) + sin(psi) sin(gamma) sin^2(phi/2)],
//   1 + cos(theta) = 2 [sin^2((psi + gamma - pi)/2) + sin(psi) sin(gamma) cos^2(phi/2)].
// HG's 1 + g^2 - 2 g cos(theta) is written without cancellation, (1 - g)^2 + 2 g (1 - cos)
// for g >= 0 and (1 + g)^2 - 2 g (1 + cos) for g < 0, so sharp lobes keep full FP32
// precision near their peak; on one ring that is A + B t_j with non-negative A, B and t_j
// = sin^2(phi_j / 2) (g >= 0) or cos^2(phi_j / 2) (g < 0), and each node costs one FMA, a
// reciprocal square root (base^(-3/2) as its cube; a few ulp) and two multiply-adds.
__device__ __forceinline__ float cap_mean(float gamma, float beta, const PhaseSpec &ph, const float *k_g,
                                          const float *__restrict__ az_s2,
                                          const float *__restrict__ az_c2) {
    float ts[kAzim], tc[kAzim];
#pragma unroll
    for (int j = 0; j < kAzim; ++j) { ts[j] = az_s2[j]; tc[j] = az_c2[j]; }
    const float sg = sinf(gamma);
    float acc = 0.f, wsum = 0.f;
    for (int i = 0; i < kRings; ++i) {
        const float psi = beta * ((i + 0.5f) / kRings);
        const float s = sinf(psi);
        const float hm = sinf(0.5f * (psi - gamma)), hp = sinf(0.5f * (psi + gamma) - 1.5707963267949f);
        const float hm2 = hm * hm, hp2 = hp * hp, ss = s * sg;
        float ring = 0.f;
        for (int l = 0; l < ph.n; ++l) {
            const float g = ph.g[l];
            float sum = 0.f;
            if (g >= 0.f) {
                const float A = fmaf(4.f * g, hm2, (1.f - g) * (1.f - g)), B = 4.f * g * ss;
#pragma unroll
                for (int j = 0; j < kAzim; ++j) {
                    const float r = rsqrtf(fmaf(B, ts[j], A));
                    sum = fmaf(r * r, r, sum);
                }
            } else {
                const float A = fmaf(-4.f * g, hp2, (1.f + g) * (1.f + g)), B = -4.f * g * ss;
#pragma unroll
                for (int j = 0; j < kAzim; ++j) {
                    const float r = rsqrtf(fmaf(B, tc[j], A));
                    sum = fmaf(r * r, r, sum);
                }
            }
            ring = fmaf(ph.w[l] * k_g[l], sum, ring);
        }
        acc += s * ring;
        wsum += s * kAzim;
    }
    return acc / wsum;
}

// Features of one template point at offset q = (qa, qb, qc) spacings from p in the light
// frame (e_z toward the light) over the 1024 view angles, written to col[a * stride].  In
// that frame l = (0, 0, -1) and omega = (sin alpha, 0, -cos alpha); the direction from the
// template point toward p is n = -q/|q|, and f = capmean(n, l) * capmean(n, omega) (Eq. 8)
// with the cap half-angle atan((1/2)/|q|).  The angles between n and l or omega come from
// atan2 of exact cross and dot products of q.  The light factor does not depend on alpha
// and is computed once by thread 0; the CTA's threads then sweep the view angles.
__device__ void phase_column(float qa, float qb, float qc, const PhaseSpec &ph, float *col,
                             size_t stride, float *az_s2, float *az_c2, float *f_light) {
    if (threadIdx.x < kAzim) {
        float h = sinpif((2.0f * threadIdx.x + 1.0f) / (2.0f * kAzim));   // sin(phi_j / 2)
        float c = cospif((2.0f * threadIdx.x + 1.0f) / (2.0f * kAzim));
        az_s2[threadIdx.x] = h * h;
        az_c2[threadIdx.x] = c * c;
    }
    const float r2 = qa * qa + qb * qb + qc * qc;
    if (r2 == 0.f) {                                      // the point itself: isotropic value
        for (int a = threadIdx.x; a < kAlpha; a += blockDim.x)
            col[(size_t)a * stride] = 1.0f / (16.0f * 3.14159265358979f * 3.14159265358979f);
        return;
    }
    const float r = sqrtf(r2);
    const float beta = atanf(0.5f / r);
    float k_g[3];
    for (int i = 0; i < 3; ++i) k_g[i] = (1.0f - ph.g[i] * ph.g[i]) / (4.0f * 3.14159265358979f);
    __syncthreads();                                      // azimuth tables ready
    if (threadIdx.x == 0) {
        // n . l = qc / r, |n x l| = sqrt(qa^2 + qb^2) / r
        const float gam_l = atan2f(sqrtf(qa * qa + qb * qb), qc);
        *f_light = cap_mean(gam_l, beta, ph, k_g, az_s2, az_c2);
    }
    __syncthreads();
    const float f_l = *f_light;
    for (int a = threadIdx.x; a < kAlpha; a += blockDim.x) {
        const float alpha = (float)a * (3.14159265358979f / (kAlpha - 1));
        float sa, ca;
        sincosf(alpha, &sa, &ca);
        // n . omega = (qc cos a - qa sin a) / r, |n x omega|^2 = qb^2 + (qc sin a + qa cos a)^2
        const float cr = qc * sa + qa * ca;
        const float gam_w = atan2f(sqrtf(qb * qb + cr * cr), qc * ca - qa * sa);
        col[(size_t)a * stride] = f_l * cap_mean(gam_w, beta, ph, k_g, az_s2, az_c2);
    }
}

// table[a][set][t]: feature of lattice point t of point set `set` at alpha_a = a pi/1023;
// the highlight set j is shifted 9 (j + 1/2) spacings toward the light.  One CTA per (set, t).
__global__ void phase_table_kernel(const PhaseSpec ph, float *__restrict__ table) {
    __shared__ float az_s2[kAzim], az_c2[kAzim];
    __shared__ float f_light;
    const int set = blockIdx.x / kLat, t = blockIdx.x % kLat;
    float qa = (float)(t / 45 - 2), qb = (float)((t / 9) % 5 - 2), qc = (float)(t % 9 - 4);
    if (set > 0) qc += 9.0f * ((set - 1) + 0.5f);
    phase_column(qa, qb, qc, ph, table + (size_t)set * kLat + t, (size_t)kPhaseSets * kLat,
                 az_s2, az_c2, &f_light);
}

// table[a][t] for the template points of the paper model (offsets given).  One CTA per point.
struct PhasePoints {
    float q[kPaperPts][3];
};
__global__ void phase_points_kernel(const PhaseSpec ph, const __grid_constant__ PhasePoints pts,
                                    int n_pts, float *__restrict__ table) {
    __shared__ float az_s2[kAzim], az_c2[kAzim];
    __shared__ float f_light;
    const int t = blockIdx.x;
    phase_column(pts.q[t][0], pts.q[t][1], pts.q[t][2], ph, table + t, (size_t)n_pts, az_s2,
                 az_c2, &f_light);
}

void launch_phase_points(const PhaseSpec &ph, const float (*q)[3], int n_pts, float *table,
                         cudaStream_t s) {
    PhasePoints pts{};
    for (int t = 0; t < n_pts && t < kPaperPts; ++t)
        for (int c = 0; c < 3; ++c) pts.q[t][c] = q[t][c];
    note_launch();
    phase_points_kernel<<<n_pts, 256, 0, s>>>(ph, pts, n_pts, table);
}

void launch_phase_table(const PhaseSpec &ph, float *table, cudaStream_t s) {
    note_launch();
    phase_table_kernel<<<kPhaseSets * kLat, 256, 0, s>>>(ph, table);
}

}  // namespace nis
