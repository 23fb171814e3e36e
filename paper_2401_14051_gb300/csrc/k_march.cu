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

// ---- shear-warp transmittance ------------------------------------------------------------
// An O(N^3) approximation of the march for large grids (not in the paper).  Rays toward
// the light are parallel, so the slices normal to the dominant axis a of u meet them at
// positions shifted by the same fraction per slice: ray (rho_p, rho_q) crosses slice k
// (counted from the light side) at rho - k r, r = u_perp / |u_a|.  Every ray keeps its
// optical depth and its length inside the cube from its crossing toward the light.  Step
// k advances every ray from slice k-1 to slice k (the part of that move inside the cube,
// its density taken at the part's midpoint); once a ray has crossed slice k, slice k can
// be filled: a voxel centre lies between four rays and takes their bilinearly weighted mean
// density (depth / length; for a ray that has not met the cube, the density at its
// crossing) times its own exit distance.  The interpolation happens once per voxel, so its
// error does not build up along the rays; a light along an axis gives the march's sums and
// a homogeneous medium the exact depth.
//
// A ray's state depends on nothing but its own previous state, so the sweep runs in chunks
// of S steps with two launches each: one thread per ray advances it through the S steps in
// registers, storing its state after each; then one thread per voxel fills the chunk's S
// slices from those states.  2 ceil(N / S) launches instead of one per step.
namespace {

// the work of one chunk (steps k0 .. k0 + steps - 1), per level: for the ray launch the
// window of rays whose crossing of any slice k0 - 1 .. k0 + steps - 1 lies within two
// voxels of the cube (the others are read by no voxel of the chunk and keep their state:
// rays move monotonically across the windows, so one not yet in it has not met the cube
// and one past it is read no more); for the voxel launch the chunk's slices
struct SwChunk {
    int k0, n_seg;
    unsigned total;
    unsigned start[kMaxLevels];
    int width[kMaxLevels];            // threads per row: window width (rays) or n (voxels)
    float inv_width[kMaxLevels];
    int ip0[kMaxLevels], iq0[kMaxLevels];   // ray index of the window's first row and column
    int steps[kMaxLevels];
    unsigned char level[kMaxLevels];
};

__device__ __forceinline__ int sw_segment(const SwChunk &c, unsigned t) {
    int s = 0;
    while (s + 1 < c.n_seg && t >= c.start[s + 1]) ++s;
    return s;
}

// (i / w, i % w) for i < 2^24 through a float reciprocal, corrected by one step
__device__ __forceinline__ void sw_divmod(unsigned i, int w, float inv_w, int &q, int &r) {
    q = (int)((float)i * inv_w);
    r = (int)i - q * w;
    if (r >= w) { ++q; r -= w; } else if (r < 0) { --q; r += w; }
}

__device__ __forceinline__ void sw_xyz(const ShearWarpArgs &a, float ga, float gp, float gq,
                                       float &x, float &y, float &z) {
    x = a.ax_a == 0 ? ga : (a.ax_p == 0 ? gp : gq);
    y = a.ax_a == 1 ? ga : (a.ax_p == 1 ? gp : gq);
    z = a.ax_a == 2 ? ga : (a.ax_p == 2 ? gp : gq);
}

// intersects the parameter range [t0, t1] of g0 + t dg with the closed cube [-1/2, n-1/2]
// (inv_dg = 1 / dg, or 0 for dg = 0)
__device__ __forceinline__ void sw_clip(float g0, float inv_dg, float nhi, float &t0, float &t1) {
    if (inv_dg != 0.f) {
        const float lo = (-0.5f - g0) * inv_dg, hi = (nhi - g0) * inv_dg;
        t0 = fmaxf(t0, fminf(lo, hi));
        t1 = fminf(t1, fmaxf(lo, hi));
    } else if (g0 < -0.5f || g0 > nhi) {
        t1 = -1.f;
    }
}

// exit distance toward the light of the grid point (gx, gy, gz), in cube units
__device__ __forceinline__ float sw_exit(const ShearWarpArgs &a, float gx, float gy, float gz,
                                         float nhi, float inv_n) {
    float t = 3.0e38f;
    if (a.ux > 0.f) t = fminf(t, (nhi - gx) * a.iux); else if (a.ux < 0.f) t = fminf(t, (gx + 0.5f) * a.iux);
    if (a.uy > 0.f) t = fminf(t, (nhi - gy) * a.iuy); else if (a.uy < 0.f) t = fminf(t, (gy + 0.5f) * a.iuy);
    if (a.uz > 0.f) t = fminf(t, (nhi - gz) * a.iuz); else if (a.uz < 0.f) t = fminf(t, (gz + 0.5f) * a.iuz);
    return fmaxf(t, 0.f) * inv_n;
}

// rays: ray (lo_p + ip, lo_q + iq) from its crossing of slice k-1 one step along
// (-sgn, -r_p, -r_q) to slice k, for each step k of the chunk.  Stored per step: (depth,
// length) once it has met the cube, (density at the crossing, 0) before.
template <typename Index>
__global__ void __launch_bounds__(256) sw_rays_kernel(const __grid_constant__ ShearWarpArgs a,
                                                      const __grid_constant__ SwChunk c) {
    // programmatic dependent launch: the previous launch's rays are read and its voxels'
    // reads of this buffer end before anything here touches it
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.total) return;
    const int s = sw_segment(c, t);
    const ShearWarpLevel &L = a.lv[c.level[s]];
    const int n = L.n;
    const Index N = (Index)n, d1 = n > 1 ? 1 : 0, dn = n > 1 ? N : 0, dnn = n > 1 ? N * N : 0;
    const float hi = (float)(n - 1), top = (float)(n > 1 ? n - 2 : 0);
    int ip, iq;
    sw_divmod(t - c.start[s], c.width[s], c.inv_width[s], iq, ip);
    ip += c.ip0[s];
    iq += c.iq0[s];
    const size_t ri = (size_t)iq * (size_t)L.P + (size_t)ip, slot = (size_t)L.P * (size_t)L.Q;
    const float sg = (float)a.sgn, nhi = (float)n - 0.5f;
    // the state after step k0 - 1: the last slot of the previous chunk (zeros: not met)
    float tau = 0.f, ell = 0.f;
    if (c.k0 > 0) {
        const float2 old = L.ray[(size_t)(a.slices - 1) * slot + ri];
        tau = old.x;
        ell = old.y;
    }
    for (int j = 0; j < c.steps[s]; ++j) {
        const int k = c.k0 + j;
        if (!(ell > 0.f)) { tau = 0.f; ell = 0.f; }     // not met: nothing carried
        const float ga = a.sgn > 0 ? (float)(n - k) : (float)(k - 1);
        const float gp = (float)(L.lo_p + ip) - (float)(k - 1) * L.r_p;
        const float gq = (float)(L.lo_q + iq) - (float)(k - 1) * L.r_q;
        float t0 = 0.f, t1 = 1.f;
        sw_clip(ga, -sg, nhi, t0, t1);
        sw_clip(gp, -L.inv_rp, nhi, t0, t1);
        sw_clip(gq, -L.inv_rq, nhi, t0, t1);
        if (t1 > t0) {
            const float tm = 0.5f * (t0 + t1), len = (t1 - t0) * L.ts;
            float x, y, z;
            sw_xyz(a, ga - sg * tm, gp - L.r_p * tm, gq - L.r_q * tm, x, y, z);
            tau += sample_cell<Index>(L.rho, L.occ, N, hi, top, d1, dn, dnn, x, y, z) * len;
            ell += len;
        }
        if (!(ell > 0.f)) {
            // voxels read rays whose crossing is within one voxel of the cube
            const float cp = gp - L.r_p, cq = gq - L.r_q;
            tau = 0.f;
            if (cp >= -2.f && cp <= (float)n + 1.f && cq >= -2.f && cq <= (float)n + 1.f) {
                float x, y, z;
                sw_xyz(a, ga - sg, cp, cq, x, y, z);
                tau = sample_cell<Index>(L.rho, L.occ, N, hi, top, d1, dn, dnn, x, y, z);
            }
            ell = 0.f;
        }
        L.ray[(size_t)j * slot + ri] = make_float2(tau, ell);
    }
}

// voxels: voxel (jp, jq) of slice k0 + j between the rays floor(j_p + (k0 + j) r) and the
// next ones, from their states after step k0 + j
template <typename Index>
__global__ void __launch_bounds__(256) sw_voxels_kernel(const __grid_constant__ ShearWarpArgs a,
                                                        const __grid_constant__ SwChunk c) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.total) return;
    const int s = sw_segment(c, t);
    const ShearWarpLevel &L = a.lv[c.level[s]];
    const int n = L.n;
    const Index N = (Index)n;
    int row, jp, j, jq;
    sw_divmod(t - c.start[s], n, c.inv_width[s], row, jp);
    sw_divmod((unsigned)row, n, c.inv_width[s], j, jq);
    const int kk = c.k0 + j;
    const float fp = (float)jp + (float)kk * L.r_p, fq = (float)jq + (float)kk * L.r_q;
    const float p0 = floorf(fp), q0 = floorf(fq);
    const float wp = fp - p0, wq = fq - q0;
    const float2 *ray = L.ray + (size_t)j * (size_t)L.P * (size_t)L.Q;
    float mean = 0.f;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int dp = cc & 1, dq = cc >> 1;
        const float w = (dp ? wp : 1.f - wp) * (dq ? wq : 1.f - wq);
        const int ip = min(max((int)p0 + dp - L.lo_p, 0), L.P - 1);
        const int iq = min(max((int)q0 + dq - L.lo_q, 0), L.Q - 1);
        const float2 rv = ray[(size_t)iq * L.P + ip];
        mean += w * (rv.y > 0.f ? __fdividef(rv.x, rv.y) : rv.x);
    }
    const float ga = a.sgn > 0 ? (float)(n - 1 - kk) : (float)kk;
    float x, y, z;
    sw_xyz(a, ga, (float)jp, (float)jq, x, y, z);
    const float d = sw_exit(a, x, y, z, (float)n - 0.5f, 1.0f / (float)n);
    L.T[((Index)z * N + (Index)y) * N + (Index)x] = expf(-L.scale * d * mean);
}

}  // namespace

void shear_warp_setup(ShearWarpArgs &a, const int *sizes, int levels, float ux, float uy,
                      float uz, float lam, size_t *ray_floats) {
    const double u[3] = {ux, uy, uz};
    int ax = 0;
    for (int c = 1; c < 3; ++c)
        if (std::fabs(u[c]) > std::fabs(u[ax])) ax = c;
    a.levels = levels;
    a.slices = sw_slices(sizes[0]);
    a.sgn = u[ax] > 0 ? 1 : -1;
    a.ax_a = ax;
    a.ax_p = ax == 0 ? 1 : 0;
    a.ax_q = ax == 2 ? 1 : 2;
    a.ux = ux;
    a.uy = uy;
    a.uz = uz;
    a.iux = ux != 0.f ? (float)(1.0 / std::fabs(u[0])) : 0.f;
    a.iuy = uy != 0.f ? (float)(1.0 / std::fabs(u[1])) : 0.f;
    a.iuz = uz != 0.f ? (float)(1.0 / std::fabs(u[2])) : 0.f;
    const double ua = std::fabs(u[ax]);
    const double rp = u[a.ax_p] / ua, rq = u[a.ax_q] / ua;
    for (int m = 0; m < levels; ++m) {
        ShearWarpLevel &L = a.lv[m];
        const int n = sizes[m];
        L.n = n;
        L.lo_p = (int)std::floor(-1.0 + std::min(0.0, (n - 1) * rp));
        L.lo_q = (int)std::floor(-1.0 + std::min(0.0, (n - 1) * rq));
        L.P = (int)std::ceil(n + std::max(0.0, (n - 1) * rp)) - L.lo_p + 1;
        L.Q = (int)std::ceil(n + std::max(0.0, (n - 1) * rq)) - L.lo_q + 1;
        L.r_p = (float)rp;
        L.r_q = (float)rq;
        L.inv_rp = rp != 0.0 ? (float)(1.0 / rp) : 0.f;
        L.inv_rq = rq != 0.0 ? (float)(1.0 / rq) : 0.f;
        L.ts = (float)(1.0 / (n * ua));
        L.scale = powf(lam, (float)(m + 1));
        ray_floats[m] = 2 * (size_t)a.slices * L.P * L.Q;
    }
}

void launch_shear_warp(const ShearWarpArgs &a, cudaStream_t s) {
    const int n0 = a.lv[0].n, S = a.slices;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    auto launch = [&](bool rays, const SwChunk &c) {
        if (c.total == 0) return;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((c.total + 255) / 256);
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        note_launch();
        if (n0 <= 1024)
            cudaLaunchKernelEx(&cfg, rays ? sw_rays_kernel<unsigned> : sw_voxels_kernel<unsigned>, a, c);
        else
            cudaLaunchKernelEx(&cfg, rays ? sw_rays_kernel<size_t> : sw_voxels_kernel<size_t>, a, c);
    };
    for (int k0 = 0; k0 < n0; k0 += S) {
        SwChunk rc{}, vc{};
        rc.k0 = vc.k0 = k0;
        for (int m = 0; m < a.levels; ++m) {
            const ShearWarpLevel &L = a.lv[m];
            if (k0 >= L.n) continue;
            const int steps = std::min(S, L.n - k0), k1 = k0 + steps - 1;
            // rays whose crossing of a slice k0 - 1 .. k1 is within [-2, n + 1]
            auto window = [&](double r, int lo, int count, int &first, int &width) {
                const double a0 = std::min((k0 - 1) * r, k1 * r), a1 = std::max((k0 - 1) * r, k1 * r);
                const int r0 = std::max(lo, (int)std::floor(-2.0 + a0));
                const int r1 = std::min(lo + count - 1, (int)std::ceil(L.n + 1.0 + a1));
                first = r0 - lo;
                width = std::max(0, r1 - r0 + 1);
            };
            int fp, wp, fq, wq;
            window(L.r_p, L.lo_p, L.P, fp, wp);
            window(L.r_q, L.lo_q, L.Q, fq, wq);
            if (wp > 0 && wq > 0) {
                const int i = rc.n_seg++;
                rc.start[i] = rc.total;
                rc.level[i] = (unsigned char)m;
                rc.width[i] = wp;
                rc.inv_width[i] = 1.0f / (float)wp;
                rc.ip0[i] = fp;
                rc.iq0[i] = fq;
                rc.steps[i] = steps;
                rc.total += (unsigned)wp * (unsigned)wq;
            }
            const int i = vc.n_seg++;
            vc.start[i] = vc.total;
            vc.level[i] = (unsigned char)m;
            vc.width[i] = L.n;
            vc.inv_width[i] = 1.0f / (float)L.n;
            vc.steps[i] = steps;
            vc.total += (unsigned)steps * (unsigned)L.n * (unsigned)L.n;
        }
        launch(true, rc);
        launch(false, vc);
    }
}

}  // namespace nis
