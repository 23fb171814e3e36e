// The paper-template model's gathers (Sec. III.B.2, Eq. 2-4; Sec. III.B.1, Fig. 3): density,
// phase and a volume-level transmission feature at the paper's own template points, with the
// SE squeeze statistics and excitation weights (Eq. 24-26).
//
// Template (the readings of the model): diffuse layer k (0..7) holds 6, 8, 12, 16, 24, 32,
// 48, 48 points -- layer 0 the centre and five directions at half radius, the others
// spherical Fibonacci directions turned by k golden angles -- on the sphere of radius
// r_k = 2^k xi_(k+1) / (N D_k) (Eq. 4, D_k the mean nearest-neighbour distance of the
// unit-radius set, Eq. 3), so that the layer's point spacing is 2^k xi_(k+1) / N; mip level
// min(k, L-1).  Highlight layer j (0..3) holds 32, 16, 16, 8 points, a sunflower pattern on
// the disc of radius d/8 normal to the light, centred (j + 1/2) d/4 toward the light (d the
// exit distance, floored at 1/N); mip level from its spacing (d/8) D_j as for the lattice.
// Transmission feature at a point x: b + sum over the volume's levels (the 11 finest) of
// w_m T_m(x).
#include "nis_internal.h"

#include <cmath>

namespace nis {

namespace {
constexpr double kGolden = 3.14159265358979323846 * (3.0 - 2.2360679774997896964);

__device__ __forceinline__ float sigmoidf_p(float x) { return 1.0f / (1.0f + expf(-x)); }

}  // namespace

void paper_template(double unit[kPaperPts][3], double D[kLayers], float q[kPaperPts][3]) {
    for (int k = 0; k < kLayers; ++k) {
        const int n = paper_count(k), f = paper_first(k);
        for (int i = 0; i < n; ++i) {
            double *u = unit[f + i];
            if (k < kDiffuse) {
                if (k == 0 && i == 0) { u[0] = u[1] = u[2] = 0.0; continue; }
                const int m = k == 0 ? 5 : n, j = k == 0 ? i - 1 : i;
                const double z = 1.0 - (2.0 * j + 1.0) / m, r = std::sqrt(std::max(0.0, 1.0 - z * z));
                const double phi = j * kGolden + k * kGolden, sc = k == 0 ? 0.5 : 1.0;
                u[0] = sc * r * std::cos(phi); u[1] = sc * r * std::sin(phi); u[2] = sc * z;
            } else {
                const double r = std::sqrt((i + 0.5) / n), phi = i * kGolden;
                u[0] = r * std::cos(phi); u[1] = r * std::sin(phi); u[2] = 0.0;
            }
        }
        double sum = 0.0;                                   // Eq. 3
        for (int i = 0; i < n; ++i) {
            double best = 1e300;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                const double dx = unit[f + i][0] - unit[f + j][0], dy = unit[f + i][1] - unit[f + j][1],
                             dz = unit[f + i][2] - unit[f + j][2];
                best = std::min(best, std::sqrt(dx * dx + dy * dy + dz * dz));
            }
            sum += best;
        }
        D[k] = sum / n;
        for (int i = 0; i < n; ++i) {
            // offset from p over the layer spacing: diffuse unit / D; highlight (disc point
            // + 2 (j + 1/2) radii toward the light) / D, since the centre lies (j + 1/2) d/4
            // = 2 (j + 1/2) radii from p
            const double lift = k < kDiffuse ? 0.0 : 2.0 * ((k - kDiffuse) + 0.5);
            q[f + i][0] = (float)(unit[f + i][0] / D[k]);
            q[f + i][1] = (float)(unit[f + i][1] / D[k]);
            q[f + i][2] = (float)((unit[f + i][2] + lift) / D[k]);
        }
    }
}

// 16 bytes to a 16-byte aligned global address; two floats as BF16 (lo at the lower address).
__device__ __forceinline__ void st_v4p(void *p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" :: "l"(p), "r"(x), "r"(y), "r"(z),
                 "r"(w) : "memory");
}
__device__ __forceinline__ uint32_t pack_bf2p(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// The BF16 parts of 8 consecutive operand columns (x = x0 + x1 + x2 with three parts, each
// part the remainder rounded to BF16), one 16-byte store per part.
__device__ __forceinline__ void store_parts8(__nv_bfloat16 *dst, size_t part, int parts,
                                             float (&v)[8]) {
    for (int q = 0; q < parts; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            w[i] = pack_bf2p(v[2 * i], v[2 * i + 1]);
            v[2 * i] -= __uint_as_float(w[i] << 16);
            v[2 * i + 1] -= __uint_as_float(w[i] & 0xffff0000u);
        }
        st_v4p(dst + q * part, w[0], w[1], w[2], w[3]);
    }
}

constexpr int kPWarps = 4;                             // warps per CTA, 32 points each

// One lane per shading point, a warp over 32 consecutive points (neighbouring pixels of a
// frame, so a warp's samples of one template point touch few cache lines).  Each lane walks
// its point's 266 template points layer by layer: the density at the layer's level, the
// transmittance at every level, the phase column; it sums each layer's squeeze statistics
// in point order in registers, then computes the layer's SE excitation, and writes its BF16
// operand columns 8 at a time (16-byte stores).
__global__ void __launch_bounds__(kPWarps * 32, 4) gather_paper_kernel(const __grid_constant__ PaperGatherArgs a) {
    const int p = (blockIdx.x * kPWarps + (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
    if (p >= a.count) return;
    const float lx = a.lx, ly = a.ly, lz = a.lz;
    const float px = a.points[3 * p], py = a.points[3 * p + 1], pz = a.points[3 * p + 2];
    float ox = a.omega[3 * p], oy = a.omega[3 * p + 1], oz = a.omega[3 * p + 2];
    {
        float inv = 1.0f / sqrtf(ox * ox + oy * oy + oz * oz);
        ox *= inv; oy *= inv; oz *= inv;
    }
    // light frame: e_z toward the light, e_x = omega's part orthogonal to e_z
    const float ezx = -lx, ezy = -ly, ezz = -lz;
    float dz = ox * ezx + oy * ezy + oz * ezz;
    float wx = ox - dz * ezx, wy = oy - dz * ezy, wz = oz - dz * ezz;
    float nw = sqrtf(wx * wx + wy * wy + wz * wz);
    float exx, exy, exz;
    if (nw >= 1e-6f) {
        exx = wx / nw; exy = wy / nw; exz = wz / nw;
    } else {                                   // omega parallel to the light
        float tx = ezy, ty = -ezx, tz = 0.f;   // e_z x z-hat
        float tn = sqrtf(tx * tx + ty * ty);
        if (tn < 1e-6f) { tx = 0.f; ty = ezz; tz = -ezy; tn = sqrtf(ty * ty + tz * tz); }
        exx = tx / tn; exy = ty / tn; exz = tz / tn;
    }
    const float eyx = ezy * exz - ezz * exy, eyy = ezz * exx - ezx * exz,
                eyz = ezx * exy - ezy * exx;
    float cx_ = oy * lz - oz * ly, cy_ = oz * lx - ox * lz, cz_ = ox * ly - oy * lx;
    const float alpha = atan2f(sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_), ox * lx + oy * ly + oz * lz);
    float tt = fminf(fmaxf(alpha * ((kAlpha - 1) / 3.14159265358979f), 0.f), (float)(kAlpha - 1));
    const int ja = min((int)floorf(tt), kAlpha - 2);
    const float wa = tt - ja;
    const float *tab0 = a.table + (size_t)ja * kPaperPts, *tab1 = tab0 + kPaperPts;
    const int N = a.rho.n[0], L = a.rho.levels;
    const int nlv = L < kLevelWeights ? L : kLevelWeights;
    const float lb = __ldg(a.level_b);
    const bool bf = a.Hb_rho != nullptr;
    __nv_bfloat16 *row_r = bf ? a.Hb_rho + (size_t)p * a.ld_rf : nullptr;
    __nv_bfloat16 *row_f = bf ? a.Hb_f + (size_t)p * a.ld_rf : nullptr;
    __nv_bfloat16 *row_t = bf ? a.Hb_T + (size_t)p * a.ld_t : nullptr;

    for (int k = 0; k < kLayers; ++k) {
        float cx = px, cy = py, cz = pz, radius;
        int m;
        if (k < kDiffuse) {
            const float xi = 1.0f - 0.08f * (float)min(k + 1, 5);
            radius = (float)(1 << k) * xi / ((float)N * a.D[k]);
            m = min(k, L - 1);
        } else {
            const float d_exit = fmaxf(exit_distance(px, py, pz, ezx, ezy, ezz), 1.0f / N);
            const float f = ((k - kDiffuse) + 0.5f) * d_exit * 0.25f;
            cx += ezx * f; cy += ezy * f; cz += ezz * f;
            radius = d_exit * 0.125f;
            const float z = log2f(radius * a.D[k] * (float)N) + 0.5f;
            m = (int)fminf(fmaxf(floorf(z), 0.f), (float)(L - 1));
        }
        const float *rho_lv = a.rho.lv[m];
        const int rho_n = a.rho.n[m];
        const int f0 = paper_first(k), n = paper_count(k), c0 = paper_first_pad(k);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, m0 = -3.0e38f, m1 = -3.0e38f, m2 = -3.0e38f;
        for (int i0 = 0; i0 < n; i0 += 8) {
            float vr[8], vf[8], vt[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                vr[j] = vf[j] = vt[j] = 0.f;
                if (i0 + j < n) {                  // uniform over the warp
                    const int t = f0 + i0 + j;
                    const float ux = a.unit[t][0], uy = a.unit[t][1], uz = a.unit[t][2];
                    const float sx = cx + radius * (ux * exx + uy * eyx + uz * ezx);
                    const float sy = cy + radius * (ux * exy + uy * eyy + uz * ezy);
                    const float sz = cz + radius * (ux * exz + uy * eyz + uz * ezz);
                    // the density at the layer's level; the transmission feature weighs the
                    // 11 finest levels (a grid has at most 12)
                    const float rho = sample_border(rho_lv, rho_n, sx, sy, sz, 0.0f);
                    float T = lb;
                    for (int lv = 0; lv < nlv; ++lv)
                        T = fmaf(__ldg(a.level_w + lv), sample_border(a.T.lv[lv], a.T.n[lv], sx, sy, sz, 1.0f), T);
                    const float fa = __ldg(tab0 + t), fb = __ldg(tab1 + t);
                    const float f = fa + wa * (fb - fa);
                    if (a.H_rho) {
                        const size_t o = (size_t)p * kPaperPts + t;
                        a.H_rho[o] = rho;
                        a.H_f[o] = f;
                        a.H_T[o] = T;
                    }
                    s0 += rho; s1 += f; s2 += T;
                    m0 = fmaxf(m0, rho); m1 = fmaxf(m1, f); m2 = fmaxf(m2, T);
                    vr[j] = rho; vf[j] = f; vt[j] = T;
                }
            }
            if (bf) {                              // columns c0 + i0 .. + 7 (zeros past n)
                store_parts8(row_r + c0 + i0, a.part_rf, a.parts, vr);
                store_parts8(row_f + c0 + i0, a.part_rf, a.parts, vf);
                store_parts8(row_t + c0 + i0, a.part_t, a.parts, vt);
            }
        }
        const float inv_n = 1.0f / (float)n;
        const float v[8] = {s0 * inv_n, s1 * inv_n, s2 * inv_n, m0, m1, m2, a.g, alpha};
        if (a.v)
            for (int q = 0; q < 8; ++q) a.v[((size_t)p * kLayers + k) * 8 + q] = v[q];
        const float *w1 = a.se + a.se_w1[k], *b1 = a.se + a.se_b1[k];
        const float *w2 = a.se + a.se_w2[k], *b2 = a.se + a.se_b2[k];
        float z[2];
        for (int r = 0; r < 2; ++r) {
            float acc = b1[r];
            for (int q = 0; q < 8; ++q) acc += w1[r * 8 + q] * v[q];
            z[r] = fmaxf(acc, 0.f);
        }
        for (int r = 0; r < 3; ++r)
            a.w_se[((size_t)p * kLayers + k) * 3 + r] =
                sigmoidf_p(b2[r] + w2[r * 2] * z[0] + w2[r * 2 + 1] * z[1]);
        if (k == 0) {
            float *c = a.cfg + (size_t)p * kCfg;
            c[0] = a.g; c[1] = a.albedo[0]; c[2] = a.albedo[1]; c[3] = a.albedo[2]; c[4] = alpha;
        }
    }
    if (bf) {
        // the zero tail after the last layer: the MMAs read whole operand boxes, whose
        // columns beyond a layer meet zero weights and so must hold finite values
        for (int c = kPaperPad; c < kPaperPadTail; c += 8)
            for (int q = 0; q < a.parts; ++q) {
                st_v4p(row_r + c + q * a.part_rf, 0u, 0u, 0u, 0u);
                st_v4p(row_f + c + q * a.part_rf, 0u, 0u, 0u, 0u);
                st_v4p(row_t + c + q * a.part_t, 0u, 0u, 0u, 0u);
            }
    }
}

void launch_gather_paper(const PaperGatherArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    note_launch();
    gather_paper_kernel<<<(a.count + 32 * kPWarps - 1) / (32 * kPWarps), 32 * kPWarps, 0, s>>>(a);
}

}  // namespace nis
