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

// One CTA per shading point, thread t < 266 owns template point t.  Each samples the
// density at its layer's level and the transmittance at every level, reads its phase
// column; the squeeze statistics of each layer are then summed in point order by one thread
// per layer (deterministic) and the SE excitation follows.
__global__ void __launch_bounds__(288, 4) gather_paper_kernel(const __grid_constant__ PaperGatherArgs a) {
    __shared__ float s_rho[kPaperPts], s_f[kPaperPts], s_T[kPaperPts];
    __shared__ float s_alpha;
    const int p = blockIdx.x, t = threadIdx.x;
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
    const int N = a.rho.n[0], L = a.rho.levels;
    if (t < kPaperPts) {
        const int k = paper_layer_of(t);
        const float ux = a.unit[t][0], uy = a.unit[t][1], uz = a.unit[t][2];
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
        const float sx = cx + radius * (ux * exx + uy * eyx + uz * ezx);
        const float sy = cy + radius * (ux * exy + uy * eyy + uz * ezy);
        const float sz = cz + radius * (ux * exz + uy * eyz + uz * ezz);
        // the density at the layer's level; the transmission feature weighs the 11 finest
        // levels (a grid has at most 12).  Plain float grids, not the interleaved pairs: the
        // transmittance alone is read at every level (measured 2 % faster than the pairs)
        const float rho = sample_border(a.rho.lv[m], a.rho.n[m], sx, sy, sz, 0.0f);
        float T = __ldg(a.level_b);
        for (int lv = 0; lv < L && lv < kLevelWeights; ++lv)
            T = fmaf(__ldg(a.level_w + lv), sample_border(a.T.lv[lv], a.T.n[lv], sx, sy, sz, 1.0f), T);
        const float f0 = __ldg(a.table + (size_t)ja * kPaperPts + t);
        const float f1 = __ldg(a.table + (size_t)(ja + 1) * kPaperPts + t);
        const float f = f0 + wa * (f1 - f0);
        if (a.H_rho) {
            const size_t o = (size_t)p * kPaperPts + t;
            a.H_rho[o] = rho;
            a.H_f[o] = f;
            a.H_T[o] = T;
        }
        if (a.Hb_rho) {                        // BF16 parts, the layer's padded columns
            const int col = paper_first_pad(k) + (t - paper_first(k));
            __nv_bfloat16 *dr = a.Hb_rho + (size_t)p * a.ld_rf + col;
            __nv_bfloat16 *df = a.Hb_f + (size_t)p * a.ld_rf + col;
            __nv_bfloat16 *dt = a.Hb_T + (size_t)p * a.ld_t + col;
            float r0 = rho, r1 = f, r2 = T;
            for (int q = 0; q < a.parts; ++q) {
                const __nv_bfloat16 b0 = __float2bfloat16_rn(r0), b1 = __float2bfloat16_rn(r1),
                                    b2 = __float2bfloat16_rn(r2);
                dr[q * a.part_rf] = b0;
                df[q * a.part_rf] = b1;
                dt[q * a.part_t] = b2;
                r0 -= __bfloat162float(b0);
                r1 -= __bfloat162float(b1);
                r2 -= __bfloat162float(b2);
            }
        }
        s_rho[t] = rho; s_f[t] = f; s_T[t] = T;
    } else if (a.Hb_rho) {
        // zeros in the layers' padding columns and the tail: the MMAs read whole operand
        // boxes (32 or 64 columns), whose columns beyond a layer meet zero weights and so
        // must hold finite values
        for (int z = t - kPaperPts; z < kPaperPadTail - kPaperPts; z += blockDim.x - kPaperPts) {
            int col = -1, seen = 0;
            for (int k = 0; k < kLayers && col < 0; ++k) {
                const int padn = paper_count_pad(k) - paper_count(k);
                if (z < seen + padn) col = paper_first_pad(k) + paper_count(k) + (z - seen);
                seen += padn;
            }
            if (col < 0) col = kPaperPad + (z - seen);
            for (int q = 0; q < a.parts; ++q) {
                a.Hb_rho[(size_t)p * a.ld_rf + col + q * a.part_rf] = __float2bfloat16_rn(0.f);
                a.Hb_f[(size_t)p * a.ld_rf + col + q * a.part_rf] = __float2bfloat16_rn(0.f);
                a.Hb_T[(size_t)p * a.ld_t + col + q * a.part_t] = __float2bfloat16_rn(0.f);
            }
        }
    }
    if (t == 0) s_alpha = alpha;
    __syncthreads();
    if (t < kLayers) {
        const int k = t, f0 = paper_first(k), n = paper_count(k);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, m0 = -3.0e38f, m1 = -3.0e38f, m2 = -3.0e38f;
        for (int i = f0; i < f0 + n; ++i) {
            s0 += s_rho[i]; s1 += s_f[i]; s2 += s_T[i];
            m0 = fmaxf(m0, s_rho[i]); m1 = fmaxf(m1, s_f[i]); m2 = fmaxf(m2, s_T[i]);
        }
        const float inv_n = 1.0f / (float)n;
        const float v[8] = {s0 * inv_n, s1 * inv_n, s2 * inv_n, m0, m1, m2, a.g, s_alpha};
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
            c[0] = a.g; c[1] = a.albedo[0]; c[2] = a.albedo[1]; c[3] = a.albedo[2]; c[4] = s_alpha;
        }
    }
}

void launch_gather_paper(const PaperGatherArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    note_launch();
    gather_paper_kernel<<<a.count, 288, 0, s>>>(a);
}

}  // namespace nis
