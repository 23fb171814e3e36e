// Template gathers (Sec. III.B.2-5; Eq. 2-4, 8) with the SE squeeze statistics and the SE
// excitation weights (Eq. 24-26) fused in: one 256-thread CTA per shading point, thread t
// owns lattice point t of every layer.
#include "nis_internal.h"

namespace nis {

namespace {
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }
}

__global__ void __launch_bounds__(256) gather_kernel(const __grid_constant__ GatherArgs a) {
    const int p = blockIdx.x;
    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    __shared__ float red[8][6];

    const float px = a.points[3 * p], py = a.points[3 * p + 1], pz = a.points[3 * p + 2];
    float ox = a.omega[3 * p], oy = a.omega[3 * p + 1], oz = a.omega[3 * p + 2];
    {
        float inv = 1.0f / sqrtf(ox * ox + oy * oy + oz * oz);
        ox *= inv; oy *= inv; oz *= inv;
    }
    // light frame: e_z toward the light, e_x = omega's part orthogonal to e_z
    const float ezx = -a.lx, ezy = -a.ly, ezz = -a.lz;
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
    // view angle alpha = angle(omega, l), via atan2 for conditioning near 0 and pi
    float cx_ = oy * a.lz - oz * a.ly, cy_ = oz * a.lx - ox * a.lz, cz_ = ox * a.ly - oy * a.lx;
    const float alpha = atan2f(sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_),
                               ox * a.lx + oy * a.ly + oz * a.lz);
    // phase-table interpolation weights
    // (clamped so that a NaN direction cannot index outside the table)
    float tt = fminf(fmaxf(alpha * ((kAlpha - 1) / 3.14159265358979f), 0.f), (float)(kAlpha - 1));
    int ja = min((int)floorf(tt), kAlpha - 2);
    float wa = tt - ja;
    const float *row0 = a.table + (size_t)ja * kPhaseSets * kLat;
    const float *row1 = row0 + kPhaseSets * kLat;

    const int N = a.rho.n[0];
    const int L = a.rho.levels;
    const float d_exit = fmaxf(exit_distance(px, py, pz, ezx, ezy, ezz), 1.0f / N);

    const bool active = t < kLat;
    const float qa = (float)(t / 45 - 2), qb = (float)((t / 9) % 5 - 2), qc = (float)(t % 9 - 4);
    const float ox_ = qa * exx + qb * eyx + qc * ezx;
    const float oy_ = qa * exy + qb * eyy + qc * ezy;
    const float oz_ = qa * exz + qb * eyz + qc * ezz;

    for (int k = 0; k < kLayers; ++k) {
        float cxk, cyk, czk, h;
        int m, set;
        if (k < kDiffuse) {
            cxk = px; cyk = py; czk = pz;
            float xi = 1.0f - 0.08f * (float)min(k + 1, 5);
            h = (float)(1 << k) * xi / (float)N;
            m = min(k, L - 1);
            set = 0;
        } else {
            int j = k - kDiffuse;
            float f = (j + 0.5f) * d_exit * 0.25f;
            cxk = px + ezx * f; cyk = py + ezy * f; czk = pz + ezz * f;
            h = d_exit * (1.0f / 36.0f);
            float z = log2f(h * (float)N) + 0.5f;
            m = (int)fminf(fmaxf(floorf(z), 0.f), (float)(L - 1));
            set = 1 + j;
        }
        float rho = 0.f, T = 0.f, f = 0.f;
        if (active) {
            float sx = cxk + h * ox_, sy = cyk + h * oy_, sz = czk + h * oz_;
            rho = sample_border(a.rho.lv[m], a.rho.n[m], sx, sy, sz, 0.0f);
            T = sample_border(a.T.lv[m], a.T.n[m], sx, sy, sz, 1.0f);
            float f0 = __ldg(row0 + set * kLat + t), f1 = __ldg(row1 + set * kLat + t);
            f = f0 + wa * (f1 - f0);
            size_t o = ((size_t)p * kLayers + k) * kLat + t;
            a.H_T[o] = T;
            if (a.Hb_rho) {
                size_t ob = ((size_t)p * kLayers + k) * kLatPad + t;
                a.Hb_rho[ob] = __float2bfloat16_rn(rho);
                a.Hb_f[ob] = __float2bfloat16_rn(f);
            } else {
                a.H_rho[o] = rho;
                a.H_f[o] = f;
            }
        } else if (a.Hb_rho && t < kLatPad) {     // zero the BF16 row padding
            size_t ob = ((size_t)p * kLayers + k) * kLatPad + t;
            a.Hb_rho[ob] = __float2bfloat16_rn(0.f);
            a.Hb_f[ob] = __float2bfloat16_rn(0.f);
        }
        // squeeze statistics (mean and max pooling over the layer's points)
        float s0 = rho, s1 = f, s2 = T;
        float m0 = active ? rho : -3.0e38f, m1 = active ? f : -3.0e38f, m2 = active ? T : -3.0e38f;
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(~0u, s0, o);
            s1 += __shfl_xor_sync(~0u, s1, o);
            s2 += __shfl_xor_sync(~0u, s2, o);
            m0 = fmaxf(m0, __shfl_xor_sync(~0u, m0, o));
            m1 = fmaxf(m1, __shfl_xor_sync(~0u, m1, o));
            m2 = fmaxf(m2, __shfl_xor_sync(~0u, m2, o));
        }
        if (lane == 0) {
            red[warp][0] = s0; red[warp][1] = s1; red[warp][2] = s2;
            red[warp][3] = m0; red[warp][4] = m1; red[warp][5] = m2;
        }
        __syncthreads();
        if (t == 0) {
            float v[8];
            for (int q = 0; q < 3; ++q) {
                float s = 0.f, mx = -3.0e38f;
                for (int w = 0; w < 8; ++w) { s += red[w][q]; mx = fmaxf(mx, red[w][3 + q]); }
                v[q] = s * (1.0f / kLat);
                v[3 + q] = mx;
            }
            v[6] = a.g;
            v[7] = alpha;
            if (a.v)
                for (int q = 0; q < 8; ++q) a.v[((size_t)p * kLayers + k) * 8 + q] = v[q];
            // SE excitation: w = sigmoid(W2 ReLU(W1 v + b1) + b2)
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
                    sigmoidf_(b2[r] + w2[r * 2] * z[0] + w2[r * 2 + 1] * z[1]);
        }
        __syncthreads();
    }
    if (t == 0) {
        float *c = a.cfg + (size_t)p * kCfg;
        c[0] = a.g; c[1] = a.albedo[0]; c[2] = a.albedo[1]; c[3] = a.albedo[2]; c[4] = alpha;
    }
}

void launch_gather(const GatherArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    note_launch();
    gather_kernel<<<a.count, 256, 0, s>>>(a);
}

}  // namespace nis
