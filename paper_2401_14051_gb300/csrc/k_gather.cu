// Template gathers (Sec. III.B.2-5; Eq. 2-4, 8) with the SE squeeze statistics and the SE
// excitation weights (Eq. 24-26) fused in: one CTA per shading point, one warp per template
// layer; lane l owns lattice points l, l + 32, ... and the squeeze statistics are reduced
// with warp shuffles, so the layers proceed independently without block barriers.
#include <cuda_fp8.h>

#include "nis_internal.h"

namespace nis {

namespace {
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }
}

// kF8: the FP8 path, which keeps every sample of the layer to scale them by its maximum.
template <bool kF8>
__global__ void __launch_bounds__(kLayers * 32, kF8 ? 2 : 3) gather_kernel(const __grid_constant__ GatherArgs a) {
    const int p = blockIdx.x;
    const int k = threadIdx.x >> 5;            // one warp per template layer
    const int lane = threadIdx.x & 31;
    // lattice offsets (a, b, c) of the 225 template points, in spacings
    __shared__ float4 s_lat[kLat];
    for (int t = threadIdx.x; t < kLat; t += blockDim.x)
        s_lat[t] = make_float4((float)(t / 45 - 2), (float)((t / 9) % 5 - 2), (float)(t % 9 - 4), 0.f);
    __syncthreads();

    // single request, or this point's request in a mixed batch
    const ReqDesc *d = a.descs ? a.descs + a.req_of_point[p] : nullptr;
    const PairView &RT = d ? d->rt : a.rt;
    const float lx = d ? d->l[0] : a.lx, ly = d ? d->l[1] : a.ly, lz = d ? d->l[2] : a.lz;
    const float gg = d ? d->g : a.g;
    const float *table = d ? d->table : a.table;
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
    // view angle alpha = angle(omega, l), via atan2 for conditioning near 0 and pi
    float cx_ = oy * lz - oz * ly, cy_ = oz * lx - ox * lz, cz_ = ox * ly - oy * lx;
    const float alpha = atan2f(sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_), ox * lx + oy * ly + oz * lz);
    // phase-table interpolation weights
    // (clamped so that a NaN direction cannot index outside the table)
    float tt = fminf(fmaxf(alpha * ((kAlpha - 1) / 3.14159265358979f), 0.f), (float)(kAlpha - 1));
    int ja = min((int)floorf(tt), kAlpha - 2);
    float wa = tt - ja;

    const int N = RT.n[0];
    const int L = RT.levels;
    // this warp's layer: centre, spacing, mip level and phase point set
    float cxk, cyk, czk, h;
    int m, set;
    if (k < kDiffuse) {
        cxk = px; cyk = py; czk = pz;
        float xi = 1.0f - 0.08f * (float)min(k + 1, 5);
        h = (float)(1 << k) * xi / (float)N;
        m = min(k, L - 1);
        set = 0;
    } else {
        const float d_exit = fmaxf(exit_distance(px, py, pz, ezx, ezy, ezz), 1.0f / N);
        int j = k - kDiffuse;
        float f = (j + 0.5f) * d_exit * 0.25f;
        cxk = px + ezx * f; cyk = py + ezy * f; czk = pz + ezz * f;
        h = d_exit * (1.0f / 36.0f);
        float z = log2f(h * (float)N) + 0.5f;
        m = (int)fminf(fmaxf(floorf(z), 0.f), (float)(L - 1));
        set = 1 + j;
    }
    const float4 *rt_lv = RT.lv[m];
    const int nm = RT.n[m];
    const float *row0 = table + ((size_t)ja * kPhaseSets + set) * kLat;
    const float *row1 = row0 + kPhaseSets * kLat;
    const size_t obase = ((size_t)p * kLayers + k) * kLat;
    // BF16 rows per layer: kLatPad, or kFuseLatLd with the fused backbone's configuration
    // operand after the features
    const size_t obase_b = ((size_t)p * kLayers + k) * (a.fused ? kFuseLatLd : kLatPad);

    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float m0 = -3.0e38f, m1 = -3.0e38f, m2 = -3.0e38f;
    float keep_rho[kF8 ? 8 : 1], keep_f[kF8 ? 8 : 1];   // this lane's samples (FP8 only)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int t = lane + 32 * i;
        if (kF8) keep_rho[i] = keep_f[i] = 0.f;
        if (t < kLat) {
            const float4 ql = s_lat[t];
            const float qa = ql.x, qb = ql.y, qc = ql.z;
            const float sx = cxk + h * (qa * exx + qb * eyx + qc * ezx);
            const float sy = cyk + h * (qa * exy + qb * eyy + qc * ezy);
            const float sz = czk + h * (qa * exz + qb * eyz + qc * ezz);
            const float2 rt = sample_pair(rt_lv, nm, sx, sy, sz);
            const float rho = rt.x, T = rt.y;
            const float f0 = __ldg(row0 + t), f1 = __ldg(row1 + t);
            const float f = f0 + wa * (f1 - f0);
            a.H_T[obase + t] = T;
            if (a.H_rho) {                        // FP32 copies (FP32 SIMT path, or debug)
                a.H_rho[obase + t] = rho;
                a.H_f[obase + t] = f;
            }
            if (a.Hb_rho) {
                if (a.split) {                    // three-way BF16 split (FP32-accurate mode)
                    float r0 = rho, r1 = f;
                    for (int q = 0; q < 3; ++q) {
                        __nv_bfloat16 b0 = __float2bfloat16_rn(r0), b1 = __float2bfloat16_rn(r1);
                        a.Hb_rho[obase_b + t + q * a.part] = b0;
                        a.Hb_f[obase_b + t + q * a.part] = b1;
                        r0 -= __bfloat162float(b0);
                        r1 -= __bfloat162float(b1);
                    }
                } else {
                    a.Hb_rho[obase_b + t] = __float2bfloat16_rn(rho);
                    a.Hb_f[obase_b + t] = __float2bfloat16_rn(f);
                }
            }
            s0 += rho; s1 += f; s2 += T;
            m0 = fmaxf(m0, rho); m1 = fmaxf(m1, f); m2 = fmaxf(m2, T);
            if (kF8) {
                keep_rho[i] = rho;
                keep_f[i] = f;
            }
        } else if (a.Hb_rho && t < kLatPad && !a.fused) {     // zero the BF16 row padding
            for (int q = 0; q < (a.split ? 3 : 1); ++q) {
                a.Hb_rho[obase_b + t + q * a.part] = __float2bfloat16_rn(0.f);
                a.Hb_f[obase_b + t + q * a.part] = __float2bfloat16_rn(0.f);
            }
        }
    }
    // squeeze statistics (mean and max pooling over the layer's points)
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(~0u, s0, o);
        s1 += __shfl_xor_sync(~0u, s1, o);
        s2 += __shfl_xor_sync(~0u, s2, o);
        m0 = fmaxf(m0, __shfl_xor_sync(~0u, m0, o));
        m1 = fmaxf(m1, __shfl_xor_sync(~0u, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(~0u, m2, o));
    }
    if (kF8) {
        // e4m3 features scaled per (point, layer, type) by max / 448
        const float sr = m0 > 0.f ? m0 / 448.f : 1.f, sf = m1 > 0.f ? m1 / 448.f : 1.f;
        const size_t ob8 = ((size_t)p * kLayers + k) * kLatPad8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int t = lane + 32 * i;
            if (t < kLatPad8) {
                a.H8_rho[ob8 + t] = __nv_cvt_float_to_fp8(keep_rho[i] / sr, __NV_SATFINITE, __NV_E4M3);
                a.H8_f[ob8 + t] = __nv_cvt_float_to_fp8(keep_f[i] / sf, __NV_SATFINITE, __NV_E4M3);
            }
        }
        if (lane == 0) {
            a.f8_scale[((size_t)p * kLayers + k) * 2] = sr;
            a.f8_scale[((size_t)p * kLayers + k) * 2 + 1] = sf;
        }
    }
    if (lane == 0) {
        float v[8] = {s0 * (1.0f / kLat), s1 * (1.0f / kLat), s2 * (1.0f / kLat), m0, m1, m2, gg, alpha};
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
        float wse[3];
        for (int r = 0; r < 3; ++r) {
            wse[r] = sigmoidf_(b2[r] + w2[r * 2] * z[0] + w2[r * 2 + 1] * z[1]);
            a.w_se[((size_t)p * kLayers + k) * 3 + r] = wse[r];
        }
        const float *alb = d ? d->albedo : a.albedo;
        if (k == 0) {
            float *c = a.cfg + (size_t)p * kCfg;
            c[0] = gg; c[1] = alb[0]; c[2] = alb[1]; c[3] = alb[2]; c[4] = alpha;
        }
        if (a.fused) {
            // the fused backbone's configuration operand of this layer, per type: c / w and
            // 1 / w as two BF16 parts each (hi, lo), then zeros to the end of the row; rho and
            // f in their feature rows after the 225 features, T ahead of the CNN's 80 outputs
            const float c5[5] = {gg, alb[0], alb[1], alb[2], alpha};
            for (int r = 0; r < 3; ++r) {
                const float u = 1.0f / fmaxf(wse[r], kSeFloor);
                float row[16];
                for (int q = 0; q < 5; ++q) {
                    const float x = c5[q] * u;
                    const float hi = __bfloat162float(__float2bfloat16_rn(x));
                    row[q] = hi;
                    row[5 + q] = x - hi;
                }
                const float uh = __bfloat162float(__float2bfloat16_rn(u));
                row[10] = uh; row[11] = uh; row[12] = u - uh;
                row[13] = row[14] = row[15] = 0.f;
                __nv_bfloat16 *dst = r == 0 ? a.Hb_rho + obase_b + kLat
                                   : r == 1 ? a.Hb_f + obase_b + kLat
                                            : a.XT_cfg + ((size_t)p * kLayers + k) * kFuseXtLd + kDT;
                const int n = r == 2 ? kFuseXtLd - kDT : kFuseLatLd - kLat;
                for (int q = 0; q < n; ++q) dst[q] = __float2bfloat16_rn(row[q]);
            }
        }
    }
}

void launch_gather(const GatherArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    note_launch();
    if (a.H8_rho) gather_kernel<true><<<a.count, kLayers * 32, 0, s>>>(a);
    else gather_kernel<false><<<a.count, kLayers * 32, 0, s>>>(a);
}

// Mixed batches: row -> request descriptor, and each row's decode scale.
__global__ void fill_segments_kernel(const int *__restrict__ seg_start,
                                     const int *__restrict__ seg_desc, int nseg, int count,
                                     int *__restrict__ req_of_point, float *__restrict__ dec_rows,
                                     const ReqDesc *__restrict__ descs) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    int lo = 0, hi = nseg - 1;                // last segment whose start <= r
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg_start[mid] <= r) lo = mid; else hi = mid - 1;
    }
    int d = seg_desc[lo];
    req_of_point[r] = d;
    for (int c = 0; c < 3; ++c) dec_rows[3 * (size_t)r + c] = descs[d].dec[c];
}

void launch_fill_segments(const int *seg_start, const int *seg_desc, int nseg, int count,
                          int *req_of_point, float *dec_rows, const ReqDesc *descs,
                          cudaStream_t s) {
    if (count <= 0) return;
    note_launch();
    fill_segments_kernel<<<(count + 255) / 256, 256, 0, s>>>(seg_start, seg_desc, nseg, count,
                                                             req_of_point, dec_rows, descs);
}

}  // namespace nis
