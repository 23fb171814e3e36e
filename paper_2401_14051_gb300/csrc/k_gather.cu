// Template gathers (Sec. III.B.2-5; Eq. 2-4, 8) with the SE squeeze statistics and the SE
// excitation weights (Eq. 24-26) fused in.
//
// gather_kernel (FP32, BF16 and three-part BF16 outputs): one lane per shading point, one
// warp per template layer over 32 consecutive points, four layers per CTA.  Consecutive
// shading points of a frame are neighbouring pixels, so a warp's 32 samples of one lattice
// point fall on the same or adjacent voxels and each load touches few cache lines.  Each lane
// walks its point's 225 lattice points in order, keeps the squeeze statistics in registers
// (no reduction), and packs its outputs in registers into whole 32-byte pieces of its rows,
// written with single vector stores.
//
// gather8_kernel (FP8 outputs): one CTA per shading point, one warp per layer, lane l owns
// lattice points l, l + 32, ...; it keeps all of a lane's samples to scale the layer's e4m3
// row by the layer's maximum.
#include <cuda_fp8.h>

#include "nis_internal.h"

namespace nis {

namespace {
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// Per shading point: its position, the light frame (e_z toward the light, e_x the part of
// omega orthogonal to e_z), the view angle alpha and the phase table's interpolation node.
struct PointFrame {
    float px, py, pz;
    float ex[3], ey[3], ez[3];
    float alpha, wa;
    int ja;
};

__device__ __forceinline__ PointFrame point_frame(const float *points, const float *omega, int p,
                                                  float lx, float ly, float lz) {
    PointFrame f;
    f.px = points[3 * p]; f.py = points[3 * p + 1]; f.pz = points[3 * p + 2];
    float ox = omega[3 * p], oy = omega[3 * p + 1], oz = omega[3 * p + 2];
    {
        float inv = 1.0f / sqrtf(ox * ox + oy * oy + oz * oz);
        ox *= inv; oy *= inv; oz *= inv;
    }
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
    f.ex[0] = exx; f.ex[1] = exy; f.ex[2] = exz;
    f.ez[0] = ezx; f.ez[1] = ezy; f.ez[2] = ezz;
    f.ey[0] = ezy * exz - ezz * exy;
    f.ey[1] = ezz * exx - ezx * exz;
    f.ey[2] = ezx * exy - ezy * exx;
    // alpha = angle(omega, l) via atan2, well conditioned near 0 and pi
    float cx_ = oy * lz - oz * ly, cy_ = oz * lx - ox * lz, cz_ = ox * ly - oy * lx;
    f.alpha = atan2f(sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_), ox * lx + oy * ly + oz * lz);
    // phase-table node and weight (clamped so that a NaN direction cannot leave the table)
    float tt = fminf(fmaxf(f.alpha * ((kAlpha - 1) / 3.14159265358979f), 0.f), (float)(kAlpha - 1));
    f.ja = min((int)floorf(tt), kAlpha - 2);
    f.wa = tt - f.ja;
    return f;
}

// Layer k of a point: template centre, spacing h, mip level m and phase point set.  Diffuse
// layers sit at the point with h = 2^k xi_(k+1) / N on level k; highlight layer j sits at
// (j + 1/2) d / 4 toward the light with h = d / 36 on the level whose voxel matches h.
struct LayerGeom {
    float cx, cy, cz, h;
    int m, set;
};

__device__ __forceinline__ LayerGeom layer_geom(int k, const PointFrame &f, int N, int L) {
    LayerGeom g;
    if (k < kDiffuse) {
        g.cx = f.px; g.cy = f.py; g.cz = f.pz;
        float xi = 1.0f - 0.08f * (float)min(k + 1, 5);
        g.h = (float)(1 << k) * xi / (float)N;
        g.m = min(k, L - 1);
        g.set = 0;
    } else {
        const float d_exit = fmaxf(exit_distance(f.px, f.py, f.pz, f.ez[0], f.ez[1], f.ez[2]), 1.0f / N);
        int j = k - kDiffuse;
        float s = (j + 0.5f) * d_exit * 0.25f;
        g.cx = f.px + f.ez[0] * s; g.cy = f.py + f.ez[1] * s; g.cz = f.pz + f.ez[2] * s;
        g.h = d_exit * (1.0f / 36.0f);
        float z = log2f(g.h * (float)N) + 0.5f;
        g.m = (int)fminf(fmaxf(floorf(z), 0.f), (float)(L - 1));
        g.set = 1 + j;
    }
    return g;
}

// The squeeze vector of (point p, layer k), its SE excitation w = sigmoid(W2 ReLU(W1 v + b1)
// + b2) (to w_se and wse) and, for k = 0, the point's configuration vector.
__device__ __forceinline__ void se_epilogue(const GatherArgs &a, const ReqDesc *d, int p, int k,
                                            float s0, float s1, float s2, float m0, float m1,
                                            float m2, float gg, float alpha, float (&wse)[3]) {
    float v[8] = {s0 * (1.0f / kLat), s1 * (1.0f / kLat), s2 * (1.0f / kLat), m0, m1, m2, gg, alpha};
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
    for (int r = 0; r < 3; ++r) {
        wse[r] = sigmoidf_(b2[r] + w2[r * 2] * z[0] + w2[r * 2 + 1] * z[1]);
        a.w_se[((size_t)p * kLayers + k) * 3 + r] = wse[r];
    }
    if (k == 0) {
        const float *alb = d ? d->albedo : a.albedo;
        float *c = a.cfg + (size_t)p * kCfg;
        c[0] = gg; c[1] = alb[0]; c[2] = alb[1]; c[3] = alb[2]; c[4] = alpha;
    }
}

// Two floats as BF16 (round to nearest even), lo at the lower address.
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float bf_lo(uint32_t r) { return __uint_as_float(r << 16); }
__device__ __forceinline__ float bf_hi(uint32_t r) { return __uint_as_float(r & 0xffff0000u); }

// 16 bytes to a 16-byte aligned global address.
__device__ __forceinline__ void st_v4(void *p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" :: "l"(p), "r"(x), "r"(y), "r"(z),
                 "r"(w) : "memory");
}
// 32 bytes to a 32-byte aligned global address.
__device__ __forceinline__ void st_v8(void *p, const uint32_t (&v)[8]) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                    "r"(v[6]), "r"(v[7]) : "memory");
}

// The fused backbone's configuration operand of a layer for one type: c / w and 1 / w as two
// BF16 parts each (hi, lo) in columns 0-12, zeros in 13-15; as packed pairs.
__device__ __forceinline__ void fused_cfg_row(float gg, const float *alb, float alpha, float w,
                                              uint32_t (&row)[8]) {
    const float c5[5] = {gg, alb[0], alb[1], alb[2], alpha};
    const float u = 1.0f / fmaxf(w, kSeFloor);
    float x[16];
    for (int q = 0; q < 5; ++q) {
        const float v = c5[q] * u;
        const float hi = __bfloat162float(__float2bfloat16_rn(v));
        x[q] = hi;
        x[5 + q] = v - hi;
    }
    const float uh = __bfloat162float(__float2bfloat16_rn(u));
    x[10] = uh; x[11] = uh; x[12] = u - uh;
    x[13] = x[14] = x[15] = 0.f;
    for (int q = 0; q < 8; ++q) row[q] = pack_bf2(x[2 * q], x[2 * q + 1]);
}

// One 32-byte PairView entry (two float4: the y0 and y1 rows of a cell's z slice) in one
// full-sector load.
__device__ __forceinline__ void ld_entry(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Trilinear (density, transmittance) at grid coordinates (gx, gy, gz) = position * n - 1/2 of
// a PairView level (entry (z, j, i) holds both fields at y = j - 1, j and x = i - 1, i), zero
// density and unit transmittance outside the grid: two 32-byte loads, one per z slice.
__device__ __forceinline__ float2 sample_pair_grid(const float4 *__restrict__ g, int n, float gx,
                                                   float gy, float gz) {
    int ix = __float2int_rd(gx), iy = __float2int_rd(gy), iz = __float2int_rd(gz);
    const float fx = gx - (float)ix, fy = gy - (float)iy, fz = gz - (float)iz;
    const int m = n + 1;
    float4 q[4];                                 // (y, z) corners; .x .y at ix, .z .w at ix + 1
    // entry (z, iy + 1, ix + 1) exists for iy, ix in [-1, n - 1]
    const bool xy_in = (unsigned)(ix + 1) <= (unsigned)n && (unsigned)(iy + 1) <= (unsigned)n;
    if (xy_in && (unsigned)iz < (unsigned)(n - 1) && n <= 1024) {
        const float4 *p = g + 2 * (((unsigned)iz * (unsigned)m + (unsigned)(iy + 1)) * (unsigned)m + (unsigned)(ix + 1));
        ld_entry(p, q[0], q[1]);
        ld_entry(p + 2 * (unsigned)m * (unsigned)m, q[2], q[3]);
    } else {
        iz = min(max(iz, -2), n + 1);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int cz = iz + c;
            if (xy_in && (unsigned)cz < (unsigned)n) {
                ld_entry(g + 2 * (((size_t)cz * m + (iy + 1)) * m + (ix + 1)), q[2 * c], q[2 * c + 1]);
            } else {
                q[2 * c] = q[2 * c + 1] = make_float4(0.0f, 1.0f, 0.0f, 1.0f);
            }
        }
    }
    const float2 c00 = lerp2(make_float2(q[0].x, q[0].y), make_float2(q[0].z, q[0].w), fx);
    const float2 c01 = lerp2(make_float2(q[1].x, q[1].y), make_float2(q[1].z, q[1].w), fx);
    const float2 c10 = lerp2(make_float2(q[2].x, q[2].y), make_float2(q[2].z, q[2].w), fx);
    const float2 c11 = lerp2(make_float2(q[3].x, q[3].y), make_float2(q[3].z, q[3].w), fx);
    return lerp2(lerp2(c00, c01, fy), lerp2(c10, c11, fy), fz);
}

// Lattice offsets (a, b, c) of the 225 template points in spacings: t = 45 (a + 2) +
// 9 (b + 2) + (c + 4), a, b in -2..2, c in -4..4.
__device__ __forceinline__ float4 lattice_offset(int t) {
    return make_float4((float)(t / 45 - 2), (float)((t / 9) % 5 - 2), (float)(t % 9 - 4), 0.f);
}
}  // namespace

constexpr int kGWarps = 4;                       // layers (warps) per gather_kernel CTA

// kParts 1: BF16 feature rows; 3: the three-part BF16 split; 8: e4m3 rows of the fused
// network's e4m3 mode.  Rows are written in chunks of 16 BF16 columns (32 e4m3; 8 FP32 for
// H_T), one 32-byte store each.
template <int kParts>
__global__ void __launch_bounds__(kGWarps * 32, 4) gather_kernel(const __grid_constant__ GatherArgs a) {
    __shared__ float4 s_lat[kLat];
    for (int t = threadIdx.x; t < kLat; t += blockDim.x) s_lat[t] = lattice_offset(t);
    __syncthreads();
    const int k = blockIdx.y * kGWarps + (threadIdx.x >> 5);   // this warp's template layer
    const int p = blockIdx.x * 32 + (threadIdx.x & 31);        // this lane's shading point
    if (p >= a.count) return;                                  // no block barrier follows

    const ReqDesc *d = a.descs ? a.descs + a.req_of_point[p] : nullptr;
    const PairView &RT = d ? d->rt : a.rt;
    const float lx = d ? d->l[0] : a.lx, ly = d ? d->l[1] : a.ly, lz = d ? d->l[2] : a.lz;
    const float gg = d ? d->g : a.g;
    const float *table = d ? d->table : a.table;
    const PointFrame f = point_frame(a.points, a.omega, p, lx, ly, lz);
    const LayerGeom lg = layer_geom(k, f, RT.n[0], RT.levels);
    const float4 *rt_lv = RT.lv[lg.m];
    const int nm = RT.n[lg.m];
    // sample position in the level's grid coordinates: G0 + a A + b B + c C
    const float sc = lg.h * (float)nm;
    const float g0x = lg.cx * nm - 0.5f, g0y = lg.cy * nm - 0.5f, g0z = lg.cz * nm - 0.5f;
    const float Ax = sc * f.ex[0], Ay = sc * f.ex[1], Az = sc * f.ex[2];
    const float Bx = sc * f.ey[0], By = sc * f.ey[1], Bz = sc * f.ey[2];
    const float Cx = sc * f.ez[0], Cy = sc * f.ez[1], Cz = sc * f.ez[2];
    const float wa = f.wa;
    const float *row0 = table + ((size_t)f.ja * kPhaseSets + lg.set) * kLat;
    const float *row1 = row0 + kPhaseSets * kLat;
    const size_t rk = (size_t)p * kLayers + k;
    float *hT = a.H_T + rk * kLatT;
    float *hR = a.H_rho ? a.H_rho + rk * kLat : nullptr;      // FP32 copies (SIMT path, debug)
    float *hF = a.H_f ? a.H_f + rk * kLat : nullptr;
    __nv_bfloat16 *bR = a.Hb_rho ? a.Hb_rho + rk * kLatPad : nullptr;
    __nv_bfloat16 *bF = a.Hb_f ? a.Hb_f + rk * kLatPad : nullptr;
    const size_t part = a.part;
    // e4m3 mode: x / s with s = sigma_max / 448 (density) and the phase set's table maximum /
    // 448 (phase); both bound their feature from above, so nothing saturates
    uint8_t *qR = kParts == 8 ? a.F8_rho + rk * kF8LatLd : nullptr;
    uint8_t *qF = kParts == 8 ? a.F8_f + rk * kF8LatLd : nullptr;
    float s_r = 1.f, s_f = 1.f;
    if (kParts == 8) {
        const float sg = __ldg(a.f8_sigma), tm = __ldg(a.f8_tabmax + lg.set);
        if (sg > 0.f) s_r = sg * (1.0f / 448.f);
        if (tm > 0.f) s_f = tm * (1.0f / 448.f);
    }
    const float inv_r = 1.0f / s_r, inv_f = 1.0f / s_f;
    auto q2 = [](float x0, float x1) -> uint32_t {   // two values as e4m3, x0 in the low byte
        return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(x0, x1), __NV_SATFINITE, __NV_E4M3);
    };

    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float m0 = -3.0e38f, m1 = -3.0e38f, m2 = -3.0e38f;
    auto sample = [&](int t, float &rho, float &T, float &fv) {
        const float4 ql = s_lat[t];
        const float gx = g0x + ql.x * Ax + ql.y * Bx + ql.z * Cx;
        const float gy = g0y + ql.x * Ay + ql.y * By + ql.z * Cy;
        const float gz = g0z + ql.x * Az + ql.y * Bz + ql.z * Cz;
        const float2 rt = sample_pair_grid(rt_lv, nm, gx, gy, gz);
        rho = rt.x; T = rt.y;
        const float f0 = __ldg(row0 + t), f1 = __ldg(row1 + t);
        fv = f0 + wa * (f1 - f0);
        if (hR) { hR[t] = rho; hF[t] = fv; }
        s0 += rho; s1 += fv; s2 += T;
        m0 = fmaxf(m0, rho); m1 = fmaxf(m1, fv); m2 = fmaxf(m2, T);
    };
    // BF16 parts of a pair of values: x = p0 + p1 + p2 (kParts 3) or p0 (kParts 1)
    auto split2 = [&](float x0, float x1, uint32_t (&out)[3]) {
        out[0] = pack_bf2(x0, x1);
        if constexpr (kParts == 3) {
            x0 -= bf_lo(out[0]); x1 -= bf_hi(out[0]);
            out[1] = pack_bf2(x0, x1);
            x0 -= bf_lo(out[1]); x1 -= bf_hi(out[1]);
            out[2] = pack_bf2(x0, x1);
        }
    };
    constexpr int CH = 16;                                  // columns per chunk
    for (int t0 = 0; t0 < kLat - 1; t0 += CH) {             // lattice points 0..223
        // kParts 1: packed BF16 pairs; kParts 3: the FP32 values, split after the chunk;
        // kParts 8: packed e4m3 quadruples (16 bytes per chunk)
        uint32_t rb[CH / 2], fb[CH / 2];
        float rv[kParts == 3 ? CH : 1], fvv[kParts == 3 ? CH : 1];
        float tb[8];
#pragma unroll
        for (int u = 0; u < CH; u += 2) {
            float r0, T0, f0, r1, T1, f1;
            sample(t0 + u, r0, T0, f0);
            sample(t0 + u + 1, r1, T1, f1);
            tb[u & 7] = T0;
            tb[(u + 1) & 7] = T1;
            if ((u & 7) == 6) {                              // 8 transmittance values
                uint32_t v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = __float_as_uint(tb[q]);
                st_v8(hT + t0 + u - 6, v);
            }
            if constexpr (kParts == 1) {
                rb[u / 2] = pack_bf2(r0, r1);
                fb[u / 2] = pack_bf2(f0, f1);
            } else if constexpr (kParts == 8) {
                const uint32_t qr = q2(r0 * inv_r, r1 * inv_r), qf = q2(f0 * inv_f, f1 * inv_f);
                if ((u & 2) == 0) { rb[u / 4] = qr; fb[u / 4] = qf; }
                else { rb[u / 4] |= qr << 16; fb[u / 4] |= qf << 16; }
            } else {
                rv[u] = r0; rv[u + 1] = r1;
                fvv[u] = f0; fvv[u + 1] = f1;
            }
        }
        if constexpr (kParts == 8) {
            st_v4(qR + t0, rb[0], rb[1], rb[2], rb[3]);
            st_v4(qF + t0, fb[0], fb[1], fb[2], fb[3]);
        } else if (bR) {
            if constexpr (kParts == 1) {
                st_v8(bR + t0, rb);
                st_v8(bF + t0, fb);
            } else {
                // three-way split x = x0 + x1 + x2: each part rounds the remainder to BF16
#pragma unroll
                for (int q = 0; q < 3; ++q) {
#pragma unroll
                    for (int i = 0; i < CH / 2; ++i) {
                        rb[i] = pack_bf2(rv[2 * i], rv[2 * i + 1]);
                        fb[i] = pack_bf2(fvv[2 * i], fvv[2 * i + 1]);
                        rv[2 * i] -= bf_lo(rb[i]); rv[2 * i + 1] -= bf_hi(rb[i]);
                        fvv[2 * i] -= bf_lo(fb[i]); fvv[2 * i + 1] -= bf_hi(fb[i]);
                    }
                    st_v8(bR + q * part + t0, rb);
                    st_v8(bF + q * part + t0, fb);
                }
            }
        }
    }
    // the last lattice point (224), then the squeeze and excitation, then the rows' tails:
    // columns 224..231 of H_T (zeros after 224) and 224..239 of the BF16 rows (zeros, or the
    // fused backbone's configuration operand in 225..237)
    float rl, Tl, fl;
    sample(kLat - 1, rl, Tl, fl);
    {
        uint32_t v[8] = {__float_as_uint(Tl), 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        st_v8(hT + kLat - 1, v);
    }
    float wse[3];
    se_epilogue(a, d, p, k, s0, s1, s2, m0, m1, m2, gg, f.alpha, wse);
    if constexpr (kParts == 8) {
        // the e4m3 rows' tails (columns 224..255), the configuration operands c / u and 1 / u
        // of density and phase (u = w_se s S_w) and of the transmittance (u = w_se), and the
        // epilogue's row factors u
        {
            uint32_t vr[8] = {q2(rl * inv_r, 0.f), 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            uint32_t vf[8] = {q2(fl * inv_f, 0.f), 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            st_v8(qR + kLat - 1, vr);
            st_v8(qF + kLat - 1, vf);
        }
        const float *alb = d ? d->albedo : a.albedo;
        const float u_r = fmaxf(wse[0] * s_r * a.f8_sw[k][0], kSeFloor);
        const float u_f = fmaxf(wse[1] * s_f * a.f8_sw[k][1], kSeFloor);
        uint32_t row[8];
        fused_cfg_row(gg, alb, f.alpha, u_r, row);
        st_v8(a.F8_cfg + rk * kF8CfgLd, row);
        fused_cfg_row(gg, alb, f.alpha, u_f, row);
        st_v8(a.F8_cfg + rk * kF8CfgLd + 16, row);
        fused_cfg_row(gg, alb, f.alpha, wse[2], row);
        st_v8(a.XT_cfg + rk * kFuseXtLd + kDT, row);
        a.fc1_scale[rk * 3] = u_r;
        a.fc1_scale[rk * 3 + 1] = u_f;
        a.fc1_scale[rk * 3 + 2] = fmaxf(wse[2], kSeFloor);
    } else if (bR) {
        if (a.fused) {                                       // BF16 only (kParts 1)
            const float *alb = d ? d->albedo : a.albedo;
            uint32_t row[8], out[8];
            fused_cfg_row(gg, alb, f.alpha, wse[0], row);
            out[0] = (pack_bf2(rl, 0.f) & 0xffffu) | (row[0] << 16);
            for (int q = 1; q < 8; ++q) out[q] = (row[q - 1] >> 16) | (row[q] << 16);
            st_v8(bR + kLat - 1, out);
            fused_cfg_row(gg, alb, f.alpha, wse[1], row);
            out[0] = (pack_bf2(fl, 0.f) & 0xffffu) | (row[0] << 16);
            for (int q = 1; q < 8; ++q) out[q] = (row[q - 1] >> 16) | (row[q] << 16);
            st_v8(bF + kLat - 1, out);
            fused_cfg_row(gg, alb, f.alpha, wse[2], row);
            st_v8(a.XT_cfg + rk * kFuseXtLd + kDT, row);
        } else {
            uint32_t pr[3], pf[3];
            split2(rl, 0.f, pr);
            split2(fl, 0.f, pf);
#pragma unroll
            for (int q = 0; q < kParts; ++q) {
                uint32_t vr[8] = {pr[q], 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                uint32_t vf[8] = {pf[q], 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                st_v8(bR + q * part + kLat - 1, vr);
                st_v8(bF + q * part + kLat - 1, vf);
            }
        }
    }
}

__global__ void __launch_bounds__(kLayers * 32, 2) gather8_kernel(const __grid_constant__ GatherArgs a) {
    __shared__ float4 s_lat[kLat];
    for (int t = threadIdx.x; t < kLat; t += blockDim.x) s_lat[t] = lattice_offset(t);
    __syncthreads();
    const int p = blockIdx.x;
    const int k = threadIdx.x >> 5;              // one warp per template layer
    const int lane = threadIdx.x & 31;
    const ReqDesc *d = a.descs ? a.descs + a.req_of_point[p] : nullptr;
    const PairView &RT = d ? d->rt : a.rt;
    const float lx = d ? d->l[0] : a.lx, ly = d ? d->l[1] : a.ly, lz = d ? d->l[2] : a.lz;
    const float gg = d ? d->g : a.g;
    const float *table = d ? d->table : a.table;
    const PointFrame f = point_frame(a.points, a.omega, p, lx, ly, lz);
    const LayerGeom lg = layer_geom(k, f, RT.n[0], RT.levels);
    const float4 *rt_lv = RT.lv[lg.m];
    const int nm = RT.n[lg.m];
    const float sc = lg.h * (float)nm;
    const float g0x = lg.cx * nm - 0.5f, g0y = lg.cy * nm - 0.5f, g0z = lg.cz * nm - 0.5f;
    const float *row0 = table + ((size_t)f.ja * kPhaseSets + lg.set) * kLat;
    const float *row1 = row0 + kPhaseSets * kLat;
    const size_t rk = (size_t)p * kLayers + k;

    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    float m0 = -3.0e38f, m1 = -3.0e38f, m2 = -3.0e38f;
    float keep_rho[8], keep_f[8];                // this lane's samples
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int t = lane + 32 * i;
        keep_rho[i] = keep_f[i] = 0.f;
        if (t < kLat) {
            const float4 ql = s_lat[t];
            const float gx = g0x + sc * (ql.x * f.ex[0] + ql.y * f.ey[0] + ql.z * f.ez[0]);
            const float gy = g0y + sc * (ql.x * f.ex[1] + ql.y * f.ey[1] + ql.z * f.ez[1]);
            const float gz = g0z + sc * (ql.x * f.ex[2] + ql.y * f.ey[2] + ql.z * f.ez[2]);
            const float2 rt = sample_pair_grid(rt_lv, nm, gx, gy, gz);
            const float rho = rt.x, T = rt.y;
            const float f0 = __ldg(row0 + t), f1 = __ldg(row1 + t);
            const float fv = f0 + f.wa * (f1 - f0);
            a.H_T[rk * kLatT + t] = T;
            if (a.H_rho) {                       // FP32 copies (debug)
                a.H_rho[rk * kLat + t] = rho;
                a.H_f[rk * kLat + t] = fv;
            }
            s0 += rho; s1 += fv; s2 += T;
            m0 = fmaxf(m0, rho); m1 = fmaxf(m1, fv); m2 = fmaxf(m2, T);
            keep_rho[i] = rho;
            keep_f[i] = fv;
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
    // e4m3 features scaled per (point, layer, type) by max / 448
    const float sr = m0 > 0.f ? m0 / 448.f : 1.f, sf = m1 > 0.f ? m1 / 448.f : 1.f;
    const size_t ob8 = rk * kLatPad8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int t = lane + 32 * i;
        if (t < kLatPad8) {
            a.H8_rho[ob8 + t] = __nv_cvt_float_to_fp8(keep_rho[i] / sr, __NV_SATFINITE, __NV_E4M3);
            a.H8_f[ob8 + t] = __nv_cvt_float_to_fp8(keep_f[i] / sf, __NV_SATFINITE, __NV_E4M3);
        }
    }
    if (lane == 0) {
        a.f8_scale[rk * 2] = sr;
        a.f8_scale[rk * 2 + 1] = sf;
        float wse[3];
        se_epilogue(a, d, p, k, s0, s1, s2, m0, m1, m2, gg, f.alpha, wse);
    }
}

void launch_gather(const GatherArgs &a, cudaStream_t s) {
    if (a.count <= 0) return;
    note_launch();
    if (a.H8_rho) {
        gather8_kernel<<<a.count, kLayers * 32, 0, s>>>(a);
    } else {
        const dim3 grid((a.count + 31) / 32, kLayers / kGWarps);
        if (a.F8_rho) gather_kernel<8><<<grid, kGWarps * 32, 0, s>>>(a);
        else if (a.Hb_rho && a.split) gather_kernel<3><<<grid, kGWarps * 32, 0, s>>>(a);
        else gather_kernel<1><<<grid, kGWarps * 32, 0, s>>>(a);
    }
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

namespace nis {

// Largest value of each of the phase table's point sets ([kAlpha][kPhaseSets][kLat], all
// entries >= 0): blocks of 256 threads over slices of the alpha nodes, a shared-memory
// reduction, then an atomic max on the value's bits (order-preserving for non-negative
// floats) into out[set], cleared first.
constexpr int kTabSlices = 64;
__global__ void __launch_bounds__(256) table_set_max_kernel(const float *__restrict__ table,
                                                            float *__restrict__ out) {
    __shared__ float red[256];
    const int set = blockIdx.y;
    constexpr int per = kAlpha / kTabSlices;
    float m = 0.f;
    for (int i = threadIdx.x; i < per * kLat; i += 256) {
        const int al = blockIdx.x * per + i / kLat, t = i % kLat;
        m = fmaxf(m, table[((size_t)al * kPhaseSets + set) * kLat + t]);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<int *>(out) + set, __float_as_int(fmaxf(red[0], 0.f)));
}

void launch_table_set_max(const float *table, float *out, cudaStream_t s) {
    cudaMemsetAsync(out, 0, kPhaseSets * sizeof(float), s);
    note_launch();
    table_set_max_kernel<<<dim3(kTabSlices, kPhaseSets), 256, 0, s>>>(table, out);
}

}  // namespace nis
