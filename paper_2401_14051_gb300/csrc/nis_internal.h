// Internal declarations shared by the library's translation units: device-side helpers
// (voxel lookups, geometry), the constants of the method, and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "nis.h"

namespace nis {

// ---- method constants (Sec. III.B-C) ----------------------------------------------------
constexpr int kLayers = 12;          // 8 diffuse + 4 highlight template layers
constexpr int kDiffuse = 8;
constexpr int kHighlight = 4;
constexpr int kLatA = 5, kLatB = 5, kLatC = 9;
constexpr int kLat = 225;            // lattice points per layer
constexpr int kLatPad = 240;         // BF16 feature row per layer: 480 bytes, 32-byte aligned
constexpr int kLatT = 232;           // FP32 transmittance lattice row (H_T): 928 bytes, 32-byte aligned
constexpr int kPhaseSets = 5;        // all diffuse layers share one set; one per highlight
constexpr int kAlpha = 1024;         // alpha nodes of the phase table
constexpr int kRings = 16;           // cap quadrature: rings (angle midpoints) ...
constexpr int kAzim = 24;            // ... times azimuths
constexpr float kTauMax = 30.0f;     // march stops past this scaled optical depth
constexpr float kHitFraction = 0.05f;
constexpr int kWidth = 200;          // backbone width
constexpr int kCnnCh = 16;
constexpr int kDT = 80;              // CNN output per layer
constexpr int kCfg = 5;              // [g, albedo rgb, alpha]
constexpr int kMaxLevels = 16;

// ---- weight blob layout ------------------------------------------------------------------
// The two networks a weight blob can hold (header word 2): the lattice model (5x5x9
// lattices, per-layer 3D-CNN) and the paper-template model (the paper's own point sets of
// 6..48 and 32..8 points per layer, a volume-level transmission feature from per-level
// weights, no per-layer CNN).
constexpr int kModelLattice = 0, kModelPaper = 1;
constexpr int kPaperPts = 266;        // 194 diffuse + 72 highlight template points
constexpr int kLevelWeights = 11;
// points of the paper model's layer k, and the index of its first point
__host__ __device__ constexpr int paper_count(int k) {
    return k == 0 ? 6 : k == 1 ? 8 : k == 2 ? 12 : k == 3 ? 16 : k == 4 ? 24 : k == 5 ? 32
         : k == 6 ? 48 : k == 7 ? 48 : k == 8 ? 32 : k == 9 ? 16 : k == 10 ? 16 : 8;
}
// First point of layer k (0..12) in template order.  Closed forms rather than recursion:
// device code calls a recursive function through a stack frame at every use.
__host__ __device__ constexpr int paper_first(int k) {
    return k <= 0 ? 0 : k == 1 ? 6 : k == 2 ? 14 : k == 3 ? 26 : k == 4 ? 42 : k == 5 ? 66
         : k == 6 ? 98 : k == 7 ? 146 : k == 8 ? 194 : k == 9 ? 226 : k == 10 ? 242
         : k == 11 ? 258 : 266;
}
// The layer of template point t (0..265): the k with paper_first(k) <= t < paper_first(k + 1).
__host__ __device__ constexpr int paper_layer_of(int t) {
    return (t >= 6) + (t >= 14) + (t >= 26) + (t >= 42) + (t >= 66) + (t >= 98) + (t >= 146) +
           (t >= 194) + (t >= 226) + (t >= 242) + (t >= 258);
}
// tensor-core operand layout of the paper model's features: each layer's columns padded to a
// multiple of 8 (16-byte TMA coordinates), 272 in all, then a zero tail as wide as the
// widest operand box (64 columns: a layer's box reaches past its end into zero weights)
__host__ __device__ constexpr int paper_count_pad(int k) { return (paper_count(k) + 7) & ~7; }
__host__ __device__ constexpr int paper_first_pad(int k) {
    return k <= 0 ? 0 : k == 1 ? 8 : k == 2 ? 16 : k == 3 ? 32 : k == 4 ? 48 : k == 5 ? 72
         : k == 6 ? 104 : k == 7 ? 152 : k == 8 ? 200 : k == 9 ? 232 : k == 10 ? 248
         : k == 11 ? 264 : 272;
}
constexpr bool paper_layout_consistent() {
    if (paper_first(0) != 0 || paper_first_pad(0) != 0) return false;
    for (int k = 0; k < kLayers; ++k) {
        if (paper_first(k + 1) != paper_first(k) + paper_count(k)) return false;
        if (paper_first_pad(k + 1) != paper_first_pad(k) + paper_count_pad(k)) return false;
        for (int t = paper_first(k); t < paper_first(k + 1); ++t)
            if (paper_layer_of(t) != k) return false;
    }
    return true;
}
static_assert(paper_layout_consistent(), "paper template offsets are the counts' prefix sums");
static_assert(paper_first(kLayers) == kPaperPts, "paper template size");
constexpr int kPaperPad = paper_first_pad(kLayers);           // 272
constexpr int kPaperPadTail = kPaperPad + 64;

struct WeightOffsets {                // float offsets into the FP32 weight buffer
    int model = kModelLattice;
    size_t level_w = 0, level_b = 0;  // paper model: transmission weights per level, bias
    size_t cnn_w1[kLayers], cnn_b1[kLayers], cnn_w2[kLayers], cnn_b2[kLayers];
    size_t se_w1[kLayers], se_b1[kLayers], se_w2[kLayers], se_b2[kLayers];
    size_t blk_w1[3][kLayers], blk_b1[3][kLayers], blk_w2[3][kLayers], blk_b2[3][kLayers];
    size_t mrg_w[3], mrg_b[3];
    size_t head_w[3], head_b[3];
    size_t total;
};
void weight_offsets(WeightOffsets *o);   // fills the fixed blob order
void weight_offsets_paper(WeightOffsets *o);   // ... of the paper-template model
int weights_model(::nis_ctx *ctx, nis_weights w);   // kModel* of a weight set, -1 if unknown
inline int feat_dim(int type) { return type == 2 ? kDT : kLat; }

// ---- device helpers ---------------------------------------------------------------------
struct Level {                       // one voxel-centred cubic grid level
    const float *data;
    int n;
};

// Trilinear lookup with clamp-to-edge indices (used by the march, inside the cube).
__device__ __forceinline__ float sample_clamped(const float *__restrict__ g, int n, float x,
                                                float y, float z) {
    const float hi = (float)(n - 1);
    float gx = fminf(fmaxf(x * n - 0.5f, 0.0f), hi);
    float gy = fminf(fmaxf(y * n - 0.5f, 0.0f), hi);
    float gz = fminf(fmaxf(z * n - 0.5f, 0.0f), hi);
    const int top = n > 1 ? n - 2 : 0;
    int ix = min((int)floorf(gx), top), iy = min((int)floorf(gy), top),
        iz = min((int)floorf(gz), top);
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

// Trilinear lookup where voxels outside the grid read `border` (template gathers, hits).
// occ (optional): the grid's cell occupancy (cell (i, j, k) flagged when one of its eight
// corners is nonzero); an interior cell that is not flagged returns 0 after one byte load,
// the value its eight zero corners interpolate to.
__device__ __forceinline__ float sample_border(const float *__restrict__ g, int n, float x,
                                               float y, float z, float border,
                                               const unsigned char *__restrict__ occ = nullptr) {
    float gx = x * n - 0.5f, gy = y * n - 0.5f, gz = z * n - 0.5f;
    float flx = floorf(gx), fly = floorf(gy), flz = floorf(gz);
    float fx = gx - flx, fy = gy - fly, fz = gz - flz;
    // coordinates far outside: clamp the integer base so index math cannot overflow
    int ix = (int)fminf(fmaxf(flx, -2.0f), (float)n + 1.0f);
    int iy = (int)fminf(fmaxf(fly, -2.0f), (float)n + 1.0f);
    int iz = (int)fminf(fmaxf(flz, -2.0f), (float)n + 1.0f);
    // interior cells only (0 <= index <= n - 2; a 1^3 grid has none)
    if (occ && n >= 2 && (unsigned)ix <= (unsigned)(n - 2) && (unsigned)iy <= (unsigned)(n - 2) &&
        (unsigned)iz <= (unsigned)(n - 2) && !__ldg(occ + ((size_t)iz * n + iy) * n + ix))
        return 0.f;
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int cx = ix + (c & 1), cy = iy + ((c >> 1) & 1), cz = iz + (c >> 2);
        bool in = (unsigned)cx < (unsigned)n && (unsigned)cy < (unsigned)n &&
                  (unsigned)cz < (unsigned)n;
        v[c] = in ? __ldg(g + ((size_t)cz * n + cy) * n + cx) : border;
    }
    float c00 = v[0] + fx * (v[1] - v[0]);
    float c01 = v[2] + fx * (v[3] - v[2]);
    float c10 = v[4] + fx * (v[5] - v[4]);
    float c11 = v[6] + fx * (v[7] - v[6]);
    float c0 = c00 + fy * (c01 - c00);
    float c1 = c10 + fy * (c11 - c10);
    return c0 + fz * (c1 - c0);
}

// (a + f (b - a)) for the two lanes of a pair at once (packed FP32: sub.rn / fma.rn .f32x2,
// the same roundings as the scalar form).
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float f) {
    float2 r;
    asm("{\n\t.reg .b64 A, B, F, D;\n\t"
        "mov.b64 A, {%2, %3};\n\tmov.b64 B, {%4, %5};\n\tmov.b64 F, {%6, %6};\n\t"
        "sub.rn.f32x2 D, B, A;\n\tfma.rn.f32x2 D, F, D, A;\n\tmov.b64 {%0, %1}, D;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(f));
    return r;
}

// Distance from (x, y, z) along unit u to the boundary of the unit cube (>= 0).
__device__ __forceinline__ float exit_distance(float x, float y, float z, float ux, float uy,
                                               float uz) {
    float t = 3.0e38f;
    if (ux > 0.f) t = fminf(t, (1.f - x) / ux); else if (ux < 0.f) t = fminf(t, -x / ux);
    if (uy > 0.f) t = fminf(t, (1.f - y) / uy); else if (uy < 0.f) t = fminf(t, -y / uy);
    if (uz > 0.f) t = fminf(t, (1.f - z) / uz); else if (uz < 0.f) t = fminf(t, -z / uz);
    return fmaxf(t, 0.f);
}

// ---- device-side error word bits (read back by nis_sync) ----------------------------------
constexpr unsigned kErrBadDensity = 1u;
constexpr unsigned kErrBadIndex = 2u;
constexpr unsigned kErrTimeout = 4u;     // a bounded wait in a tensor-core kernel gave up

// ---- launchers (all enqueue on `s`) ----------------------------------------------------------
void note_launch();                  // counts every kernel launch of the library
// volume
void launch_convert_density(const void *src, int dtype, float scale, size_t count,
                            float *dst, unsigned *err, float *sigma_max, cudaStream_t s);
void launch_downsample(const float *src, int n, float *dst, int m, cudaStream_t s);
// one PairView level of size n from the density and transmittance levels
void launch_pack_pairs(const float *rho, const float *T, int n, float4 *out, cudaStream_t s);
// float4 count of a PairView level of size n
inline size_t pair_level_float4(int n) { return 2 * (size_t)n * (size_t)(n + 1) * (size_t)(n + 1); }
// occupancy of the trilinear cells of an n^3 level, one byte per base voxel (i, j, k):
// occ = 0 guarantees that the cell's corners (i..min(i+1, n-1), likewise j, k) are all zero
void launch_occupancy(const float *level, int n, unsigned char *occ, cudaStream_t s);
// out[c][r] = in[r][c] for an R x C row-major float matrix (R / 32 * C / 32 < 2^31 tiles)
void launch_transpose(const float *in, size_t R, size_t C, float *out, cudaStream_t s);
// transmittance of one level
void launch_march(const float *level, const unsigned char *occ, int n, int m, float ux,
                  float uy, float uz, float lam, float *out, cudaStream_t s);
// shear-warp transmittance, an O(N^3) approximation of the march (all levels, one light):
// parallel rays toward the light cross the slices normal to the dominant axis a of u at
// perpendicular positions rho - k r (rho integer, r = u_perp / |u_a|, k the slice count
// from the light side); each ray keeps a running optical depth and in-cube length, and
// each voxel centre takes the mean density of its four nearest rays times its own exit
// distance
struct ShearWarpLevel {
    const float *rho;             // density level, [z][y][x]
    const unsigned char *occ;     // its cell occupancy
    float *T;                     // transmittance out, [z][y][x]
    float2 *ray;                  // ray (depth, length) [slice of the chunk][q][p]
    int n, P, Q, lo_p, lo_q;      // P x Q rays, ray (lo_p + ip, lo_q + iq) at index iq P + ip
    float r_p, r_q, ts, scale;    // shifts per slice, step length 1/(n |u_a|), lambda^(m+1)
    float inv_rp, inv_rq;         // 1 / r (0 where r = 0)
};
struct ShearWarpArgs {
    int levels, sgn;              // sgn = sign(u_a): slice a-index of step k is n-1-k or k
    int slices;                   // steps per launch pair (sw_slices of the finest size)
    int ax_a, ax_p, ax_q;         // coordinate (0 x, 1 y, 2 z) of the axes a, p < q in the
                                  // arrays the kernel reads and writes
    float ux, uy, uz;             // unit direction toward the light, in those coordinates
    float iux, iuy, iuz;          // 1 / |u| per coordinate (0 where u = 0)
    ShearWarpLevel lv[kMaxLevels];
};
// Steps the sweep takes per pair of launches for a finest level of n voxels a side: the
// ray states of every step of a chunk are kept (2 n + 3 rays a side at most), up to 256 MB
// of them at the finest level, 2 to 32 steps, and a chunk's voxel indices stay below 2^24
// (the kernels split indices through a float reciprocal).
inline int sw_slices(int n) {
    const double side = 2.0 * n + 3.0;
    int s = (int)((256.0 * 1024 * 1024) / (8.0 * side * side));
    s = s < 2 ? 2 : (s > 32 ? 32 : s);
    const long long cap = ((1LL << 24) - 1) / ((long long)n * n);
    return (int)(cap < 1 ? 1 : (cap < s ? cap : s));
}
// fills the geometry of `a` (axes, shifts, ray ranges, slices; not the pointers) for levels
// of the given sizes and returns the ray-buffer floats each level needs (2 per ray and step
// of a chunk) in ray_floats
void shear_warp_setup(ShearWarpArgs &a, const int *sizes, int levels, float ux, float uy,
                      float uz, float lam, size_t *ray_floats);
// enqueues the sweep: per chunk of a.slices steps one launch that advances the rays through
// them and one that fills those slices' voxels (the ray pointers of `a` set by the caller)
void launch_shear_warp(const ShearWarpArgs &a, cudaStream_t s);
// phase function of the phase features: one HG lobe, or a mixture of up to 3 (Eq. 6)
struct PhaseSpec {
    int n;
    float g[3], w[3];
};
// phase table [kAlpha][kPhaseSets][kLat]
void launch_phase_table(const PhaseSpec &ph, float *table, cudaStream_t s);

struct PyramidView {                 // device pointers of all levels of a pyramid
    const float *lv[kMaxLevels];
    int n[kMaxLevels];
    int levels;
};

// Density and transmittance of a (volume, light) pair side by side for the gathers: entry
// (z, j, i) of a level of size n, j, i = 0..n, holds {rho, T} at the four (y, x) of y = j - 1,
// j and x = i - 1, i (each outside the volume as its border value, rho 0 and T 1), ordered
// (y0 x0, y0 x1, y1 x0, y1 x1): 32 bytes, so that one full-sector load brings a trilinear
// cell's four corners of one z slice for both fields.  [z][n + 1][n + 1] entries per level,
// each two float4.
struct PairView {
    const float4 *lv[kMaxLevels];
    int n[kMaxLevels];
    int levels;
};

// Per-request inputs of a mixed batch (continuous batching): point p uses
// descs[req_of_point[p]] instead of the single-request fields of GatherArgs.
struct ReqDesc {
    PyramidView rho, T;
    PairView rt;                     // what the gathers read
    const float *table;
    float l[3];
    float g;
    float albedo[3];
    float dec[3];                    // I * albedo^4 (decode scale)
};

struct GatherArgs {
    const ReqDesc *descs;            // mixed batch (may be null)
    const int *req_of_point;
    PyramidView rho, T;
    PairView rt;                     // what the gathers read
    const float *table;              // phase table of the material's g
    const float *points, *omega;     // [n][3]
    int count;
    float lx, ly, lz;                // unit light propagation direction
    float g;
    float albedo[3];
    const float *se;                 // FP32 weights base; SE offsets below
    size_t se_w1[kLayers], se_b1[kLayers], se_w2[kLayers], se_b2[kLayers];
    float *H_rho, *H_T, *H_f;        // H_T [count][12][kLatT]; H_rho, H_f [count][12][225], may be
                                     // null when Hb_* are set
    __nv_bfloat16 *Hb_rho, *Hb_f;    // optional BF16 copies [count][12][kLatPad] (pad zeroed)
    uint8_t *H8_rho, *H8_f;          // optional e4m3 copies [count][12][kLatPad8], each layer's
    float *f8_scale;                 // row scaled by f8_scale[count][12][2] = max / 448
    int split; size_t part;          // BF16 copies as 3 split parts, part stride in elements
    float *v;                        // [count][12][8] (may be null)
    float *w_se;                     // [count][12][3]
    float *cfg;                      // [count][5]
    // fused backbone (BF16): Hb_* rows of kFuseLatLd per layer with the configuration
    // operand in columns 225..237, and the same operand of type T in XT_cfg (rows of
    // kFuseXtLd per layer, columns 80..92) ahead of the CNN's outputs
    int fused;
    __nv_bfloat16 *XT_cfg;
    // e4m3 mode of the fused network: the density and phase rows as e4m3 [count][12][kF8LatLd]
    // scaled by 448 / sigma_max and 448 / the phase set's table maximum, their configuration
    // operands [count][12][kF8CfgLd] BF16 and the FC-1 row factors [count][12][3]
    uint8_t *F8_rho, *F8_f;
    __nv_bfloat16 *F8_cfg;
    float *fc1_scale;
    const float *f8_sigma;                   // device: sigma_max of the volume
    const float *f8_tabmax;                  // device: [5] maxima of the phase table's sets
    float f8_sw[kLayers][2];                 // weight scales of FC-1 (rho, f)
};
void launch_gather(const GatherArgs &a, cudaStream_t s);
// out[set] = the largest entry of the phase table's point set (kPhaseSets of them)
void launch_table_set_max(const float *table, float *out, cudaStream_t s);

// ---- paper-template model (k_gather_paper.cu) -----------------------------------------------
// Unit-radius point sets of the 12 layers (light-frame coordinates; Fibonacci sphere,
// sunflower disc), their mean nearest-neighbour distances D[12] (Eq. 3) and every point's
// offset from the shading point over its layer's spacing, q[266][3] (the phase offsets).
void paper_template(double unit[kPaperPts][3], double D[kLayers], float q[kPaperPts][3]);
struct PaperGatherArgs {
    PyramidView rho, T;              // density and transmittance levels (plain float grids)
    const float *table;              // [kAlpha][266] phase features of the material
    const float *points, *omega;     // [n][3]
    int count;
    float lx, ly, lz;                // unit light propagation direction
    float g;
    float albedo[3];
    float D[kLayers];                // unit-set spacings
    float unit[kPaperPts][3];        // unit-radius template points (from paper_template)
    const float *level_w, *level_b;  // device: per-level transmission weights, bias
    const float *se;                 // FP32 weights base; SE offsets below
    size_t se_w1[kLayers], se_b1[kLayers], se_w2[kLayers], se_b2[kLayers];
    float *H_rho, *H_f, *H_T;        // [count][266] FP32 (may be null)
    // tensor-core operands (may be null): BF16 [parts][count][row] in the padded layout, the
    // parts of the three-way split `part` elements apart; rows of ld_rf (rho, f), ld_t (T)
    __nv_bfloat16 *Hb_rho, *Hb_f, *Hb_T;
    int parts; size_t part_rf, part_t; int ld_rf, ld_t;
    float *v;                        // [count][12][8] (may be null)
    float *w_se;                     // [count][12][3]
    float *cfg;                      // [count][5]
};
void launch_gather_paper(const PaperGatherArgs &a, cudaStream_t s);
// phase features of arbitrary template offsets q (in spacings, light frame) over the alpha
// nodes: table[a][t], t < n_pts <= kPaperPts
void launch_phase_points(const PhaseSpec &ph, const float (*q)[3], int n_pts, float *table,
                         cudaStream_t s);

// FP32 CNN (FP32 FFMA): outputs X_T (FP32, optional) and X_T_bf (BF16, optional; three
// split parts `split_part` elements apart when split_part != 0), [count][12][80].
void launch_cnn_f32(const float *H_T, int count, const float *wbase, const WeightOffsets &o,
                    float *X_T, __nv_bfloat16 *X_T_bf, cudaStream_t s, size_t split_part = 0,
                    const CUtensorMap *map_ht = nullptr, unsigned *err = nullptr);
// The same CNN with BF16 operands on the tensor cores (FP32 accumulation): outputs X_T
// (FP32, optional), X_T_bf (BF16, optional), X_T_f8 (e4m3, optional), [count][12][80].
void launch_cnn_tc(const CUtensorMap &map_ht, int count, const float *wbase, const WeightOffsets &o,
                   float *X_T, __nv_bfloat16 *X_T_bf, uint8_t *X_T_f8, unsigned *err, int num_sms,
                   cudaStream_t s, int xt_ld = kDT);   // xt_ld: X_T_bf row per layer
// FP8 weights: scale[n] = max_k |W[n][k]| / 448 (1 for empty rows), dst = e4m3(W / scale)
void launch_pack_fp8(const float *src, int N, int K, int ld_src, uint8_t *dst, float *scale,
                     int Np, int Kp, cudaStream_t s);
bool make_tmap_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                  uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);
// dst[n][k] = bf16(src[n * ld_src + k]) for n < N, k < K, zero elsewhere in [Np][Kp]
void launch_pack_bf16(const float *src, int N, int K, int ld_src, __nv_bfloat16 *dst, int Np,
                      int Kp, cudaStream_t s, int split_part = -1);
// Part `part` (0, 1, 2) of the three-way BF16 split x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)); part -1 is plain bf16(x).
__host__ __device__ inline float split_residual(float x, int part) {
    float r = x;
    for (int i = 0; i < part; ++i) r = r - __bfloat162float(__float2bfloat16_rn(r));
    return r;
}

// One dense layer out[r][j] = epilogue(sum_k A[r][k] W[j][k] + b[j]) over rows r < count.
struct FcArgs {
    int mode;                        // kFcFeat, kFcSum, kFcCat
    int count, K, N;
    // kFcFeat: A[r] = [ w_se[r*36 + layer*3 + type] * X[r*ldx + 0..d), cfg[r*5 + 0..5) ]
    const float *X; int ldx; int d; const float *w_se; int layer, type; const float *cfg;
    // kFcSum: A[r] = a0[r] + a1[r] (a0 may be null);  kFcCat: A[r] = [a0[r], a1[r], a2[r]]
    const float *a0, *a1, *a2; int seg;
    const float *W, *b;
    int relu;                        // apply ReLU to acc + b
    const float *resid;              // if set, out = act + resid[r][j]
    float *out; int ldo;
    // decode epilogue (last layer): rgb = intensity * albedo^4 * expm1(acc + b)
    int decode; float dec_scale[3]; float *y_out;
    const float *dec_rows;           // optional per-row decode scales [count][3]
};
constexpr int kFcFeat = 0, kFcSum = 1, kFcCat = 2;
void launch_fc_f32(const FcArgs &a, cudaStream_t s);

struct CameraArgs {
    int type, width, height;
    float eye[3], fwd[3], right[3], up[3];
    float tan_half, aspect, half_h;
};
// occ0: level 0's cell occupancy when it matches rho0 (skips empty cells), else null
void launch_find_hits(const float *rho0, const unsigned char *occ0, int n, const float *sigma_max,
                      const CameraArgs &c, int *hit_flag, float *points, float *omega,
                      int *pix_index, int *counter, cudaStream_t s);
// Hits in pixel order: per-pixel flag/point/direction, hit counts per 256-pixel block and
// their exclusive scan (offsets: nb + 1 ints, nb = ceil(pixels / 256); *total = the hits).
void launch_find_hits_ordered(const float *rho0, const unsigned char *occ0, int n,
                              const float *sigma_max, const CameraArgs &c, int *flag,
                              float *pts_px, float *om_px, int *block_count, int *offsets,
                              int *total, cudaStream_t s);
// Hits first .. first + count - 1 of that order, compacted into pts/om/pix.
void launch_hits_range(const int *flag, const float *pts_px, const float *om_px,
                       const int *offsets, int pixels, long long first, int count, float *pts,
                       float *om, int *pix, cudaStream_t s);
void launch_scatter_rgb(const float *rgb, const int *pix_index, int count, float *image,
                        int n_pixels, cudaStream_t s, bool accumulate = false);

// ---- tensor-core dense layer (k_mlp_tc.cu) ------------------------------------------------
constexpr int kEpiPlain = 0, kEpiFc1 = 1, kEpiFc2 = 2, kEpiRelu = 3, kEpiDecode = 4;
struct TcGemmArgs {
    int M, N, K;                      // rows, output columns, reduction length
    int n_mma;                        // N rounded up to a multiple of 16 (<= 208)
    int k_tiles;                      // ceil(K / 64)
    int a_col0;                       // first column of A inside its tensor map
    int epi;
    unsigned *err;                    // context error word (kErrTimeout)
    float *out_f32;                   // kEpiPlain [M][ldo], kEpiDecode rgb [M][3]
    __nv_bfloat16 *out_bf;            // kEpiFc2, kEpiRelu
    __nv_bfloat16 *out_e, *out_s;     // kEpiFc1: e and h_prev + e
    int ldo;
    const float *bias;                // [N]
    const float *row_scale; int row_scale_ld;   // kEpiFc1: SE weight per row
    const float *cfg;                 // kEpiFc1: [M][5] configuration vector (alpha = [4])
    const float *w_cfg; int w_cfg_ld; // kEpiFc1: weight columns of c, row n at w_cfg + n*ld
    float mat_cfg[4];                 // kEpiFc1: g, albedo rgb (the same for every row)
    const __nv_bfloat16 *h_prev; int ld_h;      // kEpiFc1 running state (may be null)
    const __nv_bfloat16 *resid; int ld_resid;   // kEpiFc2: e
    float dec_scale[3];               // kEpiDecode: I * albedo^4
    float *y_out;                     // kEpiDecode: network output before decode (may be null)
    const float *dec_rows;            // kEpiDecode: optional per-row scales [M][3]
    int cfg_per_row;                  // kEpiFc1: use every row's g and albedo from cfg (mixed
                                      // batches) instead of the folded mat_cfg
    // FP32-accurate mode: operands split into three BF16 parts, six products per K slice
    int n_pass;                       // 1 (plain BF16) or 6 (split)
    int a_part_rows, b_part_rows;     // row offset of part i of A / B inside its tensor map
    int out_split; size_t out_part;   // BF16 outputs (out_bf, out_s) as 3 parts, part stride
    float *out_e_f32;                 // kEpiFc1: e in FP32 (else BF16 out_e)
    float *out_h_f32;                 // kEpiFc2: h in FP32 (else out_bf)
    const float *pre_f32; int ld_pre; // kEpiFc1 h_prev / kEpiFc2 e in FP32 (else BF16)
    // FP8 mode: e4m3 operands (kind::f8f6f4, 128 elements per 128-byte K tile)
    int fp8;
    const float *col_scale;           // per-output-channel weight scales [N]
    const float *row_scale2; int row_scale2_ld;  // kEpiFc1: per-row feature scales
    uint8_t *out_f8, *out_s8;         // e4m3 outputs (FC-2 chain end / ReLU layers; FC-1 s)
    // Outputs written through shared memory by TMA stores (kernel arguments map_o1, map_o2)
    // instead of the pointers above: o1 = the layer's output (FC-1: e), o2 = FC-1's s.
    // Kind kOutDirect uses the pointers; parts = 3 writes the three BF16 parts of a split.
    int o1_kind, o1_parts, o2_kind, o2_parts;
    // the residual / running state read through TMA (kernel argument map_pre, [1][rows][N]
    // with 32 x 32 boxes) instead of one row per lane: 1 = FP32 (pre_f32, the split),
    // 2 = BF16 (h_prev / resid); 0 = per-lane loads
    int pre_tma;
};
constexpr int kOutDirect = 0, kOutF32 = 1, kOutBf16 = 2;
constexpr int kLatPad8 = 240;        // FP8 feature row per layer, padded to 16 bytes
constexpr int kWidth8 = 208;         // FP8 activation rows padded to 16 bytes
constexpr int kHead8 = 608;
void launch_fill_segments(const int *seg_start, const int *seg_desc, int nseg, int count,
                          int *req_of_point, float *dec_rows, const ReqDesc *descs,
                          cudaStream_t s);
void launch_tc_gemm(const TcGemmArgs &a, const CUtensorMap &map_a, const CUtensorMap &map_b,
                    int num_sms, cudaStream_t s, const CUtensorMap *map_o1 = nullptr,
                    const CUtensorMap *map_o2 = nullptr, const CUtensorMap *map_pre = nullptr);
// K width of a BF16 tensor-core box: 64 elements (128-byte swizzle) for one part,
// kSplitSlabK for the three parts of the FP32 split, whose stage holds every part of a slab
// at once: 32 (64-byte swizzle, two 63 KB stages); 16 (32-byte swizzle, four 31.5 KB
// stages) is supported and measured 18% slower (1080p frame: 18.5 against 15.7 ms).
constexpr int kSplitSlabK = 32;
inline uint32_t tc_box_k(int parts) { return parts > 1 ? kSplitSlabK : 64; }
// 2-D BF16 tensor map, inner dimension contiguous, box = box_inner x box_outer; box_inner 64,
// 32 or 16 gives 128-, 64- or 32-byte swizzled rows (other widths are refused).
// The tensor-core CNN's input map over H_T [count][12][kLatT] FP32: boxes of one layer's rows
// of 16 consecutive points (3-D: columns, layers, points; no swizzle).
bool make_tmap_ht(CUtensorMap *map, const float *H_T, uint64_t points);
bool make_tmap_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                    uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);
// 3-D output map of the tensor-core epilogue: [parts][rows][cols] FP32 (f32 = true, 128-byte
// swizzle) or BF16 (64-byte swizzle), box 32 columns x 32 rows x all parts.
bool make_tmap_out(CUtensorMap *map, const void *base, bool f32, uint64_t cols, uint64_t rows,
                   uint32_t parts, uint64_t row_bytes, uint64_t part_bytes);

// ---- fused backbone (k_mlp_fused.cu) --------------------------------------------------------
// The whole network after the features (Sec. III.C.2, Fig. 6: per type and template the
// chains of FC-1 / FC-2 blocks, the merge of each type, the head, the decode of Eq. 21) in one
// persistent tcgen05 kernel over 128-point tiles, BF16 operands and FP32 accumulation.  A
// program of ops runs per tile; the running state e / h stays on chip in FP32, the chain
// ends and merge outputs make one trip through global memory (BF16) for the next op's
// operand.  Biases ride in the operands: FC-1's bias and configuration part (W_c c + b) come
// from 13 columns after each layer's features holding c / w_se and 1 / w_se per (point,
// layer, type), so that e = w_se * ReLU(acc); the other layers read two columns of ones
// against the bias's two BF16 parts.
constexpr int kFuseFc1 = 0, kFuseFc2 = 1, kFuseMerge = 2, kFuseHead1 = 3, kFuseHead2 = 4, kFuseHead3 = 5;
// operand sources read by TMA (the features rho, f, T; the chain ends; the merge outputs) and
// the on-chip s buffer (FC-2 and the head's second and third layers)
constexpr int kSrcRho = 0, kSrcF = 1, kSrcT = 2, kSrcMrg = 3, kSrcHead = 4, kSrcS = 5;
constexpr int kFuseSrcs = 5;
constexpr int kFuseLatLd = 240;              // BF16 rho / f row per layer: 225 + 13 + 2 zeros
constexpr int kFuseXtLd = 96;                // BF16 T row per layer: 80 + 13 + 3 zeros
constexpr int kFuseCfgCols = 13;             // [c/w hi (5), c/w lo (5), 1/w hi, 1/w hi, 1/w lo]
constexpr int kFuseMrgLd = 416;              // chain-end row per type: 2 x 200, then [1, 1, 0...]
constexpr int kFuseHeadLd = 608;             // merge outputs: 3 x 200, then [1, 1, 0...]
constexpr int kFuseMaxOps = 96;
struct FusedOp {
    uint8_t kind, src, type, layer;
    uint8_t chain, flags;                    // flags: 1 first layer of its chain, 2 last, 4 on
                                             // accumulator Y, 8 merge operand complete,
                                             // 16 head operand complete, 32 e4m3 features
                                             // (kFuseF8Flag)
    uint16_t a_col0, n_mma, k;               // operand column; 208 or 16 outputs; K (x16)
    uint32_t b_off;                          // byte offset of the op's weight blocks
};
static_assert(sizeof(FusedOp) == 16, "FusedOp layout");
// Per op, how its weight blocks are made from the FP32 weights (host -> pack kernel).
struct FusedPackOp {
    const float *W; int ld;                  // weight rows [n_out][ld]
    int n_out, k_main;                       // outputs; input columns of the main operand
    const float *bias;                       // [n_out]
    int bias_main;                           // bias in columns k_main, k_main + 1
    int cfg;                                 // FC-1: W_c (the ld - k_main columns after the
                                             // features) and the bias in columns k_main..+12
    int k, n_mma, s_tail;                    // K; outputs; last block 16 wide (s buffer tail)
    uint32_t b_off;
    int fp8;                                 // e4m3 feature blocks (see kFuseF8Flag)
    float f8_inv;                            // 1 / the layer's weight scale S_w
};
struct FusedMaps {                           // per TMA source: 64-column boxes of 128 rows,
    CUtensorMap m64[kFuseSrcs];              // 128-byte swizzle (with e4m3 features: 128
                                             // columns of rho and f)
    CUtensorMap cfg8;                        // e4m3 mode: the configuration operands [rows][12
                                             // layers x 2 types x 16] BF16, 16-column boxes
};
// e4m3 mode of the fused network (the FP8 precision): FC-1 of the density and phase chains
// reads the layer's features as e4m3 (x / s, s the layer's activation scale) in two
// 128-column blocks against e4m3 weights (W / S_w, S_w the layer's weight scale), then a
// 16-column BF16 block of configuration columns c / u and 1 / u (u = w_se s S_w) against
// [W_c; W_c; b_hi; b_lo; b_hi]; the accumulator times u is W1 [w_se x; c] + b1, and the
// epilogue's row factor is u (FusedArgs::fc1_scale) instead of w_se.
constexpr int kFuseF8Flag = 32;
constexpr int kF8LatLd = 256;                  // e4m3 feature row per layer (225 + zeros)
constexpr int kF8CfgLd = 32;                   // configuration columns per layer: 2 types x 16
struct FusedArgs {
    int M, n_ops;
    const FusedOp *ops;                      // device, n_ops <= kFuseMaxOps
    const uint8_t *wpack;                    // weight blocks, pre-swizzled
    const float *w_se;                       // [M][12][3]
    __nv_bfloat16 *mrg;                      // [rows][3][kFuseMrgLd]
    __nv_bfloat16 *head;                     // [rows][kFuseHeadLd]
    float *rgb;                              // [M][3]
    float *y_out;                            // optional [M][3] network output before decode
    const float *dec_rows;                   // optional per-row decode scales [M][3]
    float dec_scale[3];                      // I * albedo^4
    unsigned *err;
    const float *fc1_scale;                  // e4m3 mode: FC-1 row factors [M][12][3], else null
};
// The op program and the pack list of a weight set (lattice model: feature columns
// k * kFuseLatLd for rho and f, k * kFuseXtLd for T).
// With sw (e4m3 mode), FC-1 of the density and phase chains takes e4m3 feature blocks with
// the weight scales sw[k][t] (host values, computed by the caller).
void fused_program(const WeightOffsets &o, const float *W, FusedOp *ops, FusedPackOp *pack,
                   int *n_ops, size_t *bytes, const float (*sw)[2] = nullptr);
void launch_fused_pack(const FusedPackOp *pack_dev, int n_ops, uint8_t *dst, cudaStream_t s);
void launch_mlp_fused(const FusedArgs &a, const FusedMaps &maps, int num_sms, cudaStream_t s);
// SE weights are floored at kSeFloor where the configuration operand divides by them.
constexpr float kSeFloor = 1e-20f;

// Device pointers of a resolved (volume, light, weights, phase table) set, for entry points
// that must not build or allocate anything.  Fails with NIS_ERR_NOT_READY if the pyramid or
// the phase table of g is missing.
struct ResolvedInputs {
    PyramidView rho, T;
    PairView rt;
    const float *table;
    const float *W;
    WeightOffsets off;
    float dir[3];
    int device;
};
nis_status resolve_built_inputs(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                                const nis_material *m, ResolvedInputs *out);
nis_status record_error(nis_ctx *ctx, nis_status s, const char *msg);
// Why a material cannot be shaded (its phase function, albedo or intensity), or nullptr.
const char *material_problem(const nis_material *m);
int ctx_device(const nis_ctx *ctx);
// First hits of a camera, compacted: points, omegas and pixel indices of the hits, and their
// number in *d_count (device).  Buffers hold width * height entries.
nis_status hits_compact(nis_ctx *ctx, nis_volume vol, const nis_camera *cam, float *pts,
                        float *om, int *pix, int *d_count, cudaStream_t s);

}  // namespace nis
