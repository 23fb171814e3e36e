// The C ABI (include/nis.h): context, handle registries, HBM budget accounting, weight-blob
// parsing and the stream-ordered orchestration of the kernels of the inference path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "nis_internal.h"

using namespace nis;

namespace {

std::string g_create_error;

struct Volume {
    int n = 0, levels = 0;
    int sizes[kMaxLevels] = {};
    size_t off[kMaxLevels] = {};      // float offsets of each level in `data`
    size_t total = 0;                 // floats in all levels
    float *data = nullptr;
    float *sigma_max = nullptr;       // device scalar (max of level 0)
    unsigned char *occ = nullptr;     // brick occupancy of every level (march skipping)
    size_t occ_off[kMaxLevels] = {};
    void *staging = nullptr;          // pageable-host updates (nis_update_volume)
    size_t staging_bytes = 0;
    bool pyramid = false;
    uint64_t version = 0;             // counts pyramid builds (lights pair with one of them)
    // x-major copy of the pyramid, [x][z][y] per level, and its occupancy: the shear-warp
    // sweep of a light along x reads its slices contiguously (built on first use, from
    // pyramid build `xmaj_version`)
    float *xmaj = nullptr;
    unsigned char *xmaj_occ = nullptr;
    uint64_t xmaj_version = 0;
};

struct Light {
    nis_handle vol = 0;
    float dir[3] = {0, 0, 0};         // unit propagation direction
    float lambda = 0.6f;
    int method = NIS_TRANSMITTANCE_MARCH;
    float *data = nullptr;            // same level layout as the volume
    // density and transmittance side by side for the gathers (PairView layout), packed
    // from the volume's pyramid of build `pair_version` (0: not packed)
    float4 *pairs = nullptr;
    size_t pair_off[kMaxLevels] = {};
    uint64_t pair_version = 0;
};

struct Weights {
    int precision = NIS_PREC_F32;
    float *f32 = nullptr;             // all tensors in blob order
    WeightOffsets off;
    // BF16 dense layers (precision BF16): zero-padded [n_mma][Kp] matrices and tensor maps
    __nv_bfloat16 *bf = nullptr;
    CUtensorMap map_fc1[3][kLayers], map_fc2[3][kLayers], map_mrg[3], map_head[3];
    // FP8 dense layers: e4m3 [n_mma][Kp] matrices and per-output-channel scales
    uint8_t *f8 = nullptr;
    float *f8_scales = nullptr;
    const float *sc_fc1[3][kLayers] = {}, *sc_fc2[3][kLayers] = {}, *sc_mrg[3] = {}, *sc_head[3] = {};
    // BF16 and FP8: the fused backbone's op program and pre-swizzled weight slabs (FP8: its
    // e4m3 mode, with the FC-1 weight scales of the density and phase chains)
    uint8_t *fused_w = nullptr;
    FusedOp *fused_ops = nullptr;
    FusedPackOp *fused_pack = nullptr;
    int fused_n_ops = 0;
    float f8_sw[kLayers][2] = {};
};

struct WorkspaceF8 {                  // scratch of the FP8 path, grow-only
    int cap = 0;
    uint8_t *H8_rho = nullptr, *H8_f = nullptr, *XT8 = nullptr, *S8 = nullptr,
            *mrg8[3] = {nullptr, nullptr, nullptr}, *head8 = nullptr, *Z1 = nullptr, *Z2 = nullptr;
    __nv_bfloat16 *E = nullptr, *H = nullptr;
    float *H_T = nullptr, *w_se = nullptr, *cfg = nullptr, *v = nullptr, *fscale = nullptr;
    CUtensorMap map_rho, map_f, map_xt, map_s, map_mrg[3], map_head, map_z1, map_z2;
    CUtensorMap map_ht;               // the tensor-core CNN's input boxes over H_T
};

struct WorkspaceBf {                  // scratch of the tensor-core paths, grow-only
    int cap = 0;
    int parts = 1;                    // 1: BF16; 3: three-way split (FP32-accurate)
    float *E32 = nullptr, *H32 = nullptr;   // split mode: e and the running state in FP32
    __nv_bfloat16 *Hb_rho = nullptr, *Hb_f = nullptr, *XTb = nullptr, *E = nullptr, *S = nullptr,
                  *H = nullptr, *mrg_in[3] = {nullptr, nullptr, nullptr}, *head_in = nullptr,
                  *Z1 = nullptr, *Z2 = nullptr;
    float *H_T = nullptr, *w_se = nullptr, *cfg = nullptr, *v = nullptr;
    CUtensorMap map_rho, map_f, map_xt, map_s, map_mrg[3], map_head, map_z1, map_z2;
    CUtensorMap map_ht;               // the tensor-core CNN's input boxes over H_T
    // epilogue output maps (TMA stores): e, h (FP32 with the split), s, the chain ends
    // (per type and chain), the merges (per type) and the head activations
    CUtensorMap out_e, out_h, out_s, out_mrg[3][2], out_head[3], out_z1, out_z2;
    // BF16 fused backbone: chain ends and merge outputs, and the operand maps of its sources
    // (the features in Hb_rho, Hb_f and XTb with rows of kFuseLatLd / kFuseXtLd per layer)
    __nv_bfloat16 *mrg_f = nullptr, *head_f = nullptr;
    FusedMaps fmaps{};
    // the fused backbone's e4m3 mode (FP8): e4m3 density and phase rows, their configuration
    // operands, the FC-1 row factors, the phase table's set maxima, and the operand maps
    // (rho, f and the configuration operands of their own; the rest shared with fmaps)
    int f8_cap = 0;
    uint8_t *F8_rho = nullptr, *F8_f = nullptr;
    __nv_bfloat16 *F8_cfg = nullptr;
    float *fc1_scale = nullptr, *tabmax = nullptr;
    FusedMaps f8maps{};
};

struct Workspace {                    // scratch of nis_shade_points, grow-only
    int cap = 0;
    float *H_rho = nullptr, *H_T = nullptr, *H_f = nullptr, *v = nullptr, *w_se = nullptr,
          *cfg = nullptr, *X_T = nullptr;
    float *act = nullptr;             // activation buffers, kActBufs x cap x kWidth
    int hit_cap = 0;                  // pixels
    float *hit_pts = nullptr, *hit_omega = nullptr, *hit_rgb = nullptr;
    int *hit_pix = nullptr, *hit_count = nullptr;
    int *host_count = nullptr;        // pinned
    int px_cap = 0;                   // pixels: the frame split's per-pixel hit list
    int *px_flag = nullptr, *px_blk = nullptr, *px_off = nullptr;
    float *px_pts = nullptr, *px_om = nullptr;
};
constexpr int kActBufs = 15;          // e, h0, h1, 6 chain ends, 3 merges, z1, z2, spare
// Shading points per pipeline pass, at most.  Each dense layer is one launch per pass, and
// a launch costs ~17 us beyond its tiles (prologue, pipeline fill, the last tile's epilogue),
// so passes are as large as the workspace allows: the 1080p frame (215,053 points) is one
// pass.  The tensor-core workspace is ~66 KB per point with the FP32 split (17 GB here).
constexpr int kChunk = 262144;
// Points per pass for n points: the passes share n equally (rounded up to whole 128-row
// tensor-core tiles), so that no pass is a small remainder that leaves most SMs idle.
int pass_size(int n) {
    if (n <= kChunk) return n;
    const int passes = (n + kChunk - 1) / kChunk;
    const int per = (n + passes - 1) / passes;
    return (per + 127) / 128 * 128;
}

}  // namespace

struct nis_ctx {
    int device = 0;
    size_t budget = 0, in_use = 0;
    nis_allocator alloc{};
    bool custom_alloc = false;
    std::string err;
    unsigned *d_err = nullptr;
    std::map<void *, size_t> allocs;
    std::map<nis_handle, Volume> vols;
    std::map<nis_handle, Light> lights;
    std::map<nis_handle, Weights> weights;
    std::map<std::vector<uint32_t>, float *> phase;   // by the bit patterns of the phase spec
    std::map<std::vector<uint32_t>, float *> phase_paper;   // the paper model's [kAlpha][266]
    Workspace ws;
    WorkspaceBf wsb, wsx;                 // BF16 and split (FP32-accurate) tensor paths
    WorkspaceF8 ws8;
    // mixed-batch buffers of nis_shade_segments (grow-only)
    int mix_cap = 0, mix_desc_cap = 0;
    float *mix_pts = nullptr, *mix_om = nullptr, *mix_rgb = nullptr, *mix_dec = nullptr;
    int *mix_req = nullptr, *mix_seg_start = nullptr, *mix_seg_desc = nullptr;
    ReqDesc *mix_descs = nullptr;
    // ray states of the shear-warp transmittance, and its x-major output before the
    // transpose (grow-only, floats)
    float *sw_rays = nullptr, *sw_T = nullptr;
    size_t sw_cap = 0, sw_T_cap = 0;
    int num_sms = 0;
    nis_handle next = 1;
    // kernel timing (nis_profile)
    bool prof_on = false;
    struct ProfRecord { cudaEvent_t e0, e1; int launches; };
    std::map<std::string, std::vector<ProfRecord>> prof;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

nis_status fail(nis_ctx *c, nis_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

nis_status cuda_fail(nis_ctx *c, cudaError_t e, const char *what) {
    return fail(c, NIS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NIS_CUDA(call)                                                 \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
    } while (0)

std::atomic<uint64_t> g_launches{0};

cudaEvent_t take_event(nis_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets the kernel launches of its scope with events on `s` when profiling is on.
// Brackets the kernels launched in its scope with two events and counts them (the
// library's launch counter: profile from one host thread).  The dense layers of a shading
// pass are one scope, so no event sits between two of their launches (programmatic
// dependent launch overlaps each with the previous one's tail).
struct ProfScope {
    nis_ctx *c;
    const char *family;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    uint64_t l0 = 0;
    ProfScope(nis_ctx *c_, const char *f, cudaStream_t s_) : c(c_), family(f), s(s_) {
        if (c->prof_on && (e0 = take_event(c))) {
            cudaEventRecord(e0, s);
            l0 = g_launches.load();
        }
    }
    ~ProfScope() {
        if (!e0) return;
        cudaEvent_t e1 = take_event(c);
        if (!e1) return;
        cudaEventRecord(e1, s);
        c->prof[family].push_back({e0, e1, (int)(g_launches.load() - l0)});
    }
};

nis_status dev_alloc(nis_ctx *ctx, size_t bytes, void **out, cudaStream_t s) {
    *out = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(ctx, NIS_ERR_BUDGET, "allocation of " + std::to_string(bytes) +
                                             " bytes exceeds the HBM budget");
    void *p = nullptr;
    if (ctx->custom_alloc) {
        p = ctx->alloc.alloc(ctx->alloc.user, bytes, s);
        if (!p) return fail(ctx, NIS_ERR_OOM, "allocator returned NULL");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, NIS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    ctx->allocs[p] = bytes;
    ctx->in_use += bytes;
    *out = p;
    return NIS_OK;
}

template <typename T>
nis_status dev_alloc_t(nis_ctx *ctx, size_t count, T **out, cudaStream_t s) {
    void *p;
    nis_status st = dev_alloc(ctx, count * sizeof(T), &p, s);
    *out = static_cast<T *>(p);
    return st;
}

void dev_free(nis_ctx *ctx, void *p) {
    if (!p) return;
    auto it = ctx->allocs.find(p);
    if (it == ctx->allocs.end()) return;
    if (ctx->custom_alloc) ctx->alloc.free(ctx->alloc.user, p, it->second, nullptr);
    else cudaFree(p);
    ctx->in_use -= it->second;
    ctx->allocs.erase(it);
}

PyramidView view_of(const Volume &v, const float *base) {
    PyramidView pv{};
    pv.levels = v.levels;
    for (int m = 0; m < v.levels; ++m) {
        pv.lv[m] = base + v.off[m];
        pv.n[m] = v.sizes[m];
    }
    return pv;
}

nis_status build_pyramid_impl(nis_ctx *ctx, Volume &v, cudaStream_t s) {
    for (int m = 1; m < v.levels; ++m) {
        ProfScope ps(ctx, "pyramid", s);
        launch_downsample(v.data + v.off[m - 1], v.sizes[m - 1], v.data + v.off[m], v.sizes[m], s);
    }
    if (!v.occ) {
        size_t total = 0;
        for (int m = 0; m < v.levels; ++m) {
            v.occ_off[m] = total;
            const size_t n = (size_t)v.sizes[m];
            total += n * n * n;
        }
        nis_status st = dev_alloc_t(ctx, total, &v.occ, s);
        if (st) return st;
    }
    for (int m = 0; m < v.levels; ++m) {
        ProfScope ps(ctx, "pyramid", s);
        launch_occupancy(v.data + v.off[m], v.sizes[m], v.occ + v.occ_off[m], s);
    }
    NIS_CUDA(cudaGetLastError());
    v.pyramid = true;
    ++v.version;
    return NIS_OK;
}

// The x-major copy of the pyramid and its occupancy, (re)built after each pyramid build.
nis_status ensure_xmajor(nis_ctx *ctx, Volume &v, cudaStream_t s) {
    if (v.xmaj && v.xmaj_version == v.version) return NIS_OK;
    nis_status st;
    if (!v.xmaj) {
        size_t occ_total = 0;
        for (int m = 0; m < v.levels; ++m) occ_total += (size_t)v.sizes[m] * v.sizes[m] * v.sizes[m];
        if ((st = dev_alloc_t(ctx, v.total, &v.xmaj, s))) return st;
        if ((st = dev_alloc_t(ctx, occ_total, &v.xmaj_occ, s))) return st;
    }
    for (int m = 0; m < v.levels; ++m) {
        const size_t n = (size_t)v.sizes[m];
        launch_transpose(v.data + v.off[m], n * n, n, v.xmaj + v.off[m], s);   // [(z,y)][x] -> [x][(z,y)]
        launch_occupancy(v.xmaj + v.off[m], (int)n, v.xmaj_occ + v.occ_off[m], s);
    }
    NIS_CUDA(cudaGetLastError());
    v.xmaj_version = v.version;
    return NIS_OK;
}

// Packs (or re-packs, after a pyramid rebuild) the light's PairView levels.
nis_status ensure_pairs(nis_ctx *ctx, const Volume &v, Light &L, cudaStream_t s) {
    if (L.pairs && L.pair_version == v.version) return NIS_OK;
    if (!L.pairs) {
        size_t total = 0;
        for (int m = 0; m < v.levels; ++m) {
            L.pair_off[m] = total;
            total += pair_level_float4(v.sizes[m]);
        }
        nis_status st = dev_alloc_t(ctx, total, &L.pairs, s);
        if (st) return st;
    }
    for (int m = 0; m < v.levels; ++m) {
        ProfScope ps(ctx, "pyramid", s);
        launch_pack_pairs(v.data + v.off[m], L.data + v.off[m], v.sizes[m], L.pairs + L.pair_off[m], s);
    }
    NIS_CUDA(cudaGetLastError());
    L.pair_version = v.version;
    return NIS_OK;
}

PairView pair_view(const Volume &v, const Light &L) {
    PairView pv{};
    pv.levels = v.levels;
    for (int m = 0; m < v.levels; ++m) {
        pv.lv[m] = L.pairs + L.pair_off[m];
        pv.n[m] = v.sizes[m];
    }
    return pv;
}

PhaseSpec phase_spec(const nis_material *m) {
    PhaseSpec ph{};
    if (m->n_lobes >= 2) {
        ph.n = m->n_lobes;
        for (int i = 0; i < 3; ++i) {
            ph.g[i] = i < ph.n ? m->lobe_g[i] : 0.f;
            ph.w[i] = i < ph.n ? m->lobe_w[i] : 0.f;
        }
    } else {
        ph.n = 1;
        ph.g[0] = m->g;
        ph.w[0] = 1.f;
    }
    return ph;
}

PhaseSpec phase_spec_g(float g) {
    nis_material m{};
    m.g = g;
    return phase_spec(&m);
}

// The paper model's template, computed once per process (thread-safe initialisation).
struct PaperTemplate {
    double unit[kPaperPts][3], D[kLayers];
    float q[kPaperPts][3];
};
const PaperTemplate &paper_tpl() {
    static const PaperTemplate tpl = [] {
        PaperTemplate t{};
        paper_template(t.unit, t.D, t.q);
        return t;
    }();
    return tpl;
}

// The phase table of a phase function: over the lattice point sets, or (paper = true) over
// the paper model's 266 template points.
nis_status ensure_phase(nis_ctx *ctx, const PhaseSpec &ph, cudaStream_t s, float **out,
                        bool rebuild = false, bool paper = false) {
    std::vector<uint32_t> key(1 + 2 * ph.n);
    key[0] = (uint32_t)ph.n;
    for (int i = 0; i < ph.n; ++i) {
        std::memcpy(&key[1 + 2 * i], &ph.g[i], 4);
        std::memcpy(&key[2 + 2 * i], &ph.w[i], 4);
    }
    auto &cache = paper ? ctx->phase_paper : ctx->phase;
    auto it = cache.find(key);
    float *t;
    if (it != cache.end()) {
        *out = it->second;
        if (!rebuild) return NIS_OK;
        t = it->second;
    } else {
        nis_status st = dev_alloc_t(ctx, (size_t)kAlpha * (paper ? kPaperPts : kPhaseSets * kLat), &t, s);
        if (st) return st;
    }
    {
        ProfScope ps(ctx, "phase", s);
        if (paper) {
            launch_phase_points(ph, paper_tpl().q, kPaperPts, t, s);
        } else {
            launch_phase_table(ph, t, s);
        }
    }
    NIS_CUDA(cudaGetLastError());
    cache[key] = t;
    *out = t;
    return NIS_OK;
}

nis_status ensure_workspace(nis_ctx *ctx, int cap, cudaStream_t s) {
    Workspace &w = ctx->ws;
    if (w.cap >= cap) return NIS_OK;
    float **bufs[] = {&w.H_rho, &w.H_T, &w.H_f, &w.v, &w.w_se, &w.cfg, &w.X_T, &w.act};
    for (float **b : bufs) { dev_free(ctx, *b); *b = nullptr; }
    w.cap = 0;
    size_t n = (size_t)cap;
    nis_status st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kLat, &w.H_rho, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kLatT, &w.H_T, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kLat, &w.H_f, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 8, &w.v, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 3, &w.w_se, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kCfg, &w.cfg, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kDT, &w.X_T, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kActBufs * kWidth, &w.act, s))) return st;
    w.cap = cap;
    return NIS_OK;
}

nis_status ensure_workspace_tc(nis_ctx *ctx, WorkspaceBf &w, int parts, int cap, cudaStream_t s) {
    if (w.cap >= cap) return NIS_OK;
    __nv_bfloat16 **bb[] = {&w.Hb_rho, &w.Hb_f, &w.XTb, &w.E, &w.S, &w.H, &w.mrg_in[0], &w.mrg_in[1],
                            &w.mrg_in[2], &w.head_in, &w.Z1, &w.Z2};
    for (auto **b : bb) { dev_free(ctx, *b); *b = nullptr; }
    float **ff[] = {&w.H_T, &w.w_se, &w.cfg, &w.v, &w.E32, &w.H32};
    for (float **f : ff) { dev_free(ctx, *f); *f = nullptr; }
    for (auto **b : {&w.mrg_f, &w.head_f}) { dev_free(ctx, *b); *b = nullptr; }
    w.cap = 0;
    w.parts = parts;
    const size_t n = (size_t)cap, P = (size_t)parts;
    nis_status st;
    // BF16 (one part): rows wide enough for the fused backbone's layout as well
    const size_t lat_ld = parts == 1 ? kFuseLatLd : kLatPad, xt_ld = parts == 1 ? kFuseXtLd : kDT;
    if ((st = dev_alloc_t(ctx, P * n * kLayers * lat_ld, &w.Hb_rho, s))) return st;
    if ((st = dev_alloc_t(ctx, P * n * kLayers * lat_ld, &w.Hb_f, s))) return st;
    if ((st = dev_alloc_t(ctx, P * n * kLayers * xt_ld, &w.XTb, s))) return st;
    for (auto **b : {&w.S, &w.Z1, &w.Z2})
        if ((st = dev_alloc_t(ctx, P * n * kWidth, b, s))) return st;
    if (parts == 1) {
        for (auto **b : {&w.E, &w.H})
            if ((st = dev_alloc_t(ctx, n * kWidth, b, s))) return st;
    } else {
        for (float **f : {&w.E32, &w.H32})
            if ((st = dev_alloc_t(ctx, n * kWidth, f, s))) return st;
    }
    for (int t = 0; t < 3; ++t)
        if ((st = dev_alloc_t(ctx, P * n * 2 * kWidth, &w.mrg_in[t], s))) return st;
    if ((st = dev_alloc_t(ctx, P * n * 3 * kWidth, &w.head_in, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kLatT, &w.H_T, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 3, &w.w_se, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kCfg, &w.cfg, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 8, &w.v, s))) return st;
    const uint64_t rows = P * n;      // the parts of a tensor stack along the row dimension
    const uint32_t bx = tc_box_k(parts);
    bool ok = make_tmap_ht(&w.map_ht, w.H_T, n) &&
              make_tmap_bf16(&w.map_rho, w.Hb_rho, kLayers * kLatPad, rows, kLayers * kLatPad * 2, bx, 128) &&
              make_tmap_bf16(&w.map_f, w.Hb_f, kLayers * kLatPad, rows, kLayers * kLatPad * 2, bx, 128) &&
              make_tmap_bf16(&w.map_xt, w.XTb, kLayers * kDT, rows, kLayers * kDT * 2, bx, 128) &&
              make_tmap_bf16(&w.map_s, w.S, kWidth, rows, kWidth * 2, bx, 128) &&
              make_tmap_bf16(&w.map_head, w.head_in, 3 * kWidth, rows, 3 * kWidth * 2, bx, 128) &&
              make_tmap_bf16(&w.map_z1, w.Z1, kWidth, rows, kWidth * 2, bx, 128) &&
              make_tmap_bf16(&w.map_z2, w.Z2, kWidth, rows, kWidth * 2, bx, 128);
    for (int t = 0; t < 3; ++t)
        ok = ok && make_tmap_bf16(&w.map_mrg[t], w.mrg_in[t], 2 * kWidth, rows, 2 * kWidth * 2, bx, 128);
    // outputs: [parts][cap][kWidth] views; FP32 e and h with the split, BF16 otherwise
    const bool f32 = parts > 1;
    const uint64_t eb = f32 ? 4 : 2;
    ok = ok && make_tmap_out(&w.out_e, f32 ? (void *)w.E32 : (void *)w.E, f32, kWidth, n, 1, kWidth * eb, n * kWidth * eb) &&
         make_tmap_out(&w.out_h, f32 ? (void *)w.H32 : (void *)w.H, f32, kWidth, n, 1, kWidth * eb, n * kWidth * eb) &&
         make_tmap_out(&w.out_s, w.S, false, kWidth, n, parts, kWidth * 2, n * kWidth * 2) &&
         make_tmap_out(&w.out_z1, w.Z1, false, kWidth, n, parts, kWidth * 2, n * kWidth * 2) &&
         make_tmap_out(&w.out_z2, w.Z2, false, kWidth, n, parts, kWidth * 2, n * kWidth * 2);
    for (int t = 0; t < 3; ++t) {
        for (int c = 0; c < 2; ++c)
            ok = ok && make_tmap_out(&w.out_mrg[t][c], w.mrg_in[t] + c * kWidth, false, kWidth, n, parts,
                                     2 * kWidth * 2, n * 2 * kWidth * 2);
        ok = ok && make_tmap_out(&w.out_head[t], w.head_in + t * kWidth, false, kWidth, n, parts,
                                 3 * kWidth * 2, n * 3 * kWidth * 2);
    }
    if (parts == 1) {
        // the fused backbone's operand sources: 64-column boxes of 128 rows (128-byte swizzle)
        if ((st = dev_alloc_t(ctx, n * 3 * kFuseMrgLd, &w.mrg_f, s))) return st;
        if ((st = dev_alloc_t(ctx, n * kFuseHeadLd, &w.head_f, s))) return st;
        struct Src { int id; const void *base; uint64_t cols; };
        const Src srcs[] = {{kSrcRho, w.Hb_rho, kLayers * kFuseLatLd},
                            {kSrcF, w.Hb_f, kLayers * kFuseLatLd},
                            {kSrcT, w.XTb, kLayers * kFuseXtLd},
                            {kSrcMrg, w.mrg_f, 3 * kFuseMrgLd},
                            {kSrcHead, w.head_f, kFuseHeadLd}};
        w.fmaps = FusedMaps{};
        for (const Src &q : srcs) ok = ok && make_tmap_bf16(&w.fmaps.m64[q.id], q.base, q.cols, n, q.cols * 2, 64, 128);
    }
    if (!ok) return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the tensor-core workspace");
    w.cap = cap;
    return NIS_OK;
}

// The e4m3 mode's buffers and operand maps (the BF16 workspace must already hold cap rows).
nis_status ensure_f8_fused(nis_ctx *ctx, WorkspaceBf &w, int cap, cudaStream_t s) {
    const size_t n = (size_t)cap;
    nis_status st;
    if (w.f8_cap < cap) {
        for (auto **b : {&w.F8_rho, &w.F8_f}) { dev_free(ctx, *b); *b = nullptr; }
        dev_free(ctx, w.F8_cfg); w.F8_cfg = nullptr;
        for (float **f : {&w.fc1_scale, &w.tabmax}) { dev_free(ctx, *f); *f = nullptr; }
        w.f8_cap = 0;
        if ((st = dev_alloc_t(ctx, n * kLayers * kF8LatLd, &w.F8_rho, s))) return st;
        if ((st = dev_alloc_t(ctx, n * kLayers * kF8LatLd, &w.F8_f, s))) return st;
        if ((st = dev_alloc_t(ctx, n * kLayers * kF8CfgLd, &w.F8_cfg, s))) return st;
        if ((st = dev_alloc_t(ctx, n * kLayers * 3, &w.fc1_scale, s))) return st;
        if ((st = dev_alloc_t(ctx, (size_t)kPhaseSets, &w.tabmax, s))) return st;
        w.f8_cap = cap;
    }
    // rebuilt every call: the shared sources move when the BF16 workspace grows
    w.f8maps = w.fmaps;
    const uint64_t rows = (uint64_t)w.f8_cap;
    const bool ok =
        make_tmap_u8(&w.f8maps.m64[kSrcRho], w.F8_rho, kLayers * kF8LatLd, rows, kLayers * kF8LatLd, 128, 128) &&
        make_tmap_u8(&w.f8maps.m64[kSrcF], w.F8_f, kLayers * kF8LatLd, rows, kLayers * kF8LatLd, 128, 128) &&
        make_tmap_bf16(&w.f8maps.cfg8, w.F8_cfg, kLayers * kF8CfgLd, rows, kLayers * kF8CfgLd * 2, 16, 128);
    if (!ok) return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the e4m3 operands");
    return NIS_OK;
}

int n_mma_of(int n) { return (n + 15) / 16 * 16; }

int k_pad_of(int k) { return (k + 63) / 64 * 64; }

// The fused backbone (lattice model): its op program and weight slabs; with sw, its e4m3 mode.
nis_status pack_fused(nis_ctx *ctx, Weights &w, const float (*sw)[2], cudaStream_t s) {
    FusedOp ops[kFuseMaxOps];
    FusedPackOp pk[kFuseMaxOps];
    int n_ops = 0;
    size_t bytes = 0;
    nis_status st;
    fused_program(w.off, w.f32, ops, pk, &n_ops, &bytes, sw);
    if ((st = dev_alloc_t(ctx, bytes, &w.fused_w, s))) return st;
    if ((st = dev_alloc_t(ctx, (size_t)n_ops, &w.fused_ops, s))) return st;
    if ((st = dev_alloc_t(ctx, (size_t)n_ops, &w.fused_pack, s))) return st;
    NIS_CUDA(cudaMemcpyAsync(w.fused_ops, ops, n_ops * sizeof(FusedOp), cudaMemcpyHostToDevice, s));
    NIS_CUDA(cudaMemcpyAsync(w.fused_pack, pk, n_ops * sizeof(FusedPackOp), cudaMemcpyHostToDevice, s));
    {
        ProfScope ps(ctx, "other", s);
        launch_fused_pack(w.fused_pack, n_ops, w.fused_w, s);
    }
    // the host arrays above are read by the copies before this returns
    NIS_CUDA(cudaStreamSynchronize(s));
    w.fused_n_ops = n_ops;
    return NIS_OK;
}

// Tensor-core weight pack: per dense layer `parts` zero-padded [n_mma][Kp] BF16 matrices
// stacked along the rows (1 part: BF16; 3 parts: the three-way split), one tensor map each.
nis_status pack_weights_tc(nis_ctx *ctx, Weights &w, int parts, cudaStream_t s) {
    struct Mat { const float *src; int N, K, ld; CUtensorMap *map; };
    std::vector<Mat> mats;
    const WeightOffsets &o = w.off;
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < kLayers; ++k) {
            int d = o.model == kModelPaper ? paper_count(k) : feat_dim(t);
            mats.push_back({w.f32 + o.blk_w1[t][k], kWidth, d, d + kCfg, &w.map_fc1[t][k]});
            mats.push_back({w.f32 + o.blk_w2[t][k], kWidth, kWidth, kWidth, &w.map_fc2[t][k]});
        }
    for (int t = 0; t < 3; ++t) mats.push_back({w.f32 + o.mrg_w[t], kWidth, 2 * kWidth, 2 * kWidth, &w.map_mrg[t]});
    mats.push_back({w.f32 + o.head_w[0], kWidth, 3 * kWidth, 3 * kWidth, &w.map_head[0]});
    mats.push_back({w.f32 + o.head_w[1], kWidth, kWidth, kWidth, &w.map_head[1]});
    mats.push_back({w.f32 + o.head_w[2], 3, kWidth, kWidth, &w.map_head[2]});
    size_t total = 0;
    for (auto &m : mats) total += (size_t)parts * n_mma_of(m.N) * k_pad_of(m.K);
    nis_status st = dev_alloc_t(ctx, total, &w.bf, s);
    if (st) return st;
    size_t off = 0;
    for (auto &m : mats) {
        int np = n_mma_of(m.N), kp = k_pad_of(m.K);
        __nv_bfloat16 *dst = w.bf + off;
        for (int q = 0; q < parts; ++q) {
            ProfScope ps(ctx, "other", s);
            launch_pack_bf16(m.src, m.N, m.K, m.ld, dst + (size_t)q * np * kp, np, kp, s,
                             parts > 1 ? q : -1);
        }
        if (!make_tmap_bf16(m.map, dst, (uint64_t)kp, (uint64_t)parts * np, (uint64_t)kp * 2, tc_box_k(parts),
                            (uint32_t)np))
            return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed for a weight matrix");
        off += (size_t)parts * np * kp;
    }
    if (parts == 1 && o.model == kModelLattice && (st = pack_fused(ctx, w, nullptr, s))) return st;
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

// FP8 weight pack: per dense layer an e4m3 [n_mma][Kp] matrix (Kp a multiple of 128) with
// per-output-channel scales, and a UINT8 tensor map.
nis_status pack_weights_fp8(nis_ctx *ctx, Weights &w, cudaStream_t s) {
    struct Mat { const float *src; int N, K, ld; CUtensorMap *map; const float **sc; };
    std::vector<Mat> mats;
    const WeightOffsets &o = w.off;
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < kLayers; ++k) {
            int d = feat_dim(t);
            mats.push_back({w.f32 + o.blk_w1[t][k], kWidth, d, d + kCfg, &w.map_fc1[t][k], &w.sc_fc1[t][k]});
            mats.push_back({w.f32 + o.blk_w2[t][k], kWidth, kWidth, kWidth, &w.map_fc2[t][k], &w.sc_fc2[t][k]});
        }
    for (int t = 0; t < 3; ++t)
        mats.push_back({w.f32 + o.mrg_w[t], kWidth, 2 * kWidth, 2 * kWidth, &w.map_mrg[t], &w.sc_mrg[t]});
    mats.push_back({w.f32 + o.head_w[0], kWidth, 3 * kWidth, 3 * kWidth, &w.map_head[0], &w.sc_head[0]});
    mats.push_back({w.f32 + o.head_w[1], kWidth, kWidth, kWidth, &w.map_head[1], &w.sc_head[1]});
    mats.push_back({w.f32 + o.head_w[2], 3, kWidth, kWidth, &w.map_head[2], &w.sc_head[2]});
    auto kp8 = [](int k) { return (k + 127) / 128 * 128; };
    size_t total = 0, nsc = 0;
    for (auto &m : mats) { total += (size_t)n_mma_of(m.N) * kp8(m.K); nsc += n_mma_of(m.N); }
    nis_status st = dev_alloc_t(ctx, total, &w.f8, s);
    if (st) return st;
    if ((st = dev_alloc_t(ctx, nsc, &w.f8_scales, s))) return st;
    size_t off = 0, soff = 0;
    for (auto &m : mats) {
        int np = n_mma_of(m.N), kp = kp8(m.K);
        {
            ProfScope ps(ctx, "other", s);
            launch_pack_fp8(m.src, m.N, m.K, m.ld, w.f8 + off, w.f8_scales + soff, np, kp, s);
        }
        if (!make_tmap_u8(m.map, w.f8 + off, (uint64_t)kp, (uint64_t)np, (uint64_t)kp, 128, (uint32_t)np))
            return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed for an FP8 weight matrix");
        *m.sc = w.f8_scales + soff;
        off += (size_t)np * kp;
        soff += np;
    }
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

nis_status ensure_workspace_fp8(nis_ctx *ctx, int cap, cudaStream_t s) {
    WorkspaceF8 &w = ctx->ws8;
    if (w.cap >= cap) return NIS_OK;
    uint8_t **bb[] = {&w.H8_rho, &w.H8_f, &w.XT8, &w.S8, &w.mrg8[0], &w.mrg8[1], &w.mrg8[2],
                      &w.head8, &w.Z1, &w.Z2};
    for (auto **b : bb) { dev_free(ctx, *b); *b = nullptr; }
    dev_free(ctx, w.E); dev_free(ctx, w.H); w.E = w.H = nullptr;
    float **ff[] = {&w.H_T, &w.w_se, &w.cfg, &w.v, &w.fscale};
    for (float **f : ff) { dev_free(ctx, *f); *f = nullptr; }
    w.cap = 0;
    const size_t n = (size_t)cap;
    nis_status st;
    struct B8 { uint8_t **p; size_t bytes; };
    B8 list[] = {{&w.H8_rho, n * kLayers * kLatPad8}, {&w.H8_f, n * kLayers * kLatPad8},
                 {&w.XT8, n * kLayers * kDT}, {&w.S8, n * kWidth8}, {&w.mrg8[0], n * 2 * kWidth},
                 {&w.mrg8[1], n * 2 * kWidth}, {&w.mrg8[2], n * 2 * kWidth}, {&w.head8, n * kHead8},
                 {&w.Z1, n * kWidth8}, {&w.Z2, n * kWidth8}};
    for (auto &b : list) {
        if ((st = dev_alloc_t(ctx, b.bytes, b.p, s))) return st;
        NIS_CUDA(cudaMemsetAsync(*b.p, 0, b.bytes, s));   // row padding stays zero
    }
    if ((st = dev_alloc_t(ctx, n * kWidth, &w.E, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kWidth, &w.H, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * kLatT, &w.H_T, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 3, &w.w_se, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kCfg, &w.cfg, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 8, &w.v, s))) return st;
    if ((st = dev_alloc_t(ctx, n * kLayers * 2, &w.fscale, s))) return st;
    bool ok = make_tmap_ht(&w.map_ht, w.H_T, n) &&
              make_tmap_u8(&w.map_rho, w.H8_rho, kLayers * kLatPad8, n, kLayers * kLatPad8, 128, 128) &&
              make_tmap_u8(&w.map_f, w.H8_f, kLayers * kLatPad8, n, kLayers * kLatPad8, 128, 128) &&
              make_tmap_u8(&w.map_xt, w.XT8, kLayers * kDT, n, kLayers * kDT, 128, 128) &&
              make_tmap_u8(&w.map_s, w.S8, kWidth8, n, kWidth8, 128, 128) &&
              make_tmap_u8(&w.map_head, w.head8, kHead8, n, kHead8, 128, 128) &&
              make_tmap_u8(&w.map_z1, w.Z1, kWidth8, n, kWidth8, 128, 128) &&
              make_tmap_u8(&w.map_z2, w.Z2, kWidth8, n, kWidth8, 128, 128);
    for (int t = 0; t < 3; ++t)
        ok = ok && make_tmap_u8(&w.map_mrg[t], w.mrg8[t], 2 * kWidth, n, 2 * kWidth, 128, 128);
    if (!ok) return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the FP8 workspace");
    w.cap = cap;
    return NIS_OK;
}

nis_status check_material(nis_ctx *ctx, const nis_material *m) {
    const char *why = material_problem(m);
    return why ? fail(ctx, NIS_ERR_INVALID_ARG, why) : NIS_OK;
}

struct Mixed {                        // per-point request descriptors of a mixed batch
    const ReqDesc *descs;
    const int *req_of_point;
    const float *dec_rows;
};

// The transmittance lattices of points off .. off + cnt - 1 from the workspace (rows of
// kLatT) to a caller's [n][12][225] buffer.
cudaError_t copy_ht(float *dst, const float *src, int off, int cnt, cudaStream_t s) {
    if (!dst || cnt <= 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst + (size_t)off * kLayers * kLat, kLat * sizeof(float), src,
                             kLatT * sizeof(float), kLat * sizeof(float), (size_t)cnt * kLayers,
                             cudaMemcpyDeviceToDevice, s);
}
nis_status shade_impl_bf16(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                           const nis_material *m, const float *table, const float *pts,
                           const float *om, int n, float *rgb, const nis_debug_out *dbg,
                           cudaStream_t s, const Mixed *mx);
nis_status shade_impl_fp8(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                          const nis_material *m, const float *table, const float *pts,
                          const float *om, int n, float *rgb, const nis_debug_out *dbg,
                          cudaStream_t s, const Mixed *mx);

// Runs steps 3-6 for `n` points already on the device.
// The paper model's gather arguments of one (volume, light, weights, material): everything
// but the points and the outputs.
PaperGatherArgs paper_gather_args(const Volume &vol, const Light &light, const Weights &wt,
                                  const nis_material *m, const float *table) {
    PaperGatherArgs ga{};
    const PaperTemplate &tpl = paper_tpl();
    for (int t = 0; t < kPaperPts; ++t)
        for (int c = 0; c < 3; ++c) ga.unit[t][c] = (float)tpl.unit[t][c];
    for (int k = 0; k < kLayers; ++k) ga.D[k] = (float)tpl.D[k];
    const WeightOffsets &o = wt.off;
    ga.rho = view_of(vol, vol.data);
    ga.T = view_of(vol, light.data);
    ga.table = table;
    ga.lx = light.dir[0]; ga.ly = light.dir[1]; ga.lz = light.dir[2];
    ga.g = m->g;
    for (int c = 0; c < 3; ++c) ga.albedo[c] = m->albedo[c];
    ga.level_w = wt.f32 + o.level_w;
    ga.level_b = wt.f32 + o.level_b;
    ga.se = wt.f32;
    for (int k = 0; k < kLayers; ++k) {
        ga.se_w1[k] = o.se_w1[k]; ga.se_b1[k] = o.se_b1[k];
        ga.se_w2[k] = o.se_w2[k]; ga.se_b2[k] = o.se_b2[k];
    }
    return ga;
}

// Steps 3-6 of the paper-template model with FP32 FFMA dense layers (NIS_PREC_F32_SIMT):
// its gathers (density, phase and the volume-level transmission feature at the 266 template
// points, SE), then the backbone on per-layer widths.
nis_status shade_impl_paper(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                            const nis_material *m, const float *table, const float *pts,
                            const float *om, int n, float *rgb, const nis_debug_out *dbg,
                            cudaStream_t s) {
    int chunk = pass_size(n);
    nis_status st;
    if ((st = ensure_workspace(ctx, chunk, s))) return st;
    Workspace &w = ctx->ws;
    const WeightOffsets &o = wt.off;
    const float *W = wt.f32;
    const size_t act_stride = (size_t)w.cap * kWidth;
    auto act = [&](int i) { return w.act + i * act_stride; };
    float dec_scale[3];
    for (int c = 0; c < 3; ++c) dec_scale[c] = m->intensity[c] * powf(m->albedo[c], 4.0f);
    PaperGatherArgs ga = paper_gather_args(vol, light, wt, m, table);
    // the features [cnt][266] of each type in the lattice model's feature buffers
    ga.H_rho = w.H_rho; ga.H_f = w.H_f; ga.H_T = w.H_T;
    ga.v = w.v; ga.w_se = w.w_se; ga.cfg = w.cfg;
    for (int off = 0; off < n; off += chunk) {
        int cnt = n - off < chunk ? n - off : chunk;
        ga.points = pts + 3 * (size_t)off;
        ga.omega = om + 3 * (size_t)off;
        ga.count = cnt;
        {
            ProfScope ps(ctx, "gather", s);
            launch_gather_paper(ga, s);
        }
        for (int t = 0; t < 3; ++t) {
            const float *X = t == 0 ? w.H_rho : (t == 1 ? w.H_f : w.H_T);
            for (int chain = 0; chain < 2; ++chain) {
                int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
                float *h = nullptr;
                int ping = 1;
                for (int k = k0; k < k1; ++k) {
                    const int d = paper_count(k);
                    FcArgs f1{};
                    f1.mode = kFcFeat; f1.count = cnt; f1.K = d + kCfg; f1.N = kWidth;
                    f1.X = X + paper_first(k); f1.ldx = kPaperPts; f1.d = d;
                    f1.w_se = w.w_se; f1.layer = k; f1.type = t; f1.cfg = w.cfg;
                    f1.W = W + o.blk_w1[t][k]; f1.b = W + o.blk_b1[t][k];
                    f1.relu = 1; f1.out = act(0); f1.ldo = kWidth;
                    { ProfScope ps(ctx, "mlp", s); launch_fc_f32(f1, s); }
                    FcArgs f2{};
                    f2.mode = kFcSum; f2.count = cnt; f2.K = kWidth; f2.N = kWidth;
                    f2.a0 = h; f2.a1 = act(0); f2.seg = kWidth;
                    f2.W = W + o.blk_w2[t][k]; f2.b = W + o.blk_b2[t][k];
                    f2.relu = 1; f2.resid = act(0); f2.ldo = kWidth;
                    float *dst = (k == k1 - 1) ? act(3 + 2 * t + chain) : act(ping);
                    f2.out = dst;
                    { ProfScope ps(ctx, "mlp", s); launch_fc_f32(f2, s); }
                    h = dst;
                    ping = 3 - ping;
                }
            }
            FcArgs mg{};
            mg.mode = kFcCat; mg.count = cnt; mg.K = 2 * kWidth; mg.N = kWidth;
            mg.a0 = act(3 + 2 * t); mg.a1 = act(4 + 2 * t); mg.seg = kWidth;
            mg.W = W + o.mrg_w[t]; mg.b = W + o.mrg_b[t]; mg.relu = 1;
            mg.out = act(9 + t); mg.ldo = kWidth;
            { ProfScope ps(ctx, "mlp", s); launch_fc_f32(mg, s); }
        }
        FcArgs h1{};
        h1.mode = kFcCat; h1.count = cnt; h1.K = 3 * kWidth; h1.N = kWidth;
        h1.a0 = act(9); h1.a1 = act(10); h1.a2 = act(11); h1.seg = kWidth;
        h1.W = W + o.head_w[0]; h1.b = W + o.head_b[0]; h1.relu = 1;
        h1.out = act(12); h1.ldo = kWidth;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h1, s); }
        FcArgs h2{};
        h2.mode = kFcSum; h2.count = cnt; h2.K = kWidth; h2.N = kWidth;
        h2.a1 = act(12); h2.seg = kWidth;
        h2.W = W + o.head_w[1]; h2.b = W + o.head_b[1]; h2.relu = 1;
        h2.out = act(13); h2.ldo = kWidth;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h2, s); }
        FcArgs h3{};
        h3.mode = kFcSum; h3.count = cnt; h3.K = kWidth; h3.N = 3;
        h3.a1 = act(13); h3.seg = kWidth;
        h3.W = W + o.head_w[2]; h3.b = W + o.head_b[2];
        h3.decode = 1;
        for (int c = 0; c < 3; ++c) h3.dec_scale[c] = dec_scale[c];
        h3.y_out = (dbg && dbg->y) ? dbg->y + 3 * (size_t)off : nullptr;
        h3.out = rgb + 3 * (size_t)off; h3.ldo = 3;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h3, s); }
        if (dbg) {
            auto cp = [&](float *dst, const float *src, size_t per) -> cudaError_t {
                if (!dst) return cudaSuccess;
                return cudaMemcpyAsync(dst + per * off, src, per * cnt * sizeof(float),
                                       cudaMemcpyDeviceToDevice, s);
            };
            NIS_CUDA(cp(dbg->H_rho, w.H_rho, (size_t)kPaperPts));
            NIS_CUDA(cp(dbg->H_T, w.H_T, (size_t)kPaperPts));
            NIS_CUDA(cp(dbg->H_f, w.H_f, (size_t)kPaperPts));
            NIS_CUDA(cp(dbg->v, w.v, (size_t)kLayers * 8));
            NIS_CUDA(cp(dbg->w_se, w.w_se, (size_t)kLayers * 3));
        }
        NIS_CUDA(cudaGetLastError());
    }
    return NIS_OK;
}

nis_status shade_impl(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                      const nis_material *m, const float *pts, const float *om, int n,
                      float *rgb, const nis_debug_out *dbg, cudaStream_t s,
                      const Mixed *mx = nullptr) {
    float *table = nullptr;
    nis_status st;
    if (wt.off.model == kModelPaper) {
        if (mx) return fail(ctx, NIS_ERR_UNIMPLEMENTED, "mixed batches need lattice-model weights");
        if ((st = ensure_phase(ctx, phase_spec(m), s, &table, false, true))) return st;
        if (n <= 0) return NIS_OK;
        if (wt.precision == NIS_PREC_F32_SIMT)
            return shade_impl_paper(ctx, vol, light, wt, m, table, pts, om, n, rgb, dbg, s);
        return shade_impl_bf16(ctx, vol, light, wt, m, table, pts, om, n, rgb, dbg, s, nullptr);
    }
    if (!mx && (st = ensure_phase(ctx, phase_spec(m), s, &table))) return st;
    if (n <= 0) return NIS_OK;
    // FP8: the fused backbone's e4m3 mode; mixed batches take the layered FP8 path
    if (wt.precision == NIS_PREC_FP8 && (mx || wt.fused_n_ops == 0))
        return shade_impl_fp8(ctx, vol, light, wt, m, table, pts, om, n, rgb, dbg, s, mx);
    if (wt.precision != NIS_PREC_F32_SIMT)
        return shade_impl_bf16(ctx, vol, light, wt, m, table, pts, om, n, rgb, dbg, s, mx);
    int chunk = pass_size(n);
    if ((st = ensure_workspace(ctx, chunk, s))) return st;
    Workspace &w = ctx->ws;
    const WeightOffsets &o = wt.off;
    const float *W = wt.f32;
    const size_t act_stride = (size_t)w.cap * kWidth;
    auto act = [&](int i) { return w.act + i * act_stride; };
    float dec_scale[3];
    for (int c = 0; c < 3; ++c) dec_scale[c] = m->intensity[c] * powf(m->albedo[c], 4.0f);

    for (int off = 0; off < n; off += chunk) {
        int cnt = n - off < chunk ? n - off : chunk;
        GatherArgs ga{};
        ga.rho = view_of(vol, vol.data);
        ga.T = view_of(vol, light.data);
        ga.rt = pair_view(vol, light);
        ga.table = table;
        ga.points = pts + 3 * (size_t)off;
        ga.omega = om + 3 * (size_t)off;
        ga.count = cnt;
        ga.lx = light.dir[0]; ga.ly = light.dir[1]; ga.lz = light.dir[2];
        ga.g = m->g;
        for (int c = 0; c < 3; ++c) ga.albedo[c] = m->albedo[c];
        ga.se = W;
        for (int k = 0; k < kLayers; ++k) {
            ga.se_w1[k] = o.se_w1[k]; ga.se_b1[k] = o.se_b1[k];
            ga.se_w2[k] = o.se_w2[k]; ga.se_b2[k] = o.se_b2[k];
        }
        ga.H_rho = w.H_rho; ga.H_T = w.H_T; ga.H_f = w.H_f;
        ga.v = w.v; ga.w_se = w.w_se; ga.cfg = w.cfg;
        if (mx) { ga.descs = mx->descs; ga.req_of_point = mx->req_of_point + off; }
        {
            ProfScope ps(ctx, "gather", s);
            launch_gather(ga, s);
        }
        {
            ProfScope ps(ctx, "cnn", s);
            launch_cnn_f32(w.H_T, cnt, W, o, w.X_T, nullptr, s);
        }

        // backbone: 3 types x (diffuse chain of 8, highlight chain of 4)
        for (int t = 0; t < 3; ++t) {
            const float *X = t == 0 ? w.H_rho : (t == 1 ? w.H_f : w.X_T);
            const int d = feat_dim(t);
            for (int chain = 0; chain < 2; ++chain) {
                int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
                float *h = nullptr;
                int ping = 1;
                for (int k = k0; k < k1; ++k) {
                    FcArgs f1{};
                    f1.mode = kFcFeat; f1.count = cnt; f1.K = d + kCfg; f1.N = kWidth;
                    f1.X = X + (size_t)k * d; f1.ldx = kLayers * d; f1.d = d;
                    f1.w_se = w.w_se; f1.layer = k; f1.type = t; f1.cfg = w.cfg;
                    f1.W = W + o.blk_w1[t][k]; f1.b = W + o.blk_b1[t][k];
                    f1.relu = 1; f1.out = act(0); f1.ldo = kWidth;
                    { ProfScope ps(ctx, "mlp", s); launch_fc_f32(f1, s); }
                    FcArgs f2{};
                    f2.mode = kFcSum; f2.count = cnt; f2.K = kWidth; f2.N = kWidth;
                    f2.a0 = h; f2.a1 = act(0); f2.seg = kWidth;
                    f2.W = W + o.blk_w2[t][k]; f2.b = W + o.blk_b2[t][k];
                    f2.relu = 1; f2.resid = act(0); f2.ldo = kWidth;
                    float *dst = (k == k1 - 1) ? act(3 + 2 * t + chain) : act(ping);
                    f2.out = dst;
                    { ProfScope ps(ctx, "mlp", s); launch_fc_f32(f2, s); }
                    h = dst;
                    ping = 3 - ping;
                }
            }
            FcArgs mg{};
            mg.mode = kFcCat; mg.count = cnt; mg.K = 2 * kWidth; mg.N = kWidth;
            mg.a0 = act(3 + 2 * t); mg.a1 = act(4 + 2 * t); mg.seg = kWidth;
            mg.W = W + o.mrg_w[t]; mg.b = W + o.mrg_b[t]; mg.relu = 1;
            mg.out = act(9 + t); mg.ldo = kWidth;
            { ProfScope ps(ctx, "mlp", s); launch_fc_f32(mg, s); }
        }
        FcArgs h1{};
        h1.mode = kFcCat; h1.count = cnt; h1.K = 3 * kWidth; h1.N = kWidth;
        h1.a0 = act(9); h1.a1 = act(10); h1.a2 = act(11); h1.seg = kWidth;
        h1.W = W + o.head_w[0]; h1.b = W + o.head_b[0]; h1.relu = 1;
        h1.out = act(12); h1.ldo = kWidth;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h1, s); }
        FcArgs h2{};
        h2.mode = kFcSum; h2.count = cnt; h2.K = kWidth; h2.N = kWidth;
        h2.a1 = act(12); h2.seg = kWidth;
        h2.W = W + o.head_w[1]; h2.b = W + o.head_b[1]; h2.relu = 1;
        h2.out = act(13); h2.ldo = kWidth;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h2, s); }
        FcArgs h3{};
        h3.mode = kFcSum; h3.count = cnt; h3.K = kWidth; h3.N = 3;
        h3.a1 = act(13); h3.seg = kWidth;
        h3.W = W + o.head_w[2]; h3.b = W + o.head_b[2];
        h3.decode = 1;
        for (int c = 0; c < 3; ++c) h3.dec_scale[c] = dec_scale[c];
        h3.y_out = (dbg && dbg->y) ? dbg->y + 3 * (size_t)off : nullptr;
        h3.out = rgb + 3 * (size_t)off; h3.ldo = 3;
        if (mx) h3.dec_rows = mx->dec_rows + 3 * (size_t)off;
        { ProfScope ps(ctx, "mlp", s); launch_fc_f32(h3, s); }

        if (dbg) {
            auto cp = [&](float *dst, const float *src, size_t per) -> cudaError_t {
                if (!dst) return cudaSuccess;
                return cudaMemcpyAsync(dst + per * off, src, per * cnt * sizeof(float),
                                       cudaMemcpyDeviceToDevice, s);
            };
            NIS_CUDA(cp(dbg->H_rho, w.H_rho, (size_t)kLayers * kLat));
            NIS_CUDA(copy_ht(dbg->H_T, w.H_T, off, cnt, s));
            NIS_CUDA(cp(dbg->H_f, w.H_f, (size_t)kLayers * kLat));
            NIS_CUDA(cp(dbg->v, w.v, (size_t)kLayers * 8));
            NIS_CUDA(cp(dbg->X_T, w.X_T, (size_t)kLayers * kDT));
            NIS_CUDA(cp(dbg->w_se, w.w_se, (size_t)kLayers * 3));
        }
        NIS_CUDA(cudaGetLastError());
    }
    return NIS_OK;
}

// Steps 3-6 with the dense layers on the tensor cores (BF16 operands, FP32 accumulation).
nis_status shade_impl_bf16(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                           const nis_material *m, const float *table, const float *pts,
                           const float *om, int n, float *rgb, const nis_debug_out *dbg,
                           cudaStream_t s, const Mixed *mx) {
    int chunk = pass_size(n);
    const bool split = wt.precision == NIS_PREC_F32;
    const bool paper = wt.off.model == kModelPaper;
    WorkspaceBf &w = split ? ctx->wsx : ctx->wsb;
    const int P = split ? 3 : 1;
    nis_status st = ensure_workspace_tc(ctx, w, P, chunk, s);
    if (st) return st;
    const size_t cap = (size_t)w.cap;
    const WeightOffsets &o = wt.off;
    const float *W = wt.f32;
    float dec_scale[3];
    for (int c = 0; c < 3; ++c) dec_scale[c] = m->intensity[c] * powf(m->albedo[c], 4.0f);
    // o1 / o2: the epilogue's output maps (TMA stores); null writes through the pointers
    auto gemm = [&](TcGemmArgs a, const CUtensorMap &ma, const CUtensorMap &mb,
                    const CUtensorMap *o1 = nullptr, const CUtensorMap *o2 = nullptr,
                    const CUtensorMap *pre = nullptr) {
        a.n_pass = split ? 6 : 1;
        a.k_tiles = (a.K + (int)tc_box_k(P) - 1) / (int)tc_box_k(P);
        a.a_part_rows = (int)cap;
        a.b_part_rows = a.n_mma;
        a.out_split = split ? 1 : 0;
        a.pre_tma = pre ? (split ? 1 : 2) : 0;
        launch_tc_gemm(a, ma, mb, ctx->num_sms, s, o1, o2, pre);
    };
    const int k_e = split ? kOutF32 : kOutBf16;     // kind of e and h
    // BF16 lattice model: the whole network after the features in one fused kernel; FP8 (no
    // mixed batch): the same kernel in its e4m3 mode
    const bool fused = !split && !paper && wt.fused_n_ops > 0;
    const bool f8 = wt.precision == NIS_PREC_FP8;
    if (f8 && (st = ensure_f8_fused(ctx, w, chunk, s))) return st;
    if (f8) {
        ProfScope ps(ctx, "gather", s);
        launch_table_set_max(table, w.tabmax, s);
    }
    for (int off = 0; off < n; off += chunk) {
        int cnt = n - off < chunk ? n - off : chunk;
        GatherArgs ga{};
        ga.rho = view_of(vol, vol.data);
        ga.T = view_of(vol, light.data);
        ga.rt = pair_view(vol, light);
        ga.table = table;
        ga.points = pts + 3 * (size_t)off;
        ga.omega = om + 3 * (size_t)off;
        ga.count = cnt;
        ga.lx = light.dir[0]; ga.ly = light.dir[1]; ga.lz = light.dir[2];
        ga.g = m->g;
        for (int c = 0; c < 3; ++c) ga.albedo[c] = m->albedo[c];
        ga.se = W;
        for (int k = 0; k < kLayers; ++k) {
            ga.se_w1[k] = o.se_w1[k]; ga.se_b1[k] = o.se_b1[k];
            ga.se_w2[k] = o.se_w2[k]; ga.se_b2[k] = o.se_b2[k];
        }
        ga.H_T = w.H_T; ga.Hb_rho = w.Hb_rho; ga.Hb_f = w.Hb_f;
        ga.split = split; ga.part = cap * kLayers * kLatPad;
        if (dbg && dbg->H_rho && dbg->H_f) {      // FP32 features straight into the debug buffers
            ga.H_rho = dbg->H_rho + (size_t)off * kLayers * kLat;
            ga.H_f = dbg->H_f + (size_t)off * kLayers * kLat;
        }
        ga.v = dbg ? w.v : nullptr; ga.w_se = w.w_se; ga.cfg = w.cfg;
        if (fused) { ga.fused = 1; ga.XT_cfg = w.XTb; }
        if (f8) {
            ga.Hb_rho = ga.Hb_f = nullptr;
            ga.F8_rho = w.F8_rho; ga.F8_f = w.F8_f; ga.F8_cfg = w.F8_cfg; ga.fc1_scale = w.fc1_scale;
            ga.f8_sigma = vol.sigma_max; ga.f8_tabmax = w.tabmax;
            for (int k = 0; k < kLayers; ++k)
                for (int t = 0; t < 2; ++t) ga.f8_sw[k][t] = wt.f8_sw[k][t];
        }
        if (mx) { ga.descs = mx->descs; ga.req_of_point = mx->req_of_point + off; }
        if (paper) {
            // the paper model: its gathers write the operands of all three types (the
            // transmission feature in the CNN output's buffer); no CNN
            PaperGatherArgs pg = paper_gather_args(vol, light, wt, m, table);
            pg.points = ga.points; pg.omega = ga.omega; pg.count = cnt;
            if (dbg && dbg->H_rho && dbg->H_f && dbg->H_T) {
                pg.H_rho = dbg->H_rho + (size_t)off * kPaperPts;
                pg.H_f = dbg->H_f + (size_t)off * kPaperPts;
                pg.H_T = dbg->H_T + (size_t)off * kPaperPts;
            }
            pg.Hb_rho = w.Hb_rho; pg.Hb_f = w.Hb_f; pg.Hb_T = w.XTb;
            pg.parts = P; pg.ld_rf = kLayers * kLatPad; pg.ld_t = kLayers * kDT;
            pg.part_rf = cap * kLayers * kLatPad; pg.part_t = cap * kLayers * kDT;
            pg.v = dbg ? w.v : nullptr; pg.w_se = w.w_se; pg.cfg = w.cfg;
            ProfScope ps(ctx, "gather", s);
            launch_gather_paper(pg, s);
        } else {
            {
                ProfScope ps(ctx, "gather", s);
                launch_gather(ga, s);
            }
            ProfScope ps(ctx, "cnn", s);
            float *xt_dbg = (dbg && dbg->X_T) ? dbg->X_T + (size_t)off * kLayers * kDT : nullptr;
            if (split)      // FP32: the FP32 CNN, its output split into three BF16 parts
                launch_cnn_f32(w.H_T, cnt, W, o, xt_dbg, w.XTb, s, cap * kLayers * kDT, &w.map_ht, ctx->d_err);
            else            // BF16: the CNN with BF16 operands on the tensor cores
                launch_cnn_tc(w.map_ht, cnt, W, o, xt_dbg, w.XTb, nullptr, ctx->d_err, ctx->num_sms, s,
                              fused ? kFuseXtLd : kDT);
        }
        if (fused) {
            ProfScope pm(ctx, "mlp", s);
            FusedArgs fa{};
            fa.M = cnt; fa.n_ops = wt.fused_n_ops; fa.ops = wt.fused_ops; fa.wpack = wt.fused_w;
            fa.w_se = w.w_se; fa.mrg = w.mrg_f; fa.head = w.head_f;
            fa.rgb = rgb + 3 * (size_t)off;
            fa.y_out = (dbg && dbg->y) ? dbg->y + 3 * (size_t)off : nullptr;
            fa.dec_rows = mx ? mx->dec_rows + 3 * (size_t)off : nullptr;
            for (int c = 0; c < 3; ++c) fa.dec_scale[c] = dec_scale[c];
            fa.err = ctx->d_err;
            fa.fc1_scale = f8 ? w.fc1_scale : nullptr;
            launch_mlp_fused(fa, f8 ? w.f8maps : w.fmaps, ctx->num_sms, s);
        } else {
            ProfScope pm(ctx, "mlp", s);   // the pass's dense layers as one timed block
            for (int t = 0; t < 3; ++t) {
                const CUtensorMap &fmap = t == 0 ? w.map_rho : (t == 1 ? w.map_f : w.map_xt);
                const int fstride = t == 2 ? kDT : kLatPad;
                for (int chain = 0; chain < 2; ++chain) {
                    int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
                    for (int k = k0; k < k1; ++k) {
                        // the layer's input width d (its weights' columns before the 5 of the
                        // configuration) and operand columns: the paper model's padded layout
                        const int d = paper ? paper_count(k) : feat_dim(t);
                        TcGemmArgs f1{};
                        f1.M = cnt; f1.N = kWidth; f1.K = paper ? paper_count_pad(k) : d;
                        f1.n_mma = 208; f1.k_tiles = (f1.K + 63) / 64;
                        f1.a_col0 = paper ? paper_first_pad(k) : k * fstride;
                        f1.epi = kEpiFc1; f1.err = ctx->d_err;
                        f1.out_e = w.E; f1.out_s = w.S; f1.ldo = kWidth;
                        f1.out_e_f32 = split ? w.E32 : nullptr;
                        f1.out_part = cap * kWidth;
                        f1.bias = W + o.blk_b1[t][k];
                        f1.row_scale = w.w_se + k * 3 + t; f1.row_scale_ld = kLayers * 3;
                        f1.cfg = w.cfg; f1.w_cfg = W + o.blk_w1[t][k] + d; f1.w_cfg_ld = d + kCfg;
                        f1.mat_cfg[0] = m->g;
                        for (int c = 0; c < 3; ++c) f1.mat_cfg[1 + c] = m->albedo[c];
                        // per-row configuration even for one request: a request's result is then
                        // bit-identical alone and inside a mixed batch
                        f1.cfg_per_row = 1;
                        f1.h_prev = (k == k0 || split) ? nullptr : w.H; f1.ld_h = kWidth;
                        f1.pre_f32 = (k == k0 || !split) ? nullptr : w.H32; f1.ld_pre = kWidth;
                        f1.o1_kind = k_e; f1.o1_parts = 1; f1.o2_kind = kOutBf16; f1.o2_parts = P;
                        // the running state h arrives by TMA (the e and h output maps read back
                        // as 32 x 32 boxes)
                        gemm(f1, fmap, wt.map_fc1[t][k], &w.out_e, &w.out_s,
                             (f1.pre_f32 || f1.h_prev) ? &w.out_h : nullptr);
                        TcGemmArgs f2{};
                        f2.M = cnt; f2.N = kWidth; f2.K = kWidth; f2.n_mma = 208; f2.k_tiles = 4;
                        f2.epi = kEpiFc2; f2.err = ctx->d_err;
                        f2.bias = W + o.blk_b2[t][k];
                        f2.resid = w.E; f2.ld_resid = kWidth;
                        if (split) { f2.pre_f32 = w.E32; f2.ld_pre = kWidth; }
                        if (k == k1 - 1) {
                            f2.out_bf = w.mrg_in[t] + chain * kWidth; f2.ldo = 2 * kWidth;
                            f2.out_part = cap * 2 * kWidth;
                        } else if (split) {
                            f2.out_h_f32 = w.H32; f2.ldo = kWidth;
                        } else {
                            f2.out_bf = w.H; f2.ldo = kWidth;
                        }
                        const bool end = k == k1 - 1;
                        f2.o1_kind = end ? kOutBf16 : k_e; f2.o1_parts = end ? P : 1;
                        gemm(f2, w.map_s, wt.map_fc2[t][k], end ? &w.out_mrg[t][chain] : &w.out_h, nullptr,
                             &w.out_e);
                    }
                }
                TcGemmArgs mg{};
                mg.M = cnt; mg.N = kWidth; mg.K = 2 * kWidth; mg.n_mma = 208; mg.k_tiles = 7;
                mg.epi = kEpiRelu; mg.err = ctx->d_err; mg.bias = W + o.mrg_b[t];
                mg.out_bf = w.head_in + t * kWidth; mg.ldo = 3 * kWidth;
                mg.out_part = cap * 3 * kWidth;
                mg.o1_kind = kOutBf16; mg.o1_parts = P;
                gemm(mg, w.map_mrg[t], wt.map_mrg[t], &w.out_head[t]);
            }
            TcGemmArgs h1{};
            h1.M = cnt; h1.N = kWidth; h1.K = 3 * kWidth; h1.n_mma = 208; h1.k_tiles = 10;
            h1.epi = kEpiRelu; h1.err = ctx->d_err; h1.bias = W + o.head_b[0];
            h1.out_bf = w.Z1; h1.ldo = kWidth;
            h1.out_part = cap * kWidth;
            h1.o1_kind = kOutBf16; h1.o1_parts = P;
            gemm(h1, w.map_head, wt.map_head[0], &w.out_z1);
            TcGemmArgs h2 = h1;
            h2.K = kWidth; h2.k_tiles = 4; h2.bias = W + o.head_b[1]; h2.out_bf = w.Z2;
            gemm(h2, w.map_z1, wt.map_head[1], &w.out_z2);
            TcGemmArgs h3{};
            h3.M = cnt; h3.N = 3; h3.K = kWidth; h3.n_mma = 16; h3.k_tiles = 4;
            h3.epi = kEpiDecode; h3.err = ctx->d_err; h3.bias = W + o.head_b[2];
            for (int c = 0; c < 3; ++c) h3.dec_scale[c] = dec_scale[c];
            h3.out_f32 = rgb + 3 * (size_t)off;
            h3.y_out = (dbg && dbg->y) ? dbg->y + 3 * (size_t)off : nullptr;
            if (mx) h3.dec_rows = mx->dec_rows + 3 * (size_t)off;
            gemm(h3, w.map_z2, wt.map_head[2]);
        }
        if (dbg) {
            auto cp = [&](float *dst, const float *src, size_t per) -> cudaError_t {
                if (!dst) return cudaSuccess;
                return cudaMemcpyAsync(dst + per * off, src, per * cnt * sizeof(float),
                                       cudaMemcpyDeviceToDevice, s);
            };
            if (!paper) NIS_CUDA(copy_ht(dbg->H_T, w.H_T, off, cnt, s));   // paper: by the gather
            NIS_CUDA(cp(dbg->v, w.v, (size_t)kLayers * 8));
            NIS_CUDA(cp(dbg->w_se, w.w_se, (size_t)kLayers * 3));
        }
        NIS_CUDA(cudaGetLastError());
    }
    return NIS_OK;
}

// Steps 3-6 with the dense layers in FP8 e4m3 on the tensor cores (FP32 accumulation):
// weights scaled per output channel, density/phase features per (point, layer), the other
// activations unscaled.
nis_status shade_impl_fp8(nis_ctx *ctx, const Volume &vol, const Light &light, const Weights &wt,
                          const nis_material *m, const float *table, const float *pts,
                          const float *om, int n, float *rgb, const nis_debug_out *dbg,
                          cudaStream_t s, const Mixed *mx) {
    int chunk = pass_size(n);
    nis_status st = ensure_workspace_fp8(ctx, chunk, s);
    if (st) return st;
    WorkspaceF8 &w = ctx->ws8;
    const WeightOffsets &o = wt.off;
    const float *W = wt.f32;
    float dec_scale[3];
    for (int c = 0; c < 3; ++c) dec_scale[c] = m->intensity[c] * powf(m->albedo[c], 4.0f);
    auto gemm = [&](TcGemmArgs a, const CUtensorMap &ma, const CUtensorMap &mb) {
        a.fp8 = 1;
        a.k_tiles = (a.K + 127) / 128;
        launch_tc_gemm(a, ma, mb, ctx->num_sms, s);
    };
    for (int off = 0; off < n; off += chunk) {
        int cnt = n - off < chunk ? n - off : chunk;
        GatherArgs ga{};
        ga.rho = view_of(vol, vol.data);
        ga.T = view_of(vol, light.data);
        ga.rt = pair_view(vol, light);
        ga.table = table;
        ga.points = pts + 3 * (size_t)off;
        ga.omega = om + 3 * (size_t)off;
        ga.count = cnt;
        ga.lx = light.dir[0]; ga.ly = light.dir[1]; ga.lz = light.dir[2];
        ga.g = m->g;
        for (int c = 0; c < 3; ++c) ga.albedo[c] = m->albedo[c];
        ga.se = W;
        for (int k = 0; k < kLayers; ++k) {
            ga.se_w1[k] = o.se_w1[k]; ga.se_b1[k] = o.se_b1[k];
            ga.se_w2[k] = o.se_w2[k]; ga.se_b2[k] = o.se_b2[k];
        }
        ga.H_T = w.H_T; ga.H8_rho = w.H8_rho; ga.H8_f = w.H8_f; ga.f8_scale = w.fscale;
        if (dbg && dbg->H_rho && dbg->H_f) {
            ga.H_rho = dbg->H_rho + (size_t)off * kLayers * kLat;
            ga.H_f = dbg->H_f + (size_t)off * kLayers * kLat;
        }
        ga.v = dbg ? w.v : nullptr; ga.w_se = w.w_se; ga.cfg = w.cfg;
        if (mx) { ga.descs = mx->descs; ga.req_of_point = mx->req_of_point + off; }
        {
            ProfScope ps(ctx, "gather", s);
            launch_gather(ga, s);
        }
        {
            ProfScope ps(ctx, "cnn", s);
            launch_cnn_tc(w.map_ht, cnt, W, o, (dbg && dbg->X_T) ? dbg->X_T + (size_t)off * kLayers * kDT : nullptr,
                          nullptr, w.XT8, ctx->d_err, ctx->num_sms, s);
        }
        {
            ProfScope pm(ctx, "mlp", s);   // the pass's dense layers as one timed block
            for (int t = 0; t < 3; ++t) {
                const int d = feat_dim(t);
                const CUtensorMap &fmap = t == 0 ? w.map_rho : (t == 1 ? w.map_f : w.map_xt);
                const int fstride = t == 2 ? kDT : kLatPad8;
                for (int chain = 0; chain < 2; ++chain) {
                    int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
                    for (int k = k0; k < k1; ++k) {
                        TcGemmArgs f1{};
                        f1.M = cnt; f1.N = kWidth; f1.K = d; f1.n_mma = 208;
                        f1.a_col0 = k * fstride; f1.epi = kEpiFc1; f1.err = ctx->d_err;
                        f1.out_e = w.E; f1.out_s8 = w.S8; f1.ldo = kWidth;
                        f1.bias = W + o.blk_b1[t][k];
                        f1.row_scale = w.w_se + k * 3 + t; f1.row_scale_ld = kLayers * 3;
                        if (t < 2) { f1.row_scale2 = w.fscale + k * 2 + t; f1.row_scale2_ld = kLayers * 2; }
                        f1.col_scale = wt.sc_fc1[t][k];
                        f1.cfg = w.cfg; f1.w_cfg = W + o.blk_w1[t][k] + d; f1.w_cfg_ld = d + kCfg;
                        f1.cfg_per_row = 1;
                        f1.h_prev = k == k0 ? nullptr : w.H; f1.ld_h = kWidth;
                        gemm(f1, fmap, wt.map_fc1[t][k]);
                        TcGemmArgs f2{};
                        f2.M = cnt; f2.N = kWidth; f2.K = kWidth; f2.n_mma = 208;
                        f2.epi = kEpiFc2; f2.err = ctx->d_err;
                        f2.bias = W + o.blk_b2[t][k];
                        f2.col_scale = wt.sc_fc2[t][k];
                        f2.resid = w.E; f2.ld_resid = kWidth;
                        if (k == k1 - 1) { f2.out_f8 = w.mrg8[t] + chain * kWidth; f2.ldo = 2 * kWidth; }
                        else { f2.out_bf = w.H; f2.ldo = kWidth; }
                        gemm(f2, w.map_s, wt.map_fc2[t][k]);
                    }
                }
                TcGemmArgs mg{};
                mg.M = cnt; mg.N = kWidth; mg.K = 2 * kWidth; mg.n_mma = 208;
                mg.epi = kEpiRelu; mg.err = ctx->d_err; mg.bias = W + o.mrg_b[t];
                mg.col_scale = wt.sc_mrg[t];
                mg.out_f8 = w.head8 + t * kWidth; mg.ldo = kHead8;
                gemm(mg, w.map_mrg[t], wt.map_mrg[t]);
            }
            TcGemmArgs h1{};
            h1.M = cnt; h1.N = kWidth; h1.K = 3 * kWidth; h1.n_mma = 208;
            h1.epi = kEpiRelu; h1.err = ctx->d_err; h1.bias = W + o.head_b[0];
            h1.col_scale = wt.sc_head[0];
            h1.out_f8 = w.Z1; h1.ldo = kWidth8;
            gemm(h1, w.map_head, wt.map_head[0]);
            TcGemmArgs h2 = h1;
            h2.K = kWidth; h2.bias = W + o.head_b[1]; h2.col_scale = wt.sc_head[1]; h2.out_f8 = w.Z2;
            gemm(h2, w.map_z1, wt.map_head[1]);
            TcGemmArgs h3{};
            h3.M = cnt; h3.N = 3; h3.K = kWidth; h3.n_mma = 16;
            h3.epi = kEpiDecode; h3.err = ctx->d_err; h3.bias = W + o.head_b[2];
            h3.col_scale = wt.sc_head[2];
            for (int c = 0; c < 3; ++c) h3.dec_scale[c] = dec_scale[c];
            h3.out_f32 = rgb + 3 * (size_t)off;
            h3.y_out = (dbg && dbg->y) ? dbg->y + 3 * (size_t)off : nullptr;
            if (mx) h3.dec_rows = mx->dec_rows + 3 * (size_t)off;
            gemm(h3, w.map_z2, wt.map_head[2]);
        }
        if (dbg) {
            auto cp = [&](float *dst, const float *src, size_t per) -> cudaError_t {
                if (!dst) return cudaSuccess;
                return cudaMemcpyAsync(dst + per * off, src, per * cnt * sizeof(float),
                                       cudaMemcpyDeviceToDevice, s);
            };
            NIS_CUDA(copy_ht(dbg->H_T, w.H_T, off, cnt, s));
            NIS_CUDA(cp(dbg->v, w.v, (size_t)kLayers * 8));
            NIS_CUDA(cp(dbg->w_se, w.w_se, (size_t)kLayers * 3));
        }
        NIS_CUDA(cudaGetLastError());
    }
    return NIS_OK;
}

template <typename T>
T *lookup(std::map<nis_handle, T> &m, nis_handle h) {
    auto it = m.find(h);
    return it == m.end() ? nullptr : &it->second;
}

nis_status resolve(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w, Volume **pv,
                   Light **pl, Weights **pw) {
    *pv = lookup(ctx->vols, vol);
    *pl = lookup(ctx->lights, light);
    *pw = lookup(ctx->weights, w);
    if (!*pv) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    if (!*pl) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released light handle");
    if (!*pw) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released weights handle");
    if ((*pl)->vol != vol) return fail(ctx, NIS_ERR_INVALID_ARG, "light belongs to another volume");
    if (!(*pv)->pyramid) return fail(ctx, NIS_ERR_NOT_READY, "pyramid not built");
    return NIS_OK;
}

nis_status camera_args(nis_ctx *ctx, const nis_camera *cam, CameraArgs *c) {
    if (!cam) return fail(ctx, NIS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0 || (long long)cam->width * cam->height > (1LL << 27))
        return fail(ctx, NIS_ERR_INVALID_ARG, "bad image size");
    if (cam->type != NIS_CAMERA_ORTHO && cam->type != NIS_CAMERA_PERSP)
        return fail(ctx, NIS_ERR_INVALID_ARG, "bad camera type");
    for (int q = 0; q < 3; ++q)
        if (!std::isfinite(cam->eye[q]) || !std::isfinite(cam->target[q]) || !std::isfinite(cam->up[q]) ||
            std::fabs(cam->eye[q]) > 1e6f || std::fabs(cam->target[q]) > 1e6f)
            return fail(ctx, NIS_ERR_INVALID_ARG, "camera vectors must be finite (|x| <= 1e6)");
    double f[3], up[3], r[3], u[3];
    for (int q = 0; q < 3; ++q) { f[q] = (double)cam->target[q] - cam->eye[q]; up[q] = cam->up[q]; }
    double nf = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(nf > 0)) return fail(ctx, NIS_ERR_INVALID_ARG, "eye equals target");
    for (double &x : f) x /= nf;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double nr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(nr > 1e-12)) return fail(ctx, NIS_ERR_INVALID_ARG, "up is parallel to the view");
    for (double &x : r) x /= nr;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    c->type = cam->type; c->width = cam->width; c->height = cam->height;
    for (int q = 0; q < 3; ++q) {
        c->eye[q] = cam->eye[q]; c->fwd[q] = (float)f[q]; c->right[q] = (float)r[q]; c->up[q] = (float)u[q];
    }
    c->tan_half = (float)std::tan(0.5 * (double)cam->fov_y);
    c->aspect = (float)((double)cam->width / cam->height);
    c->half_h = 0.5f * cam->ortho_height;
    if (cam->type == NIS_CAMERA_PERSP && !(cam->fov_y > 0.f && cam->fov_y < 3.1f))
        return fail(ctx, NIS_ERR_INVALID_ARG, "fov_y must lie in (0, 3.1) radians");
    if (cam->type == NIS_CAMERA_ORTHO && !(cam->ortho_height > 0.f))
        return fail(ctx, NIS_ERR_INVALID_ARG, "ortho_height must be positive");
    return NIS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace nis {

const char *material_problem(const nis_material *m) {
    if (!m) return "material is NULL";
    if (!(m->g > -1.f && m->g < 1.f)) return "g must lie in (-1, 1)";
    if (m->n_lobes < 0 || m->n_lobes > 3) return "n_lobes must be 0..3";
    if (m->n_lobes >= 2) {
        float sum = 0.f;
        for (int i = 0; i < m->n_lobes; ++i) {
            if (!(m->lobe_g[i] > -1.f && m->lobe_g[i] < 1.f) || !(m->lobe_w[i] >= 0.f))
                return "lobe g must lie in (-1, 1), weights >= 0";
            sum += m->lobe_w[i];
        }
        if (std::fabs(sum - 1.f) > 1e-4f) return "lobe weights must sum to 1";
    }
    for (int c = 0; c < 3; ++c)
        if (!(m->albedo[c] > 0.f && m->albedo[c] <= 1.f) || !std::isfinite(m->intensity[c]))
            return "albedo must lie in (0, 1], intensity finite";
    return nullptr;
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}
}  // namespace

bool make_tmap_u8(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                  uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_ht(CUtensorMap *map, const float *H_T, uint64_t points) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(H_T) & 15)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kLatT, (cuuint64_t)kLayers, points};
    cuuint64_t strides[2] = {(cuuint64_t)kLatT * 4, (cuuint64_t)kLayers * kLatT * 4};
    cuuint32_t box[3] = {(cuuint32_t)kLatT, 1, 16};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(H_T), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_bf16(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                    uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
    EncodeTiledFn fn = encode_tiled();
    if (box_inner != 16 && box_inner != 32 && box_inner != 64) return false;   // swizzled rows
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              box_inner == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                              : (box_inner == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B),
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_out(CUtensorMap *map, const void *base, bool f32, uint64_t cols, uint64_t rows,
                   uint32_t parts, uint64_t row_bytes, uint64_t part_bytes) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || (part_bytes & 15) ||
        parts < 1 || parts > 3)
        return false;
    cuuint64_t dims[3] = {cols, rows, parts};
    cuuint64_t strides[2] = {row_bytes, part_bytes};
    cuuint32_t box[3] = {32, 32, parts};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
              const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

nis_status record_error(nis_ctx *ctx, nis_status s, const char *msg) { return fail(ctx, s, msg); }
int ctx_device(const nis_ctx *ctx) { return ctx->device; }

nis_status hits_compact(nis_ctx *ctx, nis_volume vol, const nis_camera *cam, float *pts,
                        float *om, int *pix, int *d_count, cudaStream_t s) {
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    CameraArgs c;
    nis_status st = camera_args(ctx, cam, &c);
    if (st) return st;
    NIS_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
    {
        ProfScope ps(ctx, "hits", s);
        launch_find_hits(v->data, v->pyramid ? v->occ : nullptr, v->n, v->sigma_max, c, nullptr, pts,
                         om, pix, d_count, s);
    }
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

nis_status resolve_built_inputs(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                                const nis_material *m, ResolvedInputs *out) {
    Volume *pv; Light *pl; Weights *pw;
    nis_status st = resolve(ctx, vol, light, w, &pv, &pl, &pw);
    if (st) return st;
    const PhaseSpec ph = phase_spec(m);
    std::vector<uint32_t> key(1 + 2 * ph.n);
    key[0] = (uint32_t)ph.n;
    for (int i = 0; i < ph.n; ++i) {
        std::memcpy(&key[1 + 2 * i], &ph.g[i], 4);
        std::memcpy(&key[2 + 2 * i], &ph.w[i], 4);
    }
    auto it = ctx->phase.find(key);
    if (it == ctx->phase.end())
        return fail(ctx, NIS_ERR_NOT_READY, "phase table for this material not built "
                                            "(shade once, or call nis_build_phase_table)");
    if (!pl->pairs || pl->pair_version != pv->version)
        return fail(ctx, NIS_ERR_NOT_READY, "light older than the volume's pyramid "
                                            "(rebuild it, or shade once through nis_shade_points)");
    out->rho = view_of(*pv, pv->data);
    out->T = view_of(*pv, pl->data);
    out->rt = pair_view(*pv, *pl);
    out->table = it->second;
    out->W = pw->f32;
    out->off = pw->off;
    for (int c = 0; c < 3; ++c) out->dir[c] = pl->dir[c];
    out->device = ctx->device;
    return NIS_OK;
}

void weight_offsets_paper(WeightOffsets *o) {
    size_t p = 0;
    o->model = kModelPaper;
    o->level_w = p; p += kLevelWeights;
    o->level_b = p; p += 1;
    for (int k = 0; k < kLayers; ++k) o->cnn_w1[k] = o->cnn_b1[k] = o->cnn_w2[k] = o->cnn_b2[k] = 0;
    for (int k = 0; k < kLayers; ++k) {
        o->se_w1[k] = p; p += 2 * 8;
        o->se_b1[k] = p; p += 2;
        o->se_w2[k] = p; p += 3 * 2;
        o->se_b2[k] = p; p += 3;
    }
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < kLayers; ++k) {
            const int d = paper_count(k);
            o->blk_w1[t][k] = p; p += (size_t)kWidth * (d + kCfg);
            o->blk_b1[t][k] = p; p += kWidth;
            o->blk_w2[t][k] = p; p += (size_t)kWidth * kWidth;
            o->blk_b2[t][k] = p; p += kWidth;
        }
    for (int t = 0; t < 3; ++t) {
        o->mrg_w[t] = p; p += (size_t)kWidth * 2 * kWidth;
        o->mrg_b[t] = p; p += kWidth;
    }
    o->head_w[0] = p; p += (size_t)kWidth * 3 * kWidth;
    o->head_b[0] = p; p += kWidth;
    o->head_w[1] = p; p += (size_t)kWidth * kWidth;
    o->head_b[1] = p; p += kWidth;
    o->head_w[2] = p; p += 3 * kWidth;
    o->head_b[2] = p; p += 3;
    o->total = p;
}

void weight_offsets(WeightOffsets *o) {
    size_t p = 0;
    for (int k = 0; k < kLayers; ++k) {
        o->cnn_w1[k] = p; p += kCnnCh * 27;
        o->cnn_b1[k] = p; p += kCnnCh;
        o->cnn_w2[k] = p; p += kCnnCh * kCnnCh * 27;
        o->cnn_b2[k] = p; p += kCnnCh;
    }
    for (int k = 0; k < kLayers; ++k) {
        o->se_w1[k] = p; p += 2 * 8;
        o->se_b1[k] = p; p += 2;
        o->se_w2[k] = p; p += 3 * 2;
        o->se_b2[k] = p; p += 3;
    }
    for (int t = 0; t < 3; ++t)
        for (int k = 0; k < kLayers; ++k) {
            int d = feat_dim(t);
            o->blk_w1[t][k] = p; p += (size_t)kWidth * (d + kCfg);
            o->blk_b1[t][k] = p; p += kWidth;
            o->blk_w2[t][k] = p; p += (size_t)kWidth * kWidth;
            o->blk_b2[t][k] = p; p += kWidth;
        }
    for (int t = 0; t < 3; ++t) {
        o->mrg_w[t] = p; p += (size_t)kWidth * 2 * kWidth;
        o->mrg_b[t] = p; p += kWidth;
    }
    o->head_w[0] = p; p += (size_t)kWidth * 3 * kWidth;
    o->head_b[0] = p; p += kWidth;
    o->head_w[1] = p; p += (size_t)kWidth * kWidth;
    o->head_b[1] = p; p += kWidth;
    o->head_w[2] = p; p += 3 * kWidth;
    o->head_b[2] = p; p += 3;
    o->total = p;
}
int weights_model(nis_ctx *ctx, nis_weights w) {
    Weights *pw = lookup(ctx->weights, w);
    return pw ? pw->off.model : -1;
}

}  // namespace nis

extern "C" {

nis_status nis_create(nis_ctx **out, int device, size_t hbm_budget_bytes,
                      const nis_allocator *alloc) {
    if (!out) { g_create_error = "out is NULL"; return NIS_ERR_INVALID_ARG; }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = std::string("no CUDA device ") + std::to_string(device) +
                         (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
        cudaGetLastError();
        return NIS_ERR_CUDA;
    }
    if (alloc && (!alloc->alloc != !alloc->free)) {
        g_create_error = "allocator needs both callbacks";
        return NIS_ERR_INVALID_ARG;
    }
    nis_ctx *ctx = new nis_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    if (alloc && alloc->alloc) { ctx->alloc = *alloc; ctx->custom_alloc = true; }
    DeviceGuard g(device);
    void *p;
    if (dev_alloc(ctx, sizeof(unsigned), &p, nullptr) != NIS_OK) {
        g_create_error = ctx->err;
        delete ctx;
        return NIS_ERR_OOM;
    }
    ctx->d_err = static_cast<unsigned *>(p);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&ctx->ws.host_count, sizeof(int)) != cudaSuccess) {
        g_create_error = "device set-up failed";
        cudaGetLastError();
        dev_free(ctx, ctx->d_err);
        delete ctx;
        return NIS_ERR_CUDA;
    }
    *out = ctx;
    return NIS_OK;
}

void nis_destroy(nis_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    std::vector<void *> ptrs;
    for (auto &kv : ctx->allocs) ptrs.push_back(kv.first);
    for (void *p : ptrs) dev_free(ctx, p);
    if (ctx->ws.host_count) cudaFreeHost(ctx->ws.host_count);
    for (auto &kv : ctx->prof)
        for (auto &e : kv.second) { cudaEventDestroy(e.e0); cudaEventDestroy(e.e1); }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
}

const char *nis_last_error(const nis_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

size_t nis_bytes_in_use(const nis_ctx *ctx) { return ctx ? ctx->in_use : 0; }

nis_status nis_upload_volume(nis_ctx *ctx, const void *density, int nx, int ny, int nz,
                             int dtype, int src_is_device, float sigma_scale, nis_stream stream,
                             nis_volume *out) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!density || !out) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL density or out");
    if (nx != ny || ny != nz) return fail(ctx, NIS_ERR_INVALID_ARG, "grid must be cubic");
    if (nx < 1 || nx > 2048) return fail(ctx, NIS_ERR_INVALID_ARG, "grid size must be 1..2048");
    if (dtype != NIS_DTYPE_F32 && dtype != NIS_DTYPE_F16)
        return fail(ctx, NIS_ERR_INVALID_ARG, "dtype must be F32 or F16");
    if (!(sigma_scale >= 0.f) || !std::isfinite(sigma_scale))
        return fail(ctx, NIS_ERR_INVALID_ARG, "sigma_scale must be finite and >= 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Volume v;
    v.n = nx;
    int sz = nx;
    size_t total = 0;
    while (true) {
        v.sizes[v.levels] = sz;
        v.off[v.levels] = total;
        total += (size_t)sz * sz * sz;
        ++v.levels;
        if (sz == 1) break;
        sz = (sz + 1) / 2;
    }
    v.total = total;
    nis_status st = dev_alloc_t(ctx, total, &v.data, s);
    if (st) return st;
    if ((st = dev_alloc_t(ctx, 1, &v.sigma_max, s))) { dev_free(ctx, v.data); return st; }
    size_t count = (size_t)nx * nx * nx;
    size_t elem = dtype == NIS_DTYPE_F16 ? 2 : 4;
    const void *src = density;
    void *staging = nullptr;
    if (!src_is_device) {
        cudaPointerAttributes attr{};
        void *mapped = nullptr;
        if (cudaPointerGetAttributes(&attr, density) == cudaSuccess &&
            attr.type == cudaMemoryTypeHost &&
            cudaHostGetDevicePointer(&mapped, const_cast<void *>(density), 0) == cudaSuccess) {
            src = mapped;                   // page-locked: the conversion kernel reads it in place
        } else {
            cudaGetLastError();
            // pageable: stream-ordered staging (no device-wide synchronisation); the copy
            // has consumed the caller's buffer when cudaMemcpyAsync returns
            cudaError_t e = cudaMallocAsync(&staging, count * elem, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(staging, density, count * elem, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                if (staging) cudaFreeAsync(staging, s);
                dev_free(ctx, v.data); dev_free(ctx, v.sigma_max);
                return cuda_fail(ctx, e, "density upload");
            }
            src = staging;
        }
    }
    {
        ProfScope ps(ctx, "other", s);
        launch_convert_density(src, dtype, sigma_scale, count, v.data, ctx->d_err, v.sigma_max, s);
    }
    cudaError_t e = cudaGetLastError();
    if (staging) cudaFreeAsync(staging, s);
    if (e != cudaSuccess) {
        dev_free(ctx, v.data); dev_free(ctx, v.sigma_max);
        return cuda_fail(ctx, e, "convert_density");
    }
    nis_handle h = ctx->next++;
    ctx->vols[h] = v;
    *out = h;
    return NIS_OK;
}

nis_status nis_build_pyramid(nis_ctx *ctx, nis_volume vol, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    DeviceGuard g(ctx->device);
    return build_pyramid_impl(ctx, *v, reinterpret_cast<cudaStream_t>(stream));
}

nis_status nis_build_transmittance(nis_ctx *ctx, nis_volume vol, const float light_dir[3],
                                   float lambda, nis_stream stream, nis_light *out) {
    return nis_build_transmittance_method(ctx, vol, light_dir, lambda, NIS_TRANSMITTANCE_MARCH,
                                          stream, out);
}

nis_status nis_build_transmittance_method(nis_ctx *ctx, nis_volume vol, const float light_dir[3],
                                          float lambda, int method, nis_stream stream,
                                          nis_light *out) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!light_dir || !out) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL light_dir or out");
    if (method != NIS_TRANSMITTANCE_MARCH && method != NIS_TRANSMITTANCE_SHEAR_WARP)
        return fail(ctx, NIS_ERR_INVALID_ARG, "unknown transmittance method");
    if (!(lambda > 0.f && lambda <= 1.f)) return fail(ctx, NIS_ERR_INVALID_ARG, "lambda must lie in (0, 1]");
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    double l[3] = {light_dir[0], light_dir[1], light_dir[2]};
    double nl = std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    if (!(nl > 0) || !std::isfinite(nl)) return fail(ctx, NIS_ERR_INVALID_ARG, "light_dir must be finite and non-zero");
    float dir[3] = {(float)(l[0] / nl), (float)(l[1] / nl), (float)(l[2] / nl)};
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    nis_status st;
    if (!v->pyramid && (st = build_pyramid_impl(ctx, *v, s))) return st;
    nis_handle h = 0;
    for (auto &kv : ctx->lights)
        if (kv.second.vol == vol && kv.second.lambda == lambda && kv.second.method == method &&
            std::memcmp(kv.second.dir, dir, sizeof(dir)) == 0) { h = kv.first; break; }
    if (!h) {
        Light L;
        L.vol = vol;
        std::memcpy(L.dir, dir, sizeof(dir));
        L.lambda = lambda;
        L.method = method;
        if ((st = dev_alloc_t(ctx, v->total, &L.data, s))) return st;
        h = ctx->next++;
        ctx->lights[h] = L;
    }
    Light &L = ctx->lights[h];
    // u = -l points toward the light
    if (method == NIS_TRANSMITTANCE_MARCH) {
        for (int m = 0; m < v->levels; ++m) {
            ProfScope ps(ctx, "march", s);
            launch_march(v->data + v->off[m], v->occ + v->occ_off[m], v->sizes[m], m, -dir[0],
                         -dir[1], -dir[2], lambda, L.data + v->off[m], s);
        }
    } else {
        ShearWarpArgs sw{};
        size_t rays[kMaxLevels] = {}, total = 0;
        shear_warp_setup(sw, v->sizes, v->levels, -dir[0], -dir[1], -dir[2], lambda, rays);
        for (int m = 0; m < v->levels; ++m) total += rays[m];
        ProfScope ps(ctx, "march", s);
        // slices normal to x are strided in [z][y][x]: sweep the x-major copy instead, as a
        // cube whose (x, y, z) are the volume's (y, z, x), and transpose the result back
        const bool xmajor = sw.ax_a == 0;
        if (xmajor) {
            if ((st = ensure_xmajor(ctx, *v, s))) return st;
            if (ctx->sw_T_cap < v->total) {
                dev_free(ctx, ctx->sw_T);
                ctx->sw_T = nullptr;
                ctx->sw_T_cap = 0;
                if ((st = dev_alloc_t(ctx, v->total, &ctx->sw_T, s))) return st;
                ctx->sw_T_cap = v->total;
            }
            sw.ax_a = 2;
            sw.ax_p = 0;
            sw.ax_q = 1;
            const float ux = sw.ux, iux = sw.iux;
            sw.ux = sw.uy; sw.iux = sw.iuy;
            sw.uy = sw.uz; sw.iuy = sw.iuz;
            sw.uz = ux;    sw.iuz = iux;
        }
        if (ctx->sw_cap < total) {
            dev_free(ctx, ctx->sw_rays);
            ctx->sw_rays = nullptr;
            ctx->sw_cap = 0;
            if ((st = dev_alloc_t(ctx, total, &ctx->sw_rays, s))) return st;
            ctx->sw_cap = total;
        }
        // rays outside a step's window keep their state: all start as not having met the cube
        NIS_CUDA(cudaMemsetAsync(ctx->sw_rays, 0, total * sizeof(float), s));
        float *r = ctx->sw_rays;
        for (int m = 0; m < v->levels; ++m) {
            ShearWarpLevel &Lm = sw.lv[m];
            Lm.rho = (xmajor ? v->xmaj : v->data) + v->off[m];
            Lm.occ = (xmajor ? v->xmaj_occ : v->occ) + v->occ_off[m];
            Lm.T = (xmajor ? ctx->sw_T : L.data) + v->off[m];
            Lm.ray = reinterpret_cast<float2 *>(r);
            r += rays[m];
        }
        launch_shear_warp(sw, s);
        if (xmajor)
            for (int m = 0; m < v->levels; ++m) {
                const size_t n = (size_t)v->sizes[m];
                launch_transpose(ctx->sw_T + v->off[m], n, n * n, L.data + v->off[m], s);
            }
    }
    NIS_CUDA(cudaGetLastError());
    L.pair_version = 0;                       // new transmittance: re-pack
    if ((st = ensure_pairs(ctx, *v, L, s))) return st;
    *out = h;
    return NIS_OK;
}

nis_status nis_load_weights(nis_ctx *ctx, const void *blob, size_t bytes, int precision,
                            nis_stream stream, nis_weights *out) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!blob || !out) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL blob or out");
    if (precision != NIS_PREC_F32 && precision != NIS_PREC_BF16 && precision != NIS_PREC_F32_SIMT &&
        precision != NIS_PREC_FP8)
        return fail(ctx, NIS_ERR_INVALID_ARG, "precision must be F32, BF16, FP8 or F32_SIMT");
    if (bytes < 80) return fail(ctx, NIS_ERR_BAD_BLOB, "blob shorter than its header");
    uint32_t hd[16];
    uint64_t n_floats, checksum;
    std::memcpy(hd, blob, 64);
    std::memcpy(&n_floats, static_cast<const char *>(blob) + 64, 8);
    std::memcpy(&checksum, static_cast<const char *>(blob) + 72, 8);
    WeightOffsets o;
    const bool paper = hd[2] == (uint32_t)kModelPaper;
    if (paper) weight_offsets_paper(&o);
    else weight_offsets(&o);
    const uint32_t expect[13] = {0x5753494Eu, 1u, paper ? 1u : 0u, 80u, (uint32_t)kLayers,
                                 (uint32_t)kDiffuse, paper ? (uint32_t)kPaperPts : (uint32_t)kLat,
                                 paper ? 0u : (uint32_t)kCnnCh, 2u, (uint32_t)kWidth,
                                 (uint32_t)kCfg, 3u, paper ? (uint32_t)kLevelWeights : (uint32_t)kDT};
    for (int i = 0; i < 13; ++i)
        if (hd[i] != expect[i])
            return fail(ctx, NIS_ERR_BAD_BLOB, "blob header field " + std::to_string(i) + " mismatch");
    if (paper && precision == NIS_PREC_FP8)
        return fail(ctx, NIS_ERR_UNIMPLEMENTED, "the paper-template model runs in FP32 or BF16");
    if (n_floats != o.total || bytes != 80 + 4 * n_floats)
        return fail(ctx, NIS_ERR_BAD_BLOB, "blob size does not match the network shape");
    const uint32_t *words = reinterpret_cast<const uint32_t *>(static_cast<const char *>(blob) + 80);
    uint64_t sum = 0;
    for (uint64_t i = 0; i < n_floats; ++i) sum += (uint64_t)words[i] * (2 * i + 1);
    if (sum != checksum) return fail(ctx, NIS_ERR_BAD_BLOB, "blob checksum mismatch");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Weights w;
    w.precision = precision;
    w.off = o;
    nis_status st = dev_alloc_t(ctx, o.total, &w.f32, s);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(w.f32, words, o.total * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the caller may free the blob
    if (e != cudaSuccess) { dev_free(ctx, w.f32); return cuda_fail(ctx, e, "weights upload"); }
    if (precision == NIS_PREC_FP8) {
        st = pack_weights_fp8(ctx, w, s);
        if (!st) {
            // the fused backbone's e4m3 mode: per layer, the FC-1 weight scale of the density and
            // phase features (largest magnitude / 448, the e4m3 maximum)
            for (int k = 0; k < kLayers; ++k)
                for (int t = 0; t < 2; ++t) {
                    const int d = feat_dim(t);
                    float mx = 0.f;
                    for (int n = 0; n < kWidth; ++n)
                        for (int kk = 0; kk < d; ++kk) {
                            float x;
                            std::memcpy(&x, words + o.blk_w1[t][k] + (size_t)n * (d + kCfg) + kk, 4);
                            mx = std::max(mx, std::fabs(x));
                        }
                    w.f8_sw[k][t] = mx > 0.f ? mx / 448.f : 1.f;
                }
            st = pack_fused(ctx, w, w.f8_sw, s);
        }
    } else if (precision != NIS_PREC_F32_SIMT) st = pack_weights_tc(ctx, w, precision == NIS_PREC_F32 ? 3 : 1, s);
    if (st) {
        dev_free(ctx, w.f32);
        dev_free(ctx, w.bf);
        dev_free(ctx, w.f8);
        dev_free(ctx, w.f8_scales);
        dev_free(ctx, w.fused_w);
        dev_free(ctx, w.fused_ops);
        dev_free(ctx, w.fused_pack);
        return st;
    }
    nis_handle h = ctx->next++;
    ctx->weights[h] = w;
    *out = h;
    return NIS_OK;
}

nis_status nis_shade_points_debug(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                                  const nis_material *m, const float *d_points,
                                  const float *d_omega, int n, float *d_rgb_out,
                                  const nis_debug_out *dbg, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, NIS_ERR_INVALID_ARG, "n must be >= 0");
    if (n > 0 && (!d_points || !d_omega || !d_rgb_out))
        return fail(ctx, NIS_ERR_INVALID_ARG, "NULL points, omega or output");
    nis_status st = check_material(ctx, m);
    if (st) return st;
    Volume *pv; Light *pl; Weights *pw;
    if ((st = resolve(ctx, vol, light, w, &pv, &pl, &pw))) return st;
    if (n == 0) return NIS_OK;
    DeviceGuard g(ctx->device);
    if ((st = ensure_pairs(ctx, *pv, *pl, reinterpret_cast<cudaStream_t>(stream)))) return st;
    return shade_impl(ctx, *pv, *pl, *pw, m, d_points, d_omega, n, d_rgb_out, dbg,
                      reinterpret_cast<cudaStream_t>(stream));
}

nis_status nis_shade_points(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                            const nis_material *m, const float *d_points, const float *d_omega,
                            int n, float *d_rgb_out, nis_stream stream) {
    return nis_shade_points_debug(ctx, vol, light, w, m, d_points, d_omega, n, d_rgb_out, nullptr,
                                  stream);
}

nis_status nis_find_hits(nis_ctx *ctx, nis_volume vol, const nis_camera *cam, int *d_hit,
                         float *d_points, float *d_omega, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!d_hit || !d_points || !d_omega) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL output");
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    CameraArgs c;
    nis_status st = camera_args(ctx, cam, &c);
    if (st) return st;
    DeviceGuard g(ctx->device);
    launch_find_hits(v->data, v->pyramid ? v->occ : nullptr, v->n, v->sigma_max, c, d_hit, d_points,
                     d_omega, nullptr, nullptr,
                     reinterpret_cast<cudaStream_t>(stream));
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

// Hit-list buffers of a frame of `pixels` pixels (grow-only).
nis_status ensure_hit_ws(nis_ctx *ctx, int pixels, cudaStream_t s) {
    Workspace &ws = ctx->ws;
    if (ws.hit_cap >= pixels) return NIS_OK;
    nis_status st;
    dev_free(ctx, ws.hit_pts); dev_free(ctx, ws.hit_omega); dev_free(ctx, ws.hit_rgb);
    dev_free(ctx, ws.hit_pix); dev_free(ctx, ws.hit_count);
    ws.hit_pts = ws.hit_omega = ws.hit_rgb = nullptr;
    ws.hit_pix = ws.hit_count = nullptr;
    ws.hit_cap = 0;
    if ((st = dev_alloc_t(ctx, 3 * (size_t)pixels, &ws.hit_pts, s))) return st;
    if ((st = dev_alloc_t(ctx, 3 * (size_t)pixels, &ws.hit_omega, s))) return st;
    if ((st = dev_alloc_t(ctx, 3 * (size_t)pixels, &ws.hit_rgb, s))) return st;
    if ((st = dev_alloc_t(ctx, (size_t)pixels, &ws.hit_pix, s))) return st;
    if ((st = dev_alloc_t(ctx, 1, &ws.hit_count, s))) return st;
    ws.hit_cap = pixels;
    return NIS_OK;
}

// Per-pixel hit list of the frame split (grow-only): flags, points, directions, block counts
// and their offsets.
nis_status ensure_px_ws(nis_ctx *ctx, int pixels, cudaStream_t s) {
    Workspace &ws = ctx->ws;
    if (ws.px_cap >= pixels) return NIS_OK;
    nis_status st;
    dev_free(ctx, ws.px_flag); dev_free(ctx, ws.px_blk); dev_free(ctx, ws.px_off);
    dev_free(ctx, ws.px_pts); dev_free(ctx, ws.px_om);
    ws.px_flag = ws.px_blk = ws.px_off = nullptr;
    ws.px_pts = ws.px_om = nullptr;
    ws.px_cap = 0;
    const size_t nb = ((size_t)pixels + 255) / 256;
    if ((st = dev_alloc_t(ctx, (size_t)pixels, &ws.px_flag, s))) return st;
    if ((st = dev_alloc_t(ctx, nb, &ws.px_blk, s))) return st;
    if ((st = dev_alloc_t(ctx, nb + 1, &ws.px_off, s))) return st;
    if ((st = dev_alloc_t(ctx, 3 * (size_t)pixels, &ws.px_pts, s))) return st;
    if ((st = dev_alloc_t(ctx, 3 * (size_t)pixels, &ws.px_om, s))) return st;
    ws.px_cap = pixels;
    return NIS_OK;
}

// Frame for one or more lights: the shading points (first hits) do not depend on the light;
// each light's radiance is shaded with its own transmittance and added to the pixels.
nis_status render_impl(nis_ctx *ctx, nis_volume vol, const nis_light *lights, int n_lights,
                       nis_weights w, const nis_material *m, const nis_camera *cam,
                       float *d_rgb_out, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!d_rgb_out) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL output");
    if (!lights || n_lights < 1) return fail(ctx, NIS_ERR_INVALID_ARG, "no light");
    nis_status st = check_material(ctx, m);
    if (st) return st;
    CameraArgs c;
    if ((st = camera_args(ctx, cam, &c))) return st;
    Volume *pv; Light *pl; Weights *pw;
    std::vector<Light *> ls(n_lights);
    for (int q = 0; q < n_lights; ++q) {
        if ((st = resolve(ctx, vol, lights[q], w, &pv, &pl, &pw))) return st;
        ls[q] = pl;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (Light *l : ls)
        if ((st = ensure_pairs(ctx, *pv, *l, s))) return st;
    Workspace &ws = ctx->ws;
    int pixels = c.width * c.height;
    if ((st = ensure_hit_ws(ctx, pixels, s)) || (st = ensure_px_ws(ctx, pixels, s))) return st;
    // the shading points in pixel order: neighbouring points of the list are neighbouring
    // pixels, which the gathers' lane mapping relies on for coherent loads
    {
        ProfScope ps(ctx, "hits", s);
        launch_find_hits_ordered(pv->data, pv->pyramid ? pv->occ : nullptr, pv->n, pv->sigma_max, c,
                                 ws.px_flag, ws.px_pts,
                                 ws.px_om, ws.px_blk, ws.px_off, ws.hit_count, s);
    }
    NIS_CUDA(cudaGetLastError());
    NIS_CUDA(cudaMemcpyAsync(ws.host_count, ws.hit_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    NIS_CUDA(cudaStreamSynchronize(s));
    int count = *ws.host_count;
    if (count > 0) {
        ProfScope ps(ctx, "hits", s);
        launch_hits_range(ws.px_flag, ws.px_pts, ws.px_om, ws.px_off, pixels, 0, count,
                          ws.hit_pts, ws.hit_omega, ws.hit_pix, s);
    }
    NIS_CUDA(cudaGetLastError());
    NIS_CUDA(cudaMemsetAsync(d_rgb_out, 0, sizeof(float) * 3 * (size_t)pixels, s));
    if (count > 0) {
        for (int q = 0; q < n_lights; ++q) {
            if ((st = shade_impl(ctx, *pv, *ls[q], *pw, m, ws.hit_pts, ws.hit_omega, count, ws.hit_rgb,
                                 nullptr, s)))
                return st;
            ProfScope ps(ctx, "other", s);
            launch_scatter_rgb(ws.hit_rgb, ws.hit_pix, count, d_rgb_out, pixels, s, q > 0);
        }
        NIS_CUDA(cudaGetLastError());
    }
    return NIS_OK;
}

nis_status nis_render_frame(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                            const nis_material *m, const nis_camera *cam, float *d_rgb_out,
                            nis_stream stream) {
    return render_impl(ctx, vol, &light, 1, w, m, cam, d_rgb_out, stream);
}

nis_status nis_render_frame_lights(nis_ctx *ctx, nis_volume vol, const nis_light *lights,
                                   int n_lights, nis_weights w, const nis_material *m,
                                   const nis_camera *cam, float *d_rgb_out, nis_stream stream) {
    if (ctx && n_lights > 64) return fail(ctx, NIS_ERR_INVALID_ARG, "at most 64 lights");
    return render_impl(ctx, vol, lights, n_lights, w, m, cam, d_rgb_out, stream);
}

nis_status nis_part_range(long long n, int part, int parts, long long *first, long long *count) {
    if (n < 0 || parts < 1 || part < 0 || part >= parts || !first || !count)
        return NIS_ERR_INVALID_ARG;
    // floor(p * n / parts) without overflow: n = q * parts + r
    const long long q = n / parts, r = n % parts;
    auto start = [&](long long p) { return p * q + p * r / parts; };
    *first = start(part);
    *count = start(part + 1) - *first;
    return NIS_OK;
}

nis_status nis_render_frame_part(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                                 const nis_material *m, const nis_camera *cam, int part,
                                 int parts, float *d_rgb, int *d_pix, int capacity, int *n_hits,
                                 int *first, int *count, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (parts < 1 || part < 0 || part >= parts)
        return fail(ctx, NIS_ERR_INVALID_ARG, "part outside [0, parts)");
    if (!d_rgb || !d_pix || !n_hits || !first || !count || capacity < 0)
        return fail(ctx, NIS_ERR_INVALID_ARG, "NULL output or negative capacity");
    nis_status st = check_material(ctx, m);
    if (st) return st;
    CameraArgs c;
    if ((st = camera_args(ctx, cam, &c))) return st;
    Volume *pv; Light *pl; Weights *pw;
    if ((st = resolve(ctx, vol, light, w, &pv, &pl, &pw))) return st;
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((st = ensure_pairs(ctx, *pv, *pl, s))) return st;
    const int pixels = c.width * c.height;
    if ((st = ensure_hit_ws(ctx, pixels, s)) || (st = ensure_px_ws(ctx, pixels, s))) return st;
    Workspace &ws = ctx->ws;
    {
        ProfScope ps(ctx, "hits", s);
        launch_find_hits_ordered(pv->data, pv->pyramid ? pv->occ : nullptr, pv->n, pv->sigma_max, c,
                                 ws.px_flag, ws.px_pts,
                                 ws.px_om, ws.px_blk, ws.px_off, ws.hit_count, s);
    }
    NIS_CUDA(cudaGetLastError());
    NIS_CUDA(cudaMemcpyAsync(ws.host_count, ws.hit_count, sizeof(int), cudaMemcpyDeviceToHost, s));
    NIS_CUDA(cudaStreamSynchronize(s));
    const int hits = *ws.host_count;
    long long f, k;
    nis_part_range(hits, part, parts, &f, &k);
    *n_hits = hits;
    *first = (int)f;
    *count = (int)k;
    if (k > capacity) return fail(ctx, NIS_ERR_INVALID_ARG, "capacity below the part's hit count");
    if (k == 0) return NIS_OK;
    {
        ProfScope ps(ctx, "hits", s);
        launch_hits_range(ws.px_flag, ws.px_pts, ws.px_om, ws.px_off, pixels, f, (int)k,
                          ws.hit_pts, ws.hit_omega, d_pix, s);
    }
    NIS_CUDA(cudaGetLastError());
    return shade_impl(ctx, *pv, *pl, *pw, m, ws.hit_pts, ws.hit_omega, (int)k, d_rgb, nullptr, s);
}

nis_status nis_scatter_part(nis_ctx *ctx, const float *d_rgb, const int *d_pix, int n,
                            float *d_image, int n_pixels, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (n < 0 || n_pixels < 0 || (n > 0 && (!d_rgb || !d_pix || !d_image)))
        return fail(ctx, NIS_ERR_INVALID_ARG, "NULL buffer or negative size");
    if (n == 0) return NIS_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        ProfScope ps(ctx, "other", s);
        launch_scatter_rgb(d_rgb, d_pix, n, d_image, n_pixels, s);
    }
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

nis_status nis_release(nis_ctx *ctx, nis_handle h) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (Volume *v = lookup(ctx->vols, h)) {
        cudaDeviceSynchronize();
        std::vector<nis_handle> dead;
        for (auto &kv : ctx->lights)
            if (kv.second.vol == h) {
                dev_free(ctx, kv.second.data);
                dev_free(ctx, kv.second.pairs);
                dead.push_back(kv.first);
            }
        for (nis_handle d : dead) ctx->lights.erase(d);
        dev_free(ctx, v->data);
        dev_free(ctx, v->sigma_max);
        dev_free(ctx, v->staging);
        dev_free(ctx, v->occ);
        dev_free(ctx, v->xmaj);
        dev_free(ctx, v->xmaj_occ);
        ctx->vols.erase(h);
        return NIS_OK;
    }
    if (Light *l = lookup(ctx->lights, h)) {
        cudaDeviceSynchronize();
        dev_free(ctx, l->data);
        dev_free(ctx, l->pairs);
        ctx->lights.erase(h);
        return NIS_OK;
    }
    if (Weights *w = lookup(ctx->weights, h)) {
        cudaDeviceSynchronize();
        dev_free(ctx, w->f32);
        dev_free(ctx, w->bf);
        dev_free(ctx, w->f8);
        dev_free(ctx, w->f8_scales);
        dev_free(ctx, w->fused_w);
        dev_free(ctx, w->fused_ops);
        dev_free(ctx, w->fused_pack);
        ctx->weights.erase(h);
        return NIS_OK;
    }
    return fail(ctx, NIS_ERR_INVALID_ARG, "unknown handle");
}

nis_status nis_sync(nis_ctx *ctx, nis_stream stream, int timeout_ms) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto start = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream");
        if (timeout_ms > 0 &&
            std::chrono::steady_clock::now() - start > std::chrono::milliseconds(timeout_ms))
            return fail(ctx, NIS_ERR_TIMEOUT, "stream did not finish within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    unsigned err = 0;
    NIS_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) {
        NIS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
        if (err & kErrTimeout)
            return fail(ctx, NIS_ERR_TIMEOUT, "a tensor-core kernel's bounded wait gave up");
        if (err & kErrBadDensity)
            return fail(ctx, NIS_ERR_BAD_DATA, "density contained NaN, infinite or negative values");
        return fail(ctx, NIS_ERR_BAD_DATA, "a kernel bounds check failed");
    }
    return NIS_OK;
}

nis_status nis_volume_info(nis_ctx *ctx, nis_volume vol, int *levels, int sizes[16],
                           float *sigma_max) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    DeviceGuard g(ctx->device);
    if (levels) *levels = v->levels;
    if (sizes) for (int m = 0; m < kMaxLevels; ++m) sizes[m] = m < v->levels ? v->sizes[m] : 0;
    if (sigma_max) NIS_CUDA(cudaMemcpy(sigma_max, v->sigma_max, sizeof(float), cudaMemcpyDeviceToHost));
    return NIS_OK;
}

nis_status nis_copy_level(nis_ctx *ctx, nis_volume vol, int level, float *d_dst,
                          nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    if (level < 0 || level >= v->levels || !d_dst) return fail(ctx, NIS_ERR_INVALID_ARG, "bad level or NULL dst");
    DeviceGuard g(ctx->device);
    size_t n = (size_t)v->sizes[level] * v->sizes[level] * v->sizes[level];
    NIS_CUDA(cudaMemcpyAsync(d_dst, v->data + v->off[level], n * 4, cudaMemcpyDeviceToDevice,
                             reinterpret_cast<cudaStream_t>(stream)));
    return NIS_OK;
}

nis_status nis_copy_transmittance(nis_ctx *ctx, nis_light light, int level, float *d_dst,
                                  nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    Light *l = lookup(ctx->lights, light);
    if (!l) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released light handle");
    Volume *v = lookup(ctx->vols, l->vol);
    if (level < 0 || level >= v->levels || !d_dst) return fail(ctx, NIS_ERR_INVALID_ARG, "bad level or NULL dst");
    DeviceGuard g(ctx->device);
    size_t n = (size_t)v->sizes[level] * v->sizes[level] * v->sizes[level];
    NIS_CUDA(cudaMemcpyAsync(d_dst, l->data + v->off[level], n * 4, cudaMemcpyDeviceToDevice,
                             reinterpret_cast<cudaStream_t>(stream)));
    return NIS_OK;
}

nis_status nis_build_phase_table(nis_ctx *ctx, float g, float *d_dst, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!(g > -1.f && g < 1.f)) return fail(ctx, NIS_ERR_INVALID_ARG, "g must lie in (-1, 1)");
    DeviceGuard gd(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *t;
    nis_status st = ensure_phase(ctx, phase_spec_g(g), s, &t, /*rebuild=*/true);
    if (st) return st;
    if (d_dst)
        NIS_CUDA(cudaMemcpyAsync(d_dst, t, sizeof(float) * kAlpha * kPhaseSets * kLat,
                                 cudaMemcpyDeviceToDevice, s));
    return NIS_OK;
}

nis_status nis_update_volume(nis_ctx *ctx, nis_volume vol, const void *density, int dtype,
                             int src_is_device, float sigma_scale, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!density) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL density");
    if (dtype != NIS_DTYPE_F32 && dtype != NIS_DTYPE_F16)
        return fail(ctx, NIS_ERR_INVALID_ARG, "dtype must be F32 or F16");
    if (!(sigma_scale >= 0.f) || !std::isfinite(sigma_scale))
        return fail(ctx, NIS_ERR_INVALID_ARG, "sigma_scale must be finite and >= 0");
    Volume *v = lookup(ctx->vols, vol);
    if (!v) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume handle");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t count = (size_t)v->n * v->n * v->n;
    size_t bytes = count * (dtype == NIS_DTYPE_F16 ? 2 : 4);
    const void *src = density;
    if (!src_is_device) {
        cudaPointerAttributes attr{};
        cudaError_t e = cudaPointerGetAttributes(&attr, density);
        if (e != cudaSuccess) cudaGetLastError();
        void *mapped = nullptr;
        if (e == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            cudaHostGetDevicePointer(&mapped, const_cast<void *>(density), 0) == cudaSuccess) {
            src = mapped;                       // page-locked: the kernel reads it in place
        } else {
            cudaGetLastError();
            if (v->staging_bytes < bytes) {
                dev_free(ctx, v->staging);
                v->staging = nullptr;
                v->staging_bytes = 0;
                nis_status st = dev_alloc(ctx, bytes, &v->staging, s);
                if (st) return st;
                v->staging_bytes = bytes;
            }
            NIS_CUDA(cudaMemcpyAsync(v->staging, density, bytes, cudaMemcpyHostToDevice, s));
            src = v->staging;
        }
    }
    {
        ProfScope ps(ctx, "other", s);
        launch_convert_density(src, dtype, sigma_scale, count, v->data, ctx->d_err, v->sigma_max, s);
    }
    NIS_CUDA(cudaGetLastError());
    v->pyramid = false;
    return NIS_OK;
}

nis_status nis_profile(nis_ctx *ctx, int enable) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (enable) {
        cudaDeviceSynchronize();
        for (auto &kv : ctx->prof)
            for (auto &e : kv.second) {
                ctx->event_pool.push_back(e.e0);
                ctx->event_pool.push_back(e.e1);
            }
        ctx->prof.clear();
    }
    ctx->prof_on = enable != 0;
    return NIS_OK;
}

nis_status nis_profile_read(nis_ctx *ctx, const char *family, double *total_ms, int *launches) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!family || !total_ms || !launches) return fail(ctx, NIS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(ctx->device);
    *total_ms = 0.0;
    *launches = 0;
    auto it = ctx->prof.find(family);
    if (it == ctx->prof.end()) return NIS_OK;
    for (auto &e : it->second) {
        NIS_CUDA(cudaEventSynchronize(e.e1));
        float ms = 0.f;
        NIS_CUDA(cudaEventElapsedTime(&ms, e.e0, e.e1));
        *total_ms += ms;
        *launches += e.launches;
    }
    return NIS_OK;
}

uint64_t nis_kernel_launches(void) { return g_launches.load(); }

nis_status nis_debug_tc_gemm(nis_ctx *ctx, const void *d_a, int lda, const void *d_b, int ldb,
                             int m, int n, int k, float *d_c, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!d_a || !d_b || !d_c || m < 1 || n < 1 || n > 208 || k < 1 || lda < k || ldb < k ||
        (lda % 8) || (ldb % 8))
        return fail(ctx, NIS_ERR_INVALID_ARG, "bad GEMM arguments (n <= 208, lda/ldb >= k and % 8)");
    DeviceGuard g(ctx->device);
    TcGemmArgs a{};
    a.M = m; a.N = n; a.K = k;
    a.n_mma = (n + 15) / 16 * 16;
    a.k_tiles = (k + 63) / 64;
    a.epi = kEpiPlain;
    a.err = ctx->d_err;
    a.out_f32 = d_c; a.ldo = n;
    CUtensorMap ma, mb;
    if (!make_tmap_bf16(&ma, d_a, (uint64_t)k, (uint64_t)m, (uint64_t)lda * 2, 64, 128) ||
        !make_tmap_bf16(&mb, d_b, (uint64_t)k, (uint64_t)n, (uint64_t)ldb * 2, 64, (uint32_t)a.n_mma))
        return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    // C through the epilogue's TMA stores where its rows are whole 16-byte units
    CUtensorMap mc;
    const bool tma_c = n % 4 == 0 && make_tmap_out(&mc, d_c, true, (uint64_t)n, (uint64_t)m, 1,
                                                   (uint64_t)n * 4, (uint64_t)n * m * 4);
    if (tma_c) { a.o1_kind = kOutF32; a.o1_parts = 1; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    {
        ProfScope ps(ctx, "mlp", reinterpret_cast<cudaStream_t>(stream));
        launch_tc_gemm(a, ma, mb, sms, reinterpret_cast<cudaStream_t>(stream), tma_c ? &mc : nullptr);
    }
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}


nis_status nis_debug_tc_gemm_f32(nis_ctx *ctx, const float *d_a, int lda, const float *d_b,
                                 int ldb, int m, int n, int k, float *d_c, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (!d_a || !d_b || !d_c || m < 1 || n < 1 || n > 208 || k < 1 || lda < k || ldb < k)
        return fail(ctx, NIS_ERR_INVALID_ARG, "bad GEMM arguments (n <= 208, lda/ldb >= k)");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n_mma = (n + 15) / 16 * 16, kp = (k + 63) / 64 * 64;
    const size_t a_elems = (size_t)3 * m * kp, b_elems = (size_t)3 * n_mma * kp;
    __nv_bfloat16 *parts = nullptr;
    NIS_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&parts), (a_elems + b_elems) * 2, s));
    __nv_bfloat16 *ap = parts, *bp = parts + a_elems;
    for (int q = 0; q < 3; ++q) {
        launch_pack_bf16(d_a, m, k, lda, ap + (size_t)q * m * kp, m, kp, s, q);
        launch_pack_bf16(d_b, n, k, ldb, bp + (size_t)q * n_mma * kp, n_mma, kp, s, q);
    }
    TcGemmArgs a{};
    a.M = m; a.N = n; a.K = k;
    a.n_mma = n_mma;
    a.n_pass = 6;
    a.k_tiles = (k + (int)tc_box_k(3) - 1) / (int)tc_box_k(3);
    a.a_part_rows = m;
    a.b_part_rows = n_mma;
    a.epi = kEpiPlain;
    a.err = ctx->d_err;
    a.out_f32 = d_c; a.ldo = n;
    CUtensorMap ma, mb;
    bool ok = make_tmap_bf16(&ma, ap, (uint64_t)kp, (uint64_t)3 * m, (uint64_t)kp * 2, tc_box_k(3), 128) &&
              make_tmap_bf16(&mb, bp, (uint64_t)kp, (uint64_t)3 * n_mma, (uint64_t)kp * 2, tc_box_k(3),
                             (uint32_t)n_mma);
    CUtensorMap mc;
    const bool tma_c = n % 4 == 0 && make_tmap_out(&mc, d_c, true, (uint64_t)n, (uint64_t)m, 1,
                                                   (uint64_t)n * 4, (uint64_t)n * m * 4);
    if (tma_c) { a.o1_kind = kOutF32; a.o1_parts = 1; }
    if (ok) {
        ProfScope ps(ctx, "mlp", s);
        launch_tc_gemm(a, ma, mb, ctx->num_sms, s, tma_c ? &mc : nullptr);
    }
    cudaFreeAsync(parts, s);
    if (!ok) return fail(ctx, NIS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

nis_status nis_shade_segments(nis_ctx *ctx, nis_weights w, const nis_segment *segs, int nseg,
                              nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (nseg < 0 || (nseg > 0 && !segs)) return fail(ctx, NIS_ERR_INVALID_ARG, "bad segment list");
    Weights *pw = lookup(ctx->weights, w);
    if (!pw) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released weights handle");
    if (pw->off.model != kModelLattice)
        return fail(ctx, NIS_ERR_UNIMPLEMENTED, "mixed batches need lattice-model weights");
    DeviceGuard g(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<ReqDesc> descs(nseg);
    long long total = 0;
    Volume *v0 = nullptr;
    Light *l0 = nullptr;
    for (int i = 0; i < nseg; ++i) {
        const nis_segment &sg = segs[i];
        nis_status st = check_material(ctx, &sg.material);
        if (st) return st;
        if (sg.n < 0 || (sg.n > 0 && (!sg.d_points || !sg.d_omega || !sg.d_rgb_out)))
            return fail(ctx, NIS_ERR_INVALID_ARG, "bad segment buffers");
        Volume *pv = lookup(ctx->vols, sg.vol);
        Light *pl = lookup(ctx->lights, sg.light);
        if (!pv || !pl) return fail(ctx, NIS_ERR_NOT_READY, "unknown or released volume or light handle");
        if (pl->vol != sg.vol) return fail(ctx, NIS_ERR_INVALID_ARG, "light belongs to another volume");
        if (!pv->pyramid) return fail(ctx, NIS_ERR_NOT_READY, "pyramid not built");
        float *table;
        if ((st = ensure_phase(ctx, phase_spec(&sg.material), s, &table))) return st;
        if ((st = ensure_pairs(ctx, *pv, *pl, s))) return st;
        ReqDesc &d = descs[i];
        d.rho = view_of(*pv, pv->data);
        d.T = view_of(*pv, pl->data);
        d.rt = pair_view(*pv, *pl);
        d.table = table;
        for (int c = 0; c < 3; ++c) {
            d.l[c] = pl->dir[c];
            d.albedo[c] = sg.material.albedo[c];
            d.dec[c] = sg.material.intensity[c] * powf(sg.material.albedo[c], 4.0f);
        }
        d.g = sg.material.g;
        total += sg.n;
        if (!v0) { v0 = pv; l0 = pl; }
    }
    if (total == 0) return NIS_OK;
    // batch buffers (grow-only)
    nis_status st;
    if (ctx->mix_cap < kChunk) {
        if ((st = dev_alloc_t(ctx, 3 * (size_t)kChunk, &ctx->mix_pts, s))) return st;
        if ((st = dev_alloc_t(ctx, 3 * (size_t)kChunk, &ctx->mix_om, s))) return st;
        if ((st = dev_alloc_t(ctx, 3 * (size_t)kChunk, &ctx->mix_rgb, s))) return st;
        if ((st = dev_alloc_t(ctx, 3 * (size_t)kChunk, &ctx->mix_dec, s))) return st;
        if ((st = dev_alloc_t(ctx, (size_t)kChunk, &ctx->mix_req, s))) return st;
        ctx->mix_cap = kChunk;
    }
    if (ctx->mix_desc_cap < nseg) {
        dev_free(ctx, ctx->mix_descs); dev_free(ctx, ctx->mix_seg_start); dev_free(ctx, ctx->mix_seg_desc);
        ctx->mix_descs = nullptr; ctx->mix_seg_start = ctx->mix_seg_desc = nullptr;
        ctx->mix_desc_cap = 0;
        if ((st = dev_alloc_t(ctx, (size_t)nseg, &ctx->mix_descs, s))) return st;
        if ((st = dev_alloc_t(ctx, (size_t)nseg, &ctx->mix_seg_start, s))) return st;
        if ((st = dev_alloc_t(ctx, (size_t)nseg, &ctx->mix_seg_desc, s))) return st;
        ctx->mix_desc_cap = nseg;
    }
    // pageable-source copies are staged by the driver before the call returns
    NIS_CUDA(cudaMemcpyAsync(ctx->mix_descs, descs.data(), sizeof(ReqDesc) * nseg,
                             cudaMemcpyHostToDevice, s));
    int seg = 0, seg_off = 0;
    while (seg < nseg) {
        std::vector<int> starts, dids;
        struct Piece { int seg, off, row, n; };
        std::vector<Piece> pieces;
        int rows = 0;
        while (seg < nseg && rows < kChunk) {
            int take = std::min(segs[seg].n - seg_off, kChunk - rows);
            if (take > 0) {
                pieces.push_back({seg, seg_off, rows, take});
                starts.push_back(rows);
                dids.push_back(seg);
                rows += take;
                seg_off += take;
            }
            if (seg_off >= segs[seg].n) { ++seg; seg_off = 0; }
        }
        if (rows == 0) break;
        for (const Piece &pc : pieces) {
            const nis_segment &sg = segs[pc.seg];
            NIS_CUDA(cudaMemcpyAsync(ctx->mix_pts + 3 * (size_t)pc.row, sg.d_points + 3 * (size_t)pc.off,
                                     12 * (size_t)pc.n, cudaMemcpyDeviceToDevice, s));
            NIS_CUDA(cudaMemcpyAsync(ctx->mix_om + 3 * (size_t)pc.row, sg.d_omega + 3 * (size_t)pc.off,
                                     12 * (size_t)pc.n, cudaMemcpyDeviceToDevice, s));
        }
        NIS_CUDA(cudaMemcpyAsync(ctx->mix_seg_start, starts.data(), sizeof(int) * starts.size(),
                                 cudaMemcpyHostToDevice, s));
        NIS_CUDA(cudaMemcpyAsync(ctx->mix_seg_desc, dids.data(), sizeof(int) * dids.size(),
                                 cudaMemcpyHostToDevice, s));
        {
            ProfScope ps(ctx, "other", s);
            launch_fill_segments(ctx->mix_seg_start, ctx->mix_seg_desc, (int)starts.size(), rows,
                                 ctx->mix_req, ctx->mix_dec, ctx->mix_descs, s);
        }
        Mixed mx{ctx->mix_descs, ctx->mix_req, ctx->mix_dec};
        if ((st = shade_impl(ctx, *v0, *l0, *pw, &segs[pieces[0].seg].material, ctx->mix_pts,
                             ctx->mix_om, rows, ctx->mix_rgb, nullptr, s, &mx)))
            return st;
        for (const Piece &pc : pieces)
            NIS_CUDA(cudaMemcpyAsync(segs[pc.seg].d_rgb_out + 3 * (size_t)pc.off,
                                     ctx->mix_rgb + 3 * (size_t)pc.row, 12 * (size_t)pc.n,
                                     cudaMemcpyDeviceToDevice, s));
    }
    NIS_CUDA(cudaGetLastError());
    return NIS_OK;
}

}  // extern "C"
