// nis_shade_points_static: the shading path of nis_shade_points for callers that cannot
// allocate device memory.  Its scratch is a fixed file-scope __device__ array, so the call
// itself allocates nothing; it refuses work that does not fit and inputs it would have to
// build (pyramid, phase table).
#include <mutex>

#include "nis_internal.h"

using namespace nis;

namespace {

constexpr size_t kMaxPts = NIS_STATIC_MAX_POINTS;
constexpr size_t round64(size_t n) { return (n + 63) & ~size_t(63); }   // 256-byte steps

// float offsets of the sub-buffers inside the scratch array
constexpr size_t kOffHrho = 0;
constexpr size_t kOffHT = kOffHrho + round64(kMaxPts * kLayers * kLat);
constexpr size_t kOffHf = kOffHT + round64(kMaxPts * kLayers * kLatT);
constexpr size_t kOffV = kOffHf + round64(kMaxPts * kLayers * kLat);
constexpr size_t kOffW = kOffV + round64(kMaxPts * kLayers * 8);
constexpr size_t kOffCfg = kOffW + round64(kMaxPts * kLayers * 3);
constexpr size_t kOffXT = kOffCfg + round64(kMaxPts * kCfg);
constexpr size_t kOffAct = kOffXT + round64(kMaxPts * kLayers * kDT);
constexpr int kActs = 15;
constexpr size_t kActStride = round64(kMaxPts * kWidth);
constexpr size_t kScratchFloats = kOffAct + kActs * kActStride;
static_assert(kScratchFloats * sizeof(float) == NIS_STATIC_SCRATCH_BYTES,
              "NIS_STATIC_SCRATCH_BYTES in nis.h must match the scratch layout");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {};

}  // namespace

// One array per device that loads the library; every call on that device shares it.
static __device__ __align__(256) float g_static_scratch[kScratchFloats];

namespace {

// Device address of g_static_scratch on `device` (which must be current): looked up once
// per device.  The host-side symbol itself is not a device address.
cudaError_t scratch_address(int device, float **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" nis_status nis_shade_points_static(nis_ctx *ctx, nis_volume vol, nis_light light,
                                              nis_weights w, const nis_material *m,
                                              const float *d_points, const float *d_omega,
                                              int n, float *d_rgb_out, nis_stream stream) {
    if (!ctx) return NIS_ERR_INVALID_ARG;
    if (n < 0 || (size_t)n > kMaxPts)
        return record_error(ctx, NIS_ERR_INVALID_ARG,
                            "nis_shade_points_static takes at most NIS_STATIC_MAX_POINTS (512) "
                            "points per call");
    if (n > 0 && (!d_points || !d_omega || !d_rgb_out))
        return record_error(ctx, NIS_ERR_INVALID_ARG, "NULL points, omega or output");
    // the same material checks as every other shading call (phase lobes included)
    if (const char *why = material_problem(m)) return record_error(ctx, NIS_ERR_INVALID_ARG, why);
    if (weights_model(ctx, w) == kModelPaper)
        return record_error(ctx, NIS_ERR_UNIMPLEMENTED, "nis_shade_points_static takes lattice-model weights");
    ResolvedInputs in;
    nis_status st = resolve_built_inputs(ctx, vol, light, w, m, &in);
    if (st) return st;
    if (n == 0) return NIS_OK;
    if (in.device < 0 || in.device >= kMaxDevices)
        return record_error(ctx, NIS_ERR_INVALID_ARG, "device index beyond the static table");

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != in.device && cudaSetDevice(in.device) != cudaSuccess)
        return record_error(ctx, NIS_ERR_CUDA, "cudaSetDevice failed");
    float *scratch = nullptr;
    cudaError_t e = scratch_address(in.device, &scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0 && prev != in.device) cudaSetDevice(prev);
        return record_error(ctx, NIS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *H_rho = scratch + kOffHrho, *H_T = scratch + kOffHT, *H_f = scratch + kOffHf;
    float *v = scratch + kOffV, *w_se = scratch + kOffW, *cfg = scratch + kOffCfg;
    float *X_T = scratch + kOffXT;
    auto act = [&](int i) { return scratch + kOffAct + i * kActStride; };
    const WeightOffsets &o = in.off;
    const float *W = in.W;

    // Every scratch buffer is written before it is read within a call, so nothing needs
    // clearing between calls.
    GatherArgs ga{};
    ga.rho = in.rho;
    ga.T = in.T;
    ga.rt = in.rt;
    ga.table = in.table;
    ga.points = d_points;
    ga.omega = d_omega;
    ga.count = n;
    ga.lx = in.dir[0]; ga.ly = in.dir[1]; ga.lz = in.dir[2];
    ga.g = m->g;
    for (int c = 0; c < 3; ++c) ga.albedo[c] = m->albedo[c];
    ga.se = W;
    for (int k = 0; k < kLayers; ++k) {
        ga.se_w1[k] = o.se_w1[k]; ga.se_b1[k] = o.se_b1[k];
        ga.se_w2[k] = o.se_w2[k]; ga.se_b2[k] = o.se_b2[k];
    }
    ga.H_rho = H_rho; ga.H_T = H_T; ga.H_f = H_f; ga.v = v; ga.w_se = w_se; ga.cfg = cfg;
    launch_gather(ga, s);
    launch_cnn_f32(H_T, n, W, o, X_T, nullptr, s);
    for (int t = 0; t < 3; ++t) {
        const float *X = t == 0 ? H_rho : (t == 1 ? H_f : X_T);
        const int d = feat_dim(t);
        for (int chain = 0; chain < 2; ++chain) {
            int k0 = chain == 0 ? 0 : kDiffuse, k1 = chain == 0 ? kDiffuse : kLayers;
            float *h = nullptr;
            int ping = 1;
            for (int k = k0; k < k1; ++k) {
                FcArgs f1{};
                f1.mode = kFcFeat; f1.count = n; f1.K = d + kCfg; f1.N = kWidth;
                f1.X = X + (size_t)k * d; f1.ldx = kLayers * d; f1.d = d;
                f1.w_se = w_se; f1.layer = k; f1.type = t; f1.cfg = cfg;
                f1.W = W + o.blk_w1[t][k]; f1.b = W + o.blk_b1[t][k];
                f1.relu = 1; f1.out = act(0); f1.ldo = kWidth;
                launch_fc_f32(f1, s);
                FcArgs f2{};
                f2.mode = kFcSum; f2.count = n; f2.K = kWidth; f2.N = kWidth;
                f2.a0 = h; f2.a1 = act(0); f2.seg = kWidth;
                f2.W = W + o.blk_w2[t][k]; f2.b = W + o.blk_b2[t][k];
                f2.relu = 1; f2.resid = act(0); f2.ldo = kWidth;
                float *dst = (k == k1 - 1) ? act(3 + 2 * t + chain) : act(ping);
                f2.out = dst;
                launch_fc_f32(f2, s);
                h = dst;
                ping = 3 - ping;
            }
        }
        FcArgs mg{};
        mg.mode = kFcCat; mg.count = n; mg.K = 2 * kWidth; mg.N = kWidth;
        mg.a0 = act(3 + 2 * t); mg.a1 = act(4 + 2 * t); mg.seg = kWidth;
        mg.W = W + o.mrg_w[t]; mg.b = W + o.mrg_b[t]; mg.relu = 1;
        mg.out = act(9 + t); mg.ldo = kWidth;
        launch_fc_f32(mg, s);
    }
    FcArgs h1{};
    h1.mode = kFcCat; h1.count = n; h1.K = 3 * kWidth; h1.N = kWidth;
    h1.a0 = act(9); h1.a1 = act(10); h1.a2 = act(11); h1.seg = kWidth;
    h1.W = W + o.head_w[0]; h1.b = W + o.head_b[0]; h1.relu = 1;
    h1.out = act(12); h1.ldo = kWidth;
    launch_fc_f32(h1, s);
    FcArgs h2{};
    h2.mode = kFcSum; h2.count = n; h2.K = kWidth; h2.N = kWidth;
    h2.a1 = act(12); h2.seg = kWidth;
    h2.W = W + o.head_w[1]; h2.b = W + o.head_b[1]; h2.relu = 1;
    h2.out = act(13); h2.ldo = kWidth;
    launch_fc_f32(h2, s);
    FcArgs h3{};
    h3.mode = kFcSum; h3.count = n; h3.K = kWidth; h3.N = 3;
    h3.a1 = act(13); h3.seg = kWidth;
    h3.W = W + o.head_w[2]; h3.b = W + o.head_b[2];
    h3.decode = 1;
    for (int c = 0; c < 3; ++c) h3.dec_scale[c] = m->intensity[c] * powf(m->albedo[c], 4.0f);
    h3.out = d_rgb_out; h3.ldo = 3;
    launch_fc_f32(h3, s);
    e = cudaGetLastError();
    if (prev >= 0 && prev != in.device) cudaSetDevice(prev);
    if (e != cudaSuccess) return record_error(ctx, NIS_ERR_CUDA, cudaGetErrorString(e));
    return NIS_OK;
}
