/*
 * nis.h -- C ABI of the neural in-scattering estimator of arXiv 2401.14051
 * ("A real-time rendering method for high albedo anisotropic materials with multiple
 * scattering"), built for one GB300 (sm_103a).
 *
 * The library runs the paper's inference path per shading point and per light:
 *   1. density mip pyramid                         (Sec. III.B.1)
 *   2. graded transmittance fields, Eq. 1          (Sec. III.B.1; Eq. 15)
 *   3. diffuse + highlight template gathers of density, transmittance and
 *      cone-integrated HG phase features           (Sec. III.B.2-5; Eq. 2-5, 8, 9)
 *   4. per-layer 3D-CNN over the transmittance stencil (Sec. III.B.1, Fig. 3)
 *   5. SE channel attention                        (Sec. III.C.3; Eq. 24-26)
 *   6. backbone MLP + output decode                (Sec. III.C.2, Fig. 6; Eq. 21)
 * Every step runs in this library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions.  The medium occupies the unit cube [0,1]^3.  A grid of N^3 voxels is
 * stored x-fastest (index (k*N + j)*N + i for voxel (i, j, k)), voxel centres at
 * ((i+1/2)/N, (j+1/2)/N, (k+1/2)/N).  light_dir is the direction the light travels
 * (unit or not; the library normalises it).  omega is the direction from a shading point
 * toward the camera.  Images are row-major [height][width][3] float32, row 0 at the top.
 *
 * Errors.  Every call returns NIS_OK (0) or a negative nis_status; argument errors are
 * reported synchronously and nis_last_error() gives a message.  Calls that enqueue GPU
 * work return once it is enqueued on the caller's stream; device-side faults detected by
 * the kernels' own checks are reported by nis_sync().  A context is not thread-safe:
 * serialise calls on one context.
 *
 * Ownership.  The library copies volumes and weights into its own device memory and owns
 * every pyramid, transmittance field, phase table and scratch buffer it builds.  Input and
 * output buffers passed to a call stay owned by the caller.
 */
#ifndef NIS_H
#define NIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nis_stream; /* a cudaStream_t; NULL = legacy default stream */
typedef struct nis_ctx nis_ctx;
typedef uint64_t nis_handle;            /* 0 is never a valid handle */
typedef nis_handle nis_volume;
typedef nis_handle nis_light;
typedef nis_handle nis_weights;

typedef int nis_status;
#define NIS_OK 0
#define NIS_ERR_INVALID_ARG -1   /* bad pointer, size, enum or handle */
#define NIS_ERR_NOT_READY -2     /* handle released, or a cache the call may not build */
#define NIS_ERR_BUDGET -3        /* allocation would exceed the context's HBM budget */
#define NIS_ERR_OOM -4           /* the allocator failed */
#define NIS_ERR_CUDA -5          /* a CUDA runtime call failed */
#define NIS_ERR_TIMEOUT -6       /* a host wait passed its deadline */
#define NIS_ERR_UNIMPLEMENTED -7
#define NIS_ERR_BAD_BLOB -8      /* weight blob header, size or checksum mismatch */
#define NIS_ERR_BAD_DATA -9      /* a kernel check failed (e.g. NaN/negative density) */

#define NIS_DTYPE_F32 0
#define NIS_DTYPE_F16 1

#define NIS_PREC_F32 0           /* FP32-accurate: dense layers on the tensor cores with every
                                    operand split into three BF16 parts (x = x0 + x1 + x2,
                                    residual < 2^-24 |x|) and the six products that matter
                                    accumulated in FP32; everything else in FP32 */
#define NIS_PREC_BF16 1          /* CNN output, features and dense layers in BF16, FP32 accumulation */
#define NIS_PREC_FP8 2           /* as BF16, FC-1 of the density and phase chains on e4m3 operands
                                    (per-layer scales); mixed batches: e4m3 dense layers with
                                    per-channel weight scales */
#define NIS_PREC_F32_SIMT 3      /* FP32 everywhere on the FP32 FFMA pipes (reference path) */

#define NIS_CAMERA_ORTHO 0
#define NIS_CAMERA_PERSP 1

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns NULL
 * on failure.  Either both callbacks are set or the library uses cudaMalloc/cudaFree. */
typedef struct nis_allocator {
    void *user;
    void *(*alloc)(void *user, size_t bytes, nis_stream stream);
    void (*free)(void *user, void *ptr, size_t bytes, nis_stream stream);
} nis_allocator;

/* Material: HG asymmetry g in (-1, 1) (Eq. 5), RGB albedo in (0, 1] (Sec. III.C.2) and
 * RGB light intensity I (Eq. 16).  g is the network's configuration input and, with
 * n_lobes <= 1, the phase function of the phase features.  With n_lobes = 2 or 3 the phase
 * features use the multi-lobe mixture sum_i lobe_w[i] HG(lobe_g[i]) (Eq. 6; weights >= 0
 * summing to 1), while g stays the network input (for example the mixture's mean cosine).
 * g = 0 with n_lobes <= 1 is the isotropic phase function (Eq. 7). */
typedef struct nis_material {
    float g;
    float albedo[3];
    float intensity[3];
    int n_lobes;
    float lobe_g[3];
    float lobe_w[3];
} nis_material;

/* Pinhole (PERSP, vertical field of view fov_y in radians) or orthographic (ORTHO, view
 * height ortho_height) camera at eye looking at target; up fixes the roll. */
typedef struct nis_camera {
    int type;
    int width, height;
    float eye[3], target[3], up[3];
    float fov_y;
    float ortho_height;
} nis_camera;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the device memory the
 * context may hold (0 = no cap).  alloc may be NULL.  *out receives the context. */
nis_status nis_create(nis_ctx **out, int device, size_t hbm_budget_bytes,
                      const nis_allocator *alloc);

/* Frees every buffer the context owns (after a device synchronise) and the context. */
void nis_destroy(nis_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  Valid until the next
 * call on the context.  A NULL ctx gives the message of the last failed nis_create. */
const char *nis_last_error(const nis_ctx *ctx);

/* Bytes of device memory the context holds now. */
size_t nis_bytes_in_use(const nis_ctx *ctx);

/* Copies an nx*ny*nz density grid (sigma_t per unit length, float32 or float16, x-fastest)
 * from host or device memory (src_is_device) into a new volume, multiplied by
 * sigma_scale.  The grid must be cubic (nx = ny = nz, 1..2048).  Values are checked on the
 * device: NaN, infinite or negative densities make the next nis_sync return
 * NIS_ERR_BAD_DATA.  The caller keeps ownership of `density`.  A page-locked host source
 * is read in place by the conversion kernel (keep it valid until the stream passes the
 * call); a pageable host source has been copied when the call returns. */
nis_status nis_upload_volume(nis_ctx *ctx, const void *density, int nx, int ny, int nz,
                             int dtype, int src_is_device, float sigma_scale,
                             nis_stream stream, nis_volume *out);

/* Builds the density mip pyramid of `vol` (Sec. III.B.1): levels N, ceil(N/2), ..., 1,
 * each voxel the mean of its in-range 2x2x2 children, plus sigma_max of level 0, and each
 * level's cell occupancy (which cells have a nonzero corner).  Rebuilding an already built
 * pyramid recomputes it in place.  Once it is built, the first-hit search of the calls below
 * (nis_render_frame*, nis_find_hits, nis_render_frame_part) reads level 0's occupancy to pass
 * over empty cells (the hits are the same): order those calls after this one when they run
 * on another stream. */
nis_status nis_build_pyramid(nis_ctx *ctx, nis_volume vol, nis_stream stream);

/* Marches the graded transmittance fields of `vol` toward a distant light (Eq. 1):
 * T_m(x) = exp(-lambda^(m+1) * integral of level m's density from x to the cube exit along
 * -light_dir), midpoint rule with step 1/N_m and a partial last step, stopping once the
 * scaled optical depth exceeds 30.  lambda in (0, 1] (the paper uses 0.6).  Builds the
 * pyramid first if needed.  A light with the same volume, direction and lambda is
 * re-marched into its existing buffers and its handle returned again.  The light also keeps
 * a cell-entry copy for the template gathers: per z slice and cell (y, x), the density and
 * the transmittance at the cell's four (y, x) corners in 32 bytes (about 8x the
 * transmittance pyramid's bytes: 34 GB for a 1024^3 grid); shading calls refresh that copy
 * when the pyramid has been rebuilt since. */
nis_status nis_build_transmittance(nis_ctx *ctx, nis_volume vol, const float light_dir[3],
                                   float lambda, nis_stream stream, nis_light *out);

/* Transmittance methods of nis_build_transmittance_method. */
#define NIS_TRANSMITTANCE_MARCH 0       /* the march above, O(N^4) per level */
#define NIS_TRANSMITTANCE_SHEAR_WARP 1  /* O(N^3) approximation, below */

/* nis_build_transmittance with a choice of method (no counterpart in the paper, which
 * marches every voxel).  NIS_TRANSMITTANCE_SHEAR_WARP approximates Eq. 1's depth for large
 * grids: parallel rays toward the light cross the slices normal to the axis a where
 * |light_dir| is largest at positions that shift by r = u_perp / |u_a| per slice (u =
 * -light_dir); each ray sums, slice by slice, the part of its step that lies inside the cube
 * (its in-cube length) and that length times the density at the part's midpoint (its
 * depth); each voxel centre takes the bilinearly weighted mean density of the four rays
 * around it (depth / length, or the density at the crossing for a ray that has not met the
 * cube) times its own exit distance.  No stop rule.  A light along an axis reproduces the
 * march (to rounding), a homogeneous medium gives the exact depth, the field is continuous
 * in the light direction, and otherwise the error is an interpolation error made once per
 * voxel: second order in the voxel size on average, first order on rays through a cube
 * edge.  It takes N_0 + 1 launches of one kernel (all levels together) and a ray scratch of
 * 4 floats per ray, about (1 + |r_p|)(1 + |r_q|) N^2 rays per level, owned by the context
 * (grow-only; calls on one context that overlap on the GPU race on it).  For lights whose
 * |x| component is largest the volume also keeps an x-major copy of its pyramid (about the
 * pyramid's size, with its occupancy), and the context an output buffer of the same size.
 * A light is identified by volume, direction, lambda and method.  Unknown methods return
 * NIS_ERR_INVALID_ARG. */
nis_status nis_build_transmittance_method(nis_ctx *ctx, nis_volume vol, const float light_dir[3],
                                          float lambda, int method, nis_stream stream,
                                          nis_light *out);

/* Parses a weight blob (80-byte header, float32 tensors in the fixed order below, a
 * position-weighted word checksum) and uploads it at `precision`.  The caller keeps the
 * blob.  Header word 2 names the network:
 *   0, the lattice model: CNN[12]{w1 16x1x3x3x3, b1, w2 16x16x3x3x3, b2}, SE[12]{w1 2x8,
 *      b1, w2 3x2, b2}, blocks[type rho,f,T][layer 0..11]{W1 200x(d+5), b1, W2 200x200, b2}
 *      with d = 225, 225, 80, merge[3]{200x400, b}, head{200x600, b, 200x200, b, 3x200, b};
 *   1, the paper-template model (the paper's own template sets, Sec. III.B.2: 6, 8, 12,
 *      16, 24, 32, 48, 48 diffuse and 32, 16, 16, 8 highlight points per layer; a
 *      volume-level transmission feature b + sum_m w_m T_m at each point, Fig. 3, in place
 *      of the per-layer CNN): level w[11], level b[1], then SE, blocks with d = the layer's
 *      point count for all three types, merges and head as above.  Header words 6, 7 and 12
 *      are 266, 0 and 11.  It runs at NIS_PREC_F32, NIS_PREC_BF16 (tensor cores) or
 *      NIS_PREC_F32_SIMT (FFMA); NIS_PREC_FP8 returns NIS_ERR_UNIMPLEMENTED.  It shades
 *      through nis_shade_points, nis_shade_points_debug (features [n][266] at the start of
 *      the H buffers; no X_T) and the frame calls; mixed batches, the server and the
 *      allocation-free call take the lattice model only (NIS_ERR_UNIMPLEMENTED). */
nis_status nis_load_weights(nis_ctx *ctx, const void *blob, size_t bytes, int precision,
                            nis_stream stream, nis_weights *out);

/* Radiance at n shading points (steps 3-6; Sec. III.C.2 output layer): rgb[i] =
 * I * albedo^4 * expm1(y_i) where y_i is the network output for point d_points[i] (x, y, z)
 * seen along d_omega[i].  All three buffers are device float32 arrays of n*3 values.
 * Builds the phase table for material->g if it is not cached. */
nis_status nis_shade_points(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                            const nis_material *m, const float *d_points,
                            const float *d_omega, int n, float *d_rgb_out,
                            nis_stream stream);

/* Renders one frame: per pixel, the first sample along the camera ray (step 0.5/N from the
 * cube entry) whose level-0 density reaches 0.05 sigma_max is the shading point; its
 * radiance (as nis_shade_points, omega = -ray direction) is the pixel value, 0 for rays
 * that find none.  d_rgb_out is a device float32 [height][width][3] buffer.  Waits once on
 * the stream to read the number of shading points. */
nis_status nis_render_frame(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                            const nis_material *m, const nis_camera *cam, float *d_rgb_out,
                            nis_stream stream);

/* The same frame lit by several directional lights (no counterpart in the paper's
 * experiments, which use one; the in-scattered radiance of independent lights adds): the
 * shading points are found once, each light's radiance is estimated with its own
 * transmittance field (nis_build_transmittance per light, all of `vol`) and the per-light
 * radiances are summed per pixel in the order of `lights`.  1 <= n_lights <= 64; the light
 * handles are read before the call returns. */
nis_status nis_render_frame_lights(nis_ctx *ctx, nis_volume vol, const nis_light *lights,
                                   int n_lights, nis_weights w, const nis_material *m,
                                   const nis_camera *cam, float *d_rgb_out, nis_stream stream);

/* ---- one frame split into ranges of shading points ------------------------------------
 * The paper runs many network instances in parallel over independent shading points
 * (Sec. III.C.2, input batching).  These calls split one frame's shading points into `parts`
 * contiguous ranges, one per process (or per GPU), with the volume, light and weights
 * replicated; each range's radiance is shaded where it lies and the parts are assembled into
 * one image on one device.  The frame's hits are listed in pixel order, so every process
 * computes the same list and the ranges cover each hit exactly once. */

/* Range `part` of `parts` equal contiguous ranges over n items: *first = floor(part * n /
 * parts), *count = floor((part + 1) * n / parts) - *first.  Host only: needs no context and
 * no device.  NIS_ERR_INVALID_ARG for n < 0, parts < 1, part outside [0, parts) or a NULL
 * output. */
nis_status nis_part_range(long long n, int part, int parts, long long *first, long long *count);

/* Range `part` of `parts` of one frame (the frame of nis_render_frame with the same
 * arguments): finds the frame's hits, lists them in pixel order, and shades hits *first ..
 * *first + *count - 1 of that list (nis_part_range over the frame's hits).  Writes their
 * radiance to d_rgb (device float32, count x 3) and their pixel indices y * width + x to d_pix
 * (device int32, count); both hold `capacity` rows, and ceil(width * height / parts) always
 * suffices.  *n_hits, *first and *count (host) receive the frame's hit count and the range.
 * Each hit's radiance is bit-identical to that pixel of nis_render_frame.  NIS_ERR_INVALID_ARG
 * for part/parts out of range, NULL buffers, or capacity < count (then nothing is shaded),
 * besides the errors of nis_render_frame.  Waits once on the stream (to read the hit count). */
nis_status nis_render_frame_part(nis_ctx *ctx, nis_volume vol, nis_light light, nis_weights w,
                                 const nis_material *m, const nis_camera *cam, int part,
                                 int parts, float *d_rgb, int *d_pix, int capacity, int *n_hits,
                                 int *first, int *count, nis_stream stream);

/* Assembles one part into an image: d_image[3 * d_pix[i] + c] = d_rgb[3 * i + c] for i < n and
 * c < 3 (all device buffers; d_image float32 of n_pixels x 3).  Pixel indices outside
 * [0, n_pixels) are skipped.  Pixels that no part names keep their value, so the caller
 * clears the image once before the first part.  Asynchronous on `stream`. */
nis_status nis_scatter_part(nis_ctx *ctx, const float *d_rgb, const int *d_pix, int n,
                            float *d_image, int n_pixels, nis_stream stream);

/* Overwrites the density of an existing volume with a grid of the same size (same
 * conventions as nis_upload_volume) without allocating: device sources and page-locked
 * host sources are read in place (a GB300 kernel reads pinned host memory over
 * NVLink-C2C); pageable host sources go through a staging buffer the volume keeps.  The
 * pyramid and every transmittance field of the volume become stale until rebuilt. */
nis_status nis_update_volume(nis_ctx *ctx, nis_volume vol, const void *density, int dtype,
                             int src_is_device, float sigma_scale, nis_stream stream);

/* ---- allocation-free shading (no counterpart in the paper) ---------------------------
 * Some callers cannot allocate device memory while they shade: a renderer plug-in whose
 * host engine owns and budgets every byte of GPU memory, or a frame loop that must not call
 * cudaMalloc (it can synchronise the device and stall the frame).  This entry point gives
 * them the result of nis_shade_points for up to NIS_STATIC_MAX_POINTS points per call
 * without allocating anything: its scratch is one fixed array in the library's device
 * memory of NIS_STATIC_SCRATCH_BYTES (about 25 MB), which every GPU that loads the library
 * holds until the process exits.  Callers still pass their own inputs and output.
 *
 * - n above NIS_STATIC_MAX_POINTS returns NIS_ERR_INVALID_ARG (split larger batches).
 * - Nothing is built here: the pyramid, the light's transmittance and the phase table for
 *   m->g must exist (nis_build_pyramid / nis_build_transmittance / nis_build_phase_table),
 *   otherwise NIS_ERR_NOT_READY.  So must the light's copy of the density it shades with:
 *   after a pyramid rebuild, build the light again or shade once through nis_shade_points
 *   (which refreshes that copy), else NIS_ERR_NOT_READY.
 * - The dense layers run in FP32 on the CUDA cores (the FP32 copy of the weights), whatever
 *   precision the weights were loaded with: BF16- or FP8-loaded weights give the FP32
 *   result.  Paper-template weights are refused with NIS_ERR_UNIMPLEMENTED; materials are
 *   checked as for nis_shade_points (NIS_ERR_INVALID_ARG).
 * - The first call on a device looks up the array's device address; make that first call
 *   before any stream capture.
 * - All calls in the process share the one array and leave their intermediates in it; the
 *   path writes every scratch value before reading it, so nothing needs clearing, but two
 *   calls whose work overlaps on the GPU (different streams, no ordering) race on it and
 *   give wrong results.  Serialise them (one stream, or events). */
#define NIS_STATIC_MAX_POINTS 512
#define NIS_STATIC_SCRATCH_BYTES 25151488
nis_status nis_shade_points_static(nis_ctx *ctx, nis_volume vol, nis_light light,
                                   nis_weights w, const nis_material *m,
                                   const float *d_points, const float *d_omega, int n,
                                   float *d_rgb_out, nis_stream stream);

/* One request's share of a mixed batch: n shading points (device, n x 3) of volume `vol`
 * lit by `light` with its material; radiance goes to d_rgb_out (device, n x 3). */
typedef struct nis_segment {
    nis_volume vol;
    nis_light light;
    nis_material material;
    const float *d_points, *d_omega;
    int n;
    float *d_rgb_out;
} nis_segment;

/* Continuous batching (the paper's "multiple network instances in parallel", Sec. III.C.2,
 * across requests): shades the points of several requests -- different volumes, lights and
 * materials -- in the same gather, CNN and MLP launches.  Each point carries its request's
 * pyramid, transmittance field, phase table, light and material, so every result equals
 * what nis_shade_points gives for that request alone.  Pyramids must be built. */
nis_status nis_shade_segments(nis_ctx *ctx, nis_weights w, const nis_segment *segs, int nseg,
                              nis_stream stream);

/* ---- serving: continuous batching of render requests -----------------------------------
 * A server owns a context (no other calls on that context while the server lives) and one
 * host thread.  Requests -- each a density grid in host memory with its light, material and
 * camera -- are admitted in arrival order while the HBM budget and the in-flight limit
 * allow; an admitted request's volume upload, pyramid, transmittance and first-hit
 * search run on a preparation stream while earlier requests shade on a second stream; the
 * shading points of all ready requests are shaded together in mixed batches
 * (nis_shade_segments), so requests that arrive while others run join the next batch: of a
 * batch's max_batch_points the oldest ready request takes up to half and the other ready
 * requests share the rest equally; what a request cannot use goes to the others in
 * admission order.
 * Pyramids are cached per volume_key and transmittance fields per (volume_key, light,
 * lambda), kept on the device and evicted least-recently-used (unreferenced only) when the
 * budget needs room.  Each request's image is written to its rgb_out (host, H x W x 3
 * float32) before nis_server_wait reports it done. */
typedef struct nis_server nis_server;

typedef struct nis_server_config {
    size_t hbm_budget_bytes;      /* device memory the server may hold (0 = no limit) */
    int max_batch_points;         /* shading points per mixed batch (<= 65536) */
    int max_inflight;             /* admitted, unfinished requests at most */
    int transmittance_method;     /* NIS_TRANSMITTANCE_* of every light the server builds
                                     (0, the march, when zero-initialised) */
} nis_server_config;

typedef struct nis_request {
    const void *density;          /* host N^3 grid (NIS_DTYPE_*), kept valid until done */
    int n;
    int dtype;
    uint64_t volume_key;          /* same key = same density: the pyramid is reused */
    float light_dir[3];
    float lambda;
    nis_material material;
    nis_camera camera;
    float *rgb_out;               /* host [height][width][3] float32 */
} nis_request;

typedef struct nis_server_stats {
    uint64_t submitted, completed, failed;
    double p50_ms, p99_ms, mean_ms, max_ms;       /* submit -> image in rgb_out */
    uint64_t points_shaded, batches;
    double mean_batch_points, mean_batch_requests;
    uint64_t volume_hits, volume_misses, light_hits, light_misses, evictions;
    size_t peak_bytes;
    double span_seconds;          /* first submit -> last completion */
} nis_server_stats;

nis_status nis_server_create(nis_ctx *ctx, nis_weights w, const nis_server_config *cfg,
                             nis_server **out);
/* Queues a request (copies the struct; the buffers it points to stay the caller's).
 * NIS_ERR_INVALID_ARG, and nothing queued, for a malformed request: NULL buffers, grid
 * size outside 1..2048, dtype, image size, or a material nis_shade_points would refuse. */
nis_status nis_server_submit(nis_server *srv, const nis_request *req, uint64_t *id);
/* Waits up to timeout_ms (<= 0: no limit) for request `id`; NIS_ERR_TIMEOUT if not done.
 * latency_ms (may be NULL) receives submit-to-completion time.  A request that failed
 * returns its error: NIS_ERR_BUDGET if it can never fit the budget, else the status of the
 * step that failed (upload, builds, shading or the image read-back); its rgb_out is then
 * undefined. */
nis_status nis_server_wait(nis_server *srv, uint64_t id, int timeout_ms, double *latency_ms);
nis_status nis_server_get_stats(nis_server *srv, nis_server_stats *out);
/* Stops the loop after the admitted requests finish and frees the server's buffers. */
void nis_server_destroy(nis_server *srv);
/* Test hook (no counterpart in the paper): the next batch that shades points of request
 * `id` is treated, for that request only, as if its shading had returned `status` (< 0,
 * else NIS_ERR_INVALID_ARG).  The failure is made on the host; nothing faults on the GPU.
 * The request shades no further points and completes with `status`; the other requests
 * complete as usual.  Call it before the request's points are batched (for example right
 * after nis_server_submit; ids are 1, 2, ... in submit order). */
nis_status nis_server_inject_failure(nis_server *srv, uint64_t id, nis_status status);

/* Frees a volume (and its lights), a light or a weight set. */
nis_status nis_release(nis_ctx *ctx, nis_handle h);

/* Waits for `stream` (polling, up to timeout_ms; <= 0 waits without limit) and reports
 * any fault recorded by the kernels' own checks since the last nis_sync. */
nis_status nis_sync(nis_ctx *ctx, nis_stream stream, int timeout_ms);

/* ---- inspection (tests, benchmarks) ----------------------------------------------- */

/* Number of pyramid levels, their sizes (sizes[0..levels-1]) and, after a nis_sync, the
 * densest voxel of level 0. */
nis_status nis_volume_info(nis_ctx *ctx, nis_volume vol, int *levels, int sizes[16],
                           float *sigma_max);

/* Copies pyramid level `level` (N_m^3 float32) or transmittance level `level` of `light`
 * into a caller device buffer. */
nis_status nis_copy_level(nis_ctx *ctx, nis_volume vol, int level, float *d_dst,
                          nis_stream stream);
nis_status nis_copy_transmittance(nis_ctx *ctx, nis_light light, int level, float *d_dst,
                                  nis_stream stream);

/* (Re)builds the phase table for asymmetry g (Sec. III.B.5): 1024 alpha nodes
 * j*pi/1023 x 5 point sets (all diffuse layers; highlight layers 0..3) x 225 lattice points,
 * alpha-major, float32, and copies it to d_dst (1024*1125 floats) if d_dst is not NULL.
 * nis_shade_points builds a missing table itself; this call recomputes a cached one. */
nis_status nis_build_phase_table(nis_ctx *ctx, float g, float *d_dst, nis_stream stream);

/* Intermediate outputs of nis_shade_points for n points (any pointer may be NULL):
 * H_rho, H_T, H_f [n][12][225]; v [n][12][8] (Eq. 24 squeeze vectors); X_T [n][12][80]
 * (CNN output, position-major); w_se [n][12][3] (SE weights, order rho, f, T); y [n][3]
 * (network output before the decode).  All device float32. */
typedef struct nis_debug_out {
    float *H_rho, *H_T, *H_f, *v, *X_T, *w_se, *y;
} nis_debug_out;
nis_status nis_shade_points_debug(nis_ctx *ctx, nis_volume vol, nis_light light,
                                  nis_weights w, const nis_material *m,
                                  const float *d_points, const float *d_omega, int n,
                                  float *d_rgb_out, const nis_debug_out *dbg,
                                  nis_stream stream);

/* First-hit search alone: per pixel, hit flag (int32), shading point and omega (float32
 * x3) into caller device buffers of width*height entries.  Reads level 0 (and, once the
 * pyramid is built, its cell occupancy: see nis_build_pyramid). */
nis_status nis_find_hits(nis_ctx *ctx, nis_volume vol, const nis_camera *cam, int *d_hit,
                         float *d_points, float *d_omega, nis_stream stream);

/* Kernel timing: with profiling on, the kernels the context launches are bracketed by CUDA
 * events on their stream, accumulated per kernel family: each kernel on its own, except the
 * tensor-core dense layers of one shading pass and the launches of one shear-warp
 * transmittance build, which are one bracketed block each (no event between two of their
 * launches, which overlap as programmatic dependent launches).  nis_profile(ctx, 1)
 * clears and starts, nis_profile(ctx, 0) stops.  nis_profile_read waits for the recorded
 * events and returns the summed device time and the number of kernels launched inside the
 * brackets of one family: "pyramid", "march", "phase", "hits", "gather", "cnn", "mlp" or
 * "other".  The launch count assumes one host thread launching on the library. */
nis_status nis_profile(nis_ctx *ctx, int enable);
nis_status nis_profile_read(nis_ctx *ctx, const char *family, double *total_ms,
                            int *launches);

/* Plain GEMM on the tensor-core dense-layer kernel, for tests: C[m][n] = sum_k A[m][k] B[n][k]
 * with A (m x k, leading dimension lda) and B (n x k, leading dimension ldb) BF16 row-major
 * device arrays and C FP32 (m x n, dense).  n <= 208; lda and ldb multiples of 8. */
nis_status nis_debug_tc_gemm(nis_ctx *ctx, const void *d_a, int lda, const void *d_b, int ldb,
                             int m, int n, int k, float *d_c, nis_stream stream);

/* The FP32 form of the same kernel, as the FP32 precision mode runs it: A (m x k, leading
 * dimension lda) and B (n x k, leading dimension ldb) are FP32 device arrays; each is split
 * on the device into three BF16 parts (x = x0 + x1 + x2) and the six products of parts whose
 * indices sum to at most 2 are accumulated in FP32 tensor memory.  C FP32 (m x n, dense).
 * n <= 208.  Temporary part buffers are allocated and freed stream-ordered on `stream`. */
nis_status nis_debug_tc_gemm_f32(nis_ctx *ctx, const float *d_a, int lda, const float *d_b,
                                 int ldb, int m, int n, int k, float *d_c, nis_stream stream);

/* Number of kernels this library has launched in the process (all contexts). */
uint64_t nis_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* NIS_H */
