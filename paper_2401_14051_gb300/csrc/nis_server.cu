// Serving loop (include/nis.h, "serving"): continuous batching of render requests with
// device-resident pyramid and transmittance caches and admission by HBM budget.
//
// One host thread runs the loop.  Each iteration:
//   1. admits queued requests in arrival order while the in-flight limit and the budget
//      allow (evicting unreferenced cached volumes / lights least-recently-used), and
//      enqueues their preparation on the prep stream: upload + pyramid (cache miss),
//      transmittance (cache miss), compacted first hits, hit count read-back;
//   2. marks requests whose preparation event completed as ready;
//   3. when the previous batch has drained, shades up to max_batch_points points as one mixed
//      batch on the shade stream: the oldest ready request takes up to half of the room and
//      the other ready requests share the rest equally (so every ready request advances in
//      every batch, and the oldest at least half as fast as alone); what a request cannot use
//      goes to the others in admission order; a request whose last points are in the batch
//      gets its image scattered and copied to a page-locked staging buffer behind the batch;
//   4. retires requests whose image copy completed: copies it to rgb_out, records the
//      latency, releases its buffers (stream-ordered frees) and its cache references.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "nis_internal.h"

using namespace nis;
using Clock = std::chrono::steady_clock;

namespace {

// kFailing: every point was handed out but the image can never be produced (a shading or
// read-back error); the loop retires it as failed.
enum { kQueued = 0, kPrep = 1, kReady = 2, kFinishing = 3, kDone = 4, kFailed = 5, kFailing = 6 };

struct Req {
    uint64_t id = 0;
    nis_request r{};
    std::atomic<int> state{kQueued};   // written by the server thread, read by waiters
    Clock::time_point t_submit, t_done;
    nis_volume vol = 0;
    nis_light light = 0;
    uint64_t vkey = 0;                 // cache key (0: uncached volume owned by the request)
    int pixels = 0;
    float *pts = nullptr, *om = nullptr, *rgb = nullptr, *img = nullptr;
    int *pix = nullptr, *d_count = nullptr;
    int *h_count = nullptr;            // page-locked
    float *h_img = nullptr;            // page-locked staging of the image
    size_t h_img_bytes = 0;
    int n_points = 0, shaded = 0;
    cudaEvent_t ev_prep = nullptr, ev_done = nullptr;
    size_t dev_bytes = 0;
    nis_status err = NIS_OK;
};

struct VolEntry {
    nis_volume h = 0;
    int refs = 0;
    uint64_t last_use = 0;
    size_t bytes = 0;
};

struct LightKey {
    uint64_t vkey;
    float dir[3];
    float lam;
    bool operator<(const LightKey &o) const {
        if (vkey != o.vkey) return vkey < o.vkey;
        int c = std::memcmp(dir, o.dir, sizeof(dir));
        if (c) return c < 0;
        return lam < o.lam;
    }
};

struct LightEntry {
    nis_light h = 0;
    int refs = 0;
    uint64_t last_use = 0;
    size_t bytes = 0;
};

size_t level_floats(int n) {
    size_t total = 0;
    for (int sz = n;; sz = (sz + 1) / 2) {
        total += (size_t)sz * sz * sz;
        if (sz == 1) break;
    }
    return total;
}
// a light: its transmittance pyramid and the (density, transmittance) pairs of the gathers
size_t light_bytes(int n) {
    size_t pairs = 0;
    for (int sz = n;; sz = (sz + 1) / 2) {
        pairs += pair_level_float4(sz);
        if (sz == 1) break;
    }
    return level_floats(n) * 4 + pairs * 16;
}
// what a shear-warp build may add: the volume's x-major pyramid copy and its occupancy
// (new volumes), the context's x-major output and ray states (grow-only, bounded here by
// this grid's size)
size_t sweep_bytes(int n, bool new_volume) {
    size_t rays = 0;
    const size_t slices = (size_t)sw_slices(n);         // ray states kept per step of a chunk
    for (int sz = n;; sz = (sz + 1) / 2) {
        rays += slices * (size_t)(2 * sz + 3) * (2 * sz + 3) * 8;
        if (sz == 1) break;
    }
    return (new_volume ? level_floats(n) * 5 : 0) + level_floats(n) * 4 + rays;
}

}  // namespace

struct nis_server {
    nis_ctx *ctx = nullptr;
    nis_weights w = 0;
    nis_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::map<uint64_t, Req *> reqs;
    std::vector<Req *> active;                    // admitted, in admission order
    std::map<uint64_t, VolEntry> vols;
    std::map<LightKey, LightEntry> lights;
    uint64_t next_id = 1, tick = 0;
    cudaStream_t prep = nullptr, shade = nullptr;
    cudaEvent_t ev_batch = nullptr;
    bool batch_in_flight = false;
    size_t req_bytes = 0;                         // per-request device buffers outstanding
    std::thread th;
    std::atomic<bool> stop{false};
    // statistics
    std::vector<double> lat_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, points = 0, batches = 0;
    double batch_points_sum = 0, batch_reqs_sum = 0;
    uint64_t vhit = 0, vmiss = 0, lhit = 0, lmiss = 0, evictions = 0;
    size_t peak = 0;
    Clock::time_point t_first, t_last;
    bool any_submit = false;
    // test hook: requests whose shading is to be treated as failed, with the status
    std::map<uint64_t, nis_status> injected;
};

namespace {

size_t held_bytes(nis_server *S) { return nis_bytes_in_use(S->ctx) + S->req_bytes; }

void note_peak(nis_server *S) { S->peak = std::max(S->peak, held_bytes(S)); }

// Frees one unreferenced cache entry (lights first, then volumes), least recently used.
bool evict_one(nis_server *S) {
    auto lit = S->lights.end();
    for (auto it = S->lights.begin(); it != S->lights.end(); ++it)
        if (it->second.refs == 0 && (lit == S->lights.end() || it->second.last_use < lit->second.last_use))
            lit = it;
    if (lit != S->lights.end()) {
        nis_release(S->ctx, lit->second.h);
        S->lights.erase(lit);
        ++S->evictions;
        return true;
    }
    auto vit = S->vols.end();
    for (auto it = S->vols.begin(); it != S->vols.end(); ++it) {
        if (it->second.refs != 0) continue;
        bool lit_ref = false;
        for (auto &kv : S->lights)
            if (kv.first.vkey == it->first && kv.second.refs) lit_ref = true;
        if (!lit_ref && (vit == S->vols.end() || it->second.last_use < vit->second.last_use)) vit = it;
    }
    if (vit != S->vols.end()) {
        for (auto it = S->lights.begin(); it != S->lights.end();)
            it = it->first.vkey == vit->first ? S->lights.erase(it) : std::next(it);
        nis_release(S->ctx, vit->second.h);       // also frees its lights
        S->vols.erase(vit);
        ++S->evictions;
        return true;
    }
    return false;
}

size_t request_bytes(const Req *q) {
    return (size_t)q->pixels * (3 * 4 * 3 + 4 + 3 * 4) + 256;
}

template <typename T>
cudaError_t salloc(nis_server *S, T **p, size_t count, size_t *acc) {
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), bytes, S->prep);
    if (e == cudaSuccess) *acc += bytes;
    return e;
}

void free_request(nis_server *S, Req *q) {
    cudaStream_t s = S->shade;
    for (void *p : {(void *)q->pts, (void *)q->om, (void *)q->rgb, (void *)q->img, (void *)q->pix,
                    (void *)q->d_count})
        if (p) cudaFreeAsync(p, s);
    q->pts = q->om = q->rgb = q->img = nullptr;
    q->pix = q->d_count = nullptr;
    S->req_bytes -= q->dev_bytes;
    q->dev_bytes = 0;
    if (q->h_count) { cudaFreeHost(q->h_count); q->h_count = nullptr; }
    if (q->h_img) { cudaFreeHost(q->h_img); q->h_img = nullptr; }
    if (q->ev_prep) { cudaEventDestroy(q->ev_prep); q->ev_prep = nullptr; }
    if (q->ev_done) { cudaEventDestroy(q->ev_done); q->ev_done = nullptr; }
    if (q->vkey) {
        auto it = S->vols.find(q->vkey);
        if (it != S->vols.end()) it->second.refs--;
        LightKey k{q->vkey, {q->r.light_dir[0], q->r.light_dir[1], q->r.light_dir[2]}, q->r.lambda};
        auto lt = S->lights.find(k);
        if (lt != S->lights.end()) lt->second.refs--;
    } else if (q->vol) {
        nis_release(S->ctx, q->vol);
        q->vol = 0;
    }
}

void finish(nis_server *S, Req *q, int state, nis_status err) {
    std::lock_guard<std::mutex> lk(S->mu);
    q->state = state;
    q->err = err;
    q->t_done = Clock::now();
    S->t_last = q->t_done;
    if (state == kDone) {
        ++S->completed;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
    } else {
        ++S->failed;
    }
    S->cv_done.notify_all();
}

// Enqueues the preparation of an admitted request on the prep stream.
nis_status prepare(nis_server *S, Req *q) {
    nis_ctx *ctx = S->ctx;
    cudaStream_t ps = S->prep;
    nis_stream st = reinterpret_cast<nis_stream>(ps);
    nis_status rc;
    q->vkey = q->r.volume_key;
    // volume + pyramid (cached by key)
    if (q->vkey) {
        auto it = S->vols.find(q->vkey);
        if (it != S->vols.end()) {
            ++S->vhit;
            it->second.refs++;
            it->second.last_use = ++S->tick;
            q->vol = it->second.h;
        } else {
            ++S->vmiss;
            if ((rc = nis_upload_volume(ctx, q->r.density, q->r.n, q->r.n, q->r.n, q->r.dtype, 0, 1.0f,
                                        st, &q->vol)))
                return rc;
            if ((rc = nis_build_pyramid(ctx, q->vol, st))) return rc;
            VolEntry e;
            e.h = q->vol; e.refs = 1; e.last_use = ++S->tick; e.bytes = level_floats(q->r.n) * 4;
            S->vols[q->vkey] = e;
        }
        LightKey k{q->vkey, {q->r.light_dir[0], q->r.light_dir[1], q->r.light_dir[2]}, q->r.lambda};
        auto lt = S->lights.find(k);
        if (lt != S->lights.end()) {
            ++S->lhit;
            lt->second.refs++;
            lt->second.last_use = ++S->tick;
            q->light = lt->second.h;
        } else {
            ++S->lmiss;
            if ((rc = nis_build_transmittance_method(ctx, q->vol, q->r.light_dir, q->r.lambda,
                                                      S->cfg.transmittance_method, st, &q->light)))
                return rc;
            LightEntry e;
            e.h = q->light; e.refs = 1; e.last_use = ++S->tick; e.bytes = light_bytes(q->r.n);
            S->lights[k] = e;
        }
    } else {
        ++S->vmiss;
        ++S->lmiss;
        if ((rc = nis_upload_volume(ctx, q->r.density, q->r.n, q->r.n, q->r.n, q->r.dtype, 0, 1.0f, st,
                                    &q->vol)))
            return rc;
        if ((rc = nis_build_pyramid(ctx, q->vol, st))) return rc;
        if ((rc = nis_build_transmittance_method(ctx, q->vol, q->r.light_dir, q->r.lambda,
                                                      S->cfg.transmittance_method, st, &q->light)))
            return rc;
    }
    // per-request buffers and first hits
    size_t px = (size_t)q->pixels;
    size_t acc = 0;
    if (salloc(S, &q->pts, 3 * px, &acc) || salloc(S, &q->om, 3 * px, &acc) ||
        salloc(S, &q->rgb, 3 * px, &acc) || salloc(S, &q->img, 3 * px, &acc) ||
        salloc(S, &q->pix, px, &acc) || salloc(S, &q->d_count, 1, &acc)) {
        cudaGetLastError();
        q->dev_bytes = acc;
        S->req_bytes += acc;
        return NIS_ERR_OOM;
    }
    q->dev_bytes = acc;
    S->req_bytes += acc;
    if (cudaMallocHost(&q->h_count, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return NIS_ERR_OOM; }
    if ((rc = hits_compact(ctx, q->vol, &q->r.camera, q->pts, q->om, q->pix, q->d_count, ps))) return rc;
    if (cudaMemsetAsync(q->img, 0, 12 * px, ps) != cudaSuccess ||
        cudaMemcpyAsync(q->h_count, q->d_count, sizeof(int), cudaMemcpyDeviceToHost, ps) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_prep, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(q->ev_prep, ps) != cudaSuccess) {
        cudaGetLastError();
        return NIS_ERR_CUDA;
    }
    note_peak(S);
    return NIS_OK;
}

// Image of a finished request: scatter the shaded points and copy to page-locked staging.
nis_status schedule_output(nis_server *S, Req *q) {
    cudaStream_t s = S->shade;
    launch_scatter_rgb(q->rgb, q->pix, q->n_points, q->img, q->pixels, s);
    q->h_img_bytes = (size_t)q->pixels * 12;
    if (cudaMallocHost(&q->h_img, q->h_img_bytes) != cudaSuccess ||
        cudaMemcpyAsync(q->h_img, q->img, q->h_img_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(q->ev_done, s) != cudaSuccess) {
        cudaGetLastError();
        return NIS_ERR_CUDA;
    }
    q->state = kFinishing;
    return NIS_OK;
}

void loop(nis_server *S) {
    cudaSetDevice(ctx_device(S->ctx));
    while (true) {
        bool worked = false;
        // 1. admission
        while (true) {
            Req *q = nullptr;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (S->queue.empty() || (int)S->active.size() >= S->cfg.max_inflight) break;
                q = S->queue.front();
            }
            size_t need = request_bytes(q) + light_bytes(q->r.n);   // light, if not cached
            bool cached_vol = q->r.volume_key && S->vols.count(q->r.volume_key);
            if (!cached_vol) need += level_floats(q->r.n) * 4 + (size_t)q->r.n * q->r.n * q->r.n * 4;
            if (S->cfg.transmittance_method == NIS_TRANSMITTANCE_SHEAR_WARP)
                need += sweep_bytes(q->r.n, !cached_vol);
            if (S->cfg.hbm_budget_bytes) {
                while (held_bytes(S) + need > S->cfg.hbm_budget_bytes && evict_one(S)) {
                }
                if (held_bytes(S) + need > S->cfg.hbm_budget_bytes) {
                    if (S->active.empty()) {              // can never fit
                        { std::lock_guard<std::mutex> lk(S->mu); S->queue.pop_front(); }
                        finish(S, q, kFailed, NIS_ERR_BUDGET);
                        worked = true;
                        continue;
                    }
                    break;                                // wait for memory to free up
                }
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->queue.pop_front();
                q->state = kPrep;
                S->active.push_back(q);
            }
            nis_status rc = prepare(S, q);
            if (rc) {
                cudaStreamSynchronize(S->prep);
                free_request(S, q);
                { std::lock_guard<std::mutex> lk(S->mu);
                  S->active.erase(std::find(S->active.begin(), S->active.end(), q)); }
                finish(S, q, kFailed, rc);
            }
            worked = true;
        }
        // 2. preparation done
        for (Req *q : S->active)
            if (q->state == kPrep && cudaEventQuery(q->ev_prep) == cudaSuccess) {
                q->n_points = *q->h_count;
                q->state = kReady;
                if (q->n_points == 0 && schedule_output(S, q) != NIS_OK) {
                    q->err = NIS_ERR_CUDA;
                    q->state = kFailing;
                }
                worked = true;
            }
        // 3. one mixed batch at a time (the host prepares the next while it runs)
        if (S->batch_in_flight && cudaEventQuery(S->ev_batch) == cudaSuccess) S->batch_in_flight = false;
        if (!S->batch_in_flight) {
            std::vector<nis_segment> segs;
            std::vector<Req *> last, in_batch;
            int room = S->cfg.max_batch_points;
            std::vector<Req *> ready;
            for (Req *q : S->active) {
                if (q->state == kReady && q->err) {   // an earlier batch failed: shade no more
                    q->state = kFailing;              // of it; retired after its batches drain
                    continue;
                }
                if (q->state == kReady && q->shaded < q->n_points) ready.push_back(q);
            }
            // the next `take` points of q as a segment of the batch
            auto add = [&](Req *q, int take) {
                nis_segment sg{};
                sg.vol = q->vol; sg.light = q->light; sg.material = q->r.material;
                sg.d_points = q->pts + 3 * (size_t)q->shaded;
                sg.d_omega = q->om + 3 * (size_t)q->shaded;
                sg.n = take;
                sg.d_rgb_out = q->rgb + 3 * (size_t)q->shaded;
                segs.push_back(sg);
                if (std::find(in_batch.begin(), in_batch.end(), q) == in_batch.end()) in_batch.push_back(q);
                q->shaded += take;
                room -= take;
                if (q->shaded == q->n_points) last.push_back(q);
            };
            if (!ready.empty()) {
                // the oldest ready request takes up to half of the room (at least one point, so
                // that a batch of one point still serves it first), the others an equal share
                // of the rest; then what is left, in admission order
                Req *head = ready.front();
                add(head, std::min(head->n_points - head->shaded,
                                   ready.size() > 1 ? std::max(1, room / 2) : room));
                if (ready.size() > 1) {
                    const int share = (room + (int)ready.size() - 2) / ((int)ready.size() - 1);
                    for (size_t i = 1; i < ready.size() && room > 0; ++i)
                        add(ready[i], std::min({ready[i]->n_points - ready[i]->shaded, share, room}));
                }
                for (Req *q : ready)
                    if (room > 0 && q->shaded < q->n_points) add(q, std::min(q->n_points - q->shaded, room));
            }
            if (!segs.empty()) {
                nis_status rc = nis_shade_segments(S->ctx, S->w, segs.data(), (int)segs.size(),
                                                   reinterpret_cast<nis_stream>(S->shade));
                if (rc)                           // every request of the batch has lost points
                    for (Req *q : in_batch) q->err = rc;
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    for (Req *q : in_batch) {
                        auto it = S->injected.find(q->id);
                        if (it != S->injected.end()) { q->err = it->second; S->injected.erase(it); }
                    }
                }
                for (Req *q : last) {
                    const nis_status ro = q->err ? q->err : schedule_output(S, q);
                    if (ro) { q->err = ro; q->state = kFailing; }
                }
                cudaEventRecord(S->ev_batch, S->shade);
                S->batch_in_flight = true;
                ++S->batches;
                S->batch_points_sum += S->cfg.max_batch_points - room;
                S->batch_reqs_sum += in_batch.size();
                S->points += S->cfg.max_batch_points - room;
                worked = true;
            }
        }
        // 4. retire
        for (size_t i = 0; i < S->active.size();) {
            Req *q = S->active[i];
            if (q->state == kFinishing && cudaEventQuery(q->ev_done) == cudaSuccess) {
                std::memcpy(q->r.rgb_out, q->h_img, q->h_img_bytes);
                nis_status err = q->err;
                free_request(S, q);
                { std::lock_guard<std::mutex> lk(S->mu); S->active.erase(S->active.begin() + i); }
                finish(S, q, err ? kFailed : kDone, err);
                worked = true;
            } else if (q->state == kFailing) {
                // its buffers are freed in stream order after the batch that used them; a
                // read-back that may have been issued is waited for before its staging goes
                cudaStreamSynchronize(S->shade);
                cudaGetLastError();
                const nis_status err = q->err ? q->err : NIS_ERR_CUDA;
                free_request(S, q);
                { std::lock_guard<std::mutex> lk(S->mu); S->active.erase(S->active.begin() + i); }
                finish(S, q, kFailed, err);
                worked = true;
            } else {
                ++i;
            }
        }
        if (!worked) {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty() && S->active.empty()) break;
            S->cv_work.wait_for(lk, std::chrono::microseconds(100));
        }
    }
}

}  // namespace

extern "C" {

nis_status nis_server_inject_failure(nis_server *srv, uint64_t id, nis_status status) {
    if (!srv || status >= 0) return NIS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->injected[id] = status;
    return NIS_OK;
}

nis_status nis_server_create(nis_ctx *ctx, nis_weights w, const nis_server_config *cfg,
                             nis_server **out) {
    if (!ctx || !cfg || !out) return NIS_ERR_INVALID_ARG;
    if (cfg->max_batch_points < 1 || cfg->max_batch_points > 65536 || cfg->max_inflight < 1)
        return record_error(ctx, NIS_ERR_INVALID_ARG, "max_batch_points in [1, 65536], max_inflight >= 1");
    if (cfg->transmittance_method != NIS_TRANSMITTANCE_MARCH &&
        cfg->transmittance_method != NIS_TRANSMITTANCE_SHEAR_WARP)
        return record_error(ctx, NIS_ERR_INVALID_ARG, "unknown transmittance method");
    if (weights_model(ctx, w) != kModelLattice)
        return record_error(ctx, NIS_ERR_UNIMPLEMENTED, "the server batches lattice-model weights");
    nis_server *S = new nis_server();
    S->ctx = ctx;
    cudaSetDevice(ctx_device(ctx));
    S->w = w;
    S->cfg = *cfg;
    if (cudaStreamCreateWithFlags(&S->prep, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->shade, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->ev_batch, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return record_error(ctx, NIS_ERR_CUDA, "stream creation failed");
    }
    S->th = std::thread(loop, S);
    *out = S;
    return NIS_OK;
}

nis_status nis_server_submit(nis_server *S, const nis_request *r, uint64_t *id) {
    if (!S || !r || !id) return NIS_ERR_INVALID_ARG;
    if (!r->density || !r->rgb_out || r->n < 1 || r->n > 2048 ||
        (r->dtype != NIS_DTYPE_F32 && r->dtype != NIS_DTYPE_F16) || r->camera.width < 1 ||
        r->camera.height < 1 || (long long)r->camera.width * r->camera.height > (1LL << 26) ||
        material_problem(&r->material))          // refused here, not in a shared batch
        return NIS_ERR_INVALID_ARG;
    Req *q = new Req();
    q->r = *r;
    q->pixels = r->camera.width * r->camera.height;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->id = S->next_id++;
        S->reqs[q->id] = q;
        S->queue.push_back(q);
        ++S->submitted;
        if (!S->any_submit) { S->any_submit = true; S->t_first = q->t_submit; }
    }
    S->cv_work.notify_one();
    *id = q->id;
    return NIS_OK;
}

nis_status nis_server_wait(nis_server *S, uint64_t id, int timeout_ms, double *latency_ms) {
    if (!S) return NIS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return NIS_ERR_INVALID_ARG;
    Req *q = it->second;
    auto done = [&] { return q->state == kDone || q->state == kFailed; };
    if (timeout_ms > 0) {
        if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return NIS_ERR_TIMEOUT;
    } else {
        S->cv_done.wait(lk, done);
    }
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    return q->state == kDone ? NIS_OK : (q->err ? q->err : NIS_ERR_CUDA);
}

nis_status nis_server_get_stats(nis_server *S, nis_server_stats *o) {
    if (!S || !o) return NIS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(o, 0, sizeof(*o));
    o->submitted = S->submitted;
    o->completed = S->completed;
    o->failed = S->failed;
    std::vector<double> l = S->lat_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            size_t i = (size_t)std::min<double>(l.size() - 1, std::ceil(p * l.size()) - 1);
            return l[i];
        };
        o->p50_ms = pct(0.50);
        o->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : l) sum += x;
        o->mean_ms = sum / l.size();
        o->max_ms = l.back();
    }
    o->points_shaded = S->points;
    o->batches = S->batches;
    o->mean_batch_points = S->batches ? S->batch_points_sum / S->batches : 0;
    o->mean_batch_requests = S->batches ? S->batch_reqs_sum / S->batches : 0;
    o->volume_hits = S->vhit;
    o->volume_misses = S->vmiss;
    o->light_hits = S->lhit;
    o->light_misses = S->lmiss;
    o->evictions = S->evictions;
    o->peak_bytes = S->peak;
    if (S->any_submit && S->completed)
        o->span_seconds = std::chrono::duration<double>(S->t_last - S->t_first).count();
    return NIS_OK;
}

void nis_server_destroy(nis_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->prep);
    cudaStreamSynchronize(S->shade);
    for (auto &kv : S->lights) nis_release(S->ctx, kv.second.h);
    for (auto &kv : S->vols) nis_release(S->ctx, kv.second.h);
    for (auto &kv : S->reqs) delete kv.second;
    cudaEventDestroy(S->ev_batch);
    cudaStreamDestroy(S->prep);
    cudaStreamDestroy(S->shade);
    delete S;
}

}  // extern "C"
