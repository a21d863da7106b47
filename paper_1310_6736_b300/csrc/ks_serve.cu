// Serving: a request loop that admits volumes by their HBM footprint and
// runs the admitted requests' work together in waves.
//
//   ks_submit   copies the raw volume into pinned host memory and queues
//               the request (FIFO).
//   scheduler   (one host thread per context, own CUDA stream) repeats:
//               1. admit queued requests while their footprint fits the
//                  budget next to the requests already on the device;
//               2. set up each newly admitted request: upload + bin the
//                  volume, seed grid, device outputs;
//               3. launch one wave: a single persistent seed launch over the
//                  octant and mean-shift items of every request that joined
//                  since the last wave, plus one z-slab of every dense
//                  request in progress (dense sweeps advance slab by slab,
//                  so a large sweep never holds back later arrivals; a
//                  sweep's slab doubles every 4 waves, so it is not starved
//                  by them either);
//               4. retire finished requests: results to host, device memory
//                  released, waiters woken.
//   ks_poll     waits for a request with a timeout.
// The per-item arithmetic is the plain path's: results are identical
// whether a request runs alone or mixed with others.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "ks_ctx.h"

namespace ks {

static double now_us() {
    using namespace std::chrono;
    static const auto t0 = steady_clock::now();
    return duration<double, std::micro>(steady_clock::now() - t0).count();
}

struct Request {
    int64_t id = 0;
    ks_request desc{};
    void *pinned = nullptr;
    size_t raw_bytes = 0;
    size_t footprint = 0;
    enum State { kPending, kActive, kDone } state = kPending;
    bool canceled = false;
    int status = KS_OK;
    int64_t vol = 0;
    Volume *v = nullptr;
    // device side
    void *dmem = nullptr;
    size_t dbytes = 0;
    int32_t *d_seeds = nullptr;
    ks_seed_result *d_oct = nullptr;
    ks_ms_result *d_ms = nullptr;
    double *d_Y = nullptr;
    uint8_t *d_s = nullptr;
    int64_t n_seeds = 0, n_items = 0, n_vox = 0;
    bool seeds_launched = false;
    int dense_next_z = 0;
    int dense_waves = 0;          // waves this dense request has advanced in
    // host results
    std::vector<ks_seed_result> oct;
    std::vector<ks_ms_result> ms;
    std::vector<double> Y;
    std::vector<uint8_t> s;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::map<int64_t, std::unique_ptr<Request>> all;
    int64_t next_id = 1;
    bool stop = false;
    std::thread th;
    cudaStream_t stream = nullptr;       // uploads, binning, seed waves
    cudaStream_t stream2 = nullptr;      // dense slabs, concurrent with the seeds
    int *d_status = nullptr;
    size_t reserved = 0;
    void *qmem = nullptr;
    size_t qbytes = 0;
    int64_t waves = 0;
};

static size_t dtype_bytes(int d) { return d == KS_U8 ? 1 : d == KS_I16 ? 2 : 4; }

static size_t footprint_of(const ks_request &r) {
    const size_t nvox = (size_t)r.nx * r.ny * r.nz;
    size_t f = volume_bytes(r.nx, r.ny, r.nz) + nvox * dtype_bytes(r.dtype);   // bins + staging
    if (r.kind == KS_REQ_DENSE) {
        f += nvox * 9;
    } else {
        const int st = std::max(1, r.params.stride);
        const size_t ns = (size_t)((r.nx + st - 1) / st) * ((r.ny + st - 1) / st) * ((r.nz + st - 1) / st);
        const int S = r.params.r_max - r.params.r_min + 1;
        f += ns * (12 + sizeof(ks_seed_result) + S * sizeof(ks_ms_result));
    }
    return f + 4096;
}

static void free_device(Ctx *c, Request *r) {
    if (r->dmem) dev_free(c, r->dmem, r->dbytes);
    r->dmem = nullptr;
    r->dbytes = 0;
    if (r->vol) {
        std::unique_ptr<Volume> v;
        {
            std::lock_guard<std::mutex> g(c->mu);
            auto it = c->vols.find(r->vol);
            if (it != c->vols.end()) {
                v = std::move(it->second);
                c->vols.erase(it);
            }
        }
        if (v) dev_free(c, v->alloc, v->bytes);
        r->vol = 0;
        r->v = nullptr;
    }
    if (r->pinned) cudaFreeHost(r->pinned);
    r->pinned = nullptr;
}

// Upload + bin the volume and lay out the request's device buffers.
static int setup(Ctx *c, ServeState *S, Request *r) {
    const ks_request &q = r->desc;
    int st = create_volume_on(c, S->stream, r->pinned, 0, q.dtype, q.nx, q.ny, q.nz, &q.binning,
                              &r->vol);
    if (st) return st;
    r->v = find_volume(c, r->vol);
    r->n_vox = (int64_t)q.nx * q.ny * q.nz;
    std::vector<int32_t> seeds;
    size_t bytes = 256;
    if (q.kind == KS_REQ_DENSE) {
        bytes += r->n_vox * 8 + r->n_vox + 256;
    } else {
        seeds = seed_grid(q.nx, q.ny, q.nz, q.params.stride);
        r->n_seeds = (int64_t)seeds.size() / 3;
        r->n_items = r->n_seeds * (q.params.r_max - q.params.r_min + 1);
        bytes += seeds.size() * 4 + 256 + r->n_seeds * sizeof(ks_seed_result) + 256 +
                 r->n_items * sizeof(ks_ms_result);
    }
    void *p;
    cudaError_t e = dev_alloc(c, &p, bytes);
    if (e != cudaSuccess) return cuda_err(c, e, "serving buffers");
    r->dmem = p;
    r->dbytes = bytes;
    uint8_t *m = (uint8_t *)p;
    if (q.kind == KS_REQ_DENSE) {
        r->d_Y = (double *)m;
        r->d_s = m + (r->n_vox * 8 + 255) / 256 * 256;
    } else {
        r->d_seeds = (int32_t *)m;
        size_t o = (seeds.size() * 4 + 255) / 256 * 256;
        r->d_oct = (ks_seed_result *)(m + o);
        o += (r->n_seeds * sizeof(ks_seed_result) + 255) / 256 * 256;
        r->d_ms = (ks_ms_result *)(m + o);
        if (!seeds.empty()) {
            e = cudaMemcpyAsync(r->d_seeds, seeds.data(), seeds.size() * 4, cudaMemcpyHostToDevice,
                                S->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
            if (e != cudaSuccess) return cuda_err(c, e, "serving seeds");
        }
    }
    return KS_OK;
}

// Dense slab height for one wave: about 3e10 window-voxel updates (roughly
// 12 ms of the dense kernel), so a large sweep advances in a few waves while
// requests that arrive meanwhile still join within one slab's time.
static int dense_slab(const Request *r) {
    const ks_request &q = r->desc;
    const double per_plane = (double)q.nx * q.ny * ball_size_host(q.params.r_max);
    int planes = (int)std::max(1.0, 3e10 / per_plane);
    return std::min(planes, q.nz);
}

static void retire(Ctx *c, ServeState *S, Request *r) {
    const ks_request &q = r->desc;
    if (!r->canceled && r->status == KS_OK) {
        cudaError_t e = cudaSuccess;
        if (q.kind == KS_REQ_DENSE) {
            r->Y.resize(r->n_vox);
            r->s.resize(r->n_vox);
            e = cudaMemcpyAsync(r->Y.data(), r->d_Y, r->n_vox * 8, cudaMemcpyDeviceToHost, S->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->s.data(), r->d_s, r->n_vox, cudaMemcpyDeviceToHost, S->stream);
        } else {
            if (q.seed_kinds & 1) {
                r->oct.resize(r->n_seeds);
                e = cudaMemcpyAsync(r->oct.data(), r->d_oct, r->n_seeds * sizeof(ks_seed_result),
                                    cudaMemcpyDeviceToHost, S->stream);
            }
            if (e == cudaSuccess && (q.seed_kinds & 2)) {
                r->ms.resize(r->n_items);
                e = cudaMemcpyAsync(r->ms.data(), r->d_ms, r->n_items * sizeof(ks_ms_result),
                                    cudaMemcpyDeviceToHost, S->stream);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) r->status = cuda_err(c, e, "serving results");
    }
    if (r->canceled) r->status = KS_ECANCELED;
    free_device(c, r);
    std::lock_guard<std::mutex> g(S->mu);
    r->t_done = now_us();
    r->state = Request::kDone;
    S->reserved -= r->footprint;
    S->cv_done.notify_all();
}

static int launch_wave_seeds(Ctx *c, ServeState *S, std::vector<Request *> &joiners) {
    std::vector<SeedJob> jobs;
    std::vector<std::pair<int, int>> segs;
    for (Request *r : joiners) {
        const ks_request &q = r->desc;
        SeedJob J{};
        J.vol = r->v->desc;
        J.r_min = q.params.r_min;
        J.r_max = q.params.r_max;
        J.S = q.params.r_max - q.params.r_min + 1;
        J.max_iter = q.params.max_iter;
        J.w_norm = q.params.w_norm;
        J.seeds = r->d_seeds;
        J.n_seeds = r->n_seeds;
        J.oct_out = r->d_oct;
        J.ms_out = r->d_ms;
        J.traj = nullptr;
        const int ji = (int)jobs.size();
        jobs.push_back(J);
        if ((q.seed_kinds & 1) && r->n_seeds) segs.push_back({ji, kOctant});
        if ((q.seed_kinds & 2) && r->n_items) segs.push_back({ji, kMeanShift});
    }
    if (segs.empty()) return KS_OK;
    const size_t jobs_bytes = (jobs.size() * sizeof(SeedJob) + 255) / 256 * 256;
    const size_t need = jobs_bytes + plan_bytes_bound(segs.size());
    if (S->qbytes < need) {
        cudaStreamSynchronize(S->stream);
        dev_free(c, S->qmem, S->qbytes);
        S->qmem = nullptr;
        S->qbytes = 0;
        void *p;
        cudaError_t e = dev_alloc(c, &p, need * 2);
        if (e != cudaSuccess) return cuda_err(c, e, "serving queue");
        S->qmem = p;
        S->qbytes = need * 2;
    }
    std::vector<uint8_t> h(jobs_bytes, 0);
    uint8_t *m = (uint8_t *)S->qmem;
    std::memcpy(h.data(), jobs.data(), jobs.size() * sizeof(SeedJob));
    const std::vector<ClassLaunch> cls =
        plan_class_queues(c, jobs, (const SeedJob *)m, segs, h, jobs_bytes, m);
    cudaError_t e = cudaMemcpyAsync(m, h.data(), h.size(), cudaMemcpyHostToDevice, S->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "serving queue upload");
    ProfRec rec;
    prof_begin(c, "ks_seeds_persistent", S->stream, &rec);
    e = launch_class_queues(c, S->stream, S->d_status, cls);
    prof_end(c, &rec, S->stream);
    return cuda_err(c, e, "serving seed wave");
}

static void scheduler(Ctx *c) {
    ServeState *S = c->serve;
    cudaSetDevice(c->device);
    const size_t budget = c->budget ? c->budget : (size_t)60 << 30;
    for (;;) {
        std::vector<Request *> joiners;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop) return;
            while (!S->pending.empty()) {
                Request *r = S->pending.front();
                if (r->canceled) {
                    S->pending.pop_front();
                    r->status = KS_ECANCELED;
                    r->state = Request::kDone;
                    r->t_done = now_us();
                    if (r->pinned) cudaFreeHost(r->pinned);
                    r->pinned = nullptr;
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->reserved + r->footprint > budget && !S->active.empty()) break;
                S->pending.pop_front();
                S->reserved += r->footprint;
                r->state = Request::kActive;
                r->t_admit = now_us();
                S->active.push_back(r);
                joiners.push_back(r);
            }
        }
        // set up the newcomers (outside the lock: uploads and binning)
        std::vector<Request *> seed_joiners;
        for (Request *r : joiners) {
            r->status = setup(c, S, r);
            if (r->status == KS_OK && r->desc.kind == KS_REQ_SEEDS) seed_joiners.push_back(r);
        }
        // one wave
        int wst = launch_wave_seeds(c, S, seed_joiners);
        for (Request *r : seed_joiners) {
            r->seeds_launched = true;
            if (wst) r->status = wst;
        }
        std::vector<Request *> act;
        {
            std::lock_guard<std::mutex> g(S->mu);
            act = S->active;
        }
        for (Request *r : act) {
            if (r->status || r->desc.kind != KS_REQ_DENSE || r->canceled) continue;
            // a sweep's slab doubles every 4 waves it has taken part in (up to
            // 64 times the base slab), so a large sweep that keeps sharing
            // waves with new arrivals still finishes in a few more waves
            const int grow = std::min(r->dense_waves / 4, 6);
            r->dense_waves++;
            const int z0 = r->dense_next_z,
                      z1 = std::min(r->desc.nz, z0 + (dense_slab(r) << grow));
            if (z0 >= z1) continue;
            const DenseOut o{r->d_Y, r->d_s, nullptr, nullptr};
            r->status = run_dense(c, S->stream2, r->v, &r->desc.params, o, z0, z1);
            r->dense_next_z = z1;
        }
        cudaError_t e = cudaStreamSynchronize(S->stream);
        const cudaError_t e2 = cudaStreamSynchronize(S->stream2);
        if (e == cudaSuccess) e = e2;
        int h = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&h, S->d_status, 4, cudaMemcpyDeviceToHost);
        S->waves++;
        // retire
        std::vector<Request *> done;
        for (Request *r : act) {
            if (e != cudaSuccess && r->status == KS_OK) r->status = cuda_err(c, e, "serving wave");
            if (h && r->status == KS_OK) r->status = KS_ETIMEDOUT;
            const bool finished = r->status != KS_OK || r->canceled ||
                                  (r->desc.kind == KS_REQ_SEEDS ? r->seeds_launched
                                                                : r->dense_next_z >= r->desc.nz);
            if (finished) done.push_back(r);
        }
        if (h) cudaMemset(S->d_status, 0, 4);
        {
            std::lock_guard<std::mutex> g(S->mu);
            for (Request *r : done)
                S->active.erase(std::find(S->active.begin(), S->active.end(), r));
        }
        for (Request *r : done) retire(c, S, r);
    }
}

static ServeState *ensure_serve(Ctx *c) {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->serve) return c->serve;
    auto S = std::make_unique<ServeState>();
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithFlags(&S->stream2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(S->stream);
        return nullptr;
    }
    void *p;
    if (cudaMalloc(&p, 256) != cudaSuccess) {
        cudaStreamDestroy(S->stream);
        cudaStreamDestroy(S->stream2);
        return nullptr;
    }
    cudaMemset(p, 0, 256);
    S->d_status = (int *)p;
    c->serve = S.release();
    c->serve->th = std::thread(scheduler, c);
    return c->serve;
}

void serve_shutdown(Ctx *c) {
    if (!c->serve) return;
    ServeState *S = c->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->stream);
    cudaStreamSynchronize(S->stream2);
    for (auto &kv : S->all) free_device(c, kv.second.get());
    dev_free(c, S->qmem, S->qbytes);
    cudaFree(S->d_status);
    cudaStreamDestroy(S->stream);
    cudaStreamDestroy(S->stream2);
    delete S;
    c->serve = nullptr;
}

}  // namespace ks

using namespace ks;

extern "C" {

int ks_submit(ks_ctx *ctx, const ks_request *req, ks_req *out) {
    if (!ctx || !req || !out || !req->data) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_binning(req->dtype, &req->binning, &why);
    if (!st) st = validate_params(&req->params, &why);
    if (st) return set_err(c, st, why);
    if (req->nx < 1 || req->ny < 1 || req->nz < 1 || req->nx > 4096 || req->ny > 4096 ||
        req->nz > 4096)
        return set_err(c, KS_EINVAL, "dims must be in [1, 4096]");
    if (req->kind != KS_REQ_SEEDS && req->kind != KS_REQ_DENSE)
        return set_err(c, KS_EINVAL, "unknown request kind");
    if (req->kind == KS_REQ_SEEDS && !(req->seed_kinds & 3))
        return set_err(c, KS_EINVAL, "seed request with no scheme selected");
    auto r = std::make_unique<Request>();
    r->desc = *req;
    r->footprint = footprint_of(*req);
    const size_t budget = c->budget ? c->budget : (size_t)60 << 30;
    if (r->footprint > budget)
        return set_err(c, KS_ENOMEM, "request footprint exceeds the HBM budget");
    r->raw_bytes = (size_t)req->nx * req->ny * req->nz * dtype_bytes(req->dtype);
    if (cudaMallocHost(&r->pinned, r->raw_bytes) != cudaSuccess)
        return set_err(c, KS_ENOMEM, "pinned staging");
    std::memcpy(r->pinned, req->data, r->raw_bytes);
    r->desc.data = nullptr;
    r->t_submit = now_us();
    ServeState *S = ensure_serve(c);
    if (!S) {
        cudaFreeHost(r->pinned);
        return set_err(c, KS_ECUDA, "serving start-up");
    }
    std::lock_guard<std::mutex> g(S->mu);
    r->id = S->next_id++;
    *out = r->id;
    S->pending.push_back(r.get());
    S->all[r->id] = std::move(r);
    S->cv_work.notify_all();
    return KS_OK;
}

int ks_poll(ks_ctx *ctx, ks_req id, int64_t timeout_us, ks_result *out) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (!c->serve) return KS_ENOTFOUND;
    ServeState *S = c->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return KS_ENOTFOUND;
    Request *r = it->second.get();
    auto done = [&] { return r->state == Request::kDone; };
    if (!done()) {
        if (timeout_us == 0) return KS_PENDING;
        if (timeout_us < 0)
            S->cv_done.wait(lk, done);
        else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
            return KS_ETIMEDOUT;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->status = r->status;
        out->kind = r->desc.kind;
        out->n_seeds = r->n_seeds;
        out->n_items = r->n_items;
        out->n_voxels = r->n_vox;
        out->oct = r->oct.empty() ? nullptr : r->oct.data();
        out->ms = r->ms.empty() ? nullptr : r->ms.data();
        out->Y_best = r->Y.empty() ? nullptr : r->Y.data();
        out->s_best = r->s.empty() ? nullptr : r->s.data();
        out->t_submit_us = r->t_submit;
        out->t_admit_us = r->t_admit;
        out->t_done_us = r->t_done;
    }
    return r->status == KS_OK ? KS_OK : r->status;
}

int ks_cancel(ks_ctx *ctx, ks_req id) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (!c->serve) return KS_ENOTFOUND;
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return KS_ENOTFOUND;
    if (it->second->state != Request::kDone) it->second->canceled = true;
    S->cv_work.notify_all();
    return KS_OK;
}

int ks_release_result(ks_ctx *ctx, ks_req id) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (!c->serve) return KS_ENOTFOUND;
    ServeState *S = c->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return KS_ENOTFOUND;
    if (it->second->state != Request::kDone) return set_err(c, KS_EINVAL, "request not finished");
    S->all.erase(it);
    return KS_OK;
}

}  // extern "C"
