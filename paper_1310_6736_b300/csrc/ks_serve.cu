// Serving: continuous batching of saliency requests (volumes of different
// sizes arriving over time) on one device.
//
//   ks_submit   copies the raw volume (and, for seed requests, its seed
//               grid) into pinned host memory from a pool and queues the
//               request (FIFO).
//   scheduler   one host thread per context; it never waits for the device
//               as a whole, only polls events, and repeats:
//     admit     queued requests while their footprint fits the HBM budget
//               next to the requests on the device;
//     set up    each admitted request on the upload stream: device buffers
//               from an arena (no cudaMalloc once the arena has grown),
//               upload, binning, zeroed item state -- asynchronously, with
//               an event;
//     seeds     iteration-level waves on the seed stream: one persistent
//               launch per (bins, scales, kind) class over the items of
//               every seed request that is set up and not finished; each
//               item advances at most `wave_iters` iterations from its
//               state in device memory (centre, iteration, flags) and, when
//               its search ends, writes its record and counts itself in its
//               request's finished counter.  A request that becomes ready
//               joins the next wave; up to two waves are queued on the
//               stream, so the device never idles between them;
//     dense     sweeps run whole on their own stream, one at a time from a
//               host queue in the order they became ready, at the seed
//               waves' priority: blocks of both take SMs as others retire,
//               and each fills the SMs the other leaves idle.  (Handing
//               every ready sweep to the stream at once raised the median
//               latency of 2000 requests at 50 /s from 1.1 to 10.3 s and the
//               99th percentile from 40 to 58 s.  Sweeps at the lowest
//               priority gave a median of 0.21 s against 1.08 s, but 37.7
//               against 40.1 volumes/s and a 99th percentile of 19.7 against
//               14.9 s);
//     results   a finished request's records go to pinned host memory on
//               the download stream; when that copy's event has completed
//               the request is done and its device memory returns to the
//               arena (after the last wave that listed it).
//   ks_poll     waits for a request with a timeout.
// The per-item arithmetic is the plain path's and a resumed search takes
// the same steps as a whole one, so results are identical whether a
// request runs alone or mixed with others, in waves of any length.
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

static size_t round256(size_t n) { return (n + 255) / 256 * 256; }

// ------------------------------------------------------------ device arena
// Device memory for requests, carved out of large chunks with a first-fit
// free list; chunks are only returned at shutdown, so a steady stream of
// requests makes no cudaMalloc / cudaFree (each of which synchronises the
// device).
struct Arena {
    struct Chunk {
        uint8_t *base = nullptr;
        size_t size = 0;
        std::map<size_t, size_t> free;   // offset -> bytes
    };
    std::vector<Chunk> chunks;
    static constexpr size_t kChunkMin = size_t(512) << 20;

    void *alloc(Ctx *c, size_t bytes) {
        bytes = round256(std::max<size_t>(bytes, 256));
        for (Chunk &ch : chunks)
            for (auto it = ch.free.begin(); it != ch.free.end(); ++it)
                if (it->second >= bytes) {
                    const size_t off = it->first, sz = it->second;
                    ch.free.erase(it);
                    if (sz > bytes) ch.free[off + bytes] = sz - bytes;
                    return ch.base + off;
                }
        Chunk ch;
        ch.size = std::max(bytes, kChunkMin);
        void *p = nullptr;
        if (dev_alloc(c, &p, ch.size) != cudaSuccess) {
            // no room for a whole chunk: try exactly what is needed
            ch.size = bytes;
            if (dev_alloc(c, &p, ch.size) != cudaSuccess) return nullptr;
        }
        ch.base = (uint8_t *)p;
        if (ch.size > bytes) ch.free[bytes] = ch.size - bytes;
        chunks.push_back(std::move(ch));
        return p;
    }
    void release(void *p, size_t bytes) {
        if (!p) return;
        bytes = round256(std::max<size_t>(bytes, 256));
        for (Chunk &ch : chunks) {
            uint8_t *q = (uint8_t *)p;
            if (q < ch.base || q >= ch.base + ch.size) continue;
            size_t off = (size_t)(q - ch.base), sz = bytes;
            auto nx = ch.free.lower_bound(off);
            if (nx != ch.free.end() && off + sz == nx->first) {     // merge with the next block
                sz += nx->second;
                nx = ch.free.erase(nx);
            }
            if (nx != ch.free.begin()) {                           // and with the previous one
                auto pv = std::prev(nx);
                if (pv->first + pv->second == off) {
                    pv->second += sz;
                    return;
                }
            }
            ch.free[off] = sz;
            return;
        }
    }
    void destroy(Ctx *c) {
        for (Chunk &ch : chunks) dev_free(c, ch.base, ch.size);
        chunks.clear();
    }
};

// --------------------------------------------------------- pinned host pool
// Pinned buffers in power-of-two sizes, kept for reuse (cudaMallocHost is
// slow and may synchronise); at most kKeep bytes are kept.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, void *> free;
    size_t kept = 0;
    static constexpr size_t kKeep = size_t(8) << 30;

    static size_t bucket(size_t n) {
        size_t b = 64 << 10;
        while (b < n) b <<= 1;
        return b;
    }
    void *get(size_t n, size_t *got) {
        const size_t b = bucket(n);
        *got = b;
        {
            std::lock_guard<std::mutex> g(mu);
            auto it = free.find(b);
            if (it != free.end()) {
                void *p = it->second;
                free.erase(it);
                kept -= b;
                return p;
            }
        }
        void *p = nullptr;
        return cudaMallocHost(&p, b) == cudaSuccess ? p : nullptr;
    }
    void put(void *p, size_t b) {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu);
        if (kept + b > kKeep) {
            cudaFreeHost(p);
            return;
        }
        free.emplace(b, p);
        kept += b;
    }
    void destroy() {
        std::lock_guard<std::mutex> g(mu);
        for (auto &kv : free) cudaFreeHost(kv.second);
        free.clear();
        kept = 0;
    }
};

// ----------------------------------------------------------------- requests
constexpr int kMaxSlots = 4096;        // finished-item counters (requests on the device)
constexpr int kMaxWavesInFlight = 2;
constexpr int kDefaultWaveIters = 0;      // whole searches: measured best at 20-100 requests/s

struct Request {
    int64_t id = 0;
    ks_request desc{};
    void *pinned = nullptr;            // raw volume, then the seed grid (pool buffer)
    size_t pin_bytes = 0;
    size_t raw_bytes = 0;
    size_t footprint = 0;
    enum State { kPending, kSetup, kReady, kRunning, kDownload, kDone } state = kPending;
    bool canceled = false;
    int status = KS_OK;
    Volume vol;
    void *dmem = nullptr;              // arena block holding every device buffer
    size_t dbytes = 0;
    int slot = -1;
    int32_t *d_seeds = nullptr;
    ks_seed_result *d_oct = nullptr;
    ks_ms_result *d_ms = nullptr;
    int4 *d_state = nullptr;
    double *d_Y = nullptr;
    uint8_t *d_s = nullptr;
    int64_t n_seeds = 0, n_items = 0, n_vox = 0, n_total = 0;
    int64_t last_wave = -1;            // sequence number of the last wave that listed it

    cudaEvent_t ev = nullptr;          // completion of the current stage
    void *res = nullptr;               // pinned results
    size_t res_bytes = 0;
    ks_seed_result *oct = nullptr;
    ks_ms_result *ms = nullptr;
    double *Y = nullptr;
    uint8_t *s = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Wave {
    int64_t seq = 0;
    std::vector<Request *> members;
    cudaEvent_t ev = nullptr;
    int buf = 0;                       // queue buffer in use
};

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> active;     // admitted, not done (scheduler thread only after admission)
    std::map<int64_t, std::unique_ptr<Request>> all;
    int64_t next_id = 1;
    bool stop = false;
    std::thread th;
    cudaStream_t s_up = nullptr, s_seed = nullptr, s_dense = nullptr, s_down = nullptr;
    std::deque<Request *> dense_ready;        // set up, not started (oldest first)
    Request *dense_on = nullptr;              // the sweep in flight on s_dense
    int *d_status = nullptr;
    unsigned int *d_counters = nullptr;     // kMaxSlots finished-item counters
    std::vector<int> free_slots;
    size_t reserved = 0;
    Arena arena;
    PinnedPool pool;
    // double-buffered queue images of the waves (device + pinned host)
    void *qdev[kMaxWavesInFlight] = {};
    size_t qdev_bytes[kMaxWavesInFlight] = {};
    void *qhost[kMaxWavesInFlight] = {};
    size_t qhost_bytes[kMaxWavesInFlight] = {};
    // per wave: counters and the status word, copied back after the wave
    unsigned int *h_counts[kMaxWavesInFlight] = {};
    std::deque<Wave> waves;
    int64_t wave_seq = 0, waves_done = 0;
    int next_buf = 0;
    int wave_iters = kDefaultWaveIters;
    std::vector<cudaEvent_t> ev_pool;
};

static size_t dtype_bytes(int d) { return d == KS_U8 ? 1 : d == KS_I16 ? 2 : 4; }

static int64_t seeds_of(const ks_request &r) {
    const int st = std::max(1, r.params.stride);
    auto cnt = [&](int n) { return (int64_t)(n > st / 2 ? (n - st / 2 + st - 1) / st : 0); };
    return cnt(r.nx) * cnt(r.ny) * cnt(r.nz);
}

// Device bytes a request occupies while admitted.
static size_t footprint_of(const ks_request &r, int num_sms) {
    const size_t nvox = (size_t)r.nx * r.ny * r.nz;
    size_t f = round256(volume_bytes(r.nx, r.ny, r.nz)) + round256(nvox * dtype_bytes(r.dtype)) +
               round256((size_t)bin_f32_scratch_blocks(num_sms) * sizeof(float2));
    if (r.kind == KS_REQ_DENSE) {
        f += round256(nvox * 8) + round256(nvox);
    } else {
        const int64_t ns = seeds_of(r);
        const int S = r.params.r_max - r.params.r_min + 1;
        f += round256(ns * 12) + round256(ns * sizeof(ks_seed_result)) +
             round256(ns * S * sizeof(ks_ms_result)) + round256((ns + ns * S) * sizeof(int4));
    }
    return f + 4096;
}

static cudaEvent_t take_event(ServeState *S) {
    if (!S->ev_pool.empty()) {
        cudaEvent_t e = S->ev_pool.back();
        S->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

static void give_event(ServeState *S, cudaEvent_t &e) {
    if (e) S->ev_pool.push_back(e);
    e = nullptr;
}

// Upload, binning and zeroed item state, all on the upload stream; records
// r->ev.  Returns KS_ENOMEM when the arena has no room yet (the request
// stays queued), another error for a failed request.
static int setup(Ctx *c, ServeState *S, Request *r) {
    const ks_request &q = r->desc;
    Volume &v = r->vol;
    v.nx = q.nx;
    v.ny = q.ny;
    v.nz = q.nz;
    v.binning = q.binning;
    v.pitch = ((int64_t)q.nx + 2 * kHalo + 15) / 16 * 16;
    v.plane = v.pitch * (q.ny + 2 * kHalo);
    v.bytes = volume_bytes(q.nx, q.ny, q.nz);
    r->n_vox = (int64_t)q.nx * q.ny * q.nz;
    const int S_ = q.params.r_max - q.params.r_min + 1;
    const size_t parts = (size_t)bin_f32_scratch_blocks(c->num_sms);
    size_t off[8] = {};
    size_t at = 0;
    auto place = [&](int k, size_t n) {
        off[k] = at;
        at += round256(std::max<size_t>(n, 1));
    };
    place(0, v.bytes);                       // bins (padded)
    place(1, r->raw_bytes);                  // raw staging
    place(2, parts * sizeof(float2));        // min/max partials
    if (q.kind == KS_REQ_DENSE) {
        place(3, (size_t)r->n_vox * 8);
        place(4, (size_t)r->n_vox);
    } else {
        r->n_items = r->n_seeds * S_;
        place(3, (size_t)r->n_seeds * 12);
        place(4, (size_t)r->n_seeds * sizeof(ks_seed_result));
        place(5, (size_t)r->n_items * sizeof(ks_ms_result));
        place(6, (size_t)(r->n_seeds + r->n_items) * sizeof(int4));
    }
    uint8_t *m = (uint8_t *)S->arena.alloc(c, at);
    if (!m) return KS_ENOMEM;
    r->dmem = m;
    r->dbytes = at;
    v.alloc = m + off[0];
    uint8_t *base = v.alloc + kHalo * v.plane + kHalo * v.pitch + kHalo;
    v.desc = VolDesc{base, q.nx, q.ny, q.nz, q.binning.bins, v.pitch, v.plane};
    v.tmap_ok = false;
    void *raw = m + off[1];
    cudaError_t e = cudaMemsetAsync(v.alloc, 0, v.bytes, S->s_up);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(raw, r->pinned, r->raw_bytes, cudaMemcpyHostToDevice, S->s_up);
    if (e == cudaSuccess) {
        if (q.binning.kind == KS_BIN_AFFINE_F32) {
            c->launches += 2;
            e = launch_bin_f32(c->lc(S->s_up), (const float *)raw, q.nx, q.ny, q.nz, q.binning.bins,
                               base, v.pitch, v.plane, (float2 *)(m + off[2]), (int)parts);
        } else {
            c->launches++;
            e = launch_bin_int(c->lc(S->s_up), raw, q.dtype, q.nx, q.ny, q.nz, q.binning, base,
                               v.pitch, v.plane);
        }
    }
    if (q.kind == KS_REQ_DENSE) {
        r->d_Y = (double *)(m + off[3]);
        r->d_s = m + off[4];
    } else {
        r->d_seeds = (int32_t *)(m + off[3]);
        r->d_oct = (ks_seed_result *)(m + off[4]);
        r->d_ms = (ks_ms_result *)(m + off[5]);
        r->d_state = (int4 *)(m + off[6]);
        r->n_total = ((q.seed_kinds & 1) ? r->n_seeds : 0) + ((q.seed_kinds & 2) ? r->n_items : 0);
        if (e == cudaSuccess && r->n_seeds)
            e = cudaMemcpyAsync(r->d_seeds, (uint8_t *)r->pinned + round256(r->raw_bytes),
                                (size_t)r->n_seeds * 12, cudaMemcpyHostToDevice, S->s_up);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(r->d_state, 0, (size_t)(r->n_seeds + r->n_items) * sizeof(int4),
                                S->s_up);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(S->d_counters + r->slot, 0, sizeof(unsigned int), S->s_up);
    }
    r->ev = take_event(S);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, S->s_up);
    return e == cudaSuccess ? KS_OK : cuda_err(c, e, "serving set-up");
}

// Results of a finished request to pinned host memory on the download
// stream (after `after`, the event of the work that produced them).
static int start_download(Ctx *c, ServeState *S, Request *r, cudaEvent_t after) {
    const ks_request &q = r->desc;
    size_t need = 0;
    if (q.kind == KS_REQ_DENSE)
        need = round256((size_t)r->n_vox * 8) + round256((size_t)r->n_vox);
    else
        need = round256((size_t)r->n_seeds * sizeof(ks_seed_result)) +
               round256((size_t)r->n_items * sizeof(ks_ms_result));
    r->res = S->pool.get(std::max<size_t>(need, 1), &r->res_bytes);
    if (!r->res) return set_err(c, KS_ENOMEM, "pinned result buffer");
    uint8_t *h = (uint8_t *)r->res;
    cudaError_t e = after ? cudaStreamWaitEvent(S->s_down, after, 0) : cudaSuccess;
    if (q.kind == KS_REQ_DENSE) {
        r->Y = (double *)h;
        r->s = h + round256((size_t)r->n_vox * 8);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->Y, r->d_Y, (size_t)r->n_vox * 8, cudaMemcpyDeviceToHost, S->s_down);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->s, r->d_s, (size_t)r->n_vox, cudaMemcpyDeviceToHost, S->s_down);
    } else {
        if (q.seed_kinds & 1) {
            r->oct = (ks_seed_result *)h;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->oct, r->d_oct, (size_t)r->n_seeds * sizeof(ks_seed_result),
                                    cudaMemcpyDeviceToHost, S->s_down);
        }
        if (q.seed_kinds & 2) {
            r->ms = (ks_ms_result *)(h + round256((size_t)r->n_seeds * sizeof(ks_seed_result)));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(r->ms, r->d_ms, (size_t)r->n_items * sizeof(ks_ms_result),
                                    cudaMemcpyDeviceToHost, S->s_down);
        }
    }
    if (!r->ev) r->ev = take_event(S);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, S->s_down);
    return e == cudaSuccess ? KS_OK : cuda_err(c, e, "serving results");
}

// One wave: every listed seed request's unfinished items advance by at most
// S->wave_iters iterations; then the finished counters and the status word
// come back to pinned memory.
static int launch_wave(Ctx *c, ServeState *S, std::vector<Request *> &members, int wave_iters) {
    std::vector<SeedJob> jobs;
    std::vector<std::pair<int, int>> segs;
    for (Request *r : members) {
        const ks_request &q = r->desc;
        SeedJob J{};
        J.vol = r->vol.desc;
        J.r_min = q.params.r_min;
        J.r_max = q.params.r_max;
        J.S = q.params.r_max - q.params.r_min + 1;
        J.max_iter = q.params.max_iter;
        J.w_norm = q.params.w_norm;
        J.seeds = r->d_seeds;
        J.n_seeds = r->n_seeds;
        J.oct_out = r->d_oct;
        J.ms_out = r->d_ms;
        J.state = r->d_state;
        J.finished = S->d_counters + r->slot;
        J.iter_budget = wave_iters;
        const int ji = (int)jobs.size();
        jobs.push_back(J);
        if ((q.seed_kinds & 1) && r->n_seeds) segs.push_back({ji, kOctant});
        if ((q.seed_kinds & 2) && r->n_items) segs.push_back({ji, kMeanShift});
    }
    const int b = S->next_buf;
    S->next_buf = (b + 1) % kMaxWavesInFlight;
    const size_t jobs_bytes = round256(jobs.size() * sizeof(SeedJob));
    const size_t need = jobs_bytes + plan_bytes_bound(segs.size());
    if (S->qdev_bytes[b] < need) {
        S->arena.release(S->qdev[b], S->qdev_bytes[b]);
        S->qdev_bytes[b] = 0;
        S->qdev[b] = S->arena.alloc(c, need * 2);
        if (!S->qdev[b]) return set_err(c, KS_ENOMEM, "serving queue");
        S->qdev_bytes[b] = need * 2;
    }
    std::vector<uint8_t> img(jobs_bytes, 0);
    uint8_t *dq = (uint8_t *)S->qdev[b];
    if (!jobs.empty()) std::memcpy(img.data(), jobs.data(), jobs.size() * sizeof(SeedJob));
    const std::vector<ClassLaunch> cls =
        plan_class_queues(c, jobs, (const SeedJob *)dq, segs, img, jobs_bytes, dq);
    if (S->qhost_bytes[b] < img.size()) {
        S->pool.put(S->qhost[b], S->qhost_bytes[b]);
        S->qhost[b] = S->pool.get(img.size(), &S->qhost_bytes[b]);
        if (!S->qhost[b]) return set_err(c, KS_ENOMEM, "serving queue image");
    }
    std::memcpy(S->qhost[b], img.data(), img.size());
    cudaError_t e = cudaMemcpyAsync(dq, S->qhost[b], img.size(), cudaMemcpyHostToDevice, S->s_seed);
    ProfRec rec;
    prof_begin(c, "ks_seeds_persistent", S->s_seed, &rec);
    if (e == cudaSuccess) e = launch_class_queues(c, S->s_seed, S->d_status, cls);
    prof_end(c, &rec, S->s_seed);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->h_counts[b], S->d_counters, (kMaxSlots + 1) * sizeof(unsigned int),
                            cudaMemcpyDeviceToHost, S->s_seed);
    Wave w;
    w.seq = S->wave_seq++;
    w.members = members;
    w.buf = b;
    w.ev = take_event(S);
    if (e == cudaSuccess) e = cudaEventRecord(w.ev, S->s_seed);
    for (Request *r : members) r->last_wave = w.seq;
    S->waves.push_back(std::move(w));
    return e == cudaSuccess ? KS_OK : cuda_err(c, e, "serving seed wave");
}

// Device memory of a request back to the arena, its slot and events freed.
static void release_device(ServeState *S, Request *r) {
    S->arena.release(r->dmem, r->dbytes);
    r->dmem = nullptr;
    r->dbytes = 0;
    if (r->slot >= 0) S->free_slots.push_back(r->slot);
    r->slot = -1;
    give_event(S, r->ev);
}

static void finish(ServeState *S, Request *r) {
    if (r->pinned) S->pool.put(r->pinned, r->pin_bytes);
    r->pinned = nullptr;
    if (r->canceled && r->status == KS_OK) r->status = KS_ECANCELED;
    std::lock_guard<std::mutex> g(S->mu);
    r->t_done = now_us();
    r->state = Request::kDone;
    S->reserved -= r->footprint;
    S->cv_done.notify_all();
}

static void scheduler(Ctx *c) {
    ServeState *S = c->serve;
    cudaSetDevice(c->device);
    const size_t budget = c->budget ? c->budget : (size_t)60 << 30;
    std::vector<Request *> retiring;    // done with the device except for waves in flight
    for (;;) {
        bool progress = false;
        std::vector<Request *> admitted;
        int wave_iters;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) return;
            wave_iters = S->wave_iters;
            while (!S->pending.empty()) {
                Request *r = S->pending.front();
                if (r->canceled) {
                    S->pending.pop_front();
                    r->status = KS_ECANCELED;
                    r->state = Request::kDone;
                    r->t_done = now_us();
                    S->pool.put(r->pinned, r->pin_bytes);
                    r->pinned = nullptr;
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->reserved + r->footprint > budget && !S->active.empty()) break;
                if (r->desc.kind == KS_REQ_SEEDS && S->free_slots.empty()) break;
                S->pending.pop_front();
                S->reserved += r->footprint;
                r->state = Request::kSetup;
                r->t_admit = now_us();
                if (r->desc.kind == KS_REQ_SEEDS) {
                    r->slot = S->free_slots.back();
                    S->free_slots.pop_back();
                }
                S->active.push_back(r);
                admitted.push_back(r);
            }
        }
        for (size_t i = 0; i < admitted.size(); ++i) {
            Request *r = admitted[i];
            const int st = setup(c, S, r);
            if (st == KS_ENOMEM && r->dmem == nullptr && S->active.size() > admitted.size() - i) {
                // no arena room while other requests hold it: back to the
                // head of the queue until they finish
                std::lock_guard<std::mutex> g(S->mu);
                for (size_t k = admitted.size(); k-- > i;) {
                    Request *q = admitted[k];
                    S->active.erase(std::find(S->active.begin(), S->active.end(), q));
                    S->reserved -= q->footprint;
                    if (q->slot >= 0) S->free_slots.push_back(q->slot);
                    q->slot = -1;
                    q->state = Request::kPending;
                    S->pending.push_front(q);
                }
                break;
            }
            r->status = st;
            progress = true;
        }
        std::vector<Request *> act;
        {
            std::lock_guard<std::mutex> g(S->mu);
            act = S->active;
        }
        // set-up done -> ready; dense sweeps start at once
        for (Request *r : act) {
            if (r->state != Request::kSetup || !r->ev) continue;
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            if (q != cudaSuccess) r->status = cuda_err(c, q, "serving set-up");
            S->pool.put(r->pinned, r->pin_bytes);
            r->pinned = nullptr;
            r->state = Request::kReady;
            if (r->status || r->canceled) continue;
            if (r->desc.kind == KS_REQ_DENSE) S->dense_ready.push_back(r);
        }
        // the next dense sweep, when none is in flight
        if (!S->dense_on && !S->dense_ready.empty()) {
            Request *r = S->dense_ready.front();
            S->dense_ready.pop_front();
            const DenseOut o{r->d_Y, r->d_s, nullptr, nullptr};
            r->status = run_dense(c, S->s_dense, &r->vol, &r->desc.params, o, 0, r->vol.nz);
            if (!r->status) {
                const cudaError_t er = cudaEventRecord(r->ev, S->s_dense);
                if (er != cudaSuccess) r->status = cuda_err(c, er, "serving dense");
            }
            S->dense_on = r;
            r->state = Request::kRunning;
            progress = true;
        }
        // waves that have completed: finished requests go to download
        while (!S->waves.empty()) {
            Wave &w = S->waves.front();
            const cudaError_t q = cudaEventQuery(w.ev);
            if (q == cudaErrorNotReady) break;
            progress = true;
            const unsigned int *cnt = S->h_counts[w.buf];
            const bool timeout = cnt[kMaxSlots] != 0;
            for (Request *r : w.members) {
                if (r->state != Request::kRunning && r->state != Request::kReady) continue;
                if (q != cudaSuccess && !r->status) r->status = cuda_err(c, q, "serving wave");
                if (timeout && !r->status) r->status = KS_ETIMEDOUT;
                if (r->status || r->canceled) continue;
                if ((int64_t)cnt[r->slot] >= r->n_total) {
                    r->status = start_download(c, S, r, nullptr);   // the wave is complete
                    r->state = Request::kDownload;
                }
            }
            if (timeout) cudaMemsetAsync(S->d_status, 0, 4, S->s_seed);
            S->waves_done = w.seq + 1;
            give_event(S, w.ev);
            S->waves.pop_front();
        }
        // dense sweeps that have completed
        for (Request *r : act) {
            if (r->desc.kind != KS_REQ_DENSE || r->state != Request::kRunning || r->status) continue;
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            if (S->dense_on == r) S->dense_on = nullptr;
            if (q != cudaSuccess) {
                r->status = cuda_err(c, q, "serving dense");
                continue;
            }
            r->status = start_download(c, S, r, nullptr);
            r->state = Request::kDownload;
        }
        // the next wave: every seed request that is set up and not finished
        if ((int)S->waves.size() < kMaxWavesInFlight) {
            std::vector<Request *> members;
            for (Request *r : act)
                if (r->desc.kind == KS_REQ_SEEDS && !r->status && !r->canceled &&
                    (r->state == Request::kReady || r->state == Request::kRunning)) {
                    members.push_back(r);
                }
            if (!members.empty()) {
                const int st = launch_wave(c, S, members, wave_iters);
                for (Request *r : members) {
                    r->state = Request::kRunning;
                    if (st) r->status = st;
                }
                progress = true;
            }
        }
        // downloads that have completed, failed and cancelled requests
        std::vector<Request *> done;
        for (Request *r : act) {
            if (r->state == Request::kDownload) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess && !r->status) r->status = cuda_err(c, q, "serving results");
                done.push_back(r);
            } else if ((r->status || r->canceled) && r->state != Request::kSetup) {
                done.push_back(r);
            } else if ((r->status || r->canceled) && r->state == Request::kSetup &&
                       (!r->ev || cudaEventQuery(r->ev) != cudaErrorNotReady)) {
                done.push_back(r);
            }
        }
        if (!done.empty()) {
            progress = true;
            {
                std::lock_guard<std::mutex> g(S->mu);
                for (Request *r : done)
                    S->active.erase(std::find(S->active.begin(), S->active.end(), r));
            }
            for (Request *r : done) {
                if (r->desc.kind == KS_REQ_DENSE && r->state == Request::kRunning && r->ev)
                    cudaEventSynchronize(r->ev);   // a cancelled sweep still writes its buffers
                if (S->dense_on == r) S->dense_on = nullptr;
                S->dense_ready.erase(std::remove(S->dense_ready.begin(), S->dense_ready.end(), r),
                                     S->dense_ready.end());
                finish(S, r);
                retiring.push_back(r);
            }
        }
        // device memory back to the arena once no queued wave lists the request
        for (size_t i = 0; i < retiring.size();) {
            Request *r = retiring[i];
            if (r->last_wave < S->waves_done) {
                release_device(S, r);
                retiring[i] = retiring.back();
                retiring.pop_back();
            } else {
                ++i;
            }
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) return;
            const bool idle = S->pending.empty() && S->active.empty() && S->waves.empty();
            if (idle && retiring.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            else
                S->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

static ServeState *ensure_serve(Ctx *c) {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->serve) return c->serve;
    auto S = std::make_unique<ServeState>();
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    bool ok = cudaStreamCreateWithPriority(&S->s_up, cudaStreamNonBlocking, hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&S->s_seed, cudaStreamNonBlocking, hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&S->s_dense, cudaStreamNonBlocking, hi) == cudaSuccess &&

              cudaStreamCreateWithPriority(&S->s_down, cudaStreamNonBlocking, hi) == cudaSuccess;
    void *p = nullptr;
    ok = ok && dev_alloc(c, &p, (kMaxSlots + 64) * sizeof(unsigned int)) == cudaSuccess;
    if (ok) {
        S->d_counters = (unsigned int *)p;
        S->d_status = (int *)(S->d_counters + kMaxSlots);   // copied back with the counters
        ok = cudaMemset(p, 0, (kMaxSlots + 64) * sizeof(unsigned int)) == cudaSuccess;
    }
    for (int b = 0; ok && b < kMaxWavesInFlight; ++b)
        ok = cudaMallocHost((void **)&S->h_counts[b], (kMaxSlots + 1) * sizeof(unsigned int)) ==
             cudaSuccess;
    if (!ok) {
        for (cudaStream_t s : {S->s_up, S->s_seed, S->s_dense, S->s_down})
            if (s) cudaStreamDestroy(s);
        dev_free(c, p, (kMaxSlots + 64) * sizeof(unsigned int));
        for (int b = 0; b < kMaxWavesInFlight; ++b)
            if (S->h_counts[b]) cudaFreeHost(S->h_counts[b]);
        return nullptr;
    }
    for (int i = kMaxSlots - 1; i >= 0; --i) S->free_slots.push_back(i);
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
    for (cudaStream_t s : {S->s_up, S->s_seed, S->s_dense, S->s_down}) cudaStreamSynchronize(s);
    for (auto &kv : S->all) {
        Request *r = kv.second.get();
        S->pool.put(r->pinned, r->pin_bytes);
        S->pool.put(r->res, r->res_bytes);
        if (r->ev) cudaEventDestroy(r->ev);
    }
    for (Wave &w : S->waves)
        if (w.ev) cudaEventDestroy(w.ev);
    for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
    for (int b = 0; b < kMaxWavesInFlight; ++b) {
        S->pool.put(S->qhost[b], S->qhost_bytes[b]);
        cudaFreeHost(S->h_counts[b]);
    }
    S->pool.destroy();
    S->arena.destroy(c);
    dev_free(c, S->d_counters, (kMaxSlots + 64) * sizeof(unsigned int));
    for (cudaStream_t s : {S->s_up, S->s_seed, S->s_dense, S->s_down}) cudaStreamDestroy(s);
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
    r->footprint = footprint_of(*req, c->num_sms);
    const size_t budget = c->budget ? c->budget : (size_t)60 << 30;
    if (r->footprint > budget)
        return set_err(c, KS_ENOMEM, "request footprint exceeds the HBM budget");
    ServeState *S = ensure_serve(c);
    if (!S) return set_err(c, KS_ECUDA, "serving start-up");
    r->raw_bytes = (size_t)req->nx * req->ny * req->nz * dtype_bytes(req->dtype);
    std::vector<int32_t> seeds;
    if (req->kind == KS_REQ_SEEDS) {
        seeds = seed_grid(req->nx, req->ny, req->nz, req->params.stride);
        r->n_seeds = (int64_t)seeds.size() / 3;
    }
    r->pinned = S->pool.get(round256(r->raw_bytes) + seeds.size() * 4 + 1, &r->pin_bytes);
    if (!r->pinned) return set_err(c, KS_ENOMEM, "pinned staging");
    std::memcpy(r->pinned, req->data, r->raw_bytes);
    if (!seeds.empty())
        std::memcpy((uint8_t *)r->pinned + round256(r->raw_bytes), seeds.data(), seeds.size() * 4);
    r->desc.data = nullptr;
    r->t_submit = now_us();
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
        const bool ok = r->status == KS_OK;
        out->status = r->status;
        out->kind = r->desc.kind;
        out->n_seeds = r->n_seeds;
        out->n_items = r->n_items;
        out->n_voxels = r->n_vox;
        out->oct = ok ? r->oct : nullptr;
        out->ms = ok ? r->ms : nullptr;
        out->Y_best = ok ? r->Y : nullptr;
        out->s_best = ok ? r->s : nullptr;
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
    S->pool.put(it->second->res, it->second->res_bytes);
    it->second->res = nullptr;
    S->all.erase(it);
    return KS_OK;
}

int ks_set_serve_wave_iters(ks_ctx *ctx, int iters) {
    if (!ctx || iters < 0 || iters > 1000) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    ServeState *S = ensure_serve(c);
    if (!S) return set_err(c, KS_ECUDA, "serving start-up");
    std::lock_guard<std::mutex> g(S->mu);
    S->wave_iters = iters;
    return KS_OK;
}

}  // extern "C"
