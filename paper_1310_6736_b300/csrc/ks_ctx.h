// Host-side context of the library (not part of the C ABI).
#pragma once

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ks_internal.cuh"

namespace ks {

struct Volume {
    int nx = 0, ny = 0, nz = 0;
    ks_binning binning{};
    uint8_t *alloc = nullptr;        // padded allocation (zero halo)
    size_t bytes = 0;
    int64_t pitch = 0, plane = 0;
    VolDesc desc{};
    bool tmap_ok = false;
    CUtensorMap tmap{};
};

struct ProfRec {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
};

struct Request;        // serving (ks_serve.cu)
struct ServeState;

struct DenseTuneKey {
    int B, r_max, size_class;
    bool operator<(const DenseTuneKey &o) const {
        return B != o.B ? B < o.B : (r_max != o.r_max ? r_max < o.r_max : size_class < o.size_class);
    }
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t budget = 0;                     // 0 = unlimited
    std::atomic<size_t> used{0};
    int *d_status = nullptr;               // device status word
    double *T = nullptr, *L = nullptr;     // entropy tables
    // Ball(32) offset tables: one device allocation holding c8 entries,
    // rest entries, c8_start, rest_start and ball_size
    void *d_offsets = nullptr;
    size_t offsets_bytes = 0;
    OffsetTables ot{};
    int h_ball_size[kRmax + 1] = {};
    // f32-binning scratch: per-block min/max partials
    float2 *d_minmax = nullptr;
    int minmax_blocks = 0;
    // volumes
    std::mutex mu;                         // guards vols, next_vol, err, prof, tune, vol_pool
    // released volume allocations kept for reuse by calls on `stream`
    std::vector<std::pair<size_t, void *>> vol_pool;
    std::map<int64_t, std::unique_ptr<Volume>> vols;
    int64_t next_vol = 1;
    std::string err;
    std::atomic<int64_t> launches{0};
    bool profiling = false;
    std::vector<ProfRec> prof;
    std::map<DenseTuneKey, DenseConfig> tune;
    // seed launches: device queue buffers (queue 1 only for the mean shift
    // that ks_saliency runs beside the octant climb; each buffer is used on
    // one stream at a time)
    void *batch_mem = nullptr;
    size_t batch_mem_bytes = 0;
    void *batch_mem2 = nullptr;
    size_t batch_mem2_bytes = 0;
    unsigned long long *d_head = nullptr;
    // serving
    ServeState *serve = nullptr;           // owned; released by serve_shutdown
    // ks_saliency: the dense sweep on the device's highest-priority stream,
    // the octant climb and mean shift each on a lowest-priority stream of
    // its own, forked from and joined to `stream`
    cudaStream_t hi_stream = nullptr, lo_stream = nullptr, lo2_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_hi = nullptr, ev_lo = nullptr, ev_lo2 = nullptr;

    LaunchCtx lc(cudaStream_t s = nullptr) const {
        return LaunchCtx{s ? s : stream, d_status, num_sms};
    }
};

// Helpers shared by ks_api.cu and ks_serve.cu.
int set_err(Ctx *c, int status, const std::string &msg);
int cuda_err(Ctx *c, cudaError_t e, const char *where);
cudaError_t dev_alloc(Ctx *c, void **p, size_t bytes);
void dev_free(Ctx *c, void *p, size_t bytes);
void prof_begin(Ctx *c, const char *name, cudaStream_t s, ProfRec *rec);
void prof_end(Ctx *c, ProfRec *rec, cudaStream_t s);
int validate_binning(int dtype, const ks_binning *b, std::string *why);
int validate_params(const ks_params *p, std::string *why);
size_t volume_bytes(int nx, int ny, int nz);
int create_volume_on(Ctx *c, cudaStream_t s, const void *data, int is_device, int dtype, int nx,
                     int ny, int nz, const ks_binning *b, int64_t *out_id);
Volume *find_volume(Ctx *c, int64_t id);
std::vector<int32_t> seed_grid(int nx, int ny, int nz, int stride);
DenseConfig pick_dense_config(Ctx *c, cudaStream_t s, Volume *v, int r_min, int r_max,
                              int w_norm);
int run_dense(Ctx *c, cudaStream_t s, Volume *v, const ks_params *p, const DenseOut &dev_out,
              int z0, int z1);
void serve_shutdown(Ctx *c);

// Persistent seed launches grouped by (bins, scales, kind): each class gets
// its own ticket queue and a shared-memory layout sized for it alone.
struct ClassLaunch {
    SeedQueue q;
    int max_B, max_S, kinds, grid;
};
size_t plan_bytes_bound(size_t n_segs);
// segs: (job index, kind) pairs in processing order.  Writes each class's
// head counter and segment arrays into `image` from offset plan_at on; the
// returned queues point into dev_base (the device copy of `image`).
std::vector<ClassLaunch> plan_class_queues(Ctx *c, const std::vector<SeedJob> &jobs,
                                           const SeedJob *dev_jobs,
                                           const std::vector<std::pair<int, int>> &segs,
                                           std::vector<uint8_t> &image, size_t plan_at,
                                           uint8_t *dev_base);
// The classes run one after another on s, each a persistent launch over its
// queue.  Run side by side (octant and mean-shift classes on two streams of
// equal priority, or every class on its own stream of descending priority)
// they were slower: each class fills the GPU, and they compete for it.
cudaError_t launch_class_queues(Ctx *c, cudaStream_t s, int *d_status,
                                const std::vector<ClassLaunch> &cls);

}  // namespace ks

struct ks_ctx {
    ks::Ctx impl;
};
