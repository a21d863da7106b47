// C ABI of the library: context, budgeted device memory, offset tables,
// volumes, the dense sweep (with its autotuner), the seed searches, the
// batched persistent launch and diagnostics.  Serving lives in ks_serve.cu.
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <unordered_map>

#include "ks_ctx.h"

namespace ks {

// ------------------------------------------------------------------ errors
int set_err(Ctx *c, int status, const std::string &msg) {
    if (c) {
        std::lock_guard<std::mutex> g(c->mu);
        c->err = msg;
    }
    return status;
}

int cuda_err(Ctx *c, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return KS_OK;
    const int st = (e == cudaErrorMemoryAllocation) ? KS_ENOMEM : KS_ECUDA;
    return set_err(c, st, std::string(where) + ": " + cudaGetErrorString(e));
}

#define KS_TRY_CUDA(c, expr)                                    \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return cuda_err((c), _e, #expr); \
    } while (0)

// ---------------------------------------------------------------- memory
cudaError_t dev_alloc(Ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    size_t cur = c->used.load();
    do {
        if (c->budget && cur + bytes > c->budget) return cudaErrorMemoryAllocation;
    } while (!c->used.compare_exchange_weak(cur, cur + bytes));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        c->used -= bytes;
        *p = nullptr;
    }
    return e;
}

void dev_free(Ctx *c, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->used -= bytes;
}

// Growable per-context scratch buffers (device), one per purpose.
struct Scratch {
    void *p = nullptr;
    size_t bytes = 0;
};
enum ScratchSlot {
    kScRaw, kScSeeds, kScOct, kScMs, kScTraj, kScY, kScS, kScH, kScW, kScTune, kScPts,
    kScSelIn, kScSelOut, kScAb, kScTicket, kScCand, kScSeeds2, kScCount
};
static std::mutex g_scratch_mu;
static std::unordered_map<Ctx *, std::vector<Scratch>> g_scratch;

static void *scratch(Ctx *c, int slot, size_t bytes, cudaError_t *err) {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    auto &v = g_scratch[c];
    if (v.empty()) v.resize(kScCount);
    Scratch &s = v[slot];
    *err = cudaSuccess;
    if (s.bytes >= bytes && s.p) return s.p;
    if (s.p) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, s.p, s.bytes);
        s.p = nullptr;
        s.bytes = 0;
    }
    const size_t want = std::max<size_t>(bytes, 256);
    *err = dev_alloc(c, &s.p, want);
    if (*err != cudaSuccess) return nullptr;
    s.bytes = want;
    return s.p;
}

// Volume allocations released through the API go to a small pool and are
// reused by the next volume of exactly the same size created on the
// context's stream, so a loop over same-sized volumes allocates (and frees,
// which synchronises the device) only once.
constexpr size_t kVolPoolMax = 4;
constexpr size_t kVolPoolBytes = size_t(2) << 30;

static void *vol_pool_take(Ctx *c, size_t bytes) {
    std::lock_guard<std::mutex> g(c->mu);
    for (size_t i = 0; i < c->vol_pool.size(); ++i)
        if (c->vol_pool[i].first == bytes) {
            void *p = c->vol_pool[i].second;
            c->vol_pool.erase(c->vol_pool.begin() + i);
            return p;
        }
    return nullptr;
}

static void vol_pool_put(Ctx *c, void *p, size_t bytes) {
    {
        std::lock_guard<std::mutex> g(c->mu);
        size_t held = 0;
        for (auto &e : c->vol_pool) held += e.first;
        if (c->vol_pool.size() < kVolPoolMax && held + bytes <= kVolPoolBytes) {
            c->vol_pool.emplace_back(bytes, p);
            return;
        }
    }
    dev_free(c, p, bytes);
}

static void vol_pool_flush(Ctx *c) {
    std::vector<std::pair<size_t, void *>> all;
    {
        std::lock_guard<std::mutex> g(c->mu);
        all.swap(c->vol_pool);
    }
    for (auto &e : all) dev_free(c, e.second, e.first);
}

static void scratch_release_all(Ctx *c) {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    auto it = g_scratch.find(c);
    if (it == g_scratch.end()) return;
    for (auto &s : it->second) dev_free(c, s.p, s.bytes);
    g_scratch.erase(it);
}

// -------------------------------------------------------------- profiling
void prof_begin(Ctx *c, const char *name, cudaStream_t s, ProfRec *rec) {
    c->launches++;
    rec->name = name;
    rec->a = rec->b = nullptr;
    if (!c->profiling) return;
    cudaEventCreate(&rec->a);
    cudaEventCreate(&rec->b);
    cudaEventRecord(rec->a, s);
}

void prof_end(Ctx *c, ProfRec *rec, cudaStream_t s) {
    if (!rec->a) return;
    cudaEventRecord(rec->b, s);
    std::lock_guard<std::mutex> g(c->mu);
    c->prof.push_back(*rec);
}

// ------------------------------------------------------------- validation
int validate_binning(int dtype, const ks_binning *b, std::string *why) {
    if (!b) return *why = "binning is NULL", KS_EINVAL;
    if (b->bins < 2 || b->bins > kMaxBins) return *why = "bins must be in [2, 64]", KS_EINVAL;
    if (dtype != KS_U8 && dtype != KS_I16 && dtype != KS_F32)
        return *why = "unknown dtype", KS_EINVAL;
    if (b->kind == KS_BIN_AFFINE_F32) {
        if (dtype != KS_F32) return *why = "AFFINE_F32 binning needs float32 data", KS_EINVAL;
        return KS_OK;
    }
    if (b->kind == KS_BIN_STORED) {
        if (dtype != KS_U8) return *why = "STORED binning needs uint8 data", KS_EINVAL;
        return KS_OK;
    }
    if (b->kind != KS_BIN_CLAMP_SHIFT && b->kind != KS_BIN_WINDOW)
        return *why = "unknown binning kind", KS_EINVAL;
    if (dtype == KS_F32) return *why = "integer binning needs uint8 or int16 data", KS_EINVAL;
    if (b->shift < 0 || b->shift > 16 || b->lo > b->hi)
        return *why = "binning needs 0 <= shift <= 16 and lo <= hi", KS_EINVAL;
    if (((int64_t)b->hi - b->lo) >> b->shift > b->bins - 1)
        return *why = "(hi - lo) >> shift exceeds bins - 1", KS_EINVAL;
    return KS_OK;
}

int validate_params(const ks_params *p, std::string *why) {
    if (!p) return *why = "params is NULL", KS_EINVAL;
    if (p->r_min < 1 || p->r_max > kRmax || p->r_min >= p->r_max)
        return *why = "scales need 1 <= r_min < r_max <= 32", KS_EINVAL;
    if (p->stride < 1) return *why = "stride must be >= 1", KS_EINVAL;
    if (p->max_iter < 0 || p->max_iter > 64) return *why = "max_iter must be in [0, 64]", KS_EINVAL;
    if (p->w_norm != KS_WNORM_KB && p->w_norm != KS_WNORM_ONE)
        return *why = "unknown w_norm", KS_EINVAL;
    return KS_OK;
}

// ------------------------------------------------------------ ball tables
static int rho_of(int d2) {
    int r = 0;
    while (r * r < d2) ++r;
    return r;
}

static int build_ball_tables(Ctx *c) {
    struct O {
        int dx, dy, dz, rho;
    };
    std::vector<O> ball;
    for (int dz = -kRmax; dz <= kRmax; ++dz)
        for (int dy = -kRmax; dy <= kRmax; ++dy)
            for (int dx = -kRmax; dx <= kRmax; ++dx) {
                const int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 <= kRmax * kRmax) ball.push_back({dx, dy, dz, rho_of(d2)});
            }
    std::stable_sort(ball.begin(), ball.end(), [](const O &a, const O &b) {
        if (a.rho != b.rho) return a.rho < b.rho;
        if (a.dz != b.dz) return a.dz < b.dz;
        if (a.dy != b.dy) return a.dy < b.dy;
        return a.dx < b.dx;
    });
    for (int r = 0; r <= kRmax; ++r) {
        int n = 0;
        for (auto &o : ball) n += o.rho <= r;
        c->h_ball_size[r] = n;
    }
    // Offset tables (see OffsetTables): three-nonzero offsets once per 8 sign
    // mirrors, then the plane/axis offsets, each part sorted by rho.
    std::vector<uint32_t> h8, hr;
    int s8[kRmax + 2], sr[kRmax + 2];
    for (int rho = 0; rho <= kRmax; ++rho) {
        s8[rho] = (int)h8.size();
        sr[rho] = (int)hr.size();
        for (auto &o : ball) {
            if (o.rho != rho) continue;
            if (o.dx > 0 && o.dy > 0 && o.dz > 0)
                h8.push_back((uint32_t)o.dx | ((uint32_t)o.dy << 8) | ((uint32_t)o.dz << 16) |
                             ((uint32_t)rho << 24));
            else if (o.dx == 0 || o.dy == 0 || o.dz == 0)
                hr.push_back((uint32_t)(o.dx + 64) | ((uint32_t)(o.dy + 64) << 8) |
                             ((uint32_t)(o.dz + 64) << 16) | ((uint32_t)rho << 24));
        }
    }
    s8[kRmax + 1] = (int)h8.size();
    sr[kRmax + 1] = (int)hr.size();
    for (int r = 0; r <= kRmax; ++r)
        if (8 * s8[r + 1] + sr[r + 1] != c->h_ball_size[r])
            return set_err(c, KS_ECUDA, "internal: offset tables inconsistent");
    if ((int)ball.size() != kTableN) return set_err(c, KS_ECUDA, "internal: ball size");
    // x-rows of every Ball(r): rows off both planes y = 0 and z = 0 first,
    // then the rows on one of them; longest first within each group (a
    // block hands rows out round robin, so a warp takes rows of one kind
    // and of similar length)
    std::vector<uint32_t> hw;
    int swr[kRmax + 2];
    for (int r = 0; r <= kRmax; ++r) {
        swr[r] = (int)hw.size();
        struct Row {
            int dy, dz, w;
        };
        std::vector<Row> rows;
        int n = 0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy) {
                const int q = r * r - dy * dy - dz * dz;
                if (q < 0) continue;
                int w = 0;
                while ((w + 1) * (w + 1) <= q) ++w;
                rows.push_back({dy, dz, w});
                n += 2 * w + 1;
            }
        if (n != c->h_ball_size[r]) return set_err(c, KS_ECUDA, "internal: row tables inconsistent");
        std::stable_sort(rows.begin(), rows.end(), [](const Row &a, const Row &b) {
            const bool pa = a.dy == 0 || a.dz == 0, pb = b.dy == 0 || b.dz == 0;
            return pa != pb ? pb : a.w > b.w;
        });
        for (auto &rw : rows)
            hw.push_back((uint32_t)(rw.dy + 64) | ((uint32_t)(rw.dz + 64) << 8) |
                         ((uint32_t)rw.w << 16));
    }
    swr[kRmax + 1] = (int)hw.size();
    // mean-shift block path: may its per-voxel sums go into two 32-bit
    // words for radius r?  Column c of a bin sees the rows i = c mod NC
    // (threads t = c mod NC walk rows t, t + 256, ...); a row adds 2w + 1 to
    // the count, (2w + 1) r to sum(dx + r), (2w + 1)(dy + r) and
    // (2w + 1)(dz + r) to the other two.
    uint8_t ms32[kRmax + 1];
    for (int r = 0; r <= kRmax; ++r) {
        const int NC = ms_columns(c->h_ball_size[r]);
        std::vector<int64_t> sc(NC, 0), sx(NC, 0), sy(NC, 0), sz(NC, 0);
        for (int i = swr[r]; i < swr[r + 1]; ++i) {
            const uint32_t e = hw[i];
            const int dy = (int)(e & 0xffu) - 64, dz = (int)((e >> 8) & 0xffu) - 64;
            const int n = 2 * (int)(e >> 16) + 1, col = (i - swr[r]) % NC;
            sc[col] += n;
            sx[col] += (int64_t)n * r;
            sy[col] += (int64_t)n * (dy + r);
            sz[col] += (int64_t)n * (dz + r);
        }
        bool ok = true;
        for (int col = 0; col < NC; ++col)
            ok = ok && sc[col] < (1 << 11) && sx[col] < (1 << 17) && sy[col] < (1 << 16) &&
                 sz[col] < (1 << 16);
        ms32[r] = ok ? 1 : 0;
    }
    // Ball(r)'s entries of each kind once more per r, sorted by row (dz, dy,
    // dx) for walks that take the whole ball at once
        auto by_rows = [](const std::vector<uint32_t> &h, const int *st, std::vector<uint32_t> &out,
                      int *ost) {
        for (int r = 0; r <= kRmax; ++r) {
            ost[r] = (int)out.size();
            std::vector<uint32_t> e(h.begin(), h.begin() + st[r + 1]);
            std::stable_sort(e.begin(), e.end(), [](uint32_t a, uint32_t b) {
                return (a & 0xffffffu) < (b & 0xffffffu);     // (dz, dy, dx)
            });
            out.insert(out.end(), e.begin(), e.end());
        }
        ost[kRmax + 1] = (int)out.size();
    };
    // rest offsets once per set of sign mirrors: the all-non-negative member
    std::vector<uint32_t> hm;
    int sm[kRmax + 2];
    for (int rho = 0; rho <= kRmax; ++rho) {
        sm[rho] = (int)hm.size();
        for (int k = sr[rho]; k < sr[rho + 1]; ++k) {
            const uint32_t f = hr[k];
            const int dx = (int)(f & 0xffu) - 64, dy = (int)((f >> 8) & 0xffu) - 64,
                      dz = (int)((f >> 16) & 0xffu) - 64;
            if (dx >= 0 && dy >= 0 && dz >= 0)
                hm.push_back((uint32_t)dx | ((uint32_t)dy << 8) | ((uint32_t)dz << 16) |
                             ((uint32_t)rho << 24));
        }
    }
    sm[kRmax + 1] = (int)hm.size();
    std::vector<uint32_t> h8r, hrr;
    int s8r[kRmax + 2], srr[kRmax + 2];
    by_rows(h8, s8, h8r, s8r);
    by_rows(hm, sm, hrr, srr);
    // one allocation: c8 | rest | rows | c8_rows | restm_rows | c8_start | rest_start |
    // rows_start | ball_size | ms32 | c8_rows_start | restm_rows_start
    const size_t b8 = h8.size() * 4, br = hr.size() * 4, bw = hw.size() * 4, bs = sizeof(s8);
    const size_t b8r = h8r.size() * 4, brr = hrr.size() * 4;
    const size_t at_r = (b8 + 255) / 256 * 256, at_w = at_r + (br + 255) / 256 * 256;
    const size_t at_8r = at_w + (bw + 255) / 256 * 256, at_rr = at_8r + (b8r + 255) / 256 * 256;
    const size_t at_s8 = at_rr + (brr + 255) / 256 * 256;
    const size_t at_sr = at_s8 + 256, at_sw = at_sr + 256, at_bs = at_sw + 256;
    const size_t at_m32 = at_bs + 256, at_s8r = at_m32 + 256, at_srr = at_s8r + 256;
    c->offsets_bytes = at_srr + 256;
    void *p;
    KS_TRY_CUDA(c, dev_alloc(c, &p, c->offsets_bytes));
    c->d_offsets = p;
    uint8_t *m = (uint8_t *)p;
    KS_TRY_CUDA(c, cudaMemcpy(m, h8.data(), b8, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_r, hr.data(), br, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_s8, s8, bs, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_sr, sr, bs, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_w, hw.data(), bw, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_sw, swr, bs, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_bs, c->h_ball_size, sizeof(c->h_ball_size),
                              cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_m32, ms32, sizeof(ms32), cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_8r, h8r.data(), b8r, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_rr, hrr.data(), brr, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_s8r, s8r, bs, cudaMemcpyHostToDevice));
    KS_TRY_CUDA(c, cudaMemcpy(m + at_srr, srr, bs, cudaMemcpyHostToDevice));
    c->ot = OffsetTables{(const uint32_t *)m,          (const int *)(m + at_s8),
                         (const uint32_t *)(m + at_r),  (const int *)(m + at_sr),
                         (const int *)(m + at_bs),      (const uint32_t *)(m + at_w),
                         (const int *)(m + at_sw),      (const uint8_t *)(m + at_m32),
                         (const uint32_t *)(m + at_8r), (const int *)(m + at_s8r),
                         (const uint32_t *)(m + at_rr), (const int *)(m + at_srr)};
    // the classes up to dense_const_rmax() also go to constant memory
    KS_TRY_CUDA(c, dense_upload_constant_table(h8.data(), s8, hr.data(), sr));
    return KS_OK;
}


// ----------------------------------------------------------------- volumes
size_t volume_bytes(int nx, int ny, int nz) {
    const int64_t pitch = ((int64_t)nx + 2 * kHalo + 15) / 16 * 16;
    // + 256 bytes of slack: row walks read whole aligned 8-byte words
    return (size_t)(pitch * (ny + 2 * kHalo) * (nz + 2 * kHalo)) + 256;
}

static size_t dtype_size(int dtype) { return dtype == KS_U8 ? 1 : dtype == KS_I16 ? 2 : 4; }

Volume *find_volume(Ctx *c, int64_t id) {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->vols.find(id);
    return it == c->vols.end() ? nullptr : it->second.get();
}

int create_volume_on(Ctx *c, cudaStream_t s, const void *data, int is_device, int dtype, int nx,
                     int ny, int nz, const ks_binning *b, int64_t *out_id) {
    std::string why;
    if (!data || !out_id) return set_err(c, KS_EINVAL, "data / out is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
        return set_err(c, KS_EINVAL, "dims must be in [1, 4096]");
    int st = validate_binning(dtype, b, &why);
    if (st) return set_err(c, st, why);
    auto v = std::make_unique<Volume>();
    v->nx = nx;
    v->ny = ny;
    v->nz = nz;
    v->binning = *b;
    v->pitch = ((int64_t)nx + 2 * kHalo + 15) / 16 * 16;
    v->plane = v->pitch * (ny + 2 * kHalo);
    v->bytes = volume_bytes(nx, ny, nz);
    const bool own = s == c->stream;       // API call on the context's stream
    void *p = own ? vol_pool_take(c, v->bytes) : nullptr;
    if (!p) {
        cudaError_t ea = dev_alloc(c, &p, v->bytes);
        if (ea == cudaErrorMemoryAllocation) {     // the pool may hold the room
            vol_pool_flush(c);
            ea = dev_alloc(c, &p, v->bytes);
        }
        KS_TRY_CUDA(c, ea);
    }
    v->alloc = (uint8_t *)p;
    cudaError_t e = cudaMemsetAsync(v->alloc, 0, v->bytes, s);
    uint8_t *base = v->alloc + kHalo * v->plane + kHalo * v->pitch + kHalo;
    const void *raw = data;
    const size_t raw_bytes = (size_t)nx * ny * nz * dtype_size(dtype);
    void *staging = nullptr;
    if (e == cudaSuccess && !is_device) {
        // the context's stream keeps a staging buffer; other streams (the
        // serving loop) take a fresh one
        if (own)
            raw = scratch(c, kScRaw, raw_bytes, &e);
        else if ((e = dev_alloc(c, &staging, raw_bytes)) == cudaSuccess)
            raw = staging;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(const_cast<void *>(raw), data, raw_bytes, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        ProfRec rec;
        prof_begin(c, "ks_bin", s, &rec);
        if (b->kind == KS_BIN_AFFINE_F32) {
            c->launches++;   // two kernels: partials, then binning
            e = launch_bin_f32(c->lc(s), (const float *)raw, nx, ny, nz, b->bins, base, v->pitch,
                               v->plane, c->d_minmax, c->minmax_blocks);
        } else {
            e = launch_bin_int(c->lc(s), raw, dtype, nx, ny, nz, *b, base, v->pitch, v->plane);
        }
        prof_end(c, &rec, s);
    }
    if (staging) {
        cudaStreamSynchronize(s);
        dev_free(c, staging, raw_bytes);
    }
    if (e != cudaSuccess) {
        dev_free(c, v->alloc, v->bytes);
        return cuda_err(c, e, "ks_create_volume");
    }
    v->desc = VolDesc{base, nx, ny, nz, b->bins, v->pitch, v->plane};
    std::lock_guard<std::mutex> g(c->mu);
    const int64_t id = c->next_vol++;
    c->vols[id] = std::move(v);
    *out_id = id;
    return KS_OK;
}

// ------------------------------------------------------------- seed grid
std::vector<int32_t> seed_grid(int nx, int ny, int nz, int stride) {
    std::vector<int32_t> s;
    for (int z = stride / 2; z < nz; z += stride)
        for (int y = stride / 2; y < ny; y += stride)
            for (int x = stride / 2; x < nx; x += stride) {
                s.push_back(x);
                s.push_back(y);
                s.push_back(z);
            }
    return s;
}

// ------------------------------------------------------------ TMA tensor map
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

static bool make_tmap(Volume *v, int bx, int by, int bz, CUtensorMap *out) {
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)v->pitch, (cuuint64_t)(v->ny + 2 * kHalo),
                                (cuuint64_t)(v->nz + 2 * kHalo)};
    const cuuint64_t strides[2] = {(cuuint64_t)v->pitch, (cuuint64_t)v->plane};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, v->alloc, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------- dense sweep
static std::vector<DenseConfig> dense_candidates(int B, int r_max) {
    std::vector<DenseConfig> out;
    const int shapes[][3] = {{1, 1, 1}, {2, 2, 1}, {2, 1, 2}, {4, 4, 1}, {4, 2, 2}, {8, 8, 1}, {8, 4, 2}, {8, 2, 4},
                             {16, 16, 1}, {16, 4, 4}, {16, 8, 2}, {16, 2, 8}};
    // r_max > 25: only the TMEM paths where they fit (a 16-, 32- or 64-bin
    // template), in the three shapes that won on the MR-shaped volumes
    // (paths 1 and 2 took about twice as long there, and every candidate
    // costs a timed sweep)
    if (r_max > 25) {
        const int wide_shapes[][3] = {{4, 4, 1}, {4, 2, 2}, {8, 4, 2}};
        for (int path : {6, 7, 8, 9})
            for (auto &s : wide_shapes) {
                DenseConfig c{path, s[0], s[1], s[2]};
                if (dense_config_fits(c, B, r_max)) out.push_back(c);
            }
        if (!out.empty()) return out;
    }
    for (int path : {0, 1, 2, 3, 4, 6, 7, 8, 9})
        for (auto &s : shapes) {
            DenseConfig c{path, s[0], s[1], s[2]};
            if (dense_config_fits(c, B, r_max)) out.push_back(c);
        }
    // sliding windows: one warp per block, runs of 16 planes (the fastest
    // run length on the PET-shaped workload; 32 and 64 were slower)
    const DenseConfig slide{5, 1, 1, 16};
    if (dense_config_fits(slide, B, r_max)) out.push_back(slide);
    return out;
}

static int g_forced_path = -1, g_forced_warps = 0, g_forced_ty = 0, g_forced_tz = 0;
// ABMSOD: items with a starting radius >= this run on a whole block when
// the launch has few items per resident warp (0: decided per launch).
constexpr int kAbmsodTeamRadius = 12;
static int g_abmsod_team_radius = 0;

static int launch_dense_cfg(Ctx *c, cudaStream_t s, Volume *v, int r_min, int r_max, int w_norm,
                            const DenseConfig &cfg, const DenseOut &out, int z0, int z1) {
    CUtensorMap tm{};
    if (cfg.path == 0) {
        const int padx = (r_max + 15) / 16 * 16;
        const int bx = (padx + 32 + r_max + 15) / 16 * 16;
        if (!make_tmap(v, bx, cfg.ty + 2 * r_max, cfg.tz + 2 * r_max, &tm))
            return set_err(c, KS_ECUDA, "cuTensorMapEncodeTiled failed");
    }
    ProfRec rec;
    prof_begin(c, "ks_dense", s, &rec);
    cudaError_t e = launch_dense(c->lc(s), v->desc, cfg.path == 0 ? &tm : nullptr, c->ot, c->T,
                                 c->L, r_min, r_max, w_norm, cfg, out, z0, z1);
    prof_end(c, &rec, s);
    return cuda_err(c, e, "dense launch");
}

// The dense autotuner's measurements, shared by every context of the
// process (keyed by device as well): per candidate, its time per computed
// centre on the tuning slab.  A volume then takes the candidate with the
// least time for its own computed centres, so a width that leaves part of
// a wide tile idle (128 centres per warp row in paths 3, 4 and 9) is
// charged for it without timing the candidates again.
struct TuneEntry {
    DenseConfig cfg;
    double ms_per_centre;
};
static std::mutex g_tune_mu;
static std::map<std::pair<int, DenseTuneKey>, std::vector<TuneEntry>> g_tune;

static DenseConfig tune_pick(const std::vector<TuneEntry> &t, const Volume *v) {
    DenseConfig best = t[0].cfg;
    double best_ms = 1e300;
    for (const TuneEntry &e : t) {
        const double ms = e.ms_per_centre * (double)dense_computed_centres(e.cfg, v->nx, v->ny, v->nz);
        if (ms < best_ms) {
            best_ms = ms;
            best = e.cfg;
        }
    }
    return best;
}

DenseConfig pick_dense_config(Ctx *c, cudaStream_t s, Volume *v, int r_min, int r_max,
                              int w_norm) {
    if (g_forced_path >= 0) {
        DenseConfig f{g_forced_path, g_forced_warps, g_forced_ty, g_forced_tz};
        if (dense_config_fits(f, v->binning.bins, r_max)) return f;
    }
    const int64_t nvox = (int64_t)v->nx * v->ny * v->nz;
    const DenseTuneKey key{v->binning.bins, r_max, nvox < (1 << 18) ? 0 : 1};
    std::vector<TuneEntry> table;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find({c->device, key});
        if (it != g_tune.end()) table = it->second;
    }
    if (table.empty()) {
        auto cands = dense_candidates(v->binning.bins, r_max);
        if (cands.size() == 1) table.push_back({cands[0], 1.0});
        if (cands.size() > 1) {
            // Time every candidate on the same slab of the volume (outputs to
            // a temporary buffer).  The slab holds about 2^20 centres (at
            // most 64 planes, at least 4): enough that every candidate's grid
            // spans several waves of resident blocks (a thin slab favours
            // shapes with a small tail), few enough that a wide sweep (r_max
            // = 32: 137 065 updates per centre) times each candidate in tens
            // of milliseconds.
            const int64_t plane_c = std::max<int64_t>(1, (int64_t)v->nx * v->ny);
            const int z_budget = (int)std::max<int64_t>(4, ((int64_t)1 << 20) / plane_c);
            const int z1 = std::min({v->nz, 64, z_budget});
            const size_t n = (size_t)v->nx * v->ny * z1;
            void *buf = nullptr;
            if (dev_alloc(c, &buf, n * 9 + 256) == cudaSuccess) {
                DenseOut o{(double *)buf, (uint8_t *)buf + n * 8, nullptr, nullptr};
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                for (auto &cfg : cands) {
                    // one untimed launch first: the first launch of a kernel
                    // variant also loads its module
                    bool ok = launch_dense_cfg(c, s, v, r_min, r_max, w_norm, cfg, o, 0, z1) == KS_OK;
                    cudaEventRecord(e0, s);
                    for (int rep = 0; rep < 2 && ok; ++rep)
                        ok = launch_dense_cfg(c, s, v, r_min, r_max, w_norm, cfg, o, 0, z1) == KS_OK;
                    cudaEventRecord(e1, s);
                    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    table.push_back(
                        {cfg, ms / 2.0 / (double)dense_computed_centres(cfg, v->nx, v->ny, z1)});
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaStreamSynchronize(s);
                dev_free(c, buf, n * 9 + 256);
            }
        }
        if (table.empty()) table.push_back({cands.empty() ? DenseConfig{1, 8, 8, 1} : cands[0], 1.0});
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[{c->device, key}] = table;
    }
    const DenseConfig best = tune_pick(table, v);
    std::lock_guard<std::mutex> g(c->mu);
    c->tune[key] = best;
    return best;
}

int run_dense(Ctx *c, cudaStream_t s, Volume *v, const ks_params *p, const DenseOut &dev_out,
              int z0, int z1) {
    const DenseConfig cfg = pick_dense_config(c, s, v, p->r_min, p->r_max, p->w_norm);
    return launch_dense_cfg(c, s, v, p->r_min, p->r_max, p->w_norm, cfg, dev_out, z0, z1);
}

// Waits for stream s (the context's stream by default) and reports the
// device status word.
static int check_status(Ctx *c, cudaStream_t s = nullptr) {
    if (!s) s = c->stream;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(c, e, "sync");
    if (h) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        if (h & kStatusBadInput)
            return set_err(c, KS_EINVAL, "a listed centre lies outside the volume");
        if (h & kStatusMisaligned)
            return set_err(c, KS_ECUDA, "dense brick: misaligned shared-memory layout (no copy issued)");
        return set_err(c, KS_ETIMEDOUT, "a bounded device wait gave up (status " +
                                            std::to_string(h) + ")");
    }
    return KS_OK;
}

}  // namespace ks

using namespace ks;

namespace ks {
// at most one class per segment; a class is 4 arrays, each 256-byte aligned
size_t plan_bytes_bound(size_t n_segs) { return 2048 + n_segs * (4 * 256 + 32); }

std::vector<ClassLaunch> plan_class_queues(Ctx *c, const std::vector<SeedJob> &jobs,
                                           const SeedJob *dev_jobs,
                                           const std::vector<std::pair<int, int>> &segs,
                                           std::vector<uint8_t> &image, size_t plan_at,
                                           uint8_t *dev_base) {
    // classes in order of first appearance
    std::vector<std::array<int, 3>> keys;      // (bins, scales, kind)
    std::vector<std::vector<int>> members;
    for (size_t s = 0; s < segs.size(); ++s) {
        const SeedJob &J = jobs[segs[s].first];
        const std::array<int, 3> k{J.vol.B, J.S, segs[s].second};
        size_t ci = 0;
        while (ci < keys.size() && keys[ci] != k) ++ci;
        if (ci == keys.size()) {
            keys.push_back(k);
            members.emplace_back();
        }
        members[ci].push_back((int)s);
    }
    std::vector<ClassLaunch> out;
    size_t off = plan_at;
    auto put = [&](const void *src, size_t n) {
        const size_t at = off;
        if (image.size() < at + n) image.resize(at + n, 0);
        if (n) std::memcpy(image.data() + at, src, n);
        off = (at + n + 255) / 256 * 256;
        return dev_base + at;
    };
    for (size_t ci = 0; ci < keys.size(); ++ci) {
        std::vector<int64_t> ss{0};
        std::vector<int> sk, sj;
        auto add = [&](int job, int kind) {
            ss.push_back(ss.back() + seed_tickets(kind, jobs[job].n_seeds, jobs[job].r_min,
                                                  jobs[job].S, jobs[job].vol.B));
            sk.push_back(kind);
            sj.push_back(job);
        };
        // a mean-shift job becomes a block-path and a warp-path segment; the
        // warp-path segments of the class go last
        for (int s : members[ci]) add(segs[s].first, segs[s].second);
        if (keys[ci][2] == kMeanShift)
            for (int s : members[ci]) add(segs[s].first, kMsWarp);
        ClassLaunch L{};
        const unsigned long long zero = 0;
        L.q.head = (unsigned long long *)put(&zero, sizeof(zero));
        L.q.jobs = dev_jobs;
        L.q.seg_start = (const int64_t *)put(ss.data(), ss.size() * 8);
        L.q.seg_kind = (const int *)put(sk.data(), sk.size() * 4);
        L.q.seg_job = (const int *)put(sj.data(), sj.size() * 4);
        L.q.n_segs = (int)sk.size();
        L.q.n_tickets = ss.back();
        L.max_B = keys[ci][0];
        L.max_S = keys[ci][1];
        L.kinds = 1 << keys[ci][2];
        L.grid = c->num_sms * seed_blocks_per_sm(L.max_B, L.max_S, L.kinds);
        out.push_back(L);
    }
    return out;
}

cudaError_t launch_class_queues(Ctx *c, cudaStream_t s, int *d_status,
                                const std::vector<ClassLaunch> &cls) {
    cudaError_t e = cudaSuccess;
    for (const ClassLaunch &L : cls) {
        if (L.q.n_tickets == 0) continue;
        e = cudaMemsetAsync(L.q.head, 0, 8, s);
        if (e == cudaSuccess)
            e = launch_seeds(LaunchCtx{s, d_status, c->num_sms}, L.q, c->ot, c->T, c->L, L.max_B,
                             L.max_S, L.kinds, true, L.grid);
        if (e != cudaSuccess) break;
    }
    return e;
}

struct BatchGraph {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
    void *mem = nullptr;
    size_t bytes = 0;
    size_t oct_off = 0, ms_off = 0;
    std::vector<int64_t> n_oct, n_ms;
    std::vector<size_t> oct_at, ms_at;
    std::vector<ClassLaunch> classes;
};
}  // namespace ks
static std::mutex g_graph_mu;
static std::unordered_map<Ctx *, std::vector<std::unique_ptr<ks::BatchGraph>>> g_graphs;

// ====================================================================== ABI
extern "C" {

const char *ks_strerror(int s) {
    switch (s) {
        case KS_OK: return "ok";
        case KS_PENDING: return "pending";
        case KS_EINVAL: return "invalid argument";
        case KS_ENOMEM: return "out of device memory or over the HBM budget";
        case KS_ECUDA: return "CUDA error";
        case KS_ETIMEDOUT: return "timed out";
        case KS_ECANCELED: return "cancelled";
        case KS_ENOTFOUND: return "unknown handle";
        case KS_ENODEV: return "no CUDA device";
        default: return "unknown status";
    }
}

const char *ks_last_error(ks_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->impl.err.c_str();
}

int ks_init(ks_ctx **out, size_t budget, void *stream, int device) {
    if (!out) return KS_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) return KS_ENODEV;
    auto *h = new ks_ctx();
    Ctx *c = &h->impl;
    c->device = device;
    c->budget = budget;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    void *p = nullptr;
    if (e == cudaSuccess) e = dev_alloc(c, &p, 256);
    c->d_status = (int *)p;
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 256);
    if (e == cudaSuccess) e = dev_alloc(c, &p, (kTableN + 1) * sizeof(double));
    c->T = (double *)p;
    if (e == cudaSuccess) e = dev_alloc(c, &p, (kTableN + 1) * sizeof(double));
    c->L = (double *)p;
    if (e == cudaSuccess) {
        c->minmax_blocks = bin_f32_scratch_blocks(c->num_sms);
        e = dev_alloc(c, &p, c->minmax_blocks * sizeof(float2));
        c->d_minmax = (float2 *)p;
    }
    if (e == cudaSuccess) {
        ProfRec rec;
        prof_begin(c, "ks_tables", c->stream, &rec);
        e = launch_tables(c->lc(), c->T, c->L, kTableN);
        prof_end(c, &rec, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    int st = e == cudaSuccess ? KS_OK : (e == cudaErrorMemoryAllocation ? KS_ENOMEM : KS_ECUDA);
    if (st == KS_OK) st = build_ball_tables(c);
    if (st != KS_OK) {
        ks_destroy(h);
        return st;
    }
    *out = h;
    return KS_OK;
}

int ks_destroy(ks_ctx *ctx) {
    if (!ctx) return KS_OK;
    Ctx *c = &ctx->impl;
    serve_shutdown(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &kv : c->vols) dev_free(c, kv.second->alloc, kv.second->bytes);
    c->vols.clear();
    scratch_release_all(c);
    vol_pool_flush(c);
    for (auto &r : c->prof) {
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    dev_free(c, c->d_status, 256);
    dev_free(c, c->T, (kTableN + 1) * sizeof(double));
    dev_free(c, c->L, (kTableN + 1) * sizeof(double));
    dev_free(c, c->d_minmax, c->minmax_blocks * sizeof(float2));
    dev_free(c, c->d_offsets, c->offsets_bytes);
    {
        std::lock_guard<std::mutex> g(g_graph_mu);
        auto it = g_graphs.find(c);
        if (it != g_graphs.end()) {
            for (auto &bg : it->second) {
                if (bg->exec) cudaGraphExecDestroy(bg->exec);
                dev_free(c, bg->mem, bg->bytes);
            }
            g_graphs.erase(it);
        }
    }
    dev_free(c, c->batch_mem, c->batch_mem_bytes);
    dev_free(c, c->batch_mem2, c->batch_mem2_bytes);
    for (cudaEvent_t ev : {c->ev_fork, c->ev_hi, c->ev_lo, c->ev_lo2})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t ps : {c->hi_stream, c->lo_stream, c->lo2_stream})
        if (ps) {
            cudaStreamSynchronize(ps);
            cudaStreamDestroy(ps);
        }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete ctx;
    return KS_OK;
}

int ks_sync(ks_ctx *ctx) {
    if (!ctx) return KS_EINVAL;
    return check_status(&ctx->impl);
}

int ks_create_volume(ks_ctx *ctx, const void *data, int is_device_ptr, int dtype, int nx, int ny,
                     int nz, const ks_binning *binning, ks_vol *out) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    int st = create_volume_on(c, c->stream, data, is_device_ptr, dtype, nx, ny, nz, binning, out);
    if (st) return st;
    KS_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return KS_OK;
}

int ks_release_volume(ks_ctx *ctx, ks_vol vol) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::unique_ptr<Volume> v;
    {
        std::lock_guard<std::mutex> g(c->mu);
        auto it = c->vols.find(vol);
        if (it == c->vols.end()) return KS_ENOTFOUND;
        v = std::move(it->second);
        c->vols.erase(it);
    }
    cudaStreamSynchronize(c->stream);
    vol_pool_put(c, v->alloc, v->bytes);
    return KS_OK;
}

int ks_volume_bins(ks_ctx *ctx, ks_vol vol, uint8_t *out, int out_on_device) {
    if (!ctx || !out) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    cudaMemcpy3DParms prm{};
    prm.srcPtr = make_cudaPitchedPtr(v->alloc, v->pitch, v->pitch, v->ny + 2 * kHalo);
    prm.srcPos = make_cudaPos(kHalo, kHalo, kHalo);
    prm.dstPtr = make_cudaPitchedPtr(out, v->nx, v->nx, v->ny);
    prm.dstPos = make_cudaPos(0, 0, 0);
    prm.extent = make_cudaExtent(v->nx, v->ny, v->nz);
    prm.kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    KS_TRY_CUDA(c, cudaMemcpy3DAsync(&prm, c->stream));
    KS_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return KS_OK;
}

int ks_dense_saliency_ex(ks_ctx *ctx, ks_vol vol, const ks_params *params, double *Y,
                         uint8_t *s_best, double *H, double *W, int out_on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (!Y || !s_best) return set_err(c, KS_EINVAL, "Y_best / s_best is NULL");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    const size_t n = (size_t)v->nx * v->ny * v->nz;
    const int S = params->r_max - params->r_min + 1;
    DenseOut o{Y, s_best, H, W};
    cudaError_t e = cudaSuccess;
    if (!out_on_device) {
        o.Y = (double *)scratch(c, kScY, n * 8, &e);
        if (o.Y) o.s = (uint8_t *)scratch(c, kScS, n, &e);
        if (o.s && H) o.H = (double *)scratch(c, kScH, n * S * 8, &e);
        if (e == cudaSuccess && W) o.W = (double *)scratch(c, kScW, n * S * 8, &e);
        if (e != cudaSuccess) return cuda_err(c, e, "dense outputs");
    }
    st = run_dense(c, c->stream, v, params, o, 0, v->nz);
    if (st) return st;
    if (!out_on_device) {
        KS_TRY_CUDA(c, cudaMemcpyAsync(Y, o.Y, n * 8, cudaMemcpyDeviceToHost, c->stream));
        KS_TRY_CUDA(c, cudaMemcpyAsync(s_best, o.s, n, cudaMemcpyDeviceToHost, c->stream));
        if (H) KS_TRY_CUDA(c, cudaMemcpyAsync(H, o.H, n * S * 8, cudaMemcpyDeviceToHost, c->stream));
        if (W) KS_TRY_CUDA(c, cudaMemcpyAsync(W, o.W, n * S * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    return check_status(c);
}

int ks_dense_saliency_range(ks_ctx *ctx, ks_vol vol, const ks_params *params, int z0, int z1,
                            double *Y, uint8_t *s_best, int out_on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (!Y || !s_best) return set_err(c, KS_EINVAL, "Y_best / s_best is NULL");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (z0 < 0 || z1 > v->nz || z0 >= z1) return set_err(c, KS_EINVAL, "need 0 <= z0 < z1 <= nz");
    const int64_t plane = (int64_t)v->nx * v->ny;
    const size_t n = (size_t)(plane * (z1 - z0));
    cudaError_t e = cudaSuccess;
    double *dY = Y;
    uint8_t *ds = s_best;
    if (!out_on_device) {
        dY = (double *)scratch(c, kScY, n * 8, &e);
        if (dY) ds = (uint8_t *)scratch(c, kScS, n, &e);
        if (e != cudaSuccess) return cuda_err(c, e, "dense outputs");
    }
    // the kernels index outputs by the voxel's index in the whole volume and
    // write only planes [z0, z1): shift the bases back by z0 planes
    const DenseOut o{dY - plane * z0, ds - plane * z0, nullptr, nullptr};
    st = run_dense(c, c->stream, v, params, o, z0, z1);
    if (st) return st;
    if (!out_on_device) {
        KS_TRY_CUDA(c, cudaMemcpyAsync(Y, dY, n * 8, cudaMemcpyDeviceToHost, c->stream));
        KS_TRY_CUDA(c, cudaMemcpyAsync(s_best, ds, n, cudaMemcpyDeviceToHost, c->stream));
    }
    return check_status(c);
}

int ks_dense_saliency(ks_ctx *ctx, ks_vol vol, const ks_params *params, double *Y,
                      uint8_t *s_best, int out_on_device) {
    return ks_dense_saliency_ex(ctx, vol, params, Y, s_best, nullptr, nullptr, out_on_device);
}

int ks_dense_points(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *xyz,
                    int64_t n, double *Y, uint8_t *s_best, double *H, double *W, int on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (n < 0) return set_err(c, KS_EINVAL, "n < 0");
    if (n > 0 && (!xyz || !Y || !s_best)) return set_err(c, KS_EINVAL, "xyz / Y_best / s_best is NULL");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (n == 0) return KS_OK;
    const int S = params->r_max - params->r_min + 1;
    DenseOut o{Y, s_best, H, W};
    const int32_t *dxyz = xyz;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        int32_t *p = (int32_t *)scratch(c, kScPts, (size_t)n * 12, &e);
        if (p) e = cudaMemcpyAsync(p, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, c->stream);
        dxyz = p;
        if (e == cudaSuccess) o.Y = (double *)scratch(c, kScY, (size_t)n * 8, &e);
        if (o.Y) o.s = (uint8_t *)scratch(c, kScS, (size_t)n, &e);
        if (o.s && H) o.H = (double *)scratch(c, kScH, (size_t)n * S * 8, &e);
        if (e == cudaSuccess && W) o.W = (double *)scratch(c, kScW, (size_t)n * S * 8, &e);
        if (e != cudaSuccess) return cuda_err(c, e, "point inputs / outputs");
    }
    ProfRec rec;
    prof_begin(c, "ks_dense_points", c->stream, &rec);
    e = launch_dense_points(c->lc(), v->desc, c->ot, c->T, c->L, params->r_min, params->r_max,
                            params->w_norm, dxyz, n, o);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!on_device) {
        KS_TRY_CUDA(c, cudaMemcpyAsync(Y, o.Y, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
        KS_TRY_CUDA(c, cudaMemcpyAsync(s_best, o.s, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
        if (H) KS_TRY_CUDA(c, cudaMemcpyAsync(H, o.H, (size_t)n * S * 8, cudaMemcpyDeviceToHost, c->stream));
        if (W) KS_TRY_CUDA(c, cudaMemcpyAsync(W, o.W, (size_t)n * S * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    return check_status(c);
}

int ks_octant_candidates(ks_ctx *ctx, const ks_seed_result *res, int64_t n, ks_candidate *out,
                         int on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (n < 0 || (n > 0 && (!res || !out))) return set_err(c, KS_EINVAL, "bad candidate buffers");
    if (n == 0) return KS_OK;
    const ks_seed_result *dres = res;
    ks_candidate *dout = out;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        void *pin = scratch(c, kScOct, (size_t)n * sizeof(ks_seed_result), &e);
        if (pin) e = cudaMemcpyAsync(pin, res, (size_t)n * sizeof(ks_seed_result),
                                     cudaMemcpyHostToDevice, c->stream);
        dres = (const ks_seed_result *)pin;
        if (e == cudaSuccess) dout = (ks_candidate *)scratch(c, kScSelOut, (size_t)n * sizeof(ks_candidate), &e);
        if (e != cudaSuccess) return cuda_err(c, e, "candidate buffers");
    }
    ProfRec rec;
    prof_begin(c, "ks_select", c->stream, &rec);
    e = launch_oct_candidates(c->lc(), dres, n, dout);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!on_device)
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, dout, (size_t)n * sizeof(ks_candidate),
                                       cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

int ks_meanshift_candidates(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                            const ks_ms_result *res, int64_t n, ks_candidate *out, int on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (n < 0 || (n > 0 && (!res || !out))) return set_err(c, KS_EINVAL, "bad candidate buffers");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (n == 0) return KS_OK;
    const int S = params->r_max - params->r_min + 1;
    cudaError_t e = cudaSuccess;
    const ks_ms_result *dres = res;
    ks_candidate *dout = out;
    if (!on_device) {
        void *pin = scratch(c, kScMs, (size_t)n * sizeof(ks_ms_result), &e);
        if (pin) e = cudaMemcpyAsync(pin, res, (size_t)n * sizeof(ks_ms_result),
                                     cudaMemcpyHostToDevice, c->stream);
        dres = (const ks_ms_result *)pin;
        if (e == cudaSuccess) dout = (ks_candidate *)scratch(c, kScSelOut, (size_t)n * sizeof(ks_candidate), &e);
        if (e != cudaSuccess) return cuda_err(c, e, "candidate buffers");
    }
    // distinct final centres -> H and W of every scale there -> each item's
    // own scale (many items converge to the same centre)
    const size_t cb = ms_centres_scratch_bytes(n);
    uint8_t *work = (uint8_t *)scratch(c, kScPts, cb + 256, &e);
    double *Y = e == cudaSuccess ? (double *)scratch(c, kScY, (size_t)n * 8, &e) : nullptr;
    uint8_t *sb = e == cudaSuccess ? (uint8_t *)scratch(c, kScS, (size_t)n, &e) : nullptr;
    double *H = e == cudaSuccess ? (double *)scratch(c, kScH, (size_t)n * S * 8, &e) : nullptr;
    double *W = e == cudaSuccess ? (double *)scratch(c, kScW, (size_t)n * S * 8, &e) : nullptr;
    if (e != cudaSuccess) return cuda_err(c, e, "candidate scratch");
    const int32_t *xyz = nullptr;
    const int *centre = nullptr;
    int64_t m = 0;
    ProfRec rec;
    prof_begin(c, "ks_select", c->stream, &rec);
    e = launch_ms_centres(c->lc(), dres, n, work, (unsigned long long *)(work + cb), &xyz, &centre,
                          &m);
    if (e == cudaSuccess)
        e = launch_dense_points(c->lc(), v->desc, c->ot, c->T, c->L, params->r_min, params->r_max,
                                params->w_norm, xyz, m, DenseOut{Y, sb, H, W});
    if (e == cudaSuccess)
        e = launch_ms_candidates(c->lc(), dres, n, centre, H, W, params->r_min, S, dout);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!on_device)
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, dout, (size_t)n * sizeof(ks_candidate),
                                       cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

int ks_select_salient(ks_ctx *ctx, const ks_candidate *in, int64_t n, double h_min, int top_k,
                      ks_candidate *out, int64_t *n_out, int on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (!n_out || n < 0 || (n > 0 && (!in || !out)))
        return set_err(c, KS_EINVAL, "bad selection buffers");
    if (top_k < 1 || top_k > 256) return set_err(c, KS_EINVAL, "top_k must be in [1, 256]");
    if (n > (int64_t)1 << 30) return set_err(c, KS_EINVAL, "more than 2^30 candidates");
    *n_out = 0;
    if (n == 0) return KS_OK;
    cudaError_t e = cudaSuccess;
    const ks_candidate *din = in;
    if (!on_device) {
        void *p = scratch(c, kScSelIn, (size_t)n * sizeof(ks_candidate), &e);
        if (p) e = cudaMemcpyAsync(p, in, (size_t)n * sizeof(ks_candidate), cudaMemcpyHostToDevice,
                                   c->stream);
        din = (const ks_candidate *)p;
        if (e != cudaSuccess) return cuda_err(c, e, "selection input");
    }
    // scratch: hash table + two candidate lists, then top_k results and a counter
    const size_t sb = select_scratch_bytes(n);
    uint8_t *work = (uint8_t *)scratch(c, kScTune, sb + 256 * sizeof(ks_candidate) + 512, &e);
    if (e != cudaSuccess) return cuda_err(c, e, "selection scratch");
    ks_candidate *res = (ks_candidate *)(work + (sb + 255) / 256 * 256);
    unsigned long long *cnt = (unsigned long long *)(res + 256);
    int64_t k = 0;
    ProfRec rec;
    prof_begin(c, "ks_select", c->stream, &rec);
    e = launch_select(c->lc(), din, n, h_min, top_k, work, on_device ? out : res, cnt, &k);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!on_device && k)
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, res, (size_t)k * sizeof(ks_candidate),
                                       cudaMemcpyDeviceToHost, c->stream));
    *n_out = k;
    return check_status(c);
}

int ks_seed_count(ks_ctx *ctx, ks_vol vol, const ks_params *params, int64_t *n) {
    if (!ctx || !params || !n) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (params->stride < 1) return set_err(c, KS_EINVAL, "stride must be >= 1");
    auto cnt = [&](int d) { return d > params->stride / 2 ? (d - params->stride / 2 - 1) / params->stride + 1 : 0; };
    *n = (int64_t)cnt(v->nx) * cnt(v->ny) * cnt(v->nz);
    return KS_OK;
}

}  // extern "C"

namespace ks {

// Shared by ks_seed_climb, ks_meanshift and the batched launch: seeds to the
// device, one SeedJob, one queue segment.
static int seeds_to_device(Ctx *c, cudaStream_t s, Volume *v, const ks_params *p,
                           const int32_t *seeds_xyz, int64_t n_in, std::vector<int32_t> *host,
                           int32_t **dev, int slot = kScSeeds) {
    if (seeds_xyz) {
        host->assign(seeds_xyz, seeds_xyz + 3 * n_in);
        for (int64_t i = 0; i < n_in; ++i) {
            const int32_t x = seeds_xyz[3 * i], y = seeds_xyz[3 * i + 1], z = seeds_xyz[3 * i + 2];
            if (x < 0 || y < 0 || z < 0 || x >= v->nx || y >= v->ny || z >= v->nz)
                return set_err(c, KS_EINVAL, "seed outside the volume");
        }
    } else {
        *host = seed_grid(v->nx, v->ny, v->nz, p->stride);
    }
    cudaError_t e;
    *dev = (int32_t *)scratch(c, slot, std::max<size_t>(host->size() * 4, 16), &e);
    if (!*dev) return cuda_err(c, e, "seed buffer");
    if (!host->empty())
        KS_TRY_CUDA(c, cudaMemcpyAsync(*dev, host->data(), host->size() * 4,
                                       cudaMemcpyHostToDevice, s));
    return KS_OK;
}

struct QueueBuf {
    SeedJob *jobs;
    int64_t *seg_start;
    int *seg_kind, *seg_job;
};

// Lay jobs + segments out in one device buffer (queue buffer `buf`: 0 =
// c->batch_mem, 1 = c->batch_mem2, grown on demand), copy them, and fill a
// SeedQueue.  A buffer is used on one stream at a time, so growing it only
// waits for that stream.
static int upload_queue(Ctx *c, cudaStream_t s, const std::vector<SeedJob> &jobs,
                        const std::vector<int64_t> &ss, const std::vector<int> &sk,
                        const std::vector<int> &sj, SeedQueue *q, int buf = 0) {
    void *&mem = buf ? c->batch_mem2 : c->batch_mem;
    size_t &mem_bytes = buf ? c->batch_mem2_bytes : c->batch_mem_bytes;
    const size_t bj = jobs.size() * sizeof(SeedJob);
    const size_t bs = ss.size() * 8, bk = sk.size() * 4, bjj = sj.size() * 4;
    const size_t need = 256 + bj + bs + bk + bjj + 64;
    if (mem_bytes < need) {
        cudaStreamSynchronize(s);
        dev_free(c, mem, mem_bytes);
        mem = nullptr;
        mem_bytes = 0;
        void *p;
        KS_TRY_CUDA(c, dev_alloc(c, &p, need * 2));
        mem = p;
        mem_bytes = need * 2;
    }
    std::vector<uint8_t> h(need, 0);
    size_t off = 256;   // first 256 bytes: the persistent-queue head counter
    auto put = [&](const void *src, size_t n) {
        const size_t at = off;
        if (n) std::memcpy(h.data() + at, src, n);
        off += (n + 15) / 16 * 16;
        return (uint8_t *)mem + at;
    };
    q->jobs = (const SeedJob *)put(jobs.data(), bj);
    q->seg_start = (const int64_t *)put(ss.data(), bs);
    q->seg_kind = (const int *)put(sk.data(), bk);
    q->seg_job = (const int *)put(sj.data(), bjj);
    q->n_segs = (int)sk.size();
    q->n_tickets = ss.back();
    q->head = (unsigned long long *)mem;
    KS_TRY_CUDA(c, cudaMemcpyAsync(mem, h.data(), off, cudaMemcpyHostToDevice, s));
    return KS_OK;
}

static int run_queue(Ctx *c, cudaStream_t s, const SeedQueue &q, int max_B, int max_S, int kinds,
                     bool persistent) {
    if (q.n_tickets == 0) return KS_OK;
    const int grid =
        persistent ? c->num_sms * seed_blocks_per_sm(max_B, max_S, kinds) : (int)q.n_tickets;
    ProfRec rec;
    prof_begin(c, persistent ? "ks_seeds_persistent" : "ks_seeds", s, &rec);
    cudaError_t e =
        launch_seeds(c->lc(s), q, c->ot, c->T, c->L, max_B, max_S, kinds, persistent, grid);
    prof_end(c, &rec, s);
    return cuda_err(c, e, "seed launch");
}

// seeds_slot, qbuf: the scratch slot of the seed list and the queue buffer
// (another pair lets a second search run beside the first on another stream).
static int seed_common(Ctx *c, ks_vol vol, const ks_params *p, const int32_t *seeds_xyz,
                       int64_t n_seeds, int kind, void *out, int64_t capacity, int64_t *n_out,
                       int32_t *traj, int out_on_device, int planar = 0,
                       cudaStream_t s = nullptr, bool wait = true, int seeds_slot = kScSeeds,
                       int qbuf = 0) {
    if (!s) s = c->stream;
    std::string why;
    int st = validate_params(p, &why);
    if (st) return set_err(c, st, why);
    if (!out || !n_out) return set_err(c, KS_EINVAL, "out / n_out is NULL");
    if (seeds_xyz && n_seeds < 0) return set_err(c, KS_EINVAL, "n_seeds < 0");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    std::vector<int32_t> hs;
    int32_t *ds;
    st = seeds_to_device(c, s, v, p, seeds_xyz, n_seeds, &hs, &ds, seeds_slot);
    if (st) return st;
    const int64_t ns = (int64_t)hs.size() / 3;
    const int S = p->r_max - p->r_min + 1;
    const int64_t n_items = kind == kOctant ? ns : ns * S;
    *n_out = n_items;
    if (capacity < n_items) return set_err(c, KS_EINVAL, "output capacity too small");
    const size_t rec = kind == kOctant ? sizeof(ks_seed_result) : sizeof(ks_ms_result);
    cudaError_t e = cudaSuccess;
    void *dout = out;
    if (!out_on_device) dout = scratch(c, kind == kOctant ? kScOct : kScMs, n_items * rec + 16, &e);
    int32_t *dtraj = traj;
    const size_t traj_bytes = (size_t)ns * (p->max_iter + 1) * 3 * 4;
    if (traj && !out_on_device && e == cudaSuccess)
        dtraj = (int32_t *)scratch(c, kScTraj, traj_bytes + 16, &e);
    if (e != cudaSuccess) return cuda_err(c, e, "seed outputs");
    SeedJob J{};
    J.vol = v->desc;
    J.planar = planar;
    J.r_min = p->r_min;
    J.r_max = p->r_max;
    J.S = S;
    J.max_iter = p->max_iter;
    J.w_norm = p->w_norm;
    J.seeds = ds;
    J.n_seeds = ns;
    J.oct_out = kind == kOctant ? (ks_seed_result *)dout : nullptr;
    J.ms_out = kind == kMeanShift ? (ks_ms_result *)dout : nullptr;
    J.traj = kind == kOctant ? dtraj : nullptr;
    SeedQueue q{};
    if (kind == kOctant) {
        // one block per seed
        st = upload_queue(c, s, {J}, {0, ns}, {kOctant}, {0}, &q, qbuf);
        if (st) return st;
        st = run_queue(c, s, q, v->binning.bins, S, 1 << kOctant, false);
    } else {
        // block-path items, then warp-path items, on a persistent launch
        const int64_t nb = seed_tickets(kMeanShift, ns, p->r_min, S, J.vol.B);
        const int64_t nw = seed_tickets(kMsWarp, ns, p->r_min, S, J.vol.B);
        st = upload_queue(c, s, {J}, {0, nb, nb + nw}, {kMeanShift, kMsWarp}, {0, 0}, &q, qbuf);
        if (st) return st;
        st = run_queue(c, s, q, v->binning.bins, S, 1 << kMeanShift, true);
    }
    if (st) return st;
    if (!out_on_device && n_items) {
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, dout, n_items * rec, cudaMemcpyDeviceToHost, s));
        if (traj && kind == kOctant)
            KS_TRY_CUDA(c, cudaMemcpyAsync(traj, dtraj, traj_bytes, cudaMemcpyDeviceToHost, s));
    }
    // wait = false: the caller joins stream s and checks the status itself
    return wait ? check_status(c, s) : KS_OK;
}

}  // namespace ks

extern "C" {

int ks_seed_climb(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *seeds_xyz,
                  int64_t n_seeds, ks_seed_result *out, int64_t capacity, int64_t *n_out,
                  int32_t *traj, int out_on_device) {
    if (!ctx) return KS_EINVAL;
    return seed_common(&ctx->impl, vol, params, seeds_xyz, n_seeds, kOctant, out, capacity, n_out,
                       traj, out_on_device);
}

int ks_quadrant_climb(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                      const int32_t *seeds_xyz, int64_t n_seeds, ks_seed_result *out,
                      int64_t capacity, int64_t *n_out, int32_t *traj, int out_on_device) {
    if (!ctx) return KS_EINVAL;
    return seed_common(&ctx->impl, vol, params, seeds_xyz, n_seeds, kOctant, out, capacity, n_out,
                       traj, out_on_device, 1);
}

int ks_meanshift(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *seeds_xyz,
                 int64_t n_seeds, ks_ms_result *out, int64_t capacity, int64_t *n_out,
                 int out_on_device) {
    if (!ctx) return KS_EINVAL;
    return seed_common(&ctx->impl, vol, params, seeds_xyz, n_seeds, kMeanShift, out, capacity,
                       n_out, nullptr, out_on_device);
}

int ks_saliency(ks_ctx *ctx, ks_vol vol, const ks_params *params, double *Y, uint8_t *s_best,
                ks_seed_result *oct, int64_t oct_capacity, int64_t *n_oct, ks_ms_result *ms,
                int64_t ms_capacity, int64_t *n_ms, int out_on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (!Y || !s_best) return set_err(c, KS_EINVAL, "Y_best / s_best is NULL");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (!c->hi_stream) {
        int least = 0, greatest = 0;
        KS_TRY_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        KS_TRY_CUDA(c, cudaStreamCreateWithPriority(&c->hi_stream, cudaStreamNonBlocking, greatest));
        KS_TRY_CUDA(c, cudaStreamCreateWithPriority(&c->lo_stream, cudaStreamNonBlocking, least));
        KS_TRY_CUDA(c, cudaStreamCreateWithPriority(&c->lo2_stream, cudaStreamNonBlocking, least));
        for (cudaEvent_t *ev : {&c->ev_fork, &c->ev_hi, &c->ev_lo, &c->ev_lo2})
            KS_TRY_CUDA(c, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    const size_t n = (size_t)v->nx * v->ny * v->nz;
    DenseOut o{Y, s_best, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    if (!out_on_device) {
        o.Y = (double *)scratch(c, kScY, n * 8, &e);
        if (o.Y) o.s = (uint8_t *)scratch(c, kScS, n, &e);
        if (e != cudaSuccess) return cuda_err(c, e, "dense outputs");
    }
    KS_TRY_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
    KS_TRY_CUDA(c, cudaStreamWaitEvent(c->hi_stream, c->ev_fork, 0));
    KS_TRY_CUDA(c, cudaStreamWaitEvent(c->lo_stream, c->ev_fork, 0));
    KS_TRY_CUDA(c, cudaStreamWaitEvent(c->lo2_stream, c->ev_fork, 0));
    // From here on every path joins all three streams before returning, so
    // no copy into the caller's buffers is still in flight after an error.
    // The dense sweep first, at the highest priority: the seed searches'
    // blocks are dispatched as its last wave leaves SMs free.  The octant
    // climb and mean shift take a low-priority stream each, the octant
    // climb launched first: mean-shift blocks fill the SMs that the octant
    // climb's last searches leave idle instead of waiting for them (the
    // pet128 step: 9.83 ms with both on one stream, 9.75 ms).  Each has its
    // own seed list and queue buffer.
    st = run_dense(c, c->hi_stream, v, params, o, 0, v->nz);
    if (st == KS_OK && !out_on_device) {
        e = cudaMemcpyAsync(Y, o.Y, n * 8, cudaMemcpyDeviceToHost, c->hi_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s_best, o.s, n, cudaMemcpyDeviceToHost, c->hi_stream);
        if (e != cudaSuccess) st = cuda_err(c, e, "dense outputs");
    }
    if (st == KS_OK)
        st = seed_common(c, vol, params, nullptr, 0, kOctant, oct, oct_capacity, n_oct, nullptr,
                         out_on_device, 0, c->lo_stream, false);
    if (st == KS_OK)
        st = seed_common(c, vol, params, nullptr, 0, kMeanShift, ms, ms_capacity, n_ms, nullptr,
                         out_on_device, 0, c->lo2_stream, false, kScSeeds2, 1);
    e = cudaEventRecord(c->ev_hi, c->hi_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_lo, c->lo_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_lo2, c->lo2_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_hi, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_lo, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_lo2, 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->hi_stream);
        cudaStreamSynchronize(c->lo_stream);
        cudaStreamSynchronize(c->lo2_stream);
        return st != KS_OK ? st : cuda_err(c, e, "join");
    }
    const int st2 = check_status(c);
    return st != KS_OK ? st : st2;
}

int ks_abmsod(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *seeds_xyz,
              int64_t n_seeds, ks_abmsod_result *out, int64_t capacity, int64_t *n_out,
              int out_on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    int st = validate_params(params, &why);
    if (st) return set_err(c, st, why);
    if (!out || !n_out) return set_err(c, KS_EINVAL, "out / n_out is NULL");
    if (seeds_xyz && n_seeds < 0) return set_err(c, KS_EINVAL, "n_seeds < 0");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    std::vector<int32_t> hs;
    int32_t *ds;
    st = seeds_to_device(c, c->stream, v, params, seeds_xyz, n_seeds, &hs, &ds);
    if (st) return st;
    const int64_t ns = (int64_t)hs.size() / 3;
    const int S = params->r_max - params->r_min + 1;
    const int64_t n_items = ns * S;
    *n_out = n_items;
    if (capacity < n_items) return set_err(c, KS_EINVAL, "output capacity too small");
    if (n_items == 0) return KS_OK;
    cudaError_t e = cudaSuccess;
    ks_abmsod_result *dout = out;
    if (!out_on_device)
        dout = (ks_abmsod_result *)scratch(c, kScAb, n_items * sizeof(ks_abmsod_result), &e);
    unsigned long long *ticket =
        e == cudaSuccess ? (unsigned long long *)scratch(c, kScTicket, 16, &e) : nullptr;
    if (e != cudaSuccess) return cuda_err(c, e, "abmsod outputs");
    ProfRec rec;
    prof_begin(c, "ks_abmsod", c->stream, &rec);
    e = launch_abmsod(c->lc(), v->desc, ds, nullptr, nullptr, ns, params->r_min, params->r_max,
                      params->max_iter, g_abmsod_team_radius, kAbmsodTeamRadius, dout, ticket);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!out_on_device)
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, dout, n_items * sizeof(ks_abmsod_result),
                                       cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

int ks_abmsod_candidates(ks_ctx *ctx, ks_vol vol, const double *x, const double *H, int64_t n,
                         int max_iter, ks_abmsod_result *out, int on_device) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    if (n < 0 || (n > 0 && (!x || !H || !out)))
        return set_err(c, KS_EINVAL, "n < 0 or a NULL buffer");
    if (max_iter < 0 || max_iter > 1000) return set_err(c, KS_EINVAL, "max_iter outside [0, 1000]");
    Volume *v = find_volume(c, vol);
    if (!v) return set_err(c, KS_ENOTFOUND, "unknown volume");
    if (n == 0) return KS_OK;
    const double dim[3] = {(double)v->nx, (double)v->ny, (double)v->nz};
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a)
                if (!(x[3 * i + a] >= 0.0 && x[3 * i + a] <= dim[a] - 1.0))
                    return set_err(c, KS_EINVAL, "candidate centre outside the volume");
            for (int k = 0; k < 6; ++k) {
                const double h = H[6 * i + k];
                const bool diag = k == 0 || k == 3 || k == 5;
                if (!(diag ? (h >= 1.0 && h <= 1024.0) : std::fabs(h) <= 1024.0))
                    return set_err(c, KS_EINVAL, "bandwidth entry outside its range");
            }
        }
    }
    cudaError_t e = cudaSuccess;
    const double *dx = x, *dH = H;
    ks_abmsod_result *dout = out;
    if (!on_device) {
        double *buf = (double *)scratch(c, kScCand, (size_t)n * 9 * sizeof(double), &e);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf, x, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf + 3 * n, H, (size_t)n * 6 * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream);
        dx = buf;
        dH = buf + 3 * n;
        if (e == cudaSuccess)
            dout = (ks_abmsod_result *)scratch(c, kScAb, (size_t)n * sizeof(ks_abmsod_result), &e);
    }
    unsigned long long *ticket =
        e == cudaSuccess ? (unsigned long long *)scratch(c, kScTicket, 16, &e) : nullptr;
    if (e != cudaSuccess) return cuda_err(c, e, "abmsod candidates");
    ProfRec rec;
    prof_begin(c, "ks_abmsod", c->stream, &rec);
    e = launch_abmsod(c->lc(), v->desc, nullptr, dx, dH, n, 0, 0, max_iter, g_abmsod_team_radius,
                      kAbmsodTeamRadius, dout, ticket);
    prof_end(c, &rec, c->stream);
    KS_TRY_CUDA(c, e);
    if (!on_device)
        KS_TRY_CUDA(c, cudaMemcpyAsync(out, dout, (size_t)n * sizeof(ks_abmsod_result),
                                       cudaMemcpyDeviceToHost, c->stream));
    const int st = check_status(c);
    if (st == KS_EINVAL)
        return set_err(c, KS_EINVAL, "a candidate centre or bandwidth entry outside its range");
    return st;
}

}  // extern "C"


extern "C" {

int ks_batch_seeds(ks_ctx *ctx, const ks_vol *vols, const ks_params *params, int n_vols,
                   int kinds, ks_seed_result *const *oct_out, ks_ms_result *const *ms_out,
                   int use_graph) {
    if (!ctx || !vols || !params || n_vols < 1 || !(kinds & 3)) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::string why;
    std::vector<Volume *> vs(n_vols);
    for (int i = 0; i < n_vols; ++i) {
        int st = validate_params(&params[i], &why);
        if (st) return set_err(c, st, why);
        vs[i] = find_volume(c, vols[i]);
        if (!vs[i]) return set_err(c, KS_ENOTFOUND, "unknown volume");
    }
    // signature of this batch (volume handles, params, kinds)
    std::vector<int64_t> key{kinds, n_vols};
    for (int i = 0; i < n_vols; ++i) {
        key.push_back(vols[i]);
        const ks_params &p = params[i];
        key.insert(key.end(), {p.r_min, p.r_max, p.stride, p.max_iter, p.w_norm});
    }
    BatchGraph *bg = nullptr;
    {
        std::lock_guard<std::mutex> g(g_graph_mu);
        for (auto &x : g_graphs[c])
            if (x->key == key) bg = x.get();
    }
    if (!bg) {
        auto nb = std::make_unique<BatchGraph>();
        nb->key = key;
        // seeds + outputs of every volume in one allocation
        std::vector<std::vector<int32_t>> seeds(n_vols);
        size_t seed_bytes = 0, oct_bytes = 0, ms_bytes = 0;
        for (int i = 0; i < n_vols; ++i) {
            seeds[i] = seed_grid(vs[i]->nx, vs[i]->ny, vs[i]->nz, params[i].stride);
            const int64_t ns = (int64_t)seeds[i].size() / 3;
            const int S = params[i].r_max - params[i].r_min + 1;
            nb->n_oct.push_back((kinds & 1) ? ns : 0);
            nb->n_ms.push_back((kinds & 2) ? ns * S : 0);
            seed_bytes += (seeds[i].size() * 4 + 15) / 16 * 16;
            nb->oct_at.push_back(oct_bytes);
            nb->ms_at.push_back(ms_bytes);
            oct_bytes += nb->n_oct.back() * sizeof(ks_seed_result);
            ms_bytes += nb->n_ms.back() * sizeof(ks_ms_result);
        }
        std::vector<SeedJob> jobs(n_vols);
        const size_t jobs_at = 0, seg_at = (n_vols * sizeof(SeedJob) + 255) / 256 * 256;
        const size_t segs_bytes = plan_bytes_bound(2 * (size_t)n_vols);
        const size_t seeds_at = seg_at + (segs_bytes + 255) / 256 * 256;
        nb->oct_off = seeds_at + (seed_bytes + 255) / 256 * 256;
        nb->ms_off = nb->oct_off + (oct_bytes + 255) / 256 * 256;
        nb->bytes = nb->ms_off + ms_bytes + 256;
        void *p;
        cudaError_t e = dev_alloc(c, &p, nb->bytes);
        if (e != cudaSuccess) return cuda_err(c, e, "batch buffers");
        nb->mem = p;
        uint8_t *m = (uint8_t *)p;
        std::vector<uint8_t> host(nb->ms_off, 0);
        size_t so = seeds_at;
        for (int i = 0; i < n_vols; ++i) {
            std::memcpy(host.data() + so, seeds[i].data(), seeds[i].size() * 4);
            SeedJob &J = jobs[i];
            J.vol = vs[i]->desc;
            J.r_min = params[i].r_min;
            J.r_max = params[i].r_max;
            J.S = params[i].r_max - params[i].r_min + 1;
            J.max_iter = params[i].max_iter;
            J.w_norm = params[i].w_norm;
            J.seeds = (const int32_t *)(m + so);
            J.n_seeds = (int64_t)seeds[i].size() / 3;
            J.oct_out = (ks_seed_result *)(m + nb->oct_off + nb->oct_at[i]);
            J.ms_out = (ks_ms_result *)(m + nb->ms_off + nb->ms_at[i]);
            J.traj = nullptr;
            so += (seeds[i].size() * 4 + 15) / 16 * 16;
        }
        // octant segments first (the longest items), then mean shift; one
        // persistent launch per (bins, scales) class
        std::vector<std::pair<int, int>> segs;
        for (int kind = 0; kind < 2; ++kind)
            for (int i = 0; i < n_vols; ++i)
                if (kind == 0 ? nb->n_oct[i] : nb->n_ms[i])
                    segs.push_back({i, kind == 0 ? kOctant : kMeanShift});
        std::memcpy(host.data() + jobs_at, jobs.data(), n_vols * sizeof(SeedJob));
        // the plan fits [seg_at, seeds_at): plan_bytes_bound(2 n_vols) was reserved
        nb->classes = plan_class_queues(c, jobs, (const SeedJob *)(m + jobs_at), segs, host,
                                        seg_at, m);
        KS_TRY_CUDA(c, cudaMemcpyAsync(m, host.data(), host.size(), cudaMemcpyHostToDevice,
                                       c->stream));
        KS_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
        // capture [reset heads; persistent launches] as a graph
        cudaGraph_t graph;
        KS_TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = launch_class_queues(c, c->stream, c->d_status, nb->classes);
        e = cudaStreamEndCapture(c->stream, &graph);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&nb->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            dev_free(c, nb->mem, nb->bytes);
            return cuda_err(c, e, "batch graph");
        }
        bg = nb.get();
        std::lock_guard<std::mutex> g(g_graph_mu);
        g_graphs[c].push_back(std::move(nb));
    }
    ProfRec rec;
    prof_begin(c, "ks_seeds_persistent", c->stream, &rec);
    if (use_graph) {
        KS_TRY_CUDA(c, cudaGraphLaunch(bg->exec, c->stream));
    } else {
        KS_TRY_CUDA(c, launch_class_queues(c, c->stream, c->d_status, bg->classes));
    }
    prof_end(c, &rec, c->stream);
    for (int i = 0; i < n_vols; ++i) {
        if (oct_out && oct_out[i] && bg->n_oct[i])
            KS_TRY_CUDA(c, cudaMemcpyAsync(oct_out[i], (uint8_t *)bg->mem + bg->oct_off + bg->oct_at[i],
                                           bg->n_oct[i] * sizeof(ks_seed_result),
                                           cudaMemcpyDeviceToHost, c->stream));
        if (ms_out && ms_out[i] && bg->n_ms[i])
            KS_TRY_CUDA(c, cudaMemcpyAsync(ms_out[i], (uint8_t *)bg->mem + bg->ms_off + bg->ms_at[i],
                                           bg->n_ms[i] * sizeof(ks_ms_result),
                                           cudaMemcpyDeviceToHost, c->stream));
    }
    return check_status(c);
}

// ------------------------------------------------------------- diagnostics
int ks_tables(ks_ctx *ctx, int64_t nmax, double *T, double *L) {
    if (!ctx || nmax < 0 || nmax > kTableN || !T || !L) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    KS_TRY_CUDA(c, cudaMemcpy(T, c->T, (nmax + 1) * 8, cudaMemcpyDeviceToHost));
    KS_TRY_CUDA(c, cudaMemcpy(L, c->L, (nmax + 1) * 8, cudaMemcpyDeviceToHost));
    return KS_OK;
}

int64_t ks_launch_count(ks_ctx *ctx) { return ctx ? ctx->impl.launches.load() : -1; }

int ks_set_profiling(ks_ctx *ctx, int on) {
    if (!ctx) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    cudaStreamSynchronize(c->stream);
    std::lock_guard<std::mutex> g(c->mu);
    for (auto &r : c->prof) {
        if (r.a) cudaEventDestroy(r.a);
        if (r.b) cudaEventDestroy(r.b);
    }
    c->prof.clear();
    c->profiling = on != 0;
    return KS_OK;
}

int ks_kernel_time(ks_ctx *ctx, const char *prefix, double *ms_total, int64_t *launches) {
    if (!ctx || !prefix || !ms_total || !launches) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    cudaStreamSynchronize(c->stream);
    std::lock_guard<std::mutex> g(c->mu);
    double t = 0;
    int64_t n = 0;
    const size_t lp = std::strlen(prefix);
    for (auto &r : c->prof) {
        if (r.name.compare(0, lp, prefix) != 0 || !r.a) continue;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            t += ms;
            ++n;
        }
    }
    *ms_total = t;
    *launches = n;
    return KS_OK;
}

static int measure_smem(ks_ctx *ctx, double *per_s, bool red_only) {
    if (!ctx || !per_s) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    cudaError_t e;
    uint32_t *sink = (uint32_t *)scratch(c, kScTune, 4096 * 4, &e);
    if (!sink) return cuda_err(c, e, "smem peak");
    const int blocks = c->num_sms * 6, iters = 4096;    // 6 blocks of 8 warps per SM
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, c->stream);
        c->launches++;
        e = launch_smem_peak(c->lc(), sink, blocks, iters, red_only);
        cudaEventRecord(b, c->stream);
        if (e != cudaSuccess) break;
        cudaEventSynchronize(b);
        float ms;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_err(c, e, "smem peak");
    *per_s = (double)blocks * 256.0 * iters * 16.0 / (best * 1e-3);
    return KS_OK;
}

int ks_measure_smem_peak(ks_ctx *ctx, double *per_s) { return measure_smem(ctx, per_s, false); }

int ks_measure_smem_red_rate(ks_ctx *ctx, double *per_s) { return measure_smem(ctx, per_s, true); }

int ks_measure_fp64_rate(ks_ctx *ctx, double *per_s) {
    if (!ctx || !per_s) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    cudaError_t e;
    double *sink = (double *)scratch(c, kScTune, 4096 * 8, &e);
    if (!sink) return cuda_err(c, e, "fp64 rate");
    const int blocks = c->num_sms * 8, iters = 512;      // 64 warps per SM
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, c->stream);
        c->launches++;
        e = launch_fp64_peak(c->lc(), sink, blocks, iters);
        cudaEventRecord(b, c->stream);
        if (e != cudaSuccess) break;
        cudaEventSynchronize(b);
        float ms;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_err(c, e, "fp64 rate");
    *per_s = (double)blocks * 256.0 * iters * 8.0 / (best * 1e-3);
    return KS_OK;
}

int ks_dense_config(ks_ctx *ctx, int bins, int r_max, int *path, int *warps, int *ty, int *tz) {
    if (!ctx || !path || !warps || !ty || !tz) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    std::lock_guard<std::mutex> g(c->mu);
    for (auto &kv : c->tune)
        if (kv.first.B == bins && kv.first.r_max == r_max) {
            *path = kv.second.path;
            *warps = kv.second.warps;
            *ty = kv.second.ty;
            *tz = kv.second.tz;
            return KS_OK;
        }
    return KS_ENOTFOUND;
}

int ks_selftest_wait_timeout(ks_ctx *ctx, int polls) {
    if (!ctx || polls < 1 || polls > (1 << 20)) return KS_EINVAL;
    Ctx *c = &ctx->impl;
    c->launches++;
    KS_TRY_CUDA(c, launch_wait_selftest(c->lc(), polls));
    return check_status(c);
}

// Force the dense launch configuration for every context (path < 0: back
// to the autotuner).  Returns KS_EINVAL for a shape that can never fit.
int ks_set_abmsod_team_radius(int r_team) {
    if (r_team > kRmax + 1) return KS_EINVAL;
    g_abmsod_team_radius = r_team <= 0 ? 0 : r_team;
    return KS_OK;
}

int ks_force_dense_config(int path, int warps, int ty, int tz) {
    if (path < 0) {
        g_forced_path = -1;
        return KS_OK;
    }
    if (path == 5) {
        if (warps != 1 || ty != 1 || tz < 1 || tz > 1024) return KS_EINVAL;
    } else if (path >= 6 && path <= 9) {
        if ((warps != 4 && warps != 8 && (warps != 16 || path != 6)) || ty * tz != warps)
            return KS_EINVAL;
    } else if (path > 9 || warps < 1 || warps > (path >= 2 ? 8 : 16) || ty * tz != warps) {
        return KS_EINVAL;
    }
    g_forced_path = path;
    g_forced_warps = warps;
    g_forced_ty = ty;
    g_forced_tz = tz;
    return KS_OK;
}

}  // extern "C"
