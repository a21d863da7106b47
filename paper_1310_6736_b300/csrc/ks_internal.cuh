// Internal declarations shared by the library's CUDA translation units.
// Device-side descriptors, PTX helpers (mbarrier, TMA, shared-memory
// reductions) and the host-side launch functions each kernel file exports.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ks.h"

namespace ks {

// Every bin volume is stored with this many "not counted" (zero) voxels on
// each side, so a window of radius <= KS_HALO around any in-volume centre
// reads only allocated, zero-initialised memory and needs no bounds checks.
constexpr int kHalo = 32;
constexpr int kRmax = 32;            // largest supported window radius
constexpr int kTableN = 137065;      // |Ball(32)|: largest possible count
constexpr int kMaxBins = 64;
constexpr int kMaxScales = kRmax;    // r_max - r_min + 1 <= 32
constexpr int kSeedThreads = 256;    // block size of the mean-shift (and mixed) seed kernels
constexpr int kOctThreads = 256;     // block size of the octant-only seed kernel

// Device status word bits (ctx->d_status); read back by ks_sync.
constexpr int kStatusTmaTimeout = 1;
constexpr int kStatusQueueTimeout = 2;
constexpr int kStatusBadInput = 4;     // a listed centre lies outside its volume
constexpr int kStatusMisaligned = 8;   // a TMA brick's shared-memory layout was misaligned

// A resident bin volume as the kernels see it.  base points at voxel
// (0,0,0); voxel (x,y,z) is base[z*plane + y*pitch + x] for
// -kHalo <= x < nx + kHalo (same for y, z).  pitch is a multiple of 16.
struct VolDesc {
    const uint8_t *base;
    int nx, ny, nz, B;
    int64_t pitch, plane;
};

// Offsets of Ball(32), built once per context and shared by every kernel.
// rho(o) = ceil(|o|) is the radius class of offset o (the smallest r with
// |o|^2 <= r^2); both parts below are sorted by rho, so Ball(r) is a prefix
// of each.
//   c8:   offsets with three nonzero components, one entry per set of 8
//         sign mirrors: |dx| | |dy| << 8 | |dz| << 16 | rho << 24.  Mirror
//         s (bit0: -x, bit1: -y, bit2: -z) of an entry is a distinct offset
//         in the open octant s.  Class rho: [c8_start[rho], c8_start[rho+1]).
//   rest: offsets on a coordinate plane or axis, one entry each:
//         (dx+64) | (dy+64) << 8 | (dz+64) << 16 | rho << 24.
//         Class rho: [rest_start[rho], rest_start[rho+1]).
// |Ball(r)| = 8 c8_start[r+1] + rest_start[r+1] = ball_size[r].
//   rows: for every r = 0..32, the x-rows of Ball(r): (dy, dz) with
//         dy^2 + dz^2 <= r^2 and half-length w = floor(sqrt(r^2 - dy^2 -
//         dz^2)), packed (dy+64) | (dz+64) << 8 | w << 16; rows with
//         dy != 0 and dz != 0 first, then the rows on the plane y = 0 or
//         z = 0, longest first within each group.  Ball(r)'s rows:
//         [rows_start[r], rows_start[r+1]).
//   ms32: for every r = 0..32, 1 when the mean-shift block path may add
//         its per-voxel sums as two 32-bit words (every column's count,
//         sum(dx + r), sum(dy + r), sum(dz + r) below 2^11, 2^17, 2^16, 2^16
//         with the rows dealt out as the block path deals them), else 0.
//   c8_rows: for every r = 0..32, the c8 entries of Ball(r) again, sorted
//         by row (dz, dy, dx) instead of by rho, at [c8_rows_start[r],
//         c8_rows_start[r+1]).  A walk that visits all of Ball(r) at once
//         (the octant pass) gives consecutive threads neighbouring voxels
//         of one row.
//   restm_rows: the same for the rest offsets, one entry per set of sign
//         mirrors encoded like c8 (|dx| | |dy| << 8 | |dz| << 16 |
//         rho << 24, at least one component 0): its 8 mirrors name every
//         distinct offset of the set 2^z times, z = its zero components.
struct OffsetTables {
    const uint32_t *c8;
    const int *c8_start;      // [kRmax + 2]
    const uint32_t *rest;
    const int *rest_start;    // [kRmax + 2]
    const int *ball_size;     // [kRmax + 1]
    const uint32_t *rows;
    const int *rows_start;    // [kRmax + 2]
    const uint8_t *ms32;      // [kRmax + 1]
    const uint32_t *c8_rows;
    const int *c8_rows_start;     // [kRmax + 2]
    const uint32_t *restm_rows;
    const int *restm_rows_start;  // [kRmax + 2]
};

// Columns per bin of the mean-shift block path for a window of nvox voxels.
__host__ __device__ inline int ms_columns(int nvox) {
    return nvox < 2048 ? 32 : (nvox < 8192 ? 64 : 128);
}

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend the
// thread for a hardware-chosen time); returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, phase)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

// ------------------------------------------------------- exact FP64 steps
// The entropy of a window's counts.  One fixed operation order shared by
// every kernel: occupied-bin count, sum of T[c_b] in bin order (terms with
// c_b <= 1 are exactly +0 and are skipped, which leaves the sum unchanged),
// one IEEE division and one subtraction.  At most one occupied bin -> 0.
__device__ __forceinline__ double entropy_from_sum(double s, uint32_t N, int occupied,
                                                   const double *__restrict__ L) {
    if (occupied <= 1) return 0.0;
    return __dsub_rn(__ldg(L + N), __ddiv_rn(s, (double)N));
}

// W(r) = f(r) * (D / (N * Np)), f = r^2/(2r-1) or 1.
__device__ __forceinline__ double kb_weight(uint64_t D, uint32_t N, uint32_t Np, int r,
                                            int w_norm) {
    if (N == 0 || Np == 0) return 0.0;
    const double f = w_norm == KS_WNORM_ONE
                         ? 1.0
                         : __ddiv_rn((double)(r * r), (double)(2 * r - 1));
    const double q = __ddiv_rn((double)D, (double)((uint64_t)N * (uint64_t)Np));
    return __dmul_rn(f, q);
}

// --------------------------------------------------------------- launches
struct LaunchCtx {
    cudaStream_t stream;
    int *d_status;
    int num_sms;
};

// |Ball(r)| by enumeration (host).
int ball_size_host(int r);

// ks_tables.cu
cudaError_t launch_tables(const LaunchCtx &lc, double *T, double *L, int64_t n);

// ks_bin.cu
cudaError_t launch_bin_int(const LaunchCtx &lc, const void *raw, int dtype, int nx, int ny,
                           int nz, const ks_binning &b, uint8_t *base, int64_t pitch,
                           int64_t plane);
// float32 affine binning: a min/max pass writing per-block partials into
// `scratch` (scratch_blocks float2 entries), then the binning pass.
int bin_f32_scratch_blocks(int num_sms);
cudaError_t launch_bin_f32(const LaunchCtx &lc, const float *raw, int nx, int ny, int nz,
                           int bins, uint8_t *base, int64_t pitch, int64_t plane,
                           float2 *scratch, int scratch_blocks);

// ks_abmsod.cu: adaptive-bandwidth mean shift for every (seed, r) item
// (record seed * S + r - r_min); items with r >= r_team run on a whole
// block, the others on one warp each; persistent over two ticket counters
// (tickets[0..1]) that the launch zeroes.  r_team = 0: r_auto when the
// launch has fewer than 4 items per resident warp, else every item on one
// warp (the small items then fill in behind the large ones).  With cx/cH
// (device arrays, n_seeds x 3 and x 6) the items are those candidates
// instead (record i, r = 0; r_min/r_max ignored): all on blocks when
// r_team is 1..32 or, for r_team <= 0, when the launch has fewer than 4
// items per resident warp, else all on warps.  A candidate outside the
// volume or with a diagonal entry outside [1, 32^2] sets kStatusBadInput
// and is left at iteration 0.
size_t abmsod_smem_bytes(int B);
cudaError_t launch_abmsod(const LaunchCtx &lc, const VolDesc &v, const int32_t *seeds,
                          const double *cx, const double *cH, int64_t n_seeds, int r_min,
                          int r_max, int max_iter, int r_team, int r_auto, ks_abmsod_result *out,
                          unsigned long long *tickets);

// ks_dense.cu
struct DenseConfig {
    int path;      // 0 = TMA brick in shared memory, 1 = direct loads (L1/L2),
                   // 2 = direct loads, two centres per lane (x, x + 32),
                   // 3 = four adjacent centres per lane (r_max <= 25)
    int warps;     // warps per block (each warp owns one row of 32, 64 or 128 centres)
    int ty, tz;    // tile rows in y and z (ty * tz = warps)
};
struct DenseOut {
    double *Y;
    uint8_t *s;
    double *H;     // optional, voxel-major x S
    double *W;     // optional
};
// Bounded-wait self-test (see ks_selftest_wait_timeout).
cudaError_t launch_wait_selftest(const LaunchCtx &lc, int polls);
// The classes rho <= dense_const_rmax() of both parts of the offset tables
// also live in the dense kernel's constant memory.
cudaError_t dense_upload_constant_table(const uint32_t *c8, const int *c8_start,
                                        const uint32_t *rest, const int *rest_start);
int dense_const_rmax();
bool dense_config_fits(const DenseConfig &c, int B, int r_max);
size_t dense_smem_bytes(const DenseConfig &c, int B, int r_max);
// Centres a launch of shape c computes for a volume (its tiles padded to
// whole x-tiles and tile rows; centres past the volume are computed but
// not written).
int64_t dense_computed_centres(const DenseConfig &c, int nx, int ny, int nz);
// Kadir-Brady at n listed centres (xyz int32 triples on the device); a
// centre outside the volume is skipped and sets kStatusBadInput.
cudaError_t launch_dense_points(const LaunchCtx &lc, const VolDesc &v, const OffsetTables &ot,
                                const double *T, const double *L, int r_min, int r_max,
                                int w_norm, const int32_t *xyz, int64_t n, const DenseOut &out);
cudaError_t launch_dense(const LaunchCtx &lc, const VolDesc &v, const CUtensorMap *tmap,
                         const OffsetTables &ot, const double *T, const double *L, int r_min,
                         int r_max, int w_norm, const DenseConfig &cfg, const DenseOut &out,
                         int z0, int z1);

// ks_seeds.cu
// Ticket kinds of a queue segment: an octant seed; a mean-shift (seed, r)
// item run by a whole block (r > 20 or more than 32 bins); one run by a
// single warp (r <= 20 and at most 32 bins).
// A launch's kinds mask has bit kOctant and/or bit kMeanShift (the latter
// covering both mean-shift kinds).
enum ItemKind { kOctant = 0, kMeanShift = 1, kMsWarp = 2 };
struct SeedJob {
    VolDesc vol;
    int r_min, r_max, S, max_iter, w_norm;
    const int32_t *seeds;        // device xyz triples
    int64_t n_seeds;
    ks_seed_result *oct_out;     // device, n_seeds (kind octant)
    ks_ms_result *ms_out;        // device, n_seeds * S (kind mean shift)
    int32_t *traj;               // device, n_seeds * (max_iter+1) * 3, or null
    int planar;                  // octant kind: 1 = the quadrant climb (disks in the
                                 // seed's z-slice, four quadrants), 0 = octants
    // Resumable searches (the serving loop), or null / 0 for whole searches:
    // state holds one int4 per item (octant item s at [s], mean-shift item i
    // at [n_seeds + i]): the centre and it | kItemStarted | kItemDone; a
    // launch advances every unfinished item by at most iter_budget
    // iterations, keeps its state, and on finishing writes the record and
    // adds 1 to *finished.  Zeroed state = not started.  The sequence of
    // operations per item is the whole search's, so records are identical.
    int4 *state;
    unsigned int *finished;
    int iter_budget;
};
constexpr int kItemStarted = 1 << 8;
constexpr int kItemDone = 1 << 9;
// A work queue in tickets: segment k covers tickets [seg_start[k],
// seg_start[k+1]) of kind seg_kind[k] on job seg_job[k]; seed_tickets()
// tells how many tickets of a kind a job needs.  kMsWarp segments must come
// after every other segment of their queue, and a queue holding them must
// be run persistently (blocks switch to per-warp ticket draws there).
struct SeedQueue {
    const SeedJob *jobs;
    const int64_t *seg_start;
    const int *seg_kind;
    const int *seg_job;
    int n_segs;
    int64_t n_tickets;
    unsigned long long *head;    // persistent mode: next ticket counter
};
int64_t seed_tickets(int kind, int64_t n_seeds, int r_min, int S, int B);
// kinds: bit k set when a launch carries tickets of kind k
size_t seed_smem_bytes(int B, int S, int kinds);
cudaError_t launch_seeds(const LaunchCtx &lc, const SeedQueue &q, const OffsetTables &ot,
                         const double *T, const double *L, int max_B, int max_S, int kinds,
                         bool persistent, int grid);
int seed_blocks_per_sm(int max_B, int max_S, int kinds);

// ks_select.cu: candidates and the device selection (ks_select_salient).
cudaError_t launch_oct_candidates(const LaunchCtx &lc, const ks_seed_result *in, int64_t n,
                                  ks_candidate *out);
// The distinct final centres of mean-shift results (*m of them, listed at
// *xyz) and, per item, the number of its centre (*centre); both inside
// `scratch` (ms_centres_scratch_bytes(n)); synchronises the stream once.
size_t ms_centres_scratch_bytes(int64_t n);
cudaError_t launch_ms_centres(const LaunchCtx &lc, const ks_ms_result *in, int64_t n,
                              void *scratch, unsigned long long *d_count, const int32_t **xyz,
                              const int **centre, int64_t *m);
cudaError_t launch_ms_candidates(const LaunchCtx &lc, const ks_ms_result *in, int64_t n,
                                 const int *centre, const double *H, const double *W, int r_min,
                                 int S, ks_candidate *out);
size_t select_scratch_bytes(int64_t n);
// Writes the first min(top_k, #survivors) candidates to `out` (device) and
// their count to *n_out; synchronises the stream once.
cudaError_t launch_select(const LaunchCtx &lc, const ks_candidate *in, int64_t n, double h_min,
                          int top_k, void *scratch, ks_candidate *out,
                          unsigned long long *d_count, int64_t *n_out);

// Micro-kernel: shared-memory increment rate (see ks_measure_smem_peak).
cudaError_t launch_smem_peak(const LaunchCtx &lc, uint32_t *sink, int blocks, int iters,
                             bool red_only);
cudaError_t launch_fp64_peak(const LaunchCtx &lc, double *sink, int blocks, int iters);

}  // namespace ks
