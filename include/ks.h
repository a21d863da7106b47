/*
 * ks.h -- C ABI of the B300 Kadir-Brady saliency library (libks.so).
 *
 * The library evaluates intensity histograms and their Shannon entropy over
 * spherical windows Ball(r) = { o in Z^3 : |o|^2 <= r^2 } around many
 * centres and scales of a 3D volume (arXiv 1310.6736, "Fast 3D Salient
 * Region Detection in Medical Images using GPUs").  Three uses share that
 * primitive:
 *   - the dense Kadir-Brady sweep (Sec. 1 and the opening of Sec. 2.1):
 *     entropy H(r) at every voxel and scale, inter-scale pdf change W(r),
 *     saliency Y = H*W at entropy peaks in scale;
 *   - octant hill-climbing from a sparse seed grid (Sec. 2.2, Alg. 1, in 3D);
 *   - mean shift towards a uniform target pmf (Sec. 2.3, Eq. 4-6).
 *
 * Conventions (all entry points)
 *   - Return value is a ks_status; no call aborts or throws across the ABI.
 *     ks_last_error() gives a one-line message for the last failure.
 *   - Volumes are x-fastest: voxel (x,y,z) is element (z*ny + y)*nx + x.
 *     Coordinates are int32 voxel indices, 0 <= x < nx etc.
 *   - Output buffers are owned by the caller.  `out_on_device` = 1 means the
 *     pointer is device memory on the context's device, 0 means host memory.
 *   - Every call is synchronous on the context's stream: it returns after the
 *     work is complete (ks_submit/ks_poll are the asynchronous interface).
 *   - FP64 results follow one fixed operation order (below), so they are
 *     reproducible bit for bit from run to run and batch to batch.
 *
 * Arithmetic (fixed by this library; see the oracle for the plain statement)
 *   bins      stored value b+1 for bin b in [0,B); 0 = voxel not counted
 *             (outside the window level, Sec. 3.2).  Voxels outside the
 *             volume are not counted.
 *   entropy   H = ln N - (sum_{b=0..B-1} T[c_b]) / N, with T[c] = c ln c and
 *             ln N taken from correctly rounded binary64 tables, the sum in
 *             bin order; H = 0 when at most one bin is occupied.
 *   weight    W(r) = f(r) * (D / (N_r N_{r-1})), D = sum_b |c_r(b) N_{r-1} -
 *             c_{r-1}(b) N_r| in exact integers, f(r) = r^2/(2r-1)
 *             (KS_WNORM_KB) or 1 (KS_WNORM_ONE).
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ks_ctx ks_ctx;   /* opaque context: one device, one stream */
typedef int64_t ks_vol;         /* handle of a resident (binned) volume   */
typedef int64_t ks_req;         /* handle of a submitted serving request  */

typedef enum ks_status {
    KS_OK = 0,
    KS_PENDING = 1,       /* ks_poll: request not finished yet              */
    KS_EINVAL = -1,       /* bad argument (sizes, ranges, null pointers)    */
    KS_ENOMEM = -2,       /* HBM budget exceeded or cudaMalloc failed       */
    KS_ECUDA = -3,        /* CUDA runtime/driver error                      */
    KS_ETIMEDOUT = -4,    /* a bounded device wait or a poll timed out      */
    KS_ECANCELED = -5,    /* request was cancelled                          */
    KS_ENOTFOUND = -6,    /* unknown volume or request handle               */
    KS_ENODEV = -7        /* no usable CUDA device                          */
} ks_status;

typedef enum ks_dtype { KS_U8 = 0, KS_I16 = 1, KS_F32 = 2 } ks_dtype;

/* Intensity -> bin map beta(s) (Eq. 4-5: "the bin number in which pixel s
 * lies"; Sec. 3.2: the constrained window-level range).
 *   KS_BIN_CLAMP_SHIFT  integer input: b = (clamp(v, lo, hi) - lo) >> shift
 *   KS_BIN_AFFINE_F32   float input:   b = clamp(floor(bins*(v - vmin) /
 *                       ((vmax - vmin) + 1e-6f)), 0, bins-1) in binary32,
 *                       vmin/vmax = exact volume minimum/maximum
 *   KS_BIN_WINDOW       integer input: v outside [lo, hi] is not counted,
 *                       otherwise b = (v - lo) >> shift
 *   KS_BIN_STORED       uint8 input that is already a bin volume in the
 *                       stored form (ks_volume_bins): v in [1, bins] is bin
 *                       v - 1, any other value is not counted (lets ranks
 *                       that share one volume exchange its bins instead of
 *                       its raw values; shift, lo, hi unused)
 * Requirements: 2 <= bins <= 64; for CLAMP_SHIFT and WINDOW lo <= hi and
 * ((hi - lo) >> shift) <= bins - 1. */
typedef enum ks_bin_kind {
    KS_BIN_CLAMP_SHIFT = 0, KS_BIN_AFFINE_F32 = 1, KS_BIN_WINDOW = 2, KS_BIN_STORED = 3
} ks_bin_kind;

typedef struct ks_binning {
    int32_t kind, bins, shift, lo, hi;
} ks_binning;

typedef enum ks_wnorm { KS_WNORM_KB = 0, KS_WNORM_ONE = 1 } ks_wnorm;

/* Scales r_min..r_max (1 <= r_min < r_max <= 32); seed grid stride (>= 1,
 * seeds at stride/2 + i*stride per axis); max_iter iterations per climb
 * (0..64); w_norm a ks_wnorm. */
typedef struct ks_params {
    int32_t r_min, r_max, stride, max_iter, w_norm;
} ks_params;

/* One octant-climb seed (Sec. 2.2).  (x,y,z) is the final centre, iters the
 * number of window evaluations, converged = 1 when the last evaluation gave
 * no move.  s_best / Y_best / H_best / W_best: the Kadir-Brady evaluation of
 * the full ball at the final centre (s_best = 0: no entropy peak in scale). */
typedef struct ks_seed_result {
    int32_t x, y, z;
    int32_t seed_x, seed_y, seed_z;
    int32_t iters, converged;
    int32_t s_best, reserved;
    double Y_best, H_best, W_best;
} ks_seed_result;

/* One mean-shift item (Sec. 2.3): seed index `seed`, window radius r.
 * rho = Bhattacharyya coefficient with the uniform pmf and H = window
 * entropy, both at the final centre. */
typedef struct ks_ms_result {
    int32_t x, y, z, r;
    int32_t seed, iters, converged, reserved;
    double rho, H;
} ks_ms_result;

/* One adaptive-bandwidth mean-shift candidate (Sec. 2.3, Alg. 2): the best
 * centre x over the iterations (FP64 voxel coordinates), its bandwidth
 * matrix H (entries 00 01 02 11 12 22) and Bhattacharyya coefficient rho to
 * the uniform pmf; the seed index, the starting radius r (H = r^2 I at the
 * start), the iterations run, and stopped = 1 when the search ended at a
 * fall of rho (0: iteration limit or an empty window); voxels: the window
 * voxels of every kernel histogram the item evaluated (each is visited
 * again by the position or bandwidth sums of the same window).  104 bytes. */
typedef struct ks_abmsod_result {
    double x[3];
    double H[6];
    double rho;
    int32_t seed, r, iters, stopped;
    int64_t voxels;
} ks_abmsod_result;

/* A candidate salient region: centre, scale r (0 = none), the index of the
 * seed or item it came from, and the window's entropy H and inter-scale pdf
 * change W at that centre and scale.  40 bytes. */
typedef struct ks_candidate {
    int32_t x, y, z, r;
    int32_t source, reserved;
    double H, W;
} ks_candidate;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` using stream `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * library creates its own non-blocking stream).  hbm_budget_bytes caps the
 * device memory the context allocates (0 = no cap).  Builds the FP64 tables
 * T[c] = c ln c and L[n] = ln n for c, n <= |Ball(32)| on the device.
 * Errors: KS_ENODEV, KS_ENOMEM, KS_ECUDA. */
int ks_init(ks_ctx **out, size_t hbm_budget_bytes, void *cuda_stream, int device);

/* Release every volume, request and buffer of the context.  NULL is a no-op. */
int ks_destroy(ks_ctx *ctx);

const char *ks_strerror(int status);
const char *ks_last_error(ks_ctx *ctx);

/* Block until all work issued by the context is complete and report any
 * device-side error recorded by its kernels (KS_ETIMEDOUT for a bounded
 * wait that gave up). */
int ks_sync(ks_ctx *ctx);

/* ---------------------------------------------------------------- volumes */

/* Copy a raw volume (dtype, nx*ny*nz elements, x-fastest; host memory, or
 * device memory when is_device_ptr = 1) to the device and bin it (Eq. 4's
 * beta).  The library keeps only the uint8 bin volume (padded with a
 * 32-voxel "not counted" halo); the caller keeps ownership of `data`.
 * Errors: KS_EINVAL (dims < 1 or > 4096, bad binning, dtype mismatch with
 * kind), KS_ENOMEM, KS_ECUDA. */
int ks_create_volume(ks_ctx *ctx, const void *data, int is_device_ptr, int dtype,
                     int nx, int ny, int nz, const ks_binning *binning, ks_vol *out);

int ks_release_volume(ks_ctx *ctx, ks_vol vol);

/* Copy the stored bin values (b+1, 0 = not counted; nx*ny*nz bytes,
 * x-fastest, no halo) to `out`. */
int ks_volume_bins(ks_ctx *ctx, ks_vol vol, uint8_t *out, int out_on_device);

/* ------------------------------------------------------------- hot path */

/* Dense Kadir-Brady sweep (Sec. 1; Sec. 2.1 opening): at every voxel,
 * histograms of Ball(r) for r = r_min..r_max built shell by shell, H(r),
 * W(r) (r > r_min), entropy peaks at interior scales (H(r-1) < H(r) >=
 * H(r+1)), Y(r) = H(r) W(r).  Writes Y_best (double, nx*ny*nz) and s_best
 * (uint8, 0 = no peak; the first peak in r, replaced only by a strictly
 * larger Y).  Errors: KS_EINVAL, KS_ENOTFOUND, KS_ENOMEM, KS_ECUDA,
 * KS_ETIMEDOUT. */
int ks_dense_saliency(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                      double *Y_best, uint8_t *s_best, int out_on_device);

/* ks_dense_saliency for the centres of the z-planes [z0, z1) only (0 <= z0
 * < z1 <= nz): their windows still see the whole volume.  Y_best and s_best
 * hold (z1 - z0)*ny*nx values, plane z0 first; each equals the whole
 * sweep's value at the same voxel.  The split of one volume into z-slabs
 * across ranks (Sec. 2.4 runs a search path per thread block; here a slab
 * per GPU, each rank holding its slab plus r_max halo planes). */
int ks_dense_saliency_range(ks_ctx *ctx, ks_vol vol, const ks_params *params, int z0, int z1,
                            double *Y_best, uint8_t *s_best, int out_on_device);

/* As ks_dense_saliency, optionally also writing H(r) and W(r) for every
 * voxel and scale: H, W are nx*ny*nz*S doubles (S = r_max - r_min + 1),
 * voxel-major; either may be NULL. */
int ks_dense_saliency_ex(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                         double *Y_best, uint8_t *s_best, double *H, double *W,
                         int out_on_device);

/* Number of seeds of the uniform grid for `params->stride` (Sec. 2.2). */
int ks_seed_count(ks_ctx *ctx, ks_vol vol, const ks_params *params, int64_t *n_seeds);

/* Octant hill-climbing (Sec. 2.2, Alg. 1 extended to the 8 closed octants
 * of Ball(k) in 3D).  seeds_xyz: n_seeds int32 triples on the host, or NULL
 * for the uniform grid (n_seeds ignored).  Writes one ks_seed_result per
 * seed into `out` (capacity entries) and the seed count into *n_out.
 * traj: optional (NULL) host/device int32 buffer of n * (max_iter+1) * 3
 * positions: entry 0 is the seed, entry t the centre after move t, repeated
 * after the last move.  Errors: KS_EINVAL (capacity too small, seeds
 * outside the volume), KS_ENOTFOUND, KS_ENOMEM, KS_ECUDA. */
int ks_seed_climb(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                  const int32_t *seeds_xyz, int64_t n_seeds,
                  ks_seed_result *out, int64_t capacity, int64_t *n_out,
                  int32_t *traj, int out_on_device);

/* Quadrant hill-climbing: Alg. 1 as printed, in 2D (Sec. 2.2), run in the
 * z-slice of each seed.  Windows are the disks {dx^2 + dy^2 <= k^2, dz = 0};
 * the four closed quadrants j = 0..3 (bit0: x<0, bit1: y<0) give eps_j and
 * k_j as in ks_seed_climb, the step sum_j eps_j k_j sigma_j / sum_j eps_j
 * has no z component, and s_best / Y_best / H_best / W_best are evaluated
 * on the disks at the final centre.  Arguments and results as for
 * ks_seed_climb. */
int ks_quadrant_climb(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                      const int32_t *seeds_xyz, int64_t n_seeds, ks_seed_result *out,
                      int64_t capacity, int64_t *n_out, int32_t *traj, int out_on_device);

/* Mean shift to the uniform pmf (Sec. 2.3, Eq. 4-6) for every (seed, r)
 * item, r = r_min..r_max, item = seed * S + (r - r_min).  Seeds as in
 * ks_seed_climb.  Writes one ks_ms_result per item. */
int ks_meanshift(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                 const int32_t *seeds_xyz, int64_t n_seeds,
                 ks_ms_result *out, int64_t capacity, int64_t *n_out,
                 int out_on_device);

/* The whole detection pass of one volume in one call: the dense Kadir-Brady
 * sweep (as ks_dense_saliency, Sec. 1 and the opening of Sec. 2.1), the
 * octant climb (as ks_seed_climb, Alg. 1) and the uniform-target mean shift
 * (as ks_meanshift, Eq. 4-6) from the default seed grid.  The results are
 * those of the three separate calls, bit for bit.  The dense sweep runs on
 * the device's highest-priority stream, and the octant climb and mean shift
 * each on a lowest-priority stream of its own.  All three are forked from
 * the context's stream and joined to it before return, so the seed blocks
 * fill the SMs that the dense sweep's last wave leaves free, and mean-shift
 * blocks those that the octant climb's last searches leave.
 * Outputs as in the three calls (Y and s_best: nx*ny*nz each; oct: one
 * record per seed; ms: one per (seed, r)); all on the device or all on the
 * host (out_on_device).  KS_EINVAL when a capacity is too small (the
 * counts are still written to n_oct / n_ms). */
int ks_saliency(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                double *Y, uint8_t *s_best,
                ks_seed_result *oct, int64_t oct_capacity, int64_t *n_oct,
                ks_ms_result *ms, int64_t ms_capacity, int64_t *n_ms,
                int out_on_device);

/* Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 6-7) to the
 * uniform pmf HQ_b = 1/B for every (seed, r) item, r = r_min..r_max, item =
 * seed * S + (r - r_min), starting at the seed with H = r^2 I.  The window
 * is the ellipsoid d(s) = (s-x)^T H^-1 (s-x) <= 1 of counted voxels, each
 * weighted by k = exp(-d/2).  An iteration: w_b = sqrt(HQ_b / HP_b) from the
 * kernel histogram HP at (x, H); x' = x + sum k w (s-x) / sum k w, clamped
 * to the volume; HP' and w' at (x', H); H' = 5 (sum w' (s-x')(s-x')^T /
 * sum w' + I/12) (Eq. 7 with the factor n + 2 that keeps a homogeneous
 * ellipsoid's bandwidth, and the second moment I/12 of a unit voxel, which
 * keeps H' positive definite), diagonal entries raised to >= 1 and H'
 * scaled so that none exceeds 32^2; rho = sum_b sqrt(HQ_b HP'_b).  The largest rho so far keeps
 * its (x', H'); the search stops at the first fall of rho or after
 * params->max_iter iterations.  Per-voxel terms are binary32 and all voxel
 * sums are exact fixed-point int64 sums (grids chosen per window from its
 * extent), so results are reproducible bit for bit and independent of the
 * launch shape; they agree with a binary64 evaluation of the same steps to
 * about 1e-4 in H and 1e-6 in rho per iteration.  Seeds, capacity and
 * errors as in ks_meanshift. */
int ks_abmsod(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *seeds_xyz,
              int64_t n_seeds, ks_abmsod_result *out, int64_t capacity, int64_t *n_out,
              int out_on_device);

/* The same search (Alg. 2) from n given candidate ellipsoids, Alg. 2's
 * "each candidate ellipsoid W_i centred at P_i with a bandwidth matrix H_i"
 * (the paper scatters them at random with varying sizes, Sec. 2.3):
 *   x    n x 3 FP64 centres (x, y, z), each in [0, dim - 1]
 *   H    n x 6 FP64 bandwidths (00 01 02 11 12 22), diagonal entries in
 *        [1, 32^2] (the window stays within 32 voxels of its centre),
 *        off-diagonal entries of magnitude <= 32^2
 *   out  n records (seed = candidate index, r = 0), record i for candidate i
 *   on_device  x, H and out are device pointers (else host)
 * max_iter in [0, 1000].  Results are those of ks_abmsod for a candidate
 * (seed, r^2 I).  Errors: KS_EINVAL (a centre or bandwidth entry outside
 * its range: refused before the launch for host inputs; for device inputs
 * the candidate is left at iteration 0 and the call returns KS_EINVAL),
 * KS_ENOTFOUND. */
int ks_abmsod_candidates(ks_ctx *ctx, ks_vol vol, const double *x, const double *H, int64_t n,
                         int max_iter, ks_abmsod_result *out, int on_device);

/* Kadir-Brady at listed centres: the dense sweep's quantities at n centres
 * given as int32 xyz triples (0 <= x < nx etc.): Y_best, s_best and, when
 * H / W are not NULL, H(r) and W(r) for every scale (n x S, centre-major;
 * W(r_min) = 0).  `on_device` applies to xyz and to every output.  Results
 * equal the dense sweep's at the same voxels.  Errors: KS_EINVAL (a centre
 * outside the volume, bad params, NULL buffers), KS_ENOTFOUND. */
int ks_dense_points(ks_ctx *ctx, ks_vol vol, const ks_params *params, const int32_t *xyz,
                    int64_t n, double *Y_best, uint8_t *s_best, double *H, double *W,
                    int on_device);

/* Candidates from the seed searches.  Octant: one per seed result, at its
 * final centre with r = s_best, H_best and W_best (r = 0 when no entropy
 * peak was found).  Mean shift: one per item, at its final centre and its
 * radius r, with H(r) and W(r) evaluated there by ks_dense_points.
 * `on_device` applies to the results and to `out` (n entries). */
int ks_octant_candidates(ks_ctx *ctx, const ks_seed_result *res, int64_t n, ks_candidate *out,
                         int on_device);
int ks_meanshift_candidates(ks_ctx *ctx, ks_vol vol, const ks_params *params,
                            const ks_ms_result *res, int64_t n, ks_candidate *out,
                            int on_device);

/* Selection of salient regions (Sec. 2.3, end; Sec. 3.1): keep candidates
 * with r > 0 and H > h_min; merge candidates with the same (x, y, z, r) into
 * the one with the smallest source; order by W descending, then H
 * descending, then z, y, x, r ascending; write the first min(top_k, #kept)
 * to `out` and their number to *n_out.  1 <= top_k <= 256 (the paper keeps
 * 20).  `on_device` applies to `in` and `out`.  Errors: KS_EINVAL. */
int ks_select_salient(ks_ctx *ctx, const ks_candidate *in, int64_t n, double h_min, int top_k,
                      ks_candidate *out, int64_t *n_out, int on_device);

/* ---------------------------------------------------------- batched form */

/* Run the octant climb and/or mean shift (kinds: bit 0 octant, bit 1 mean
 * shift) of n_vols resident volumes, each with its own params and grid
 * seeds, as ONE persistent launch over a device work queue of
 * (volume, seed, scale) items; use_graph = 1 replays a captured CUDA graph
 * of that launch.  oct_out[i] / ms_out[i]: host arrays sized by
 * ks_seed_count (x S for mean shift); entries may be NULL to skip.  The
 * per-item arithmetic is identical to ks_seed_climb / ks_meanshift. */
int ks_batch_seeds(ks_ctx *ctx, const ks_vol *vols, const ks_params *params, int n_vols,
                   int kinds, ks_seed_result *const *oct_out, ks_ms_result *const *ms_out,
                   int use_graph);

/* -------------------------------------------------------------- serving */

typedef enum ks_req_kind { KS_REQ_SEEDS = 0, KS_REQ_DENSE = 1 } ks_req_kind;

/* A serving request: a raw host volume plus what to compute.  The library
 * copies `data` during ks_submit, so the caller may reuse it on return. */
typedef struct ks_request {
    const void *data;
    int32_t dtype, nx, ny, nz;
    ks_binning binning;
    ks_params params;
    int32_t kind;          /* ks_req_kind                                   */
    int32_t seed_kinds;    /* KS_REQ_SEEDS: bit 0 octant, bit 1 mean shift  */
} ks_request;

/* Result of a finished request.  Arrays are owned by the library and stay
 * valid until ks_release_result (or ks_destroy). */
typedef struct ks_result {
    int32_t status;                       /* KS_OK, KS_ECANCELED, ...     */
    int32_t kind;
    int64_t n_seeds, n_items, n_voxels;
    const ks_seed_result *oct;            /* n_seeds (or NULL)            */
    const ks_ms_result *ms;               /* n_items (or NULL)            */
    const double *Y_best;                 /* dense: n_voxels (or NULL)    */
    const uint8_t *s_best;
    double t_submit_us, t_admit_us, t_done_us;   /* context clock         */
} ks_result;

/* Enqueue a request.  It is admitted to the device when its HBM footprint
 * fits the budget, and its work is interleaved with the other admitted
 * requests' in iteration-level waves (continuous batching).  Errors:
 * KS_EINVAL, KS_ENOMEM (footprint larger than the whole budget). */
int ks_submit(ks_ctx *ctx, const ks_request *req, ks_req *out);

/* Wait up to timeout_us (0 = just look, < 0 = forever) for a request.
 * KS_OK: done and *out filled; KS_PENDING: still running after a 0 timeout;
 * KS_ETIMEDOUT: still running after a positive timeout; KS_ENOTFOUND. */
int ks_poll(ks_ctx *ctx, ks_req req, int64_t timeout_us, ks_result *out);

/* Cancel a request that has not finished; its later poll reports
 * KS_ECANCELED. */
int ks_cancel(ks_ctx *ctx, ks_req req);

/* Free a finished request's result arrays. */
int ks_release_result(ks_ctx *ctx, ks_req req);

/* Iterations each seed item may advance per wave of the serving loop
 * (default 0 = a whole search per wave).  Waves are one persistent
 * launch per class over the items of every admitted seed request; a
 * request that arrives joins the next wave.  Results do not depend on it.
 * Errors: KS_EINVAL (iters outside [0, 1000]). */
int ks_set_serve_wave_iters(ks_ctx *ctx, int iters);

/* ---------------------------------------------------------- diagnostics */

/* Copy the device tables T[0..nmax] and L[0..nmax] (nmax <= |Ball(32)|) to
 * host arrays. */
int ks_tables(ks_ctx *ctx, int64_t nmax, double *T, double *L);

/* Number of kernels the context has launched so far. */
int64_t ks_launch_count(ks_ctx *ctx);

/* Per-kernel CUDA-event timing on the context's stream: when enabled, every
 * launch is bracketed by events; ks_kernel_time returns the summed device
 * time (ms) and launch count of kernels whose name starts with `prefix`. */
int ks_set_profiling(ks_ctx *ctx, int on);
int ks_kernel_time(ks_ctx *ctx, const char *prefix, double *ms_total, int64_t *launches);

/* Shared-memory histogram-increment rate of this device (increments per
 * second) for the kernel's counter layout, measured by a dedicated
 * micro-kernel: the denominator of the histogram kernels' roofline. */
int ks_measure_smem_peak(ks_ctx *ctx, double *increments_per_s);

/* The same counters updated by shared-memory reductions alone (no byte
 * loads, no address arithmetic): the rate no histogram kernel with one
 * reduction per update can exceed. */
int ks_measure_smem_red_rate(ks_ctx *ctx, double *increments_per_s);

/* FP64 addition rate of this device (__dadd_rn lane operations per second):
 * a micro-kernel of independent addition chains on every SM.  The entropy
 * sums and the seed steps are FP64 additions in a fixed order. */
int ks_measure_fp64_rate(ks_ctx *ctx, double *dadd_per_s);

/* Dense-sweep launch configuration chosen for (bins, r_max) by the
 * autotuner: path 0 = TMA brick in shared memory, 1 = direct L2 reads,
 * 2 = direct L2 reads with two centres (x and x + 32) per thread, 3 = four
 * adjacent centres per thread (r_max <= 25 only), 4 = path 3 with the
 * previous-scale counts in tensor memory (r_max <= 25, bins <= 32, and not
 * 8 or fewer), 5 = sliding windows (one histogram per scale, each updated
 * by the voxels entering and leaving its ball as the centre moves along z;
 * r_max <= 25, 16 or 32 bins; one warp per block, tile_z = run length),
 * 6 = path 1 with the previous-scale counts as 32-bit words in tensor
 * memory (r_max > 25, 16, 32 or 64 template bins, 4, 8 or 16 warps),
 * 7 = path 6 with two centres (x and x + 32) per thread (4 or 8 warps),
 * 8 = path 7 with the two centres' counts in 16-bit halves of one word,
 * counted modulo 2^16 and recovered exactly from the previous scale's,
 * 9 = path 4's four adjacent centres per thread for r_max > 25, with the
 * counts of path 8 and the previous counts as 32-bit words in tensor memory
 * (16, 32 or 64 template bins, 4 or 8 warps);
 * warps per block; tile rows in y and z. */
int ks_dense_config(ks_ctx *ctx, int bins, int r_max, int *path, int *warps,
                    int *tile_y, int *tile_z);

/* Force the dense launch configuration for every context of the process
 * (tests use it to cover both paths); path < 0 returns to the autotuner.
 * KS_EINVAL: path > 9, warps outside [1, 16] ([1, 8] for paths 2 to 4;
 * 4, 8 or 16 for path 6; 4 or 8 for paths 7 to 9) or tile_y * tile_z != warps
 * (path 5: warps = tile_y = 1, tile_z in [1, 1024]).
 * A forced shape that does not fit a given (bins, r_max) is ignored for
 * that call. */
int ks_force_dense_config(int path, int warps, int tile_y, int tile_z);

/* ABMSOD work split for every context of the process: items whose starting
 * radius is at least r_team run on a whole thread block (8 warps share each
 * window pass), smaller ones on one warp each; r_team > 32 puts every item
 * on one warp.  r_team <= 0 restores the default, decided per call: r_team
 * = 12 when the call has fewer than 4 items per resident warp, else every
 * item on one warp.  Results do not depend on the split.  KS_EINVAL:
 * r_team > 33. */
int ks_set_abmsod_team_radius(int r_team);

/* Failure-detection self-test: one thread waits on a device barrier that
 * nothing will complete, gives up after `polls` polls (1..2^20), records
 * the timeout in the context's status word and exits -- the same bounded
 * wait the dense kernel uses for its TMA brick.  Returns KS_ETIMEDOUT (the
 * status the host reads back); the context stays usable and the next
 * ks_sync returns KS_OK.  The paper has no counterpart. */
int ks_selftest_wait_timeout(ks_ctx *ctx, int polls);

/* ------------------------------------------------ allocation-free binning */

/* The float32 binning of ks_create_volume (KS_BIN_AFFINE_F32) for callers
 * that may not allocate device memory: code running under an allocator that
 * owns all device memory, a loop that must not take the synchronisation a
 * cudaMalloc/cudaFree can impose, or an application whose memory budget is
 * already spent.  The paper has no counterpart; this is a library-interface
 * convenience.
 *   in     device pointer, nx*ny*nz float32 values, x-fastest
 *   out    device pointer, nx*ny*nz bytes: the stored bin value b+1 of each
 *          voxel, x-fastest, no halo (the layout of ks_volume_bins)
 *   cuda_stream  cudaStream_t the two kernels are enqueued on (NULL = the
 *          legacy default stream); the call returns without waiting.
 * No cudaMalloc, cudaFree or other allocating call is made.  The reduction
 * scratch is a 32 KB array compiled into the library (held on every device
 * that loads it, until exit) and shared by all calls: calls whose kernels
 * overlap on the GPU race on it, so serialise them (one stream, or events).
 * Every call looks up the array's device address in the calling thread's
 * current context (cudaGetSymbolAddress, which allocates nothing); the
 * first call in a context may load the library's device code there, so
 * make that first call before any stream capture.
 * Errors: KS_EINVAL for null pointers, dims outside [1, 4096] (the limit of
 * ks_create_volume; a policy limit, since the scratch does not grow with
 * the volume) or bins outside [2, 64]; KS_ECUDA for a launch failure. */
int ks_bin_f32_noalloc(const float *in, int nx, int ny, int nz, int bins, uint8_t *out,
                       void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KS_H */
