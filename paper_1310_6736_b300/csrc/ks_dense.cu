// Dense Kadir-Brady sweep (Sec. 1; the opening of Sec. 2.1): at every voxel,
// the histogram of Ball(r) for r = r_min..r_max, its entropy H(r), the
// inter-scale pdf change W(r), entropy peaks in scale and Y = H*W.
//
// Work decomposition
//   block  = a tile of 32 (x) * ty * tz centres; warp = one x-row of 32
//            centres; lane = one centre with its own histogram.
//   path 0 = the tile's brick (tile + r_max halo) is copied into shared
//            memory by one TMA 3D tile load; path 1 = bins are read through
//            L1/L2 straight from the halo-padded volume (large radii whose
//            brick does not fit in shared memory).
//   scale  = built incrementally: shell r (offsets with ceil|o| == r, and
//            everything up to r_min for the first scale) is added to the
//            counts of r-1.  Offsets come from the "canonical" table: one
//            entry per set of sign mirrors, expanded to up to 8 voxels with
//            warp-uniform address arithmetic.
//   counts = each lane owns a column of 32-bit words in shared memory,
//            stride 32 words so that the 32 lanes always hit 32 different
//            banks; words hold two 16-bit counters (stored values 2w and
//            2w+1) while |Ball(r_max)| <= 65535, else one 32-bit counter.
//            Stored value 0 (not counted) goes to a dummy counter, so the
//            update has no branch.  Updates are shared-memory reductions
//            (red.shared.add), which carry no register dependence.
//   FP64   = after each shell, one pass over the lane's counters computes
//            the bin-order entropy sum, the exact integer D of W, and
//            copies the counts to the previous-scale column.  W and Y are
//            only evaluated at entropy peaks.
#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kTmaPollLimit = 1 << 20;

struct DenseArgs {
    VolDesc vol;
    BallTables bt;
    const double *T;
    const double *L;
    int r_min, r_max, S, w_norm;
    int ty, tz;
    int z0, z1;                // centres with z0 <= z < z1 (a slab of the volume)
    int bx, by, padx;          // brick row length and rows per plane (path 0)
    uint32_t brick_bytes;
    uint32_t cnt_off, mbar_off;
    DenseOut out;
    int *status;
};

template <int B, bool WIDE>
struct Counters {
    static constexpr int kWords = WIDE ? B + 1 : B / 2 + 1;
    __device__ static __forceinline__ uint32_t word_of(uint32_t v) { return WIDE ? v : v >> 1; }
    __device__ static __forceinline__ uint32_t inc_of(uint32_t v) {
        return WIDE ? 1u : 1u << ((v & 1u) << 4);
    }
};

template <int B, bool WIDE>
__device__ __forceinline__ void add_voxel(uint32_t cnt_lane, const uint8_t *p) {
    const uint32_t v = *p;
    red_add_shared(cnt_lane + (Counters<B, WIDE>::word_of(v) << 7), Counters<B, WIDE>::inc_of(v));
}

template <int B, bool WIDE>
__global__ void __launch_bounds__(512) k_dense(const DenseArgs a,
                                               const __grid_constant__ CUtensorMap tmap,
                                               int path) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ int s_ok;
    using C = Counters<B, WIDE>;
    constexpr int NW = C::kWords;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tx0 = blockIdx.x * 32, ty0 = blockIdx.y * a.ty, tz0 = a.z0 + blockIdx.z * a.tz;
    const int R = a.r_max;

    const uint8_t *src;
    int pz, py;
    if (path == 0) {
        const uint32_t mbar = smem_u32(smem + a.mbar_off);
        if (threadIdx.x == 0) {
            mbar_init(mbar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(mbar, a.brick_bytes);
            tma_load_3d(smem_u32(smem), &tmap, kHalo + tx0 - a.padx, kHalo + ty0 - R,
                        kHalo + tz0 - R, mbar);
            s_ok = mbar_wait_bounded(mbar, 0, kTmaPollLimit) ? 1 : 0;
            if (!s_ok) {
                atomicOr(a.status, kStatusTmaTimeout);
                mbar_wait_bounded(mbar, 0, kTmaPollLimit);   // let the copy land
            }
        }
        __syncthreads();
        if (!s_ok) return;
        src = smem;
        pz = a.bx * a.by;
        py = a.bx;
    } else {
        src = a.vol.base;
        pz = (int)a.vol.plane;
        py = (int)a.vol.pitch;
    }

    // Lane's counter column: cur words at +w*128, prev words at +(NW+w)*128.
    const uint32_t cnt_lane = smem_u32(smem + a.cnt_off) + (warp * 2 * NW * 32 + lane) * 4;
    const int nrows = a.ty * a.tz;
    const int *__restrict__ cstart = a.bt.canon_start;
    const int *__restrict__ csplit = a.bt.canon_split;
    const uint32_t *__restrict__ canon = a.bt.canon;

    for (int row = warp; row < nrows; row += nwarps) {
        const int cy = ty0 + row % a.ty, cz = tz0 + row / a.ty;
        if (cy >= a.vol.ny || cz >= a.z1) continue;              // warp-uniform
        const int cx = tx0 + lane;
        const bool live = cx < a.vol.nx;
        const uint8_t *c0;
        if (path == 0)
            c0 = src + (cz - tz0 + R) * pz + (cy - ty0 + R) * py + (a.padx + lane);
        else
            c0 = src + (int64_t)cz * a.vol.plane + (int64_t)cy * a.vol.pitch +
                 (live ? cx : a.vol.nx - 1);

#pragma unroll 4
        for (int w = 0; w < 2 * NW; ++w) st_shared_u32(cnt_lane + (w << 7), 0u);

        double hm1 = 0.0, hm2 = 0.0;      // H at scale index i-1, i-2
        uint32_t nm1 = 0, nm2 = 0;        // N at i-1, i-2
        uint64_t dm1 = 0;                 // D at i-1
        double yb = 0.0;
        int sb = 0;
        const int64_t oidx = ((int64_t)cz * a.vol.ny + cy) * a.vol.nx + cx;

        for (int i = 0; i < a.S; ++i) {
            const int r = a.r_min + i;
            for (int rho = (i == 0 ? 0 : r); rho <= r; ++rho) {
                const int k0 = __ldg(cstart + rho), k1 = __ldg(csplit + rho),
                          k2 = __ldg(cstart + rho + 1);
                // entries whose 8 sign mirrors are all distinct
                for (int k = k0; k < k1; ++k) {
                    const uint32_t e = __ldg(canon + k);
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    const int zy0 = Z + Y, zy1 = Z - Y, zy2 = Y - Z, zy3 = -Z - Y;
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy0 + X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy0 - X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy1 + X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy1 - X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy2 + X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy2 - X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy3 + X);
                    add_voxel<B, WIDE>(cnt_lane, c0 + zy3 - X);
                }
                // entries on a coordinate plane or axis: distinct mirrors only
                for (int k = k1; k < k2; ++k) {
                    const uint32_t e = __ldg(canon + k);
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    const uint32_t mask = e >> 24;
#pragma unroll
                    for (int s = 0; s < 8; ++s)
                        if (mask & (1u << s))
                            add_voxel<B, WIDE>(cnt_lane, c0 + ((s & 4) ? -Z : Z) +
                                                             ((s & 2) ? -Y : Y) +
                                                             ((s & 1) ? -X : X));
                }
            }

            // ---- exact per-scale quantities from the lane's counters
            const uint32_t w0 = ld_shared_u32(cnt_lane);
            const uint32_t zero_cnt = WIDE ? w0 : (w0 & 0xffffu);
            const uint32_t N = (uint32_t)__ldg(a.bt.ball_size + r) - zero_cnt;
            double ssum = 0.0;
            int occ = 0;
            uint64_t D = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t cw = ld_shared_u32(cnt_lane + (w << 7));
                const uint32_t pw = ld_shared_u32(cnt_lane + ((NW + w) << 7));
                st_shared_u32(cnt_lane + ((NW + w) << 7), cw);
#pragma unroll
                for (int h = 0; h < (WIDE ? 1 : 2); ++h) {
                    const int v = WIDE ? w : 2 * w + h;
                    if (v < 1 || v > B) continue;                 // compile-time
                    const uint32_t c = WIDE ? cw : ((cw >> (16 * h)) & 0xffffu);
                    const uint32_t p = WIDE ? pw : ((pw >> (16 * h)) & 0xffffu);
                    occ += c > 0u;
                    if (c > 1u) ssum = __dadd_rn(ssum, __ldg(a.T + c));
                    const int64_t d = (int64_t)c * nm1 - (int64_t)p * N;
                    D += (uint64_t)(d < 0 ? -d : d);
                }
            }
            const double H = entropy_from_sum(ssum, N, occ, a.L);

            if (i >= 2 && hm2 < hm1 && hm1 >= H) {                // peak at scale i-1
                const double W = kb_weight(dm1, nm1, nm2, r - 1, a.w_norm);
                const double y = __dmul_rn(hm1, W);
                if (sb == 0 || y > yb) {
                    yb = y;
                    sb = r - 1;
                }
            }
            if (live && a.out.H) a.out.H[oidx * a.S + i] = H;
            if (live && a.out.W)
                a.out.W[oidx * a.S + i] = i == 0 ? 0.0 : kb_weight(D, N, nm1, r, a.w_norm);
            hm2 = hm1;
            hm1 = H;
            nm2 = nm1;
            nm1 = N;
            dm1 = D;
        }
        if (live) {
            a.out.Y[oidx] = yb;
            a.out.s[oidx] = (uint8_t)sb;
        }
    }
}

struct Geometry {
    int padx, bx, by, bz;
    size_t brick, cnt_off, cnt_bytes, mbar_off, total;
};

int template_bins(int B) {
    return B <= 2 ? 2 : B <= 4 ? 4 : B <= 8 ? 8 : B <= 16 ? 16 : B <= 32 ? 32 : 64;
}

Geometry geometry(const DenseConfig &c, int B_, int r_max) {
    Geometry g{};
    const int B = template_bins(B_);
    const bool wide = ball_size_host(r_max) > 65535;
    const int words = wide ? B + 1 : B / 2 + 1;
    g.padx = (r_max + 15) / 16 * 16;
    g.bx = (g.padx + 32 + r_max + 15) / 16 * 16;
    g.by = c.ty + 2 * r_max;
    g.bz = c.tz + 2 * r_max;
    g.brick = c.path == 0 ? (size_t)g.bx * g.by * g.bz : 0;
    g.cnt_off = (g.brick + 127) / 128 * 128;
    g.cnt_bytes = (size_t)c.warps * 2 * words * 32 * 4;
    g.mbar_off = g.cnt_off + g.cnt_bytes;
    g.total = g.mbar_off + 16;
    return g;
}

template <int B, bool WIDE>
cudaError_t launch_t(const LaunchCtx &lc, const DenseArgs &a, const CUtensorMap *tmap,
                     const DenseConfig &cfg, size_t smem) {
    auto kern = k_dense<B, WIDE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.vol.nx + 31) / 32, (a.vol.ny + a.ty - 1) / a.ty, (a.z1 - a.z0 + a.tz - 1) / a.tz);
    CUtensorMap dummy{};
    kern<<<grid, cfg.warps * 32, smem, lc.stream>>>(a, tmap ? *tmap : dummy, cfg.path);
    return cudaGetLastError();
}

}  // namespace

int ball_size_host(int r) {
    int n = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dx * dx + dy * dy + dz * dz <= r * r) ++n;
    return n;
}

size_t dense_smem_bytes(const DenseConfig &c, int B, int r_max) {
    return geometry(c, B, r_max).total;
}

bool dense_config_fits(const DenseConfig &c, int B, int r_max) {
    if (c.warps < 1 || c.warps > 16 || c.ty * c.tz != c.warps) return false;
    const Geometry g = geometry(c, B, r_max);
    if (c.path == 0 && (g.bx > 256 || g.by > 256 || g.bz > 256)) return false;
    return g.total + 1024 <= 227 * 1024;   // leave room for static shared memory
}

cudaError_t launch_dense(const LaunchCtx &lc, const VolDesc &v, const CUtensorMap *tmap,
                         const BallTables &bt, const double *T, const double *L, int r_min,
                         int r_max, int w_norm, const DenseConfig &cfg, const DenseOut &out,
                         int z0, int z1) {
    const Geometry g = geometry(cfg, v.B, r_max);
    DenseArgs a{};
    a.vol = v;
    a.bt = bt;
    a.T = T;
    a.L = L;
    a.r_min = r_min;
    a.r_max = r_max;
    a.S = r_max - r_min + 1;
    a.w_norm = w_norm;
    a.ty = cfg.ty;
    a.tz = cfg.tz;
    a.z0 = z0;
    a.z1 = z1;
    a.bx = g.bx;
    a.by = g.by;
    a.padx = g.padx;
    a.brick_bytes = (uint32_t)g.brick;
    a.cnt_off = (uint32_t)g.cnt_off;
    a.mbar_off = (uint32_t)g.mbar_off;
    a.out = out;
    a.status = lc.d_status;
    const bool wide = ball_size_host(r_max) > 65535;
    const CUtensorMap *tm = cfg.path == 0 ? tmap : nullptr;
    // Counter columns are sized for the next supported bin count; the extra
    // stored values never occur, so their counters stay 0 and add nothing
    // to the entropy sum or to D.
    switch (template_bins(v.B)) {
#define KS_CASE(BB)                                                                 \
    case BB:                                                                        \
        return wide ? launch_t<BB, true>(lc, a, tm, cfg, g.total)                   \
                    : launch_t<BB, false>(lc, a, tm, cfg, g.total);
        KS_CASE(2)
        KS_CASE(4)
        KS_CASE(8)
        KS_CASE(16)
        KS_CASE(32)
        KS_CASE(64)
#undef KS_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ks
