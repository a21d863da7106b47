// Dense Kadir-Brady sweep (Sec. 1; the opening of Sec. 2.1): at every voxel,
// the histogram of Ball(r) for r = r_min..r_max, its entropy H(r), the
// inter-scale pdf change W(r), entropy peaks in scale and Y = H*W.
//
// Work decomposition
//   block  = a tile of 32 (x) * ty * tz centres; warp = one x-row of 32
//            centres; lane = one centre with its own histogram.
//   PATH 0 = the tile's brick (tile + r_max halo) is copied into shared
//            memory by one TMA 3D tile load (out-of-range voxels arrive as
//            0 = not counted); PATH 1 = bins are read through L1/L2 straight
//            from the halo-padded volume.  The autotuner picks per shape.
//   scale  = built incrementally: shell r (offsets o with ceil|o| == r, and
//            everything up to r_min for the first scale) is added to the
//            counts of r-1.
//   offsets= per radius class rho, the offsets with three nonzero
//            components, stored once per set of 8 sign mirrors as (|dx|,
//            |dy|, |dz|) and expanded with warp-uniform arithmetic, then every
//            offset on a coordinate plane or axis, stored with its signs.
//            For r_max <= 25 the tables sit in constant memory (warp-uniform
//            reads through the constant cache), beyond that in global memory.
//   counts = each lane owns a column of 32-bit words in shared memory
//            (word v at +128 v bytes, so the 32 lanes of a warp always hit
//            32 different banks), one word per stored value v = 0..B;
//            v = 0 (not counted) is a dummy word, so the update has no
//            branch: it is one shared-memory reduction (red.shared.add).
//   FP64   = after each shell one pass over the lane's counters computes the
//            bin-order entropy sum and the exact integer D of W against the
//            previous scale's counts (a second column of the same layout,
//            refreshed in the same pass).  W and Y are evaluated only at
//            entropy peaks.
#include <type_traits>

#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kTmaPollLimit = 1 << 20;
constexpr int kConstRmax = 25;            // largest r_max whose tables fit
constexpr int kConstC8 = 7500;            // three-nonzero entries with rho <= 25: 7442
constexpr int kConstRest = 5800;          // plane/axis entries with rho <= 25: 5731

// Offset tables of radius classes 0..kConstRmax (layout as OffsetTables).
__constant__ uint32_t c_c8[kConstC8];
__constant__ uint32_t c_rest[kConstRest];
__constant__ int c_c8_start[kConstRmax + 2];
__constant__ int c_rest_start[kConstRmax + 2];

struct DenseArgs {
    VolDesc vol;
    OffsetTables ot;             // global copy (all classes <= 32)
    const double *T;
    const double *L;
    int r_min, r_max, S, w_norm;
    int ty, tz;
    int z0, z1;                  // centres with z0 <= z < z1 (a slab of the volume)
    int bx, by, padx;            // brick row length and rows per plane (path 0)
    uint32_t brick_bytes;
    uint32_t cnt_off, mbar_off;
    DenseOut out;
    int *status;
};

template <bool CTAB>
struct Tab {
    OffsetTables g;
    __device__ __forceinline__ uint32_t c8(int k) const {
        if constexpr (CTAB) return c_c8[k]; else return __ldg(g.c8 + k);
    }
    __device__ __forceinline__ uint32_t rest(int k) const {
        if constexpr (CTAB) return c_rest[k]; else return __ldg(g.rest + k);
    }
    __device__ __forceinline__ int c8_start(int rho) const {
        if constexpr (CTAB) return c_c8_start[rho]; else return __ldg(g.c8_start + rho);
    }
    __device__ __forceinline__ int rest_start(int rho) const {
        if constexpr (CTAB) return c_rest_start[rho]; else return __ldg(g.rest_start + rho);
    }
};

template <int PATH>
struct Src;
template <>
struct Src<0> {              // brick in shared memory, byte offsets from smem
    const uint8_t *smem;
    __device__ __forceinline__ uint32_t at(int base, int off) const { return smem[base + off]; }
};
template <>
struct Src<1> {              // halo-padded volume in global memory
    const uint8_t *vol;
    __device__ __forceinline__ uint32_t at(int64_t base, int off) const {
        return __ldg(vol + (base + off));
    }
};

template <int B, bool WIDE, int PATH>
__global__ void __launch_bounds__(512) k_dense(const DenseArgs a,
                                               const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ int s_ok;
    constexpr bool CTAB = !WIDE;                 // r_max <= 25: table in constant memory
    constexpr int NW = B + 1;                    // counter words per lane
    constexpr int NPREV = NW;                    // previous-scale words
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tx0 = blockIdx.x * 32, ty0 = blockIdx.y * a.ty, tz0 = a.z0 + blockIdx.z * a.tz;
    const int R = a.r_max;

    Src<PATH> src;
    int pz, py;
    if constexpr (PATH == 0) {
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
        src.smem = smem;
        pz = a.bx * a.by;
        py = a.bx;
    } else {
        src.vol = a.vol.base;
        pz = (int)a.vol.plane;
        py = (int)a.vol.pitch;
    }
    const Tab<CTAB> tab{a.ot};

    // Lane's counter column: word v at +128 v; previous-scale words (WIDE)
    // at +128 (NW + v).
    const uint32_t cnt_lane = smem_u32(smem + a.cnt_off) + (warp * (NW + NPREV) * 32 + lane) * 4;
    const int nrows = a.ty * a.tz;

    for (int row = warp; row < nrows; row += nwarps) {
        const int cy = ty0 + row % a.ty, cz = tz0 + row / a.ty;
        if (cy >= a.vol.ny || cz >= a.z1) continue;              // warp-uniform
        const int cx = tx0 + lane;
        const bool live = cx < a.vol.nx;
        // lane's centre as an offset into the source
        using Base = typename std::conditional<PATH == 0, int, int64_t>::type;
        Base c0;
        if constexpr (PATH == 0)
            c0 = (cz - tz0 + R) * pz + (cy - ty0 + R) * py + (a.padx + lane);
        else
            c0 = (int64_t)cz * a.vol.plane + (int64_t)cy * a.vol.pitch + (live ? cx : a.vol.nx - 1);

#pragma unroll 4
        for (int w = 0; w < NW + NPREV; ++w) st_shared_u32(cnt_lane + (w << 7), 0u);

        double hm1 = 0.0, hm2 = 0.0;      // H at scale index i-1, i-2
        uint32_t nm1 = 0, nm2 = 0;        // N at i-1, i-2
        uint64_t dm1 = 0;                 // D at i-1
        double yb = 0.0;
        int sb = 0;
        const int64_t oidx = ((int64_t)cz * a.vol.ny + cy) * a.vol.nx + cx;

        for (int i = 0; i < a.S; ++i) {
            const int r = a.r_min + i;
            for (int rho = (i == 0 ? 0 : r); rho <= r; ++rho) {
                const int k0 = tab.c8_start(rho), k1 = tab.c8_start(rho + 1);
                const int k2 = tab.rest_start(rho), k3 = tab.rest_start(rho + 1);
                // three nonzero components: 8 sign mirrors
                uint32_t e = k0 < k1 ? tab.c8(k0) : 0u;
                for (int k = k0; k < k1; ++k) {
                    const uint32_t en = k + 1 < k1 ? tab.c8(k + 1) : 0u;   // prefetch
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    const int o0 = Z + Y, o1 = Z - Y, o2 = Y - Z, o3 = -Z - Y;
                    // (the top byte of e is the radius class, unused here)
                    const uint32_t v0 = src.at(c0, o0 + X), v1 = src.at(c0, o0 - X);
                    const uint32_t v2 = src.at(c0, o1 + X), v3 = src.at(c0, o1 - X);
                    const uint32_t v4 = src.at(c0, o2 + X), v5 = src.at(c0, o2 - X);
                    const uint32_t v6 = src.at(c0, o3 + X), v7 = src.at(c0, o3 - X);
                    red_add_shared(cnt_lane + (v0 << 7), 1u);
                    red_add_shared(cnt_lane + (v1 << 7), 1u);
                    red_add_shared(cnt_lane + (v2 << 7), 1u);
                    red_add_shared(cnt_lane + (v3 << 7), 1u);
                    red_add_shared(cnt_lane + (v4 << 7), 1u);
                    red_add_shared(cnt_lane + (v5 << 7), 1u);
                    red_add_shared(cnt_lane + (v6 << 7), 1u);
                    red_add_shared(cnt_lane + (v7 << 7), 1u);
                    e = en;
                }
                // offsets on a coordinate plane or axis, one entry each
                for (int k = k2; k < k3; ++k) {
                    const uint32_t f = tab.rest(k);
                    const int off = ((int)((f >> 16) & 0xffu) - 64) * pz +
                                    ((int)((f >> 8) & 0xffu) - 64) * py + ((int)(f & 0xffu) - 64);
                    red_add_shared(cnt_lane + (src.at(c0, off) << 7), 1u);
                }
            }

            // ---- exact per-scale quantities from the lane's counters
            const uint32_t zero_cnt = ld_shared_u32(cnt_lane);
            const uint32_t N = (uint32_t)__ldg(a.ot.ball_size + r) - zero_cnt;
            double ssum = 0.0;
            int occ = 0;
            uint64_t D = 0;
#pragma unroll
            for (int v = 1; v <= B; ++v) {
                const uint32_t c = ld_shared_u32(cnt_lane + (v << 7));
                const uint32_t p = ld_shared_u32(cnt_lane + ((NW + v) << 7));
                st_shared_u32(cnt_lane + ((NW + v) << 7), c);
                occ += c > 0u;
                if (c > 1u) ssum = __dadd_rn(ssum, __ldg(a.T + c));
                const int64_t d = (int64_t)c * nm1 - (int64_t)p * N;
                D += (uint64_t)(d < 0 ? -d : d);
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

int template_bins(int B) {
    return B <= 2 ? 2 : B <= 4 ? 4 : B <= 8 ? 8 : B <= 16 ? 16 : B <= 32 ? 32 : 64;
}

bool is_wide(int r_max) { return r_max > kConstRmax; }

struct Geometry {
    int padx, bx, by, bz;
    size_t brick, cnt_off, cnt_bytes, mbar_off, total;
};

Geometry geometry(const DenseConfig &c, int B_, int r_max) {
    Geometry g{};
    const int B = template_bins(B_);
    const int words = (B + 1) * 2;          // counts + previous-scale counts
    g.padx = (r_max + 15) / 16 * 16;
    g.bx = (g.padx + 32 + r_max + 15) / 16 * 16;
    g.by = c.ty + 2 * r_max;
    g.bz = c.tz + 2 * r_max;
    g.brick = c.path == 0 ? (size_t)g.bx * g.by * g.bz : 0;
    g.cnt_off = (g.brick + 127) / 128 * 128;
    g.cnt_bytes = (size_t)c.warps * words * 32 * 4;
    g.mbar_off = g.cnt_off + g.cnt_bytes;
    g.total = g.mbar_off + 16;
    return g;
}

template <int B, bool WIDE, int PATH>
cudaError_t launch_t(const LaunchCtx &lc, const DenseArgs &a, const CUtensorMap *tmap,
                     const DenseConfig &cfg, size_t smem) {
    auto kern = k_dense<B, WIDE, PATH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.vol.nx + 31) / 32, (a.vol.ny + a.ty - 1) / a.ty, (a.z1 - a.z0 + a.tz - 1) / a.tz);
    CUtensorMap dummy{};
    kern<<<grid, cfg.warps * 32, smem, lc.stream>>>(a, tmap ? *tmap : dummy);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_b(const LaunchCtx &lc, const DenseArgs &a, const CUtensorMap *tmap,
                     const DenseConfig &cfg, size_t smem) {
    const bool wide = is_wide(a.r_max);
    if (cfg.path == 0)
        return wide ? launch_t<B, true, 0>(lc, a, tmap, cfg, smem)
                    : launch_t<B, false, 0>(lc, a, tmap, cfg, smem);
    return wide ? launch_t<B, true, 1>(lc, a, tmap, cfg, smem)
                : launch_t<B, false, 1>(lc, a, tmap, cfg, smem);
}

}  // namespace

// Exercises the bounded-wait path: thread 0 waits on an mbarrier that no
// copy will ever complete, gives up after `polls` polls, records the
// timeout in the status word and returns, exactly as k_dense does when its
// brick does not arrive.
__global__ void k_wait_selftest(int *status, int polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t mbar = smem_u32(&bar);
        mbar_init(mbar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(mbar, 0, polls)) atomicOr(status, kStatusTmaTimeout);
    }
}

cudaError_t launch_wait_selftest(const LaunchCtx &lc, int polls) {
    k_wait_selftest<<<1, 32, 0, lc.stream>>>(lc.d_status, polls);
    return cudaGetLastError();
}

int ball_size_host(int r) {
    int n = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dx * dx + dy * dy + dz * dz <= r * r) ++n;
    return n;
}

cudaError_t dense_upload_constant_table(const uint32_t *c8, const int *c8_start,
                                        const uint32_t *rest, const int *rest_start) {
    const int n8 = c8_start[kConstRmax + 1], nr = rest_start[kConstRmax + 1];
    if (n8 > kConstC8 || nr > kConstRest) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_c8, c8, n8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rest, rest, nr * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_c8_start, c8_start, (kConstRmax + 2) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_rest_start, rest_start, (kConstRmax + 2) * sizeof(int));
    return e;
}

int dense_const_rmax() { return kConstRmax; }

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
                         const OffsetTables &ot, const double *T, const double *L, int r_min,
                         int r_max, int w_norm, const DenseConfig &cfg, const DenseOut &out,
                         int z0, int z1) {
    const Geometry g = geometry(cfg, v.B, r_max);
    DenseArgs a{};
    a.vol = v;
    a.ot = ot;
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
    const CUtensorMap *tm = cfg.path == 0 ? tmap : nullptr;
    // Counter columns are sized for the next supported bin count; the extra
    // stored values never occur, so their counters stay 0 and add nothing
    // to the entropy sum or to D.
    switch (template_bins(v.B)) {
        case 2: return launch_b<2>(lc, a, tm, cfg, g.total);
        case 4: return launch_b<4>(lc, a, tm, cfg, g.total);
        case 8: return launch_b<8>(lc, a, tm, cfg, g.total);
        case 16: return launch_b<16>(lc, a, tm, cfg, g.total);
        case 32: return launch_b<32>(lc, a, tm, cfg, g.total);
        case 64: return launch_b<64>(lc, a, tm, cfg, g.total);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ks
