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
//   CPL    = centres per lane on PATH 1 (launch path 2 = two): with two, a
//            warp covers 64 centres of a row (lane l: x0 + l and x0 + l + 32)
//            so one table decode and one address serve two loads that differ
//            by an immediate.  Centres past nx are evaluated (their reads stay
//            inside the zeroed halo and the allocation's slack) but not
//            written; a tile whose second centres all lie past nx walks one
//            centre per lane.
//   PATH 3 = (launch path 3, r_max <= 25) four adjacent centres per lane,
//            128 per warp, whose four bins per offset come from two aligned
//            32-bit loads and a funnel shift (k_dense4).
//   PATH 4 = (launch path 4, 16 or 32 bins, r_max <= 25) PATH 3 with the
//            previous-scale counts in tensor memory (k_dense4<B, true>).
//   launch path 5 = one histogram per scale slid along z (k_dense_slide).
//   launch paths 6 to 8 (r_max > 25; 16, 32 or 64 template bins) = PATH 1
//            with the previous-scale counts as 32-bit words in tensor memory:
//            one centre per lane (6), two (7), or two sharing each counter
//            word as 16-bit halves counted modulo 2^16 and recovered exactly
//            from the previous counts (8, WRAP).
//   scale  = built incrementally: shell r (offsets o with ceil|o| == r, and
//            everything up to r_min for the first scale) is added to the
//            counts of r-1.
//   offsets= per radius class rho, the offsets with three nonzero
//            components, stored once per set of 8 sign mirrors as (|dx|,
//            |dy|, |dz|) and expanded with warp-uniform arithmetic, then every
//            offset on a coordinate plane or axis, stored with its signs
//            (the four-centre kernel takes the plane offsets as sets of 4
//            sign mirrors, the same way).
//            For r_max <= 25 the tables sit in constant memory (warp-uniform
//            reads through the constant cache), beyond that in global memory.
//   counts = each centre owns a column of 32-bit words in shared memory
//            (word v at +128 v bytes, so the 32 lanes of a warp always hit
//            32 different banks), one word per stored value v = 0..B;
//            v = 0 (not counted) is a dummy word, so the update has no
//            branch: it is one shared-memory reduction (red.shared.add).
//            With two centres per lane and r_max <= 25 both centres share
//            the column as 16-bit halves (every count is <= |Ball(25)| =
//            65267), which halves the counter memory and raises occupancy.
//   FP64   = after each shell one pass over the centre's counters computes
//            the bin-order entropy sum and the exact integer D of W against
//            the previous scale's counts (words after the counters, refreshed
//            in the same pass; two 16-bit counts per word when every count
//            fits, |Ball(25)| = 65267).  W and Y are evaluated only at
//            entropy peaks.
#include <type_traits>
#include <vector>

#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kTmaPollLimit = 1 << 20;
constexpr int kConstRmax = 25;            // largest r_max whose tables fit
constexpr int kConstC8 = 7500;            // three-nonzero entries with rho <= 25: 7442
constexpr int kConstRest = 5800;          // plane/axis entries with rho <= 25: 5731
constexpr int kConstC4 = 1400;            // plane entries, one per 4 sign mirrors: 1395
constexpr int kConstC1 = 160;             // axis offsets and the origin with rho <= 25: 151

// Offset tables of radius classes 0..kConstRmax (layout as OffsetTables).
__constant__ uint32_t c_c8[kConstC8];
__constant__ uint32_t c_rest[kConstRest];
__constant__ int c_c8_start[kConstRmax + 2];
__constant__ int c_rest_start[kConstRmax + 2];
// The rest entries again for the four-centre kernel, regrouped by mirrors:
//   c4: offsets with exactly two nonzero components, one entry per set of 4
//       sign mirrors: |dx| | |dy| << 8 | |dz| << 16 | plane << 24, plane 0
//       for dz = 0, 1 for dy = 0, 2 for dx = 0;
//   c1: offsets on an axis and the origin, one entry each, encoded as rest.
// 4 (c4_start[rho+1] - c4_start[rho]) + c1_start[rho+1] - c1_start[rho] =
// rest_start[rho+1] - rest_start[rho].
__constant__ uint32_t c_c4[kConstC4];
__constant__ uint32_t c_c1[kConstC1];
__constant__ int c_c4_start[kConstRmax + 2];
__constant__ int c_c1_start[kConstRmax + 2];

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
    const int32_t *pts;          // listed centres (k_points)
    int64_t npts;
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
    __device__ __forceinline__ uint32_t at(const uint8_t *p, int off) const {
        return __ldg(p + off);
    }
};

// ---- tensor memory (TMEM) as per-thread storage for launch path 4
// A block allocates 128 columns per group of four warps; warp w owns TMEM
// lanes 32 (w & 3) .. 32 (w & 3) + 31 (the lane quarter its position in the
// warpgroup may address) of columns 128 (w >> 2) .. + 127, and thread l of
// the warp owns row 32 (w & 3) + l of them.  The 32x32b shape moves one
// 32-bit word per thread and column.
__device__ __forceinline__ void tm_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(dst_smem), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// The previous-scale words of one centre: NP = 17 (32 bins) or 9 (16 bins)
// consecutive columns from ta.  A load waits for its data inside the same
// asm statement, so no use of the registers can be scheduled before it.
template <int NP>
__device__ __forceinline__ void tm_load_prev(uint32_t ta, uint32_t (&v)[NP]) {
    static_assert(NP == 17 || NP == 9, "TMEM previous words: 16 or 32 bins");
    if constexpr (NP == 17) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%17];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%16}, [%18];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16])
            : "r"(ta), "r"(ta + 16u)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%9];\n\t"
            "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%10];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8])
            : "r"(ta), "r"(ta + 8u)
            : "memory");
    }
}
// Stores complete asynchronously; tm_wait_st before the next load of the
// same columns.
template <int NP>
__device__ __forceinline__ void tm_store_prev(uint32_t ta, const uint32_t (&v)[NP]) {
    static_assert(NP == 17 || NP == 9, "TMEM previous words: 16 or 32 bins");
    if constexpr (NP == 17) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15, %16, %17};\n\t"
            "tcgen05.st.sync.aligned.32x32b.x1.b32 [%1], {%18};"
            ::"r"(ta), "r"(ta + 16u), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]),
              "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]),
              "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16])
            : "memory");
    } else {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
            "tcgen05.st.sync.aligned.32x32b.x1.b32 [%1], {%10};"
            ::"r"(ta), "r"(ta + 8u), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]),
              "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8])
            : "memory");
    }
}
__host__ __device__ constexpr int tm_columns(int warps) { return 128 * ((warps + 3) / 4); }

// Launch path 6 (r_max > 25): the previous-scale counts of a lane's centre,
// bins 1..NW (NW = 16, 32 or 64 words, 32-bit), in NW consecutive columns
// from ta.  As above, a load waits for its data in the same asm statement.
template <int NW>
__device__ __forceinline__ void tm_load_words(uint32_t ta, uint32_t (&v)[NW]);
template <int NW>
__device__ __forceinline__ void tm_store_words(uint32_t ta, const uint32_t (&v)[NW]);
#define KS_R16(o) "=r"(v[o + 0]), "=r"(v[o + 1]), "=r"(v[o + 2]), "=r"(v[o + 3]), "=r"(v[o + 4]), \
    "=r"(v[o + 5]), "=r"(v[o + 6]), "=r"(v[o + 7]), "=r"(v[o + 8]), "=r"(v[o + 9]),           \
    "=r"(v[o + 10]), "=r"(v[o + 11]), "=r"(v[o + 12]), "=r"(v[o + 13]), "=r"(v[o + 14]),      \
    "=r"(v[o + 15])
#define KS_W16(o) "r"(v[o + 0]), "r"(v[o + 1]), "r"(v[o + 2]), "r"(v[o + 3]), "r"(v[o + 4]),   \
    "r"(v[o + 5]), "r"(v[o + 6]), "r"(v[o + 7]), "r"(v[o + 8]), "r"(v[o + 9]), "r"(v[o + 10]),  \
    "r"(v[o + 11]), "r"(v[o + 12]), "r"(v[o + 13]), "r"(v[o + 14]), "r"(v[o + 15])
template <>
__device__ __forceinline__ void tm_load_words<16>(uint32_t ta, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : KS_R16(0)
        : "r"(ta)
        : "memory");
}
template <>
__device__ __forceinline__ void tm_load_words<32>(uint32_t ta, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, "
        "%25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : KS_R16(0), KS_R16(16)
        : "r"(ta), "r"(ta + 16u)
        : "memory");
}
template <>
__device__ __forceinline__ void tm_load_words<64>(uint32_t ta, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, "
        "%25, %26, %27, %28, %29, %30, %31}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, "
        "%41, %42, %43, %44, %45, %46, %47}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48, %49, %50, %51, %52, %53, %54, %55, %56, "
        "%57, %58, %59, %60, %61, %62, %63}, [%67];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : KS_R16(0), KS_R16(16), KS_R16(32), KS_R16(48)
        : "r"(ta), "r"(ta + 16u), "r"(ta + 32u), "r"(ta + 48u)
        : "memory");
}
template <>
__device__ __forceinline__ void tm_store_words<16>(uint32_t ta, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16};"
        ::"r"(ta), KS_W16(0)
        : "memory");
}
template <>
__device__ __forceinline__ void tm_store_words<32>(uint32_t ta, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%1], {%18, %19, %20, %21, %22, %23, %24, %25, "
        "%26, %27, %28, %29, %30, %31, %32, %33};"
        ::"r"(ta), "r"(ta + 16u), KS_W16(0), KS_W16(16)
        : "memory");
}
template <>
__device__ __forceinline__ void tm_store_words<64>(uint32_t ta, const uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15, %16, %17, %18, %19};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%1], {%20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31, %32, %33, %34, %35};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%2], {%36, %37, %38, %39, %40, %41, %42, %43, "
        "%44, %45, %46, %47, %48, %49, %50, %51};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%3], {%52, %53, %54, %55, %56, %57, %58, %59, "
        "%60, %61, %62, %63, %64, %65, %66, %67};"
        ::"r"(ta), "r"(ta + 16u), "r"(ta + 32u), "r"(ta + 48u), KS_W16(0), KS_W16(16), KS_W16(32),
          KS_W16(48)
        : "memory");
}
#undef KS_R16
#undef KS_W16
// TMEM columns a launch path 6 block allocates: NW per group of four warps,
// rounded up to a power of two of at least 32 (tcgen05.alloc's rule).
__host__ __device__ constexpr int tm_columns_wide(int warps, int NW) {
    int c = NW * ((warps + 3) / 4);
    int p = 32;
    while (p < c) p <<= 1;
    return p;
}

// Shared-memory words of one lane.  Counters: one word per stored value
// v = 0..B.  When every count fits in 16 bits (|Ball(r_max)| <= 65535, i.e.
// r_max <= 25) two centres of a lane share each word (centre j in bits
// 16 (j & 1) .. 16 (j & 1) + 15 of pair j >> 1, so an update adds
// 1 << 16 (j & 1)); otherwise each centre has its own 32-bit column.  After
// the counters come the previous scale's counts of each centre: 16-bit
// pairs (values 2w, 2w+1 in word w) when they fit, 32-bit words otherwise.
//
// WRAP (launch path 8, r_max > 25, previous counts in TMEM): the two centres
// of a lane share a word although a count may pass 65 535.  The word is
// x = L + 2^16 H modulo 2^32 (L, H the exact counts of centres 0 and 1 since
// the row start; a low half that wraps carries into the high half), so
// L mod 2^16 = x mod 2^16 and, once L is known, H mod 2^16 = (x - L) >> 16.
// The scale step recovers each exact count from its 16-bit residue and the
// exact previous count: c = p + ((c16 - p) mod 2^16), which holds while no
// bin gains 65 536 or more between two recoveries.  A shell adds at most
// 12 578 voxels (r = 32); the first scale is recovered once at rho =
// kWrapFold (|Ball(25)| = 65 267) when r_min is larger, after which shells
// 26..31 add at most 59 220.
template <int B, bool WIDE, int CPL, bool TM = false, bool WRAP = false>
struct Words {
    static constexpr bool kPack = CPL >= 2 && (!WIDE || WRAP);
    static constexpr int kNW = B + 1;                          // counter words per column
    static constexpr int kNP = WIDE ? B + 1 : (B + 2) / 2;     // previous words per centre
    static constexpr int kCols = kPack ? CPL / 2 : CPL;        // counter columns
    // with TM the previous counts live in tensor memory, not here
    static constexpr int kPerLane = kCols * kNW + (TM ? 0 : CPL * kNP);
    // word index of centre j's counter of value v / previous word w
    __host__ __device__ static constexpr int cnt(int j, int v) {
        return (kPack ? (j >> 1) : j) * kNW + v;
    }
    __host__ __device__ static constexpr int prev(int j, int w) {
        return kCols * kNW + j * kNP + w;
    }
    __host__ __device__ static constexpr uint32_t inc(int j) {
        return kPack ? 1u << (16 * (j & 1)) : 1u;
    }
};

// Running state of one centre over the scales: H at scale index i-1 and
// i-2, N at i-1 and i-2, D at i-1, and the best Y and its scale so far;
// with WRAP also the exact count of value 0 at the last recovery.
struct ScaleState {
    double hm1, hm2, yb;
    uint32_t nm1, nm2;
    uint64_t dm1;
    int sb;
    uint32_t c0;
};

constexpr int kWrapFold = 25;             // |Ball(25)| = 65267 < 2^16
static_assert(kRmax <= 32, "WRAP recovery bounds assume r <= 32");

// WRAP: the exact count of value v from its 16-bit half c16 and the exact
// count p at the last recovery.
__device__ __forceinline__ uint32_t wrap_count(uint32_t c16, uint32_t p) {
    return p + ((c16 - p) & 0xffffu);
}

// After the shell of scale r (index i): the centre's exact N, the bin-order
// entropy sum, D against the previous scale's counts (refreshed in the same
// pass), H, the peak test at scale r - 1 and the optional H/W outputs.
// With TM the previous counts are the NP words at TMEM address tprev.
// WRAP: tlow and low_c0 are the low-half centre's exact counts (its TMEM
// columns, already refreshed for this scale, and its value-0 count), used
// by the high-half centre (j odd).
template <int B, bool WIDE, int CPL, bool TM = false, bool WRAP = false>
__device__ __forceinline__ void scale_step(const DenseArgs &a, uint32_t cnt_lane, int j, int i,
                                           int r, ScaleState &st, int64_t oidx, bool live,
                                           uint32_t tprev = 0u, uint32_t tlow = 0u,
                                           uint32_t low_c0 = 0u) {
    using Wd = Words<B, WIDE, CPL, TM, WRAP>;
    constexpr int NP = Wd::kNP;
    auto word = [&](int w) { return cnt_lane + ((uint32_t)w << 7); };
    auto count = [&](int v) -> uint32_t {
        const uint32_t x = ld_shared_u32(word(Wd::cnt(j, v)));
        return Wd::kPack ? (x >> (16 * (j & 1))) & 0xffffu : x;
    };
    uint32_t c0;
    if constexpr (WRAP) {
        const uint32_t x = ld_shared_u32(word(Wd::cnt(j, 0)));
        c0 = wrap_count((j & 1) ? (x - low_c0) >> 16 : x & 0xffffu, st.c0);
        st.c0 = c0;
    } else {
        c0 = count(0);
    }
    const uint32_t N = (uint32_t)__ldg(a.ot.ball_size + r) - c0;
    double ssum = 0.0;
    int occ = 0;
    uint64_t D = 0;
    auto term = [&](uint32_t c, uint32_t p) {
        occ += c > 0u;
        if (c > 1u) ssum = __dadd_rn(ssum, __ldg(a.T + c));
        const int64_t d = (int64_t)c * st.nm1 - (int64_t)p * N;
        D += (uint64_t)(d < 0 ? -d : d);
    };
    if constexpr (WIDE && TM && WRAP) {
        // launch path 8: 16 bins at a time (the high half also needs the
        // low-half centre's exact counts, whose stores must have landed)
        if (j & 1) tm_wait_st();
#pragma unroll
        for (int k0 = 0; k0 < B; k0 += 16) {
            uint32_t pv[16], lv[16];
            __syncwarp();                  // tcgen05 loads and stores are warp-wide
            tm_load_words<16>(tprev + (uint32_t)k0, pv);
            if (j & 1) tm_load_words<16>(tlow + (uint32_t)k0, lv);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const uint32_t x = ld_shared_u32(word(Wd::cnt(j, k0 + t + 1)));
                const uint32_t c = wrap_count((j & 1) ? (x - lv[t]) >> 16 : x & 0xffffu, pv[t]);
                term(c, pv[t]);
                pv[t] = c;
            }
            __syncwarp();
            tm_store_words<16>(tprev + (uint32_t)k0, pv);
        }
    } else if constexpr (WIDE && TM) {
        // launch paths 6 and 7: the previous counts of bins 1..B in TMEM
        uint32_t pv[B];
        __syncwarp();                      // tcgen05 loads and stores are warp-wide
        tm_load_words<B>(tprev, pv);
#pragma unroll
        for (int vv = 1; vv <= B; ++vv) {
            const uint32_t c = count(vv);
            term(c, pv[vv - 1]);
            pv[vv - 1] = c;
        }
        __syncwarp();
        tm_store_words<B>(tprev, pv);
    } else if constexpr (WIDE) {
#pragma unroll
        for (int vv = 1; vv <= B; ++vv) {
            const uint32_t c = count(vv);
            const uint32_t p = ld_shared_u32(word(Wd::prev(j, vv)));
            st_shared_u32(word(Wd::prev(j, vv)), c);
            term(c, p);
        }
    } else {
        // previous counts as 16-bit pairs: word w holds values 2w, 2w+1
        uint32_t pv[NP];
        if constexpr (TM) {
            __syncwarp();                  // tcgen05 loads and stores are warp-wide
            tm_load_prev<NP>(tprev, pv);
        }
#pragma unroll
        for (int w = 0; w < NP; ++w) {
            const uint32_t pw = TM ? pv[w] : ld_shared_u32(word(Wd::prev(j, w)));
            uint32_t c_lo = 0, c_hi = 0;
            if (2 * w >= 1 && 2 * w <= B) {
                c_lo = count(2 * w);
                term(c_lo, pw & 0xffffu);
            }
            if (2 * w + 1 <= B) {
                c_hi = count(2 * w + 1);
                term(c_hi, pw >> 16);
            }
            if constexpr (TM)
                pv[w] = c_lo | (c_hi << 16);
            else
                st_shared_u32(word(Wd::prev(j, w)), c_lo | (c_hi << 16));
        }
        if constexpr (TM) {
            __syncwarp();
            tm_store_prev<NP>(tprev, pv);
        }
    }
    const double H = entropy_from_sum(ssum, N, occ, a.L);

    if (i >= 2 && st.hm2 < st.hm1 && st.hm1 >= H) {   // peak at scale i-1
        const double W = kb_weight(st.dm1, st.nm1, st.nm2, r - 1, a.w_norm);
        const double y = __dmul_rn(st.hm1, W);
        if (st.sb == 0 || y > st.yb) {
            st.yb = y;
            st.sb = r - 1;
        }
    }
    if (live && (a.out.H || a.out.W)) {
        if (a.out.H) a.out.H[oidx * a.S + i] = H;
        if (a.out.W) a.out.W[oidx * a.S + i] = i == 0 ? 0.0 : kb_weight(D, N, st.nm1, r, a.w_norm);
    }
    st.hm2 = st.hm1;
    st.hm1 = H;
    st.nm2 = st.nm1;
    st.nm1 = N;
    st.dm1 = D;
}

// WRAP: the recovery of scale_step without a scale (the first scale's
// counts at rho = kWrapFold when r_min is larger): the exact counts become
// the reference of the next recovery.  As in scale_step, the high-half
// centre (j odd) uses the low-half centre's freshly recovered counts at
// tlow and low_c0.
template <int B, int CPL>
__device__ __forceinline__ void wrap_fold(uint32_t cnt_lane, int j, ScaleState &st,
                                          uint32_t tprev, uint32_t tlow, uint32_t low_c0) {
    using Wd = Words<B, true, CPL, true, true>;
    auto word = [&](int v) { return ld_shared_u32(cnt_lane + ((uint32_t)Wd::cnt(j, v) << 7)); };
    const uint32_t x0 = word(0);
    st.c0 = wrap_count((j & 1) ? (x0 - low_c0) >> 16 : x0 & 0xffffu, st.c0);
    if (j & 1) tm_wait_st();
#pragma unroll
    for (int k0 = 0; k0 < B; k0 += 16) {
        uint32_t pv[16], lv[16];
        __syncwarp();
        tm_load_words<16>(tprev + (uint32_t)k0, pv);
        if (j & 1) tm_load_words<16>(tlow + (uint32_t)k0, lv);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const uint32_t x = word(k0 + t + 1);
            pv[t] = wrap_count((j & 1) ? (x - lv[t]) >> 16 : x & 0xffffu, pv[t]);
        }
        __syncwarp();
        tm_store_words<16>(tprev + (uint32_t)k0, pv);
    }
}

// TM (launch paths 6 and 7: PATH 1 with one or two centres per lane, r_max >
// 25, 16, 32 or 64 bins): each centre's previous-scale counts in B TMEM
// columns instead of shared memory, so a warp needs half the shared memory.
// A block of 4, 8 or 16 warps allocates tm_columns_wide(warps, CPL B)
// columns; warp w owns the lane quarter w & 3 of columns CPL B (w >> 2) ..
// + CPL B - 1, centre j the B of them from CPL B (w >> 2) + j B.  WRAP
// (launch path 8): path 7 with the two centres' counters in 16-bit halves of
// one column (Words), so a warp needs half the shared memory again.
template <int B, bool WIDE, int PATH, int CPL, bool TM = false, bool WRAP = false>
__global__ void __launch_bounds__(CPL == 1 ? 512 : 256)
    k_dense(const DenseArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ int s_ok;
    __shared__ uint32_t s_tmem;
    static_assert(!TM || (WIDE && PATH == 1 && (CPL == 1 || CPL == 2) &&
                          (B == 16 || B == 32 || B == 64)),
                  "launch paths 6 and 7: path 1, one or two centres per lane, 16, 32 or 64 "
                  "bins, r_max > 25");
    static_assert(!WRAP || (TM && CPL == 2), "launch path 8: path 7 with 16-bit counters");
    using Wd = Words<B, WIDE, CPL, TM, WRAP>;
    constexpr bool CTAB = !WIDE;                 // r_max <= 25: table in constant memory
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tx0 = blockIdx.x * 32 * CPL, ty0 = blockIdx.y * a.ty, tz0 = a.z0 + blockIdx.z * a.tz;
    const int R = a.r_max;
    uint32_t tm_base = 0u;
    if constexpr (TM) {
        if (warp == 0) tm_alloc(smem_u32(&s_tmem), (uint32_t)tm_columns_wide(nwarps, CPL * B));
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        tm_base = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(CPL * B * (warp >> 2));
    }

    Src<PATH> src;
    int pz, py;
    if constexpr (PATH == 0) {
        const uint32_t mbar = smem_u32(smem + a.mbar_off);
        // the TMA destination must be 128-byte aligned, the mbarrier 8-byte
        // aligned and the tensor map 64-byte aligned: checked once per block,
        // reported instead of issuing a copy that would fault
        if (((smem_u32(smem) & 127u) | (mbar & 7u) |
             (uint32_t)(reinterpret_cast<uintptr_t>(&tmap) & 63u)) != 0u) {
            if (threadIdx.x == 0) atomicOr(a.status, kStatusMisaligned);
            return;
        }
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
        pz = (int)a.vol.plane;
        py = (int)a.vol.pitch;
    }
    const Tab<CTAB> tab{a.ot};

    // Lane's words: word w at cnt_lane + 128 w (the 32 lanes of a warp sit
    // in 32 different banks).
    const uint32_t cnt_lane = smem_u32(smem + a.cnt_off) + (warp * Wd::kPerLane * 32 + lane) * 4;
    auto word = [&](int w) { return cnt_lane + ((uint32_t)w << 7); };
    const int nrows = a.ty * a.tz;

    // One row of the tile with CE centres per lane (CE = CPL, or 1 in a
    // tile whose second centres x + 32 all lie past nx: then they are not
    // computed at all).
    auto sweep_row = [&](int row, auto ce) {
        constexpr int CE = decltype(ce)::value;
        const int cy = ty0 + row % a.ty, cz = tz0 + row / a.ty;
        // Lane centres cx + 32 j.  The source address of centre j is the
        // centre-0 address plus 32 j (an immediate); centres past nx are
        // computed but not written.
        const int cx = tx0 + lane;
        using Base = typename std::conditional<PATH == 0, int, const uint8_t *>::type;
        Base c0;
        if constexpr (PATH == 0)
            c0 = (cz - tz0 + R) * pz + (cy - ty0 + R) * py + (a.padx + lane);
        else
            c0 = a.vol.base + (int64_t)cz * a.vol.plane + (int64_t)cy * a.vol.pitch +
                 (CE == 1 && cx >= a.vol.nx ? a.vol.nx - 1 : cx);

#pragma unroll 4
        for (int w = 0; w < Wd::kPerLane; ++w) st_shared_u32(word(w), 0u);
        if constexpr (TM) {
            uint32_t z[B];
#pragma unroll
            for (int w = 0; w < B; ++w) z[w] = 0u;
            __syncwarp();
            tm_wait_st();                  // the previous row's last stores
#pragma unroll
            for (int j = 0; j < CE; ++j) tm_store_words<B>(tm_base + (uint32_t)(j * B), z);
        }

        ScaleState st[CE];
#pragma unroll
        for (int j = 0; j < CE; ++j) st[j] = ScaleState{0.0, 0.0, 0.0, 0u, 0u, 0ull, 0};
        const int64_t orow = ((int64_t)cz * a.vol.ny + cy) * a.vol.nx;

        for (int i = 0; i < a.S; ++i) {
            const int r = a.r_min + i;
            for (int rho = (i == 0 ? 0 : r); rho <= r; ++rho) {
                const int k0 = tab.c8_start(rho), k1 = tab.c8_start(rho + 1);
                const int k2 = tab.rest_start(rho), k3 = tab.rest_start(rho + 1);
                // three nonzero components: 8 sign mirrors
                // (an entry after the last one of a class always exists, in
                // the constant and in the global table, so the prefetch of
                // entry k + 1 needs no guard)
                uint32_t e = tab.c8(k0);
                // four entries unrolled, their loads in flight together (the
                // 32-bit-counter sweep of r <= 32: 84.6 -> 82.6 ms on a 64 x 128 x
                // 128 MR crop)
#pragma unroll 4
                for (int k = k0; k < k1; ++k) {
                    const uint32_t en = tab.c8(k + 1);
                    // (the top byte of e is the radius class, unused here)
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    const int o[8] = {Z + Y + X, Z + Y - X, Z - Y + X, Z - Y - X,
                                      Y - Z + X, Y - Z - X, -Z - Y + X, -Z - Y - X};
                    uint32_t v[8][CE];
#pragma unroll
                    for (int m = 0; m < 8; ++m)
#pragma unroll
                        for (int j = 0; j < CE; ++j) v[m][j] = src.at(c0, o[m] + 32 * j);
#pragma unroll
                    for (int m = 0; m < 8; ++m)
#pragma unroll
                        for (int j = 0; j < CE; ++j)
                            red_add_shared(word(Wd::cnt(j, v[m][j])), Wd::inc(j));
                    e = en;
                }
                // offsets on a coordinate plane or axis, one entry each
#pragma unroll 2
                for (int k = k2; k < k3; ++k) {
                    const uint32_t f = tab.rest(k);
                    const int off = ((int)((f >> 16) & 0xffu) - 64) * pz +
                                    ((int)((f >> 8) & 0xffu) - 64) * py + ((int)(f & 0xffu) - 64);
                    uint32_t v[CE];
#pragma unroll
                    for (int j = 0; j < CE; ++j) v[j] = src.at(c0, off + 32 * j);
#pragma unroll
                    for (int j = 0; j < CE; ++j) red_add_shared(word(Wd::cnt(j, v[j])), Wd::inc(j));
                }
                if constexpr (WRAP) {
                    if (i == 0 && rho == kWrapFold && r > kWrapFold) {
                        __syncwarp();
                        tm_wait_st();      // the row start's stores
#pragma unroll
                        for (int j = 0; j < CE; ++j)
                            wrap_fold<B, CPL>(cnt_lane, j, st[j], tm_base + (uint32_t)(j * B),
                                              tm_base + (uint32_t)((j ^ 1) * B),
                                              st[(j ^ 1) & (CE - 1)].c0);
                    }
                }
            }
            // ---- exact per-scale quantities from each centre's counters
            if constexpr (TM) {
                __syncwarp();
                tm_wait_st();              // the previous scale's stores
            }
#pragma unroll
            for (int j = 0; j < CE; ++j)
                scale_step<B, WIDE, CPL, TM, WRAP>(a, cnt_lane, j, i, r, st[j], orow + cx + 32 * j,
                                                   cx + 32 * j < a.vol.nx, tm_base + (uint32_t)(j * B),
                                                   tm_base + (uint32_t)((j ^ 1) * B),
                                                   st[(j ^ 1) & (CE - 1)].c0);
        }
#pragma unroll
        for (int j = 0; j < CE; ++j) {
            const int cxj = cx + 32 * j;
            if (cxj < a.vol.nx) {
                a.out.Y[orow + cxj] = st[j].yb;
                a.out.s[orow + cxj] = (uint8_t)st[j].sb;
            }
        }
    };
    // second centres past nx in the whole tile: one centre per lane
    const bool single = CPL == 2 && tx0 + 32 >= a.vol.nx;
    for (int row = warp; row < nrows; row += nwarps) {
        if (ty0 + row % a.ty >= a.vol.ny || tz0 + row / a.ty >= a.z1) continue;   // warp-uniform
        if (single)
            sweep_row(row, std::integral_constant<int, 1>{});
        else
            sweep_row(row, std::integral_constant<int, CPL>{});
    }
    if constexpr (TM) {
        tm_wait_st();
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (warp == 0) tm_dealloc(s_tmem, (uint32_t)tm_columns_wide(nwarps, CPL * B));
    }
}

// Launch path 3 (r_max <= 25): lane l of a warp takes the four adjacent
// centres x0 + 4l .. x0 + 4l + 3 of a row, so a warp covers 128 centres.
// For an offset o the four bins are the bytes x0 + 4l + o .. + 3: two
// aligned 32-bit loads (the row start is 16-byte aligned, so the
// misalignment s = o & 3 is the same for every lane) and a funnel shift
// give all four, and one warp-wide load fetches 128 consecutive bytes
// instead of 32.  The centres' counters are packed in pairs.  Reads reach
// from 3 bytes before x0 + o to 7 bytes after x0 + 127 + o: for |o| <= r_max
// that stays inside the zeroed halo, the neighbouring row or the
// allocation's 256 bytes of slack.
//
// Launch path 4 (TM, 16 or 32 bins): the same kernel with each centre's
// previous-scale counts in tensor memory (32 columns per centre, rows as
// described at tm_alloc) instead of shared memory.  That halves the shared
// memory per lane (66 instead of 134 words for 32 bins), so 16 warps fit on
// an SM instead of 12; the host keeps the blocks per SM within the 512
// TMEM columns, so the allocation never waits.
//
// W (launch path 9, r_max > 25, 16, 32 or 64 bins): the same walk with the
// counters of centres (0, 1) and (2, 3) in 16-bit halves counted modulo 2^16
// (WRAP, as launch path 8) and each centre's B previous counts as 32-bit
// words in TMEM: warp w owns the lane quarter w & 3 of columns 4 B (w >> 2)
// .. + 4 B - 1, centre j the B of them from 4 B (w >> 2) + j B.  The tables
// come from global memory: the three-nonzero entries as above, the plane and
// axis offsets one entry each.
template <int B, bool TM, bool W = false>
__global__ void __launch_bounds__(256, TM ? 2 : 1) k_dense4(const DenseArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t s_tmem;
    constexpr int CPL = 4;
    static_assert(!W || (TM && (B == 16 || B == 32 || B == 64)),
                  "launch path 9: TMEM previous counts, 16, 32 or 64 bins");
    using Wd = Words<B, W, CPL, TM, W>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t tm_base = 0u;
    constexpr int kCols4 = W ? 4 * B : 128;     // TMEM columns of a warp's lane quarter
    const uint32_t tm_cols =
        (uint32_t)(W ? tm_columns_wide(nwarps, 4 * B) : tm_columns(nwarps));
    if constexpr (TM) {
        if (warp == 0) tm_alloc(smem_u32(&s_tmem), tm_cols);
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        tm_base = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kCols4 * (warp >> 2));
    }
    const int tx0 = blockIdx.x * 128, ty0 = blockIdx.y * a.ty, tz0 = a.z0 + blockIdx.z * a.tz;
    const int pz = (int)a.vol.plane, py = (int)a.vol.pitch;
    const Tab<!W> tab{a.ot};
    const uint32_t cnt_lane = smem_u32(smem + a.cnt_off) + (warp * Wd::kPerLane * 32 + lane) * 4;
    auto word = [&](int w) { return cnt_lane + ((uint32_t)w << 7); };
    // the four bins of offset o, centre j in byte j
    auto bins4 = [](const uint8_t *p, int o) -> uint32_t {
        const int s = o & 3;
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p + (o - s));
        return __funnelshift_r(__ldg(q), __ldg(q + 1), 8 * s);
    };
    auto add4 = [&](uint32_t b4) {
#pragma unroll
        for (int j = 0; j < CPL; ++j)       // byte j of b4, zero-extended
            red_add_shared(word(Wd::cnt(j, __byte_perm(b4, 0u, 0x4440u + j))), Wd::inc(j));
    };
    const int nrows = a.ty * a.tz;

    for (int row = warp; row < nrows; row += nwarps) {
        const int cy = ty0 + row % a.ty, cz = tz0 + row / a.ty;
        if (cy >= a.vol.ny || cz >= a.z1) continue;              // warp-uniform
        const int cx = tx0 + 4 * lane;                           // centres cx .. cx + 3
        const uint8_t *c0 = a.vol.base + (int64_t)cz * a.vol.plane + (int64_t)cy * a.vol.pitch + cx;

#pragma unroll 4
        for (int w = 0; w < Wd::kPerLane; ++w) st_shared_u32(word(w), 0u);
        if constexpr (W) {
            uint32_t z[B];
#pragma unroll
            for (int w = 0; w < B; ++w) z[w] = 0u;
            __syncwarp();
            tm_wait_st();                  // the previous row's last stores
#pragma unroll
            for (int j = 0; j < CPL; ++j) tm_store_words<B>(tm_base + (uint32_t)(j * B), z);
        } else if constexpr (TM) {
            constexpr int NP = Wd::kNP;
            uint32_t z[NP];
#pragma unroll
            for (int w = 0; w < NP; ++w) z[w] = 0u;
            __syncwarp();
            tm_wait_st();                  // the previous row's last stores
#pragma unroll
            for (int j = 0; j < CPL; ++j) tm_store_prev<NP>(tm_base + 32u * j, z);
        }

        ScaleState st[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) st[j] = ScaleState{0.0, 0.0, 0.0, 0u, 0u, 0ull, 0};
        const int64_t orow = ((int64_t)cz * a.vol.ny + cy) * a.vol.nx;

        for (int i = 0; i < a.S; ++i) {
            const int r = a.r_min + i;
            for (int rho = (i == 0 ? 0 : r); rho <= r; ++rho) {
                const int k0 = tab.c8_start(rho), k1 = tab.c8_start(rho + 1);
                uint32_t e = tab.c8(k0);
                // four entries unrolled: 64 loads of the next entries are issued
                // while earlier ones are counted (7.86 -> 7.55 ms on pet128)
#pragma unroll 4
                for (int k = k0; k < k1; ++k) {
                    const uint32_t en = tab.c8(k + 1);
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    // pitch and plane are multiples of 16, so the
                    // misalignment of a mirror depends only on the sign of X
                    const int sp = X & 3, sm = (-X) & 3;
                    const int Xa = X - sp, Xc = X + sm;          // X rounded down / up to 4
                    const int oa[8] = {Z + Y + Xa, Z + Y - Xc, Z - Y + Xa, Z - Y - Xc,
                                       Y - Z + Xa, Y - Z - Xc, -Z - Y + Xa, -Z - Y - Xc};
                    uint32_t b[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const uint32_t *q = reinterpret_cast<const uint32_t *>(c0 + oa[m]);
                        b[m] = __funnelshift_r(__ldg(q), __ldg(q + 1), 8 * ((m & 1) ? sm : sp));
                    }
#pragma unroll
                    for (int m = 0; m < 8; ++m) add4(b[m]);
                    e = en;
                }
                if constexpr (W) {
                    // offsets on a coordinate plane or axis, one entry each
                    for (int k = tab.rest_start(rho); k < tab.rest_start(rho + 1); ++k) {
                        const uint32_t f = tab.rest(k);
                        const int off = ((int)((f >> 16) & 0xffu) - 64) * pz +
                                        ((int)((f >> 8) & 0xffu) - 64) * py +
                                        ((int)(f & 0xffu) - 64);
                        add4(bins4(c0, off));
                    }
                    if (i == 0 && rho == kWrapFold && r > kWrapFold) {
                        __syncwarp();
                        tm_wait_st();      // the row start's stores
#pragma unroll
                        for (int j = 0; j < CPL; ++j)
                            wrap_fold<B, CPL>(cnt_lane, j, st[j], tm_base + (uint32_t)(j * B),
                                              tm_base + (uint32_t)((j ^ 1) * B), st[j ^ 1].c0);
                    }
                    continue;
                }
                // offsets on a coordinate plane: 4 sign mirrors per entry,
                // +-A +-C with C the component along the row when it is
                // nonzero (plane 0 or 1), else the y part (a multiple of 16)
                const int k4 = c_c4_start[rho], k5 = c_c4_start[rho + 1];
                uint32_t g = c_c4[k4];
                for (int k = k4; k < k5; ++k) {
                    const uint32_t gn = c_c4[k + 1];
                    const int pl = (int)(g >> 24);
                    const int Yv = (int)((g >> 8) & 0xffu) * py;
                    const int Zv = (int)((g >> 16) & 0xffu) * pz;
                    const int A = pl == 0 ? Yv : Zv;
                    const int C = pl == 2 ? Yv : (int)(g & 0xffu);
                    const int sp = C & 3, sm = (-C) & 3;
                    const int Ca = C - sp, Cc = C + sm;
                    const int oa[4] = {A + Ca, A - Cc, -A + Ca, -A - Cc};
                    uint32_t b[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t *q = reinterpret_cast<const uint32_t *>(c0 + oa[m]);
                        b[m] = __funnelshift_r(__ldg(q), __ldg(q + 1), 8 * ((m & 1) ? sm : sp));
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) add4(b[m]);
                    g = gn;
                }
                // offsets on an axis and the origin, one entry each
                for (int k = c_c1_start[rho]; k < c_c1_start[rho + 1]; ++k) {
                    const uint32_t f = c_c1[k];
                    const int off = ((int)((f >> 16) & 0xffu) - 64) * pz +
                                    ((int)((f >> 8) & 0xffu) - 64) * py + ((int)(f & 0xffu) - 64);
                    add4(bins4(c0, off));
                }
            }
            if constexpr (TM) {
                __syncwarp();
                tm_wait_st();              // the previous scale's stores
            }
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                if constexpr (W)
                    scale_step<B, true, CPL, true, true>(
                        a, cnt_lane, j, i, r, st[j], orow + cx + j, cx + j < a.vol.nx,
                        tm_base + (uint32_t)(j * B), tm_base + (uint32_t)((j ^ 1) * B),
                        st[j ^ 1].c0);
                else
                    scale_step<B, false, CPL, TM>(a, cnt_lane, j, i, r, st[j], orow + cx + j,
                                                  cx + j < a.vol.nx, tm_base + 32u * j);
            }
        }
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            if (cx + j < a.vol.nx) {
                a.out.Y[orow + cx + j] = st[j].yb;
                a.out.s[orow + cx + j] = (uint8_t)st[j].sb;
            }
        }
    }
    if constexpr (TM) {
        tm_wait_st();
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (warp == 0) tm_dealloc(s_tmem, tm_cols);
    }
}

// Launch path 5 (sliding windows, r_max <= 25, 16 or 32 bins): a warp
// takes 32 consecutive x-centres of one y and slides them along z over a
// run of tz planes, keeping one histogram per scale (not a running one, as
// the other paths do).  Moving a centre from z to z + 1 changes Ball(r) by
// one voxel at each end of every z-row (dx, dy) of the ball: the voxel at
// z + 1 + w(dx, dy) enters, the one at z - w leaves.  That is 2 rows(r)
// updates per scale, sum over r of 2 rows(r) ~ 2 pi sum r^2 per centre
// (17 945 for r = 4..20 against 33 401 for the shell-incremental paths).
// The histograms of scales 2p and 2p + 1 share a word (16-bit halves:
// |Ball(25)| < 2^16); a removal adds -inc, which borrows nothing because
// the count it lowers is at least 1.  The first centre of a run builds its
// histograms shell by shell in a scratch column and copies each scale's
// counts out.  Each centre's scales are evaluated with the same FP64 steps,
// in the same order, as scale_step, so Y and s_best are identical.
template <int B>
__global__ void __launch_bounds__(32) k_dense_slide(const DenseArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int NW = B + 1;
    const int lane = threadIdx.x & 31;
    const int S = a.S, npair = (S + 1) / 2;
    const uint32_t col = smem_u32(smem) + lane * 4;               // word w at col + 128 w
    const uint32_t scr = col + ((uint32_t)(npair * NW) << 7);     // scratch column
    const int xg = blockIdx.x * 32 + lane;
    const bool live = xg < a.vol.nx;
    const int x = live ? xg : a.vol.nx - 1;     // idle lanes repeat the last column
    const int y = blockIdx.y;
    const int zs = a.z0 + blockIdx.z * a.tz;
    const int ze = min(zs + a.tz, a.z1);
    if (zs >= ze) return;
    const int pz = (int)a.vol.plane, py = (int)a.vol.pitch;
    const uint8_t *c0 = a.vol.base + (int64_t)zs * a.vol.plane + (int64_t)y * a.vol.pitch + x;
    const Tab<true> tab{a.ot};
    for (int w = 0; w < (npair + 1) * NW; ++w) st_shared_u32(col + ((uint32_t)w << 7), 0u);
    // the first centre: shells into the scratch column, each scale copied out
    for (int rho = 0; rho <= a.r_max; ++rho) {
        for (int k = tab.c8_start(rho); k < tab.c8_start(rho + 1); ++k) {
            const uint32_t e = tab.c8(k);
            const int X = (int)(e & 0xffu);
            const int Y = (int)((e >> 8) & 0xffu) * py;
            const int Z = (int)((e >> 16) & 0xffu) * pz;
            const int o[8] = {Z + Y + X, Z + Y - X, Z - Y + X, Z - Y - X,
                              Y - Z + X, Y - Z - X, -Z - Y + X, -Z - Y - X};
            uint32_t v[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = __ldg(c0 + o[m]);
#pragma unroll
            for (int m = 0; m < 8; ++m) red_add_shared(scr + (v[m] << 7), 1u);
        }
        for (int k = tab.rest_start(rho); k < tab.rest_start(rho + 1); ++k) {
            const uint32_t f = tab.rest(k);
            const int off = ((int)((f >> 16) & 0xffu) - 64) * pz + ((int)((f >> 8) & 0xffu) - 64) * py +
                            ((int)(f & 0xffu) - 64);
            red_add_shared(scr + ((uint32_t)__ldg(c0 + off) << 7), 1u);
        }
        const int i = rho - a.r_min;
        if (i >= 0) {
            const uint32_t pw = col + ((uint32_t)((i >> 1) * NW) << 7);
            for (int v = 0; v < NW; ++v) {
                const uint32_t cv = ld_shared_u32(scr + ((uint32_t)v << 7));
                const uint32_t adr = pw + ((uint32_t)v << 7);
                st_shared_u32(adr, (i & 1) ? (ld_shared_u32(adr) | (cv << 16)) : cv);
            }
        }
    }
    for (int z = zs;;) {
        // the centre (x, y, z): every scale from its own histogram
        ScaleState st{0.0, 0.0, 0.0, 0u, 0u, 0ull, 0};
        const int64_t oidx = ((int64_t)z * a.vol.ny + y) * a.vol.nx + x;
        for (int i = 0; i < S; ++i) {
            const int r = a.r_min + i;
            const uint32_t pw = col + ((uint32_t)((i >> 1) * NW) << 7);
            const uint32_t qw = col + ((uint32_t)(((i - 1) >> 1) * NW) << 7);   // scale i - 1
            const int sh = 16 * (i & 1), qs = 16 * ((i - 1) & 1);
            auto count = [&](int v) { return (ld_shared_u32(pw + ((uint32_t)v << 7)) >> sh) & 0xffffu; };
            const uint32_t N = (uint32_t)__ldg(a.ot.ball_size + r) - count(0);
            double ssum = 0.0;
            int occ = 0;
            uint64_t D = 0;
#pragma unroll 4
            for (int v = 1; v <= B; ++v) {
                const uint32_t c = count(v);
                const uint32_t p =
                    i == 0 ? 0u : (ld_shared_u32(qw + ((uint32_t)v << 7)) >> qs) & 0xffffu;
                occ += c > 0u;
                if (c > 1u) ssum = __dadd_rn(ssum, __ldg(a.T + c));
                const int64_t d = (int64_t)c * st.nm1 - (int64_t)p * N;
                D += (uint64_t)(d < 0 ? -d : d);
            }
            const double H = entropy_from_sum(ssum, N, occ, a.L);
            if (i >= 2 && st.hm2 < st.hm1 && st.hm1 >= H) {   // peak at scale i-1
                const double W = kb_weight(st.dm1, st.nm1, st.nm2, r - 1, a.w_norm);
                const double yv = __dmul_rn(st.hm1, W);
                if (st.sb == 0 || yv > st.yb) {
                    st.yb = yv;
                    st.sb = r - 1;
                }
            }
            if (live && (a.out.H || a.out.W)) {
                if (a.out.H) a.out.H[oidx * a.S + i] = H;
                if (a.out.W)
                    a.out.W[oidx * a.S + i] = i == 0 ? 0.0 : kb_weight(D, N, st.nm1, r, a.w_norm);
            }
            st.hm2 = st.hm1;
            st.hm1 = H;
            st.nm2 = st.nm1;
            st.nm1 = N;
            st.dm1 = D;
        }
        if (live) {
            a.out.Y[oidx] = st.yb;
            a.out.s[oidx] = (uint8_t)st.sb;
        }
        if (++z >= ze) break;
        // slide every scale's ball from z - 1 to z
        for (int i = 0; i < S; ++i) {
            const int r = a.r_min + i;
            const uint32_t pw = col + ((uint32_t)((i >> 1) * NW) << 7);
            const uint32_t inc = 1u << (16 * (i & 1)), dec = 0u - inc;
            const int k1 = __ldg(a.ot.rows_start + r + 1);
#pragma unroll 4
            for (int k = __ldg(a.ot.rows_start + r); k < k1; ++k) {
                const uint32_t e = __ldg(a.ot.rows + k);
                const int base = ((int)(e & 0xffu) - 64) + ((int)((e >> 8) & 0xffu) - 64) * py;
                const int w = (int)(e >> 16);
                const uint32_t ve = __ldg(c0 + base + (w + 1) * pz);
                const uint32_t vl = __ldg(c0 + base - w * pz);
                red_add_shared(pw + (ve << 7), inc);
                red_add_shared(pw + (vl << 7), dec);
            }
        }
        c0 += pz;
    }
}

// Kadir-Brady at listed centres: one warp per centre.  The lanes split the
// offset entries of each shell and count into lane-private columns (word v
// of lane l at +128 v + 4 l); after the shells of a scale, lane b gathers
// bin b from the 32 columns (starting at column b, so the reads fall in 32
// banks) into its running count c_b, and zeroes its column.  The scale step
// then runs on the whole warp: every lane forms the same bin-order entropy
// sum from shuffled table values (T[0] = T[1] = +0.0, so adding them leaves
// the sum as the skipping form has it), D is an exact integer reduction, and
// H, W, the peak test and Y are the same FP64 steps as in scale_step.  A
// centre outside the volume flags kStatusBadInput and is skipped.
template <int B, bool WIDE>
__global__ void __launch_bounds__(128) k_points(const DenseArgs a) {
    // (every kernel of this file declares the dynamic buffer with the same
    // 1024-byte alignment: the declarations share one symbol, and the TMA
    // brick of k_dense needs a 128-byte aligned base)
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr bool CTAB = !WIDE;
    constexpr int NB = (B + 32) / 32;               // bins 0..B, lane l holds l + 32 k
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int pz = (int)a.vol.plane, py = (int)a.vol.pitch;
    const Tab<CTAB> tab{a.ot};
    const uint32_t col = smem_u32(smem) + (warp * (B + 1) * 32 + lane) * 4;
    const uint32_t cols = smem_u32(smem) + warp * (B + 1) * 32 * 4;
    for (int w = 0; w <= B; ++w) st_shared_u32(col + ((uint32_t)w << 7), 0u);
    __syncwarp();
    for (int64_t pt = (int64_t)blockIdx.x * wpb + warp; pt < a.npts; pt += (int64_t)gridDim.x * wpb) {
        const int x = a.pts[3 * pt], y = a.pts[3 * pt + 1], z = a.pts[3 * pt + 2];
        if (x < 0 || x >= a.vol.nx || y < 0 || y >= a.vol.ny || z < 0 || z >= a.vol.nz) {
            if (lane == 0) atomicOr(a.status, kStatusBadInput);
            continue;                                                  // warp-uniform
        }
        const uint8_t *c0 = a.vol.base + (int64_t)z * a.vol.plane + (int64_t)y * a.vol.pitch + x;
        uint32_t c[NB], p[NB];                       // running and previous counts
#pragma unroll
        for (int k = 0; k < NB; ++k) c[k] = p[k] = 0u;
        ScaleState st{0.0, 0.0, 0.0, 0u, 0u, 0ull, 0};
        for (int i = 0; i < a.S; ++i) {
            const int r = a.r_min + i;
            for (int rho = (i == 0 ? 0 : r); rho <= r; ++rho) {
                const int k1 = tab.c8_start(rho + 1), k3 = tab.rest_start(rho + 1);
                for (int k = tab.c8_start(rho) + lane; k < k1; k += 32) {
                    const uint32_t e = tab.c8(k);
                    const int X = (int)(e & 0xffu);
                    const int Y = (int)((e >> 8) & 0xffu) * py;
                    const int Z = (int)((e >> 16) & 0xffu) * pz;
                    const int o[8] = {Z + Y + X, Z + Y - X, Z - Y + X, Z - Y - X,
                                      Y - Z + X, Y - Z - X, -Z - Y + X, -Z - Y - X};
                    uint32_t v[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) v[m] = __ldg(c0 + o[m]);
#pragma unroll
                    for (int m = 0; m < 8; ++m) red_add_shared(col + (v[m] << 7), 1u);
                }
                for (int k = tab.rest_start(rho) + lane; k < k3; k += 32) {
                    const uint32_t f = tab.rest(k);
                    const int off = ((int)((f >> 16) & 0xffu) - 64) * pz +
                                    ((int)((f >> 8) & 0xffu) - 64) * py + ((int)(f & 0xffu) - 64);
                    red_add_shared(col + ((uint32_t)__ldg(c0 + off) << 7), 1u);
                }
            }
            __syncwarp();
            // gather: lane b adds bin b of every column, then zeroes its own column
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int bb = lane + 32 * k;
                if (bb <= B) {
                    uint32_t sum = 0;
                    for (int l = 0; l < 32; ++l)
                        sum += ld_shared_u32(cols + ((uint32_t)bb << 7) + 4 * ((l + lane) & 31));
                    p[k] = c[k];
                    c[k] += sum;
                }
            }
            __syncwarp();
            for (int w = 0; w <= B; ++w) st_shared_u32(col + ((uint32_t)w << 7), 0u);
            __syncwarp();
            // scale step on the whole warp (bin 0 = not counted)
            const uint32_t N = (uint32_t)__ldg(a.ot.ball_size + r) - __shfl_sync(full, c[0], 0);
            int occ = 0;
            int64_t d = 0;
            double t[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int bb = lane + 32 * k;
                const bool real = bb >= 1 && bb <= B;
                occ += __popc(__ballot_sync(full, real && c[k] > 0u));
                const int64_t dd = real ? (int64_t)c[k] * st.nm1 - (int64_t)p[k] * N : 0;
                d += dd < 0 ? -dd : dd;
                t[k] = real ? __ldg(a.T + c[k]) : 0.0;
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) d += __shfl_xor_sync(full, d, off);
            const uint64_t D = (uint64_t)d;
            double ssum = 0.0;
#pragma unroll
            for (int bb = 1; bb <= B; ++bb) ssum = __dadd_rn(ssum, __shfl_sync(full, t[bb >> 5], bb & 31));
            const double H = entropy_from_sum(ssum, N, occ, a.L);
            if (i >= 2 && st.hm2 < st.hm1 && st.hm1 >= H) {      // peak at scale i-1
                const double Wp = kb_weight(st.dm1, st.nm1, st.nm2, r - 1, a.w_norm);
                const double yv = __dmul_rn(st.hm1, Wp);
                if (st.sb == 0 || yv > st.yb) {
                    st.yb = yv;
                    st.sb = r - 1;
                }
            }
            if (lane == 0) {
                if (a.out.H) a.out.H[pt * a.S + i] = H;
                if (a.out.W) a.out.W[pt * a.S + i] = i == 0 ? 0.0 : kb_weight(D, N, st.nm1, r, a.w_norm);
            }
            st.hm2 = st.hm1;
            st.hm1 = H;
            st.nm2 = st.nm1;
            st.nm1 = N;
            st.dm1 = D;
        }
        if (lane == 0) {
            a.out.Y[pt] = st.yb;
            a.out.s[pt] = (uint8_t)st.sb;
        }
    }
}

int template_bins(int B) {
    return B <= 2 ? 2 : B <= 4 ? 4 : B <= 8 ? 8 : B <= 16 ? 16 : B <= 32 ? 32 : 64;
}

bool is_wide(int r_max) { return r_max > kConstRmax; }

// shared memory of a launch path 5 block: one word per bin and pair of
// scales, plus the scratch column, for each of the 32 lanes
size_t slide_smem_bytes(int B, int S) {
    return (size_t)((S + 1) / 2 + 1) * (template_bins(B) + 1) * 128;
}

struct Geometry {
    int padx, bx, by, bz;
    size_t brick, cnt_off, cnt_bytes, mbar_off, total;
};

int centres_per_lane(const DenseConfig &c) {
    return c.path == 6 ? 1 : (c.path == 7 || c.path == 8) ? 2 : (c.path >= 3 ? 4 : (c.path == 2 ? 2 : 1));
}

Geometry geometry(const DenseConfig &c, int B_, int r_max) {
    Geometry g{};
    const int B = template_bins(B_);
    // counter columns + previous-scale counts per lane (layout of Words)
    const int cpl = centres_per_lane(c);
    const bool wide = is_wide(r_max);
    const int words = (cpl >= 2 && (!wide || c.path == 8 || c.path == 9) ? cpl / 2 : cpl) * (B + 1) +
                      (c.path == 4 || c.path >= 6 ? 0 : cpl * (wide ? B + 1 : (B + 2) / 2));
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

template <int B, bool WIDE, int PATH, int CPL>
cudaError_t launch_t(const LaunchCtx &lc, const DenseArgs &a, const CUtensorMap *tmap,
                     const DenseConfig &cfg, size_t smem) {
    auto kern = k_dense<B, WIDE, PATH, CPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.vol.nx + 32 * CPL - 1) / (32 * CPL), (a.vol.ny + a.ty - 1) / a.ty,
              (a.z1 - a.z0 + a.tz - 1) / a.tz);
    CUtensorMap dummy{};
    kern<<<grid, cfg.warps * 32, smem, lc.stream>>>(a, tmap ? *tmap : dummy);
    return cudaGetLastError();
}

// An upper bound of the blocks of `kern` that an SM can hold with `threads`
// threads and `dyn` bytes of dynamic shared memory: the register file, the
// whole shared memory (whatever carveout the driver picks), the thread and
// block limits.  cudaOccupancyMaxActiveBlocksPerMultiprocessor is not used
// here: for the TMEM kernels it reports 1 block per SM (it assumes a smaller
// shared-memory carveout) while 4 are resident.
cudaError_t max_resident_blocks(const void *kern, int threads, size_t dyn, int *out) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, regs = 0, smem = 0, thr = 0, blk = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) ||
        (e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) ||
        (e = cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) ||
        (e = cudaDeviceGetAttribute(&blk, cudaDevAttrMaxBlocksPerMultiprocessor, dev)))
        return e;
    int n = std::min(blk, thr / threads);
    if (fa.numRegs > 0) n = std::min(n, regs / (fa.numRegs * threads));
    const size_t per_block = dyn + fa.sharedSizeBytes;
    if (per_block > 0) n = std::min(n, (int)((size_t)smem / per_block));
    *out = n;
    return cudaSuccess;
}

// Launch paths 6 to 8: path 1 with one (6) or two (7, 8: 16-bit wrapping
// counters) centres per lane and the previous counts in TMEM.  The dynamic shared memory is padded until
// the blocks that fit on an SM hold at most its 512 TMEM columns, so no
// tcgen05.alloc waits for another block's.
template <int B, int CPL, bool WRAP = false>
cudaError_t launch_t_tm(const LaunchCtx &lc, const DenseArgs &a, const DenseConfig &cfg,
                        size_t smem) {
    auto kern = k_dense<B, true, 1, CPL, true, WRAP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int limit = 512 / tm_columns_wide(cfg.warps, CPL * B);
    for (;;) {
        int nb = 0;
        e = max_resident_blocks(reinterpret_cast<const void *>(kern), cfg.warps * 32, smem, &nb);
        if (e != cudaSuccess) return e;
        if (nb <= limit) break;
        smem += 1024;
        if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.vol.nx + 32 * CPL - 1) / (32 * CPL), (a.vol.ny + a.ty - 1) / a.ty,
              (a.z1 - a.z0 + a.tz - 1) / a.tz);
    CUtensorMap dummy{};
    kern<<<grid, cfg.warps * 32, smem, lc.stream>>>(a, dummy);
    return cudaGetLastError();
}

template <int B, bool TM, bool W = false>
cudaError_t launch_adj4(const LaunchCtx &lc, const DenseArgs &a, const DenseConfig &cfg,
                        size_t smem) {
    auto kern = k_dense4<B, TM, W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (TM) {
        // Pad the dynamic shared memory until the blocks that fit on an SM
        // hold at most its 512 TMEM columns, so no tcgen05.alloc waits for
        // another block's columns.
        const int limit = 512 / (W ? tm_columns_wide(cfg.warps, 4 * B) : tm_columns(cfg.warps));
        for (;;) {
            int nb = 0;
            e = max_resident_blocks(reinterpret_cast<const void *>(kern), cfg.warps * 32, smem,
                                    &nb);
            if (e != cudaSuccess) return e;
            if (nb <= limit) break;
            smem += 1024;
            if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    dim3 grid((a.vol.nx + 127) / 128, (a.vol.ny + a.ty - 1) / a.ty, (a.z1 - a.z0 + a.tz - 1) / a.tz);
    kern<<<grid, cfg.warps * 32, smem, lc.stream>>>(a);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_b(const LaunchCtx &lc, const DenseArgs &a, const CUtensorMap *tmap,
                     const DenseConfig &cfg, size_t smem) {
    const bool wide = is_wide(a.r_max);
    if (cfg.path == 5) {
        if constexpr (B == 16 || B == 32) {
            if (wide) return cudaErrorInvalidValue;
            const size_t sm = slide_smem_bytes(B, a.S);
            cudaError_t e = cudaFuncSetAttribute(k_dense_slide<B>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            dim3 grid((a.vol.nx + 31) / 32, a.vol.ny, (a.z1 - a.z0 + a.tz - 1) / a.tz);
            k_dense_slide<B><<<grid, 32, sm, lc.stream>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    if (cfg.path >= 6 && cfg.path <= 8) {
        if constexpr (B == 16 || B == 32 || B == 64) {
            if (!wide) return cudaErrorInvalidValue;
            return cfg.path == 6   ? launch_t_tm<B, 1>(lc, a, cfg, smem)
                   : cfg.path == 7 ? launch_t_tm<B, 2>(lc, a, cfg, smem)
                                   : launch_t_tm<B, 2, true>(lc, a, cfg, smem);
        }
        return cudaErrorInvalidValue;
    }
    if (cfg.path == 9) {
        if constexpr (B == 16 || B == 32 || B == 64)
            return wide ? launch_adj4<B, true, true>(lc, a, cfg, smem) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    }
    if (cfg.path == 3) return wide ? cudaErrorInvalidValue : launch_adj4<B, false>(lc, a, cfg, smem);
    if (cfg.path == 4) {
        if constexpr (B == 16 || B == 32)
            return wide ? cudaErrorInvalidValue : launch_adj4<B, true>(lc, a, cfg, smem);
        return cudaErrorInvalidValue;
    }
    if (cfg.path == 0)
        return wide ? launch_t<B, true, 0, 1>(lc, a, tmap, cfg, smem)
                    : launch_t<B, false, 0, 1>(lc, a, tmap, cfg, smem);
    if (cfg.path == 1)
        return wide ? launch_t<B, true, 1, 1>(lc, a, tmap, cfg, smem)
                    : launch_t<B, false, 1, 1>(lc, a, tmap, cfg, smem);
    return wide ? launch_t<B, true, 1, 2>(lc, a, tmap, cfg, smem)
                : launch_t<B, false, 1, 2>(lc, a, tmap, cfg, smem);
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
    // regroup the rest entries of every class into 4-mirror sets and the rest
    std::vector<uint32_t> h4, h1;
    int s4[kConstRmax + 2], s1[kConstRmax + 2];
    for (int rho = 0; rho <= kConstRmax; ++rho) {
        s4[rho] = (int)h4.size();
        s1[rho] = (int)h1.size();
        int n4 = 0;
        for (int k = rest_start[rho]; k < rest_start[rho + 1]; ++k) {
            const uint32_t f = rest[k];
            const int d[3] = {(int)(f & 0xffu) - 64, (int)((f >> 8) & 0xffu) - 64,
                              (int)((f >> 16) & 0xffu) - 64};
            const int nz = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
            if (nz <= 1) {
                h1.push_back(f);
            } else if (nz == 2) {
                ++n4;
                if (d[0] >= 0 && d[1] >= 0 && d[2] >= 0)      // the all-positive mirror
                    h4.push_back((uint32_t)d[0] | ((uint32_t)d[1] << 8) | ((uint32_t)d[2] << 16) |
                                 ((uint32_t)(d[2] == 0 ? 0 : (d[1] == 0 ? 1 : 2)) << 24));
            } else {
                return cudaErrorInvalidValue;                 // not a rest entry
            }
        }
        if (n4 != 4 * ((int)h4.size() - s4[rho])) return cudaErrorInvalidValue;
    }
    s4[kConstRmax + 1] = (int)h4.size();
    s1[kConstRmax + 1] = (int)h1.size();
    if ((int)h4.size() + 1 > kConstC4 || (int)h1.size() > kConstC1) return cudaErrorInvalidValue;
    h4.push_back(0u);                                         // the prefetch past the last entry
    cudaError_t e = cudaMemcpyToSymbol(c_c8, c8, n8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rest, rest, nr * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_c8_start, c8_start, (kConstRmax + 2) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_rest_start, rest_start, (kConstRmax + 2) * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_c4, h4.data(), h4.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_c1, h1.data(), h1.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_c4_start, s4, sizeof(s4));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_c1_start, s1, sizeof(s1));
    return e;
}

int dense_const_rmax() { return kConstRmax; }

namespace {
template <int B>
cudaError_t launch_points_b(const LaunchCtx &lc, const DenseArgs &a) {
    constexpr int kWarps = 4;                       // one centre per warp at a time
    const size_t smem = (size_t)kWarps * 32 * 4 * (B + 1);
    auto kern = is_wide(a.r_max) ? k_points<B, true> : k_points<B, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t need = (a.npts + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)lc.num_sms * 16;
    kern<<<(unsigned)(need < cap ? need : cap), kWarps * 32, smem, lc.stream>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_dense_points(const LaunchCtx &lc, const VolDesc &v, const OffsetTables &ot,
                                const double *T, const double *L, int r_min, int r_max,
                                int w_norm, const int32_t *xyz, int64_t n, const DenseOut &out) {
    if (n <= 0) return cudaSuccess;
    DenseArgs a{};
    a.vol = v;
    a.ot = ot;
    a.T = T;
    a.L = L;
    a.r_min = r_min;
    a.r_max = r_max;
    a.S = r_max - r_min + 1;
    a.w_norm = w_norm;
    a.out = out;
    a.status = lc.d_status;
    a.pts = xyz;
    a.npts = n;
    switch (template_bins(v.B)) {
        case 2: return launch_points_b<2>(lc, a);
        case 4: return launch_points_b<4>(lc, a);
        case 8: return launch_points_b<8>(lc, a);
        case 16: return launch_points_b<16>(lc, a);
        case 32: return launch_points_b<32>(lc, a);
        case 64: return launch_points_b<64>(lc, a);
        default: return cudaErrorInvalidValue;
    }
}

size_t dense_smem_bytes(const DenseConfig &c, int B, int r_max) {
    return geometry(c, B, r_max).total;
}

int64_t dense_computed_centres(const DenseConfig &c, int nx, int ny, int nz) {
    int64_t x;
    if (c.path == 5) {
        x = (int64_t)(nx + 31) / 32 * 32;
    } else {
        const int cpl = centres_per_lane(c), w = 32 * cpl;
        x = (int64_t)(nx / w) * w;
        const int rem = nx % w;
        // two centres per lane: a last tile of at most 32 centres walks one
        // per lane
        if (rem) x += cpl == 2 && rem <= 32 ? 32 : w;
    }
    const int64_t y = (int64_t)(ny + c.ty - 1) / c.ty * c.ty;
    const int64_t z = (int64_t)(nz + c.tz - 1) / c.tz * c.tz;
    return x * y * z;
}

bool dense_config_fits(const DenseConfig &c, int B, int r_max) {
    if (c.path == 5)
        return !is_wide(r_max) && (template_bins(B) == 16 || template_bins(B) == 32) &&
               c.warps == 1 && c.ty == 1 && c.tz >= 1 && c.tz <= 1024 &&
               slide_smem_bytes(B, r_max + 1) + 1024 <= 227 * 1024;
    if (c.path >= 6 && c.path <= 9) {
        // whole warpgroups (each warp its TMEM lane quarter), 16, 32 or 64
        // bins, only where the counts need 32 bits; two or four centres per
        // lane (paths 7 to 9) allow at most 8 warps (the kernels' launch
        // bounds)
        const int tb = template_bins(B);
        if (!is_wide(r_max) || (tb != 16 && tb != 32 && tb != 64)) return false;
        if ((c.warps != 4 && c.warps != 8 && (c.warps != 16 || c.path != 6)) ||
            c.ty * c.tz != c.warps)
            return false;
        return geometry(c, B, r_max).total + 1024 <= 227 * 1024;
    }
    if (c.path < 0 || c.path > 4) return false;
    if (c.path >= 3 && is_wide(r_max)) return false;      // counts need 16-bit packing
    if (c.path == 4 && template_bins(B) != 16 && template_bins(B) != 32) return false;
    if (c.warps < 1 || c.warps > (c.path >= 2 ? 8 : 16) || c.ty * c.tz != c.warps) return false;
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
