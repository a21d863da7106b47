// Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 7) towards
// the uniform target pmf HQ_b = 1/B.
//
// Items (seed, r) come from two persistent ticket queues, largest starting
// radius first: items with r >= r_team are taken by a whole block (8 warps
// share every pass, the first warp does the per-item steps), the others by
// one warp each.  An iteration makes four passes over the voxels of the
// current ellipsoid { s : (s-x)^T H^-1 (s-x) <= 1 }:
//   1. kernel histogram at (x, H) -> w_b = sqrt(HQ_b / HP_b)
//   2. Eq. 6 sums  sum k w o, sum k w            -> x'
//   3. kernel histogram at (x', H) -> w'_b, rho = sum_b sqrt(HQ_b HP'_b)
//   4. Eq. 7 sums  sum w' o o^T, sum w'         -> H' = 5 (M / sum w' + I/12)
// A pass takes the box's x-rows 32 at a time (the warps of a team take
// every T-th batch): lane j finds row j's span (the root interval of
// d <= 1 + 1/16 along x), a warp scan packs the spans end to end, and the
// lanes walk the packed voxels, two per lane per step; a lane finds its
// row from a 32-bit mask of the row starts in its half-step (one warp
// OR-reduction) and a per-warp table of the batch's rows.  Along a row d is
// (h00 o_x + 2 beta) o_x + gamma (two fused multiply-adds, beta and gamma
// once per row).  Per-voxel terms are binary32 in one fixed operation
// order; every sum over voxels is an exact integer sum of the terms rounded
// to nearest on a fixed-point grid, so the summation order does not change
// the result.  The grids are 2^-16 for k and for the weights w' of the
// bandwidth sums; the position terms k w o and the second moments w' o o^T
// take the finest grids 2^-px, 2^-pm on which no term of weight k w < 4
// (resp. w' < 4) reaches 2^22 (from the box half-width E: px = 14, pm = 9
// at E = 32, px = 18, pm = 16 at E = 2), so small windows are summed as
// finely as large ones relative to their extent; heavier rare-bin terms
// are summed in int64 on the same grids.  Histogram sums go to lane-private u32 columns in
// shared memory (shared reductions, no bank conflicts), the position and
// moment terms to int32 sums per batch of rows, then int64.  The passes are
// non-inlined functions shared by both item paths (smaller code), and the
// per-item values live in shared memory across them.  Everything per bin
// or per item is FP64, one IEEE operation at a time, done by the item's
// first warp with its lanes computing the same values, so that the warp's
// control flow stays uniform.
#include <algorithm>

#include "ks_internal.cuh"

namespace ks {

namespace {

constexpr int kAbWarps = 8;                 // warps per block, one item each
constexpr float kQK = 65536.0f;             // 2^16: kernel values
constexpr float kQW = 65536.0f;             // 2^16: weights of the bandwidth sums
constexpr double kHmax = 1024.0;            // 32^2: the window stays in the halo
constexpr double kVoxel = 5.0 / 12.0;       // (n+2) x the second moment of a unit voxel
constexpr float kSlack = 1.0625f;           // a row's span covers d <= 1 + 1/16

// exp(-d/2) for 0 <= d <= 1 by its Taylor series to degree 9 (Horner form
// with fused multiply-adds; truncation error below 3e-10, under half a
// binary32 ulp).
__device__ __forceinline__ float ab_kernel(float d) {
    const float t = __fmul_rn(-0.5f, d);
    float p = 2.755731922398589e-06f;
    p = __fmaf_rn(p, t, 2.48015873015873e-05f);
    p = __fmaf_rn(p, t, 1.984126984126984e-04f);
    p = __fmaf_rn(p, t, 0.001388888888888889f);
    p = __fmaf_rn(p, t, 0.008333333333333333f);
    p = __fmaf_rn(p, t, 0.041666666666666664f);
    p = __fmaf_rn(p, t, 0.16666666666666666f);
    p = __fmaf_rn(p, t, 0.5f);
    p = __fmaf_rn(p, t, 1.0f);
    p = __fmaf_rn(p, t, 1.0f);
    return p;
}

// Nearest integer (ties to even) of y, |y| < 2^22: adding 1.5 * 2^23 puts
// the sum in [2^23, 2^24), where the binary32 ulp is 1, so the addition
// itself rounds y to an integer; its bit pattern is 0x4B400000 + rint(y).
__device__ __forceinline__ int ab_rint_small(float y) {
    return __float_as_int(__fadd_rn(y, 12582912.0f)) - 0x4B400000;
}
// The same for any finite y (larger |y|, from heavy rare-bin weights, take
// the 64-bit conversion, which rounds the same way).
__device__ __forceinline__ int64_t ab_q(float y) {
    if (fabsf(y) < 4194304.0f) return (int64_t)ab_rint_small(y);
    return __float2ll_rn(y);
}

// Conversions between small integers (|i| < 2^21) and binary32 through the
// same bit pattern (the conversion instructions issue at a small fraction of
// the FP32 rate on this part): the float 1.5 * 2^23 + i has the bits
// 0x4B400000 + i, and subtracting 1.5 * 2^23 from it is exact.
__device__ __forceinline__ float ab_i2f(int i) {
    return __fsub_rn(__int_as_float(0x4B400000 + i), 12582912.0f);
}
__device__ __forceinline__ int ab_ceil(float y) {
    const float m = __fadd_rn(y, 12582912.0f);   // rint(y) + 1.5 * 2^23
    int r = __float_as_int(m) - 0x4B400000;
    if (__fsub_rn(m, 12582912.0f) < y) ++r;
    return r;
}
__device__ __forceinline__ int ab_floor(float y) {
    const float m = __fadd_rn(y, 12582912.0f);
    int r = __float_as_int(m) - 0x4B400000;
    if (__fsub_rn(m, 12582912.0f) > y) --r;
    return r;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The bandwidth part of a window: H^-1 rounded to binary32 (adjugate times
// 1/det in FP64) and the box half-widths E_a = ceil(sqrt(H_aa)) in
// binary32.  Returns false when H is not positive definite (det <= 0).
struct AbShape {
    float h[6];
    int E[3];
    float qx, qm;     // grids 2^px, 2^pm of the position and moment terms
    float band;       // binary32 d within band of 1: membership decided in FP64
    double adj[6];    // adjugate of H (00 01 02 11 12 22) and det H, FP64
    double det;
};

// Largest p with m 2^p <= 2^22 (m >= 2).
__device__ __forceinline__ int ab_grid_exp(int m) { return 22 - (32 - __clz(m - 1)); }

// Width of the band around d = 1 in which binary32 does not decide window
// membership: 2^-16 sum_ab |h_ab| (E_a + 1)(E_b + 1), an upper bound of
// 2^-16 |o|^T |H^-1| |o| over the box (|o_a| <= E_a + 1).  The binary32 row
// form of d is within 6.1e-7 |o|^T |H^-1| |o| of the exact value (measured
// over 1.2e8 voxels of random, elongated and oblique windows), so outside
// the band it decides as the exact test does.
__device__ __forceinline__ float ab_band(const float h[6], const int E[3]) {
    const float e0 = (float)(E[0] + 1), e1 = (float)(E[1] + 1), e2 = (float)(E[2] + 1);
    float s = __fmul_rn(__fmul_rn(fabsf(h[0]), e0), e0);
    s = __fadd_rn(s, __fmul_rn(__fmul_rn(fabsf(h[3]), e1), e1));
    s = __fadd_rn(s, __fmul_rn(__fmul_rn(fabsf(h[5]), e2), e2));
    float t = __fmul_rn(__fmul_rn(fabsf(h[1]), e0), e1);
    t = __fadd_rn(t, __fmul_rn(__fmul_rn(fabsf(h[2]), e0), e2));
    t = __fadd_rn(t, __fmul_rn(__fmul_rn(fabsf(h[4]), e1), e2));
    s = __fadd_rn(s, __fmul_rn(2.0f, t));
    return __fmul_rn(s, 1.52587890625e-05f);   // 2^-16
}
__device__ __forceinline__ bool ab_shape(const double H[6], AbShape &sh) {
    const double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
    const double c00 = __dsub_rn(__dmul_rn(a11, a22), __dmul_rn(a12, a12));
    const double c01 = __dsub_rn(__dmul_rn(a02, a12), __dmul_rn(a01, a22));
    const double c02 = __dsub_rn(__dmul_rn(a01, a12), __dmul_rn(a02, a11));
    const double c11 = __dsub_rn(__dmul_rn(a00, a22), __dmul_rn(a02, a02));
    const double c12 = __dsub_rn(__dmul_rn(a01, a02), __dmul_rn(a00, a12));
    const double c22 = __dsub_rn(__dmul_rn(a00, a11), __dmul_rn(a01, a01));
    const double det =
        __dadd_rn(__dadd_rn(__dmul_rn(a00, c00), __dmul_rn(a01, c01)), __dmul_rn(a02, c02));
    if (!(det > 0.0)) return false;
    sh.adj[0] = c00;
    sh.adj[1] = c01;
    sh.adj[2] = c02;
    sh.adj[3] = c11;
    sh.adj[4] = c12;
    sh.adj[5] = c22;
    sh.det = det;
    const double inv = __ddiv_rn(1.0, det);
    sh.h[0] = __double2float_rn(__dmul_rn(c00, inv));
    sh.h[1] = __double2float_rn(__dmul_rn(c01, inv));
    sh.h[2] = __double2float_rn(__dmul_rn(c02, inv));
    sh.h[3] = __double2float_rn(__dmul_rn(c11, inv));
    sh.h[4] = __double2float_rn(__dmul_rn(c12, inv));
    sh.h[5] = __double2float_rn(__dmul_rn(c22, inv));
    sh.E[0] = (int)ceilf(__fsqrt_rn(__double2float_rn(a00)));
    sh.E[1] = (int)ceilf(__fsqrt_rn(__double2float_rn(a11)));
    sh.E[2] = (int)ceilf(__fsqrt_rn(__double2float_rn(a22)));
    // |o_a| <= E + 1: position terms |k w o| < 4 (E + 1), moments
    // |w o o| < 4 (E + 1)^2 on the int32 path
    const int E1 = max(max(sh.E[0], sh.E[1]), sh.E[2]) + 1;
    const int px = ab_grid_exp(4 * E1), pm = ab_grid_exp(4 * E1 * E1);
    sh.qx = __int_as_float((127 + px) << 23);
    sh.qm = __int_as_float((127 + pm) << 23);
    sh.band = ab_band(sh.h, sh.E);
    return true;
}

// A window as the passes read it: H^-1, floor(x), frac(x) rounded to
// binary32, and the voxel box [floor(x) - E, floor(x) + E] clipped to the
// volume (voxels outside it are not counted).
struct AbWinS {
    double xc[3];     // the centre, FP64
    double adj[6];    // adjugate of H and det H, FP64 (the exact membership test)
    double det;
    float h[6];
    float f[3];
    int n[3];
    int lo[3], hi[3];
    int E[3];
    float qx, qm, band;
};
__device__ __forceinline__ void ab_place(const double x[3], const AbShape &sh, const int dim[3],
                                         AbWinS &w) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        w.h[k] = sh.h[k];
        w.adj[k] = sh.adj[k];
    }
    w.det = sh.det;
    w.qx = sh.qx;
    w.qm = sh.qm;
    w.band = sh.band;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.E[a] = sh.E[a];
        w.xc[a] = x[a];
        const double fl = floor(x[a]);
        w.n[a] = (int)fl;
        w.f[a] = __double2float_rn(__dsub_rn(x[a], fl));
        w.lo[a] = max(w.n[a] - sh.E[a], 0);
        w.hi[a] = min(w.n[a] + sh.E[a], dim[a] - 1);
    }
}

enum AbPass { kPassHist = 0, kPassPos = 1, kPassMom = 2 };

// Per-pass sums.  Hist: s[0] = window voxels of this lane (the sums live in
// shared memory).  Pos: s[0..2] = sum q(k w o_a), s[3] = sum q(k w) (grid
// 2^-px).  Mom: s[0..5] = sum q(w (o_a o_b)) (grid 2^-pm), s[6] = sum q(w)
// (grid 2^-16).
struct AbSums {
    int64_t s[7];
};

// Voxels whose binary32 d falls in the band around 1, kept for the exact
// test at the end of the pass: (j + 64) | (dy + 64) << 7 | (dz + 64) << 14 |
// b << 21, offsets from floor(x), b the stored bin.
constexpr int kAbQueue = 128;
struct AbQueue {
    int n;
    uint32_t e[kAbQueue];
};

// The exact membership test of the definition: (s - x)^T adj(H) (s - x) <=
// det H in FP64, one IEEE operation at a time in a fixed order (for integer
// x and H, as in the first window of a seed, every operation is exact).
__device__ __forceinline__ bool ab_exact_inside(const AbWinS &w, int j, int dy, int dz) {
    const double o0 = __dsub_rn((double)(w.n[0] + j), w.xc[0]);
    const double o1 = __dsub_rn((double)(w.n[1] + dy), w.xc[1]);
    const double o2 = __dsub_rn((double)(w.n[2] + dz), w.xc[2]);
    const double *A = w.adj;
    double q = __dadd_rn(__dmul_rn(__dmul_rn(A[0], o0), o0), __dmul_rn(__dmul_rn(A[3], o1), o1));
    q = __dadd_rn(q, __dmul_rn(__dmul_rn(A[5], o2), o2));
    double c = __dadd_rn(__dmul_rn(__dmul_rn(A[1], o0), o1), __dmul_rn(__dmul_rn(A[2], o0), o2));
    c = __dadd_rn(c, __dmul_rn(__dmul_rn(A[4], o1), o2));
    q = __dadd_rn(q, __dmul_rn(2.0, c));
    return q <= w.det;
}

// True when binary32 cannot decide d <= 1: |d - 1| <= 2^-16 |o|^T |h| |o|.
__device__ __forceinline__ bool ab_near_boundary(const AbWinS &w, float d, float o0, float o1,
                                                 float o2) {
    const float a0 = fabsf(o0), a1 = fabsf(o1), a2 = fabsf(o2);
    float m = __fmul_rn(__fmul_rn(fabsf(w.h[0]), a0), a0);
    m = __fadd_rn(m, __fmul_rn(__fmul_rn(fabsf(w.h[3]), a1), a1));
    m = __fadd_rn(m, __fmul_rn(__fmul_rn(fabsf(w.h[5]), a2), a2));
    float t = __fmul_rn(__fmul_rn(fabsf(w.h[1]), a0), a1);
    t = __fadd_rn(t, __fmul_rn(__fmul_rn(fabsf(w.h[2]), a0), a2));
    t = __fadd_rn(t, __fmul_rn(__fmul_rn(fabsf(w.h[4]), a1), a2));
    m = __fadd_rn(m, __fmul_rn(2.0f, t));
    return fabsf(__fsub_rn(d, 1.0f)) <= __fmul_rn(m, 1.52587890625e-05f);
}

// The queued voxels of one warp's pass (binary32 d within the window's band
// around 1): the exact test where binary32 cannot decide, binary32
// elsewhere; then the pass's terms on the int64 path (the same rounding as
// the int32 path, so the sums do not depend on which path a term took).
// Clears the queue.
template <int PASS>
__device__ __noinline__ AbSums ab_flush(const AbWinS &w, AbQueue *qu, uint32_t col_s,
                                        const float *wf, int lane) {
    AbSums acc;
#pragma unroll
    for (int k = 0; k < 7; ++k) acc.s[k] = 0;
    const int nq = min(qu->n, kAbQueue);
    const float h0 = w.h[0], h1 = w.h[1], h2 = w.h[2], h3 = w.h[3], h4 = w.h[4], h5 = w.h[5];
    for (int i = lane; i < nq; i += 32) {
        const uint32_t e = qu->e[i];
        const int j = (int)(e & 127u) - 64, dy = (int)((e >> 7) & 127u) - 64;
        const int dz = (int)((e >> 14) & 127u) - 64, b = (int)(e >> 21);
        const float o0 = __fsub_rn(ab_i2f(j), w.f[0]);
        const float r1 = __fsub_rn(ab_i2f(dy), w.f[1]), r2 = __fsub_rn(ab_i2f(dz), w.f[2]);
        const float beta = __fadd_rn(__fmul_rn(h1, r1), __fmul_rn(h2, r2));
        const float gamma = __fadd_rn(
            __fmul_rn(__fadd_rn(__fmul_rn(h3, r1), __fmul_rn(__fmul_rn(2.0f, h4), r2)), r1),
            __fmul_rn(__fmul_rn(h5, r2), r2));
        const float d = __fmaf_rn(__fmaf_rn(h0, o0, __fadd_rn(beta, beta)), o0, gamma);
        if (ab_near_boundary(w, d, o0, r1, r2) ? !ab_exact_inside(w, j, dy, dz) : d > 1.0f)
            continue;
        if (PASS == kPassHist) {
            red_add_shared(col_s + (uint32_t)(b - 1) * 128u,
                           (uint32_t)ab_rint_small(__fmul_rn(ab_kernel(d), kQK)));
            acc.s[0] += 1;
        } else if (PASS == kPassPos) {
            const float tk = __fmul_rn(ab_kernel(d), wf[b - 1]);
            acc.s[0] += ab_q(__fmul_rn(tk, o0));
            acc.s[1] += ab_q(__fmul_rn(tk, r1));
            acc.s[2] += ab_q(__fmul_rn(tk, r2));
            acc.s[3] += ab_q(tk);
        } else {
            const float tw = wf[b - 1];
            acc.s[0] += ab_q(__fmul_rn(tw, __fmul_rn(o0, o0)));
            acc.s[1] += ab_q(__fmul_rn(tw, __fmul_rn(o0, r1)));
            acc.s[2] += ab_q(__fmul_rn(tw, __fmul_rn(o0, r2)));
            acc.s[3] += ab_q(__fmul_rn(tw, __fmul_rn(r1, r1)));
            acc.s[4] += ab_q(__fmul_rn(tw, __fmul_rn(r1, r2)));
            acc.s[5] += ab_q(__fmul_rn(tw, __fmul_rn(r2, r2)));
            acc.s[6] += ab_q(__fmul_rn(tw, __fdiv_rn(kQW, w.qm)));
        }
    }
    __syncwarp();
    if (lane == 0) qu->n = 0;
    __syncwarp();
    return acc;
}

// One row of a batch, in the warp's table: where its voxels start in the
// packed order, and, relative to that start, its first voxel's byte offset
// from the pass base and the bit pattern of the binary32 1.5 * 2^23 + j of
// its first j = s_x - floor(x_x) (so voxel p of the packed order is at
// offp + p with j bits jp + p); the row form of d and its (o_y, o_z).
struct AbRow {
    int start;
    int offp;      // byte offset of the row's first voxel minus start
    int jp;        // 0x4B400000 + (its first j) - start
    float b2, g;   // d = (h00 o_x + b2) o_x + g along the row
    float o1, o2;
    int dyz;       // (s_y - floor(x_y) + 64) | (s_z - floor(x_z) + 64) << 7
};

// One pass of the warp over the window's voxels.
// EXACT = false: voxels in the band go to the warp's queue; if it
// overflows (only windows so oblique that the band holds many voxels), the
// pass is done again with EXACT = true, which tests them in place.
template <int PASS, bool EXACT>
__device__ __noinline__ int64_t ab_pass(const VolDesc &v, const AbWinS &w, uint32_t *col,
                                        const float *wf, AbRow *tab, AbQueue *qu, int lane,
                                        int wt, int T, int64_t *red) {
    AbSums acc;
#pragma unroll
    for (int k = 0; k < 7; ++k) acc.s[k] = 0;
    const float h0 = w.h[0], h1 = w.h[1], h2 = w.h[2], h3 = w.h[3], h4 = w.h[4], h5 = w.h[5];
    const float f0 = w.f[0], f1 = w.f[1], f2 = w.f[2];
    // int32-path limits of the weight factors (terms stay below 2^22) and
    // the factor that puts the moment pass's weights on the 2^-16 grid
    const float lim_x = __fmul_rn(4.0f, w.qx), lim_m = __fmul_rn(4.0f, w.qm);
    const float q6 = __fdiv_rn(kQW, w.qm);
    // binary32 decides membership outside [dlo, dhi]; inside it, voxels whose
    // d is within 2^-16 |o|^T |h| |o| of 1 take the exact test
    const float dlo = __fsub_rn(1.0f, w.band), dhi = __fadd_rn(1.0f, w.band);
    const int e1 = w.hi[1] - w.lo[1] + 1;
    const int nrows = e1 * (w.hi[2] - w.lo[2] + 1);
    const uint32_t col_s = PASS == kPassHist ? smem_u32(col) : 0u;
    const float jlo = ab_i2f(w.lo[0] - w.n[0]), jhi = ab_i2f(w.hi[0] - w.n[0]);
    const float ih0 = __frcp_rn(h0);
    const int pitch = (int)v.pitch, plane = (int)v.plane;
    // byte offsets below are relative to voxel (n_x, lo_y, lo_z)
    const uint8_t *base = v.base + (int64_t)w.lo[2] * v.plane + (int64_t)w.lo[1] * v.pitch + w.n[0];
    // lane's row (iy, iz) and the step of 32 T rows (this warp takes every
    // T-th batch of 32 rows)
    const int row0 = wt * 32 + lane;
    int iy = row0 % e1, iz = row0 / e1;
    const int dy = (32 * T) % e1, dz = (32 * T) / e1;
    const unsigned lt = (1u << lane) - 1u;
    for (int rb = wt * 32; rb < nrows; rb += 32 * T) {
        int len = 0, ja = 0, off = 0, dyz = 0;
        float o1 = 0.0f, o2 = 0.0f, b2 = 0.0f, g = 0.0f;
        if (rb + lane < nrows) {
            const int ry = w.lo[1] + iy - w.n[1], rz = w.lo[2] + iz - w.n[2];
            dyz = (ry + 64) | (rz + 64) << 7;
            o1 = __fsub_rn(ab_i2f(ry), f1);
            o2 = __fsub_rn(ab_i2f(rz), f2);
            const float beta = __fadd_rn(__fmul_rn(h1, o1), __fmul_rn(h2, o2));
            const float gamma = __fadd_rn(
                __fmul_rn(__fadd_rn(__fmul_rn(h3, o1), __fmul_rn(__fmul_rn(2.0f, h4), o2)), o1),
                __fmul_rn(__fmul_rn(h5, o2), o2));
            b2 = __fadd_rn(beta, beta);
            g = gamma;
            const float disc =
                __fsub_rn(__fmul_rn(beta, beta), __fmul_rn(h0, __fsub_rn(gamma, kSlack)));
            if (disc >= 0.0f) {
                const float sq = __fsqrt_rn(disc);
                // ceil / floor of the clamped roots (equal to the clamped
                // ceil / floor whenever the span is not empty)
                const float ya = fminf(
                    fmaxf(__fadd_rn(__fmul_rn(__fsub_rn(-beta, sq), ih0), f0), jlo),
                    __fadd_rn(jhi, 1.0f));
                const float yb = fmaxf(
                    fminf(__fadd_rn(__fmul_rn(__fsub_rn(sq, beta), ih0), f0), jhi),
                    __fsub_rn(jlo, 1.0f));
                const int a = ab_ceil(ya), b = ab_floor(yb);
                if (a <= b) {
                    ja = a;
                    len = b - a + 1;
                    off = iz * plane + iy * pitch + ja;
                }
            }
        }
        iy += dy;
        iz += dz;
        if (iy >= e1) {
            iy -= e1;
            ++iz;
        }
        // pack the spans end to end: exclusive start of each row
        int incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int start = incl - len;
        const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
        if (len > 0) {
            AbRow &rw = tab[__popc(nonempty & lt)];
            rw.start = start;
            rw.offp = off - start;
            rw.jp = 0x4B400000 + ja - start;
            rw.o1 = o1;
            rw.o2 = o2;
            rw.b2 = b2;
            rw.g = g;
            rw.dyz = dyz;
        }
        __syncwarp();
        // int32 partial sums of the batch: a batch has at most 32 rows of at
        // most 65 voxels, so a lane adds at most 65 terms below 2^22 here.
        // Each term is added as the bit pattern of y + 1.5 * 2^23 (that is
        // 0x4B400000 + rint(y)); the n * 0x4B400000 is taken off at the end
        // of the batch, modulo 2^32, which is exact as the sum fits int32.
        uint32_t a32[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t n32 = 0u;
        // one window voxel: packed position p of row rw, stored bin b > 0
        auto voxel = [&](const AbRow &rw, int p, int b) {
            const float o0 = __fsub_rn(__fsub_rn(__int_as_float(rw.jp + p), 12582912.0f), f0);
            const float d = __fmaf_rn(__fmaf_rn(h0, o0, rw.b2), o0, rw.g);
            if (!(d >= -0.0625f && d <= dhi)) return;
            const float r1 = rw.o1, r2 = rw.o2;
            if (d > dlo) {
                const int j = rw.jp + p - 0x4B400000;
                if (EXACT) {
                    if (ab_near_boundary(w, d, o0, r1, r2)
                            ? !ab_exact_inside(w, j, (rw.dyz & 127) - 64, (rw.dyz >> 7) - 64)
                            : d > 1.0f)
                        return;
                } else {
                    const int slot = atomicAdd(&qu->n, 1);
                    if (slot < kAbQueue)
                        qu->e[slot] = (uint32_t)(j + 64) | (uint32_t)rw.dyz << 7 | (uint32_t)b << 21;
                    return;
                }
            }
            // |o_a| <= E + 1, so on the window's grids the terms stay below
            // 2^22 when k w < 4 (position) or w < 4 (moments); heavier
            // rare-bin terms go straight to the int64 sums
            if (PASS == kPassHist) {
                red_add_shared(col_s + (uint32_t)(b - 1) * 128u,
                               (uint32_t)ab_rint_small(__fmul_rn(ab_kernel(d), kQK)));
                n32 += 1u;
            } else if (PASS == kPassPos) {
                // wf holds 2^px w (exact scaling, so (k w o) 2^px = k (2^px w) o)
                const float tk = __fmul_rn(ab_kernel(d), wf[b - 1]);
                const float y0 = __fmul_rn(tk, o0);
                const float y1 = __fmul_rn(tk, r1);
                const float y2 = __fmul_rn(tk, r2);
                const float y3 = tk;
                if (tk < lim_x) {
                    a32[0] += __float_as_uint(__fadd_rn(y0, 12582912.0f));
                    a32[1] += __float_as_uint(__fadd_rn(y1, 12582912.0f));
                    a32[2] += __float_as_uint(__fadd_rn(y2, 12582912.0f));
                    a32[3] += __float_as_uint(__fadd_rn(y3, 12582912.0f));
                    n32 += 1u;
                } else {
                    acc.s[0] += ab_q(y0);
                    acc.s[1] += ab_q(y1);
                    acc.s[2] += ab_q(y2);
                    acc.s[3] += ab_q(y3);
                }
            } else {
                // wf holds 2^pm w (exact scaling)
                const float tw = wf[b - 1];
                const float y0 = __fmul_rn(tw, __fmul_rn(o0, o0));
                const float y1 = __fmul_rn(tw, __fmul_rn(o0, r1));
                const float y2 = __fmul_rn(tw, __fmul_rn(o0, r2));
                const float y3 = __fmul_rn(tw, __fmul_rn(r1, r1));
                const float y4 = __fmul_rn(tw, __fmul_rn(r1, r2));
                const float y5 = __fmul_rn(tw, __fmul_rn(r2, r2));
                const float y6 = __fmul_rn(tw, q6);
                if (tw < lim_m) {
                    a32[0] += __float_as_uint(__fadd_rn(y0, 12582912.0f));
                    a32[1] += __float_as_uint(__fadd_rn(y1, 12582912.0f));
                    a32[2] += __float_as_uint(__fadd_rn(y2, 12582912.0f));
                    a32[3] += __float_as_uint(__fadd_rn(y3, 12582912.0f));
                    a32[4] += __float_as_uint(__fadd_rn(y4, 12582912.0f));
                    a32[5] += __float_as_uint(__fadd_rn(y5, 12582912.0f));
                    a32[6] += __float_as_uint(__fadd_rn(y6, 12582912.0f));
                    n32 += 1u;
                } else {
                    acc.s[0] += ab_q(y0);
                    acc.s[1] += ab_q(y1);
                    acc.s[2] += ab_q(y2);
                    acc.s[3] += ab_q(y3);
                    acc.s[4] += ab_q(y4);
                    acc.s[5] += ab_q(y5);
                    acc.s[6] += ab_q(y6);
                }
            }
        };
        // walk the packed voxels 64 at a time (two per lane, both loads in
        // flight together); a lane's row is found from the 32-bit masks of
        // the row starts in each half
        const unsigned le = lt | (1u << lane);
        int before = 0;        // nonempty rows that start before this step
        int sp = start;        // start - p0
        for (int p0 = 0; p0 < total; p0 += 64) {
            const unsigned m0 = __reduce_or_sync(
                0xffffffffu, len > 0 && (unsigned)sp < 32u ? 1u << sp : 0u);
            const unsigned m1 = __reduce_or_sync(
                0xffffffffu, len > 0 && (unsigned)(sp - 32) < 32u ? 1u << (sp - 32) : 0u);
            sp -= 64;
            const int c0 = __popc(m0);
            const int pa = p0 + lane, pb = pa + 32;
            int ka = 0, kb = 0, ba = 0, bb = 0;
            if (pa < total) {
                ka = before + __popc(m0 & le) - 1;
                ba = __ldg(base + tab[ka].offp + pa);
            }
            if (pb < total) {
                kb = before + c0 + __popc(m1 & le) - 1;
                bb = __ldg(base + tab[kb].offp + pb);
            }
            if (ba) voxel(tab[ka], pa, ba);
            if (bb) voxel(tab[kb], pb, bb);
            before += c0 + __popc(m1);
        }
        if (PASS == kPassHist) {
            acc.s[0] += n32;
        } else {
            const uint32_t off32 = n32 * 0x4B400000u;
#pragma unroll
            for (int k = 0; k < 7; ++k) acc.s[k] += (int32_t)(a32[k] - off32);
        }
        __syncwarp();   // the table is rewritten by the next batch
    }
    // the queued voxels (exact membership test)
    __syncwarp();
    if (!EXACT && qu->n > kAbQueue) {
        // overflow: start the pass again, testing band voxels in place
        __syncwarp();
        if (lane == 0) qu->n = 0;
        if (PASS == kPassHist)
            for (int b = 0; b < v.B; ++b) st_shared_u32(col_s + (uint32_t)b * 128u, 0u);
        __syncwarp();
        return ab_pass<PASS, true>(v, w, col, wf, tab, qu, lane, wt, T, red);
    }
    if (!EXACT && qu->n) {
        const AbSums fl = ab_flush<PASS>(w, qu, col_s, wf, lane);
#pragma unroll
        for (int k = 0; k < 7; ++k) acc.s[k] += fl.s[k];
    }
    if (PASS != kPassHist) {
        int64_t mine = 0;
#pragma unroll
        for (int k = 0; k < (PASS == kPassPos ? 4 : 7); ++k) {
            const int64_t t = warp_sum_i64(acc.s[k]);
            mine = lane == k ? t : mine;
        }
        if (lane < (PASS == kPassPos ? 4 : 7)) red[lane] = mine;
    }
    return PASS == kPassHist ? acc.s[0] : 0;
}

struct AbJob {
    VolDesc vol;
    const int32_t *seeds;
    const double *cx, *cH;         // given candidates (x, H), or null: seed x radius items
    int64_t n_seeds;
    int r_min, S, max_iter;
    int S_team;                    // radii taken by a whole block: ri >= S - S_team
    ks_abmsod_result *out;
    unsigned long long *tickets;   // [0]: block items, [1]: warp items
    int *status;
};

// Item state (the team leader's copy is the team's).
struct AbState {
    double x[3], H[6];     // current centre and bandwidth
    double xn[3], Hn[6];   // this iteration's update
    double xo[3], Ho[6];   // best so far
    double best;
    double rho;            // this iteration's rho at x'
};

// Per-warp shared memory.
struct __align__(16) AbWarpMem {
    AbRow tab[32];         // this warp's row table
    AbQueue qu;            // this warp's voxels left to the exact membership test
    AbState st;            // item state (leader's copy)
    AbWinS win;            // current window (leader's copy)
    int flag;              // leader -> team: 0 go on, 1 leave the loop, 2 stopped
    int pad;
    int64_t nv;            // this warp's window voxels of the item
    int64_t P[kMaxBins];   // this warp's per-bin sums of the last histogram
    int64_t red[8];        // this warp's pass sums
    float wf[kMaxBins];    // weights (leader's copy)
};

template <int T>
__device__ __forceinline__ void team_sync() {
    if (T == 1)
        __syncwarp();
    else
        __syncthreads();
}

// Histogram pass of one warp: the lane columns are summed (and cleared)
// into mine->P[b] for bins b = lane, lane + 32; returns this lane's window
// voxels.
__device__ __forceinline__ int64_t ab_hist_part(const VolDesc &v, const AbWinS &w, uint32_t *cols,
                                                AbRow *tab, int lane, int wt, int T, int B,
                                                AbWarpMem *mine) {
    const int64_t nv = ab_pass<kPassHist, false>(v, w, cols + lane, nullptr, tab, &mine->qu,
                                                 lane, wt, T, nullptr);
    __syncwarp();
    int64_t P0 = 0, P1 = 0;
    if (lane < B) {
        uint32_t *c = cols + lane * 32;
        for (int l = 0; l < 32; ++l) {
            const int j = (l + lane) & 31;
            P0 += c[j];
            c[j] = 0u;
        }
        mine->P[lane] = P0;
    }
    if (lane + 32 < B) {
        uint32_t *c = cols + (lane + 32) * 32;
        for (int l = 0; l < 32; ++l) {
            const int j = (l + lane) & 31;
            P1 += c[j];
            c[j] = 0u;
        }
        mine->P[lane + 32] = P1;
    }
    return nv;
}

// Leader: team totals P_b (bins lane, lane + 32), K, binary32 weights
// w_b = sqrt(K / (B P_b)) times the power of two `scale` (exact: the sums
// passes fold their fixed-point scale into the weight) into lead->wf and,
// when want_rho, rho =
// (sum_b sqrt(P_b)) / sqrt(B K) with the bins paired (b, b + 32) and then
// summed by a butterfly (the pairwise tree of the definition).  Returns K.
__device__ __forceinline__ int64_t ab_bins(AbWarpMem *team, int T, int lane, int B, bool want_rho,
                                           float scale, double &rho) {
    AbWarpMem *lead = team;
    int64_t P0 = 0, P1 = 0;
    for (int t = 0; t < T; ++t) {
        if (lane < B) P0 += team[t].P[lane];
        if (lane + 32 < B) P1 += team[t].P[lane + 32];
    }
    const int64_t K = warp_sum_i64(P0 + P1);
    rho = 0.0;
    if (K > 0) {
        const float Kf = __ll2float_rn(K), Bf = (float)B;
        if (lane < B)
            lead->wf[lane] = P0 > 0 ? __fmul_rn(__fsqrt_rn(__fdiv_rn(Kf, __fmul_rn(Bf, __ll2float_rn(P0)))), scale)
                                    : 0.0f;
        if (lane + 32 < B)
            lead->wf[lane + 32] =
                P1 > 0 ? __fmul_rn(__fsqrt_rn(__fdiv_rn(Kf, __fmul_rn(Bf, __ll2float_rn(P1)))), scale)
                       : 0.0f;
        if (want_rho) {
            double t = __dadd_rn(P0 > 0 ? __dsqrt_rn((double)P0) : 0.0,
                                 P1 > 0 ? __dsqrt_rn((double)P1) : 0.0);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, m));
            rho = __ddiv_rn(t, __dsqrt_rn(__dmul_rn((double)B, (double)K)));
        }
    }
    return K;
}

// Leader: write a window into lead->win (lane 0).
__device__ __forceinline__ void ab_publish(AbWarpMem *lead, const AbWinS &w, int lane) {
    if (lane == 0) lead->win = w;
}

// One item (seed si, radius index ri; or candidate si) by a team of T
// warps; wt = this warp's index in the team, team = the team's first warp
// memory.
template <int T>
__device__ __forceinline__ void ab_item(const AbJob &J, int64_t si, int ri, AbWarpMem *team,
                                     uint32_t *cols, int wt, int lane) {
    AbWarpMem *lead = team, *mine = team + wt;
    const bool leader = wt == 0;
    const int B = J.vol.B;
    const int r = J.cx ? 0 : J.r_min + ri;
    const int dim[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    AbState *st = &lead->st;
    if (leader) {
        if (J.cx) {
            if (lane < 3) {
                const double c = J.cx[3 * si + lane];
                st->x[lane] = c;
                st->xo[lane] = c;
            }
            if (lane < 6) {
                const double h = J.cH[6 * si + lane];
                st->H[lane] = h;
                st->Ho[lane] = h;
            }
        } else {
            const double r2 = (double)(r * r);
            if (lane < 3) {
                const double c = (double)J.seeds[3 * si + lane];
                st->x[lane] = c;
                st->xo[lane] = c;
            }
            if (lane < 6) {
                const double h = (lane == 0 || lane == 3 || lane == 5) ? r2 : 0.0;
                st->H[lane] = h;
                st->Ho[lane] = h;
            }
        }
        __syncwarp();
        if (lane == 0) {
            st->best = 0.0;
            // a given candidate must lie in the volume with 1 <= H_aa <= 32^2
            // (the window then stays inside the halo); otherwise it is
            // flagged and left at iteration 0
            bool ok = true;
            if (J.cx) {
                for (int a = 0; a < 3; ++a)
                    ok = ok && st->x[a] >= 0.0 && st->x[a] <= (double)(dim[a] - 1);
                for (int k = 0; k < 6; ++k) {
                    const double h = st->H[k];
                    const bool diag = k == 0 || k == 3 || k == 5;
                    ok = ok && (diag ? (h >= 1.0 && h <= kHmax) : fabs(h) <= kHmax);
                }
                if (!ok) atomicOr(J.status, kStatusBadInput);
            }
            lead->flag = ok ? 0 : 1;
        }
    }
    if (lane == 0) mine->nv = 0;
    team_sync<T>();
    const bool skip = lead->flag != 0;
    team_sync<T>();   // the flag is rewritten inside the loop
    int it = 0, stopped = 0;
    // the per-item values live in shared memory across the window passes
    // (the passes are calls; registers held across them would be spilled)
    while (!skip && it < J.max_iter) {
        // window at (x, H)
        if (leader) {
            __syncwarp();
            AbShape sh;
            const bool ok = ab_shape(st->H, sh);
            if (ok) {
                AbWinS w;
                ab_place(st->x, sh, dim, w);
                ab_publish(lead, w, lane);
            }
            if (lane == 0) lead->flag = ok ? 0 : 1;
        }
        team_sync<T>();
        if (lead->flag) break;
        const AbWinS &w = lead->win;   // rewritten only after the next team sync
        {
            const int64_t nv = warp_sum_i64(ab_hist_part(J.vol, w, cols, mine->tab, lane, wt, T, B, mine));
            if (lane == 0) mine->nv += nv;
        }
        team_sync<T>();
        if (leader) {
            double rho;
            const int64_t K = ab_bins(team, T, lane, B, false, lead->win.qx, rho);
            if (lane == 0) lead->flag = K == 0 ? 1 : 0;
        }
        team_sync<T>();
        if (lead->flag) break;
        {
            ab_pass<kPassPos, false>(J.vol, w, nullptr, lead->wf, mine->tab, &mine->qu, lane, wt,
                                     T, mine->red);
        }
        team_sync<T>();
        if (leader) {
            if (lane < 3) {
                int64_t num = 0, den = 0;
                for (int t = 0; t < T; ++t) {
                    num += team[t].red[lane];
                    den += team[t].red[3];
                }
                const int dm = lane == 0 ? dim[0] : (lane == 1 ? dim[1] : dim[2]);
                const double dl = den > 0 ? __ddiv_rn((double)num, (double)den) : 0.0;
                double vv = __dadd_rn(st->x[lane], dl);
                if (vv < 0.0) vv = 0.0;
                if (vv > (double)(dm - 1)) vv = (double)(dm - 1);
                st->xn[lane] = vv;
            }
            __syncwarp();
            AbShape sh;   // the bandwidth part of the current window
#pragma unroll
            for (int k = 0; k < 6; ++k) sh.h[k] = lead->win.h[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) sh.E[a] = lead->win.E[a];
            sh.qx = lead->win.qx;
            sh.qm = lead->win.qm;
            sh.band = lead->win.band;
#pragma unroll
            for (int k = 0; k < 6; ++k) sh.adj[k] = lead->win.adj[k];
            sh.det = lead->win.det;
            __syncwarp();
            AbWinS w2;
            ab_place(st->xn, sh, dim, w2);
            ab_publish(lead, w2, lane);
        }
        team_sync<T>();
        {
            const int64_t nv = warp_sum_i64(ab_hist_part(J.vol, w, cols, mine->tab, lane, wt, T, B, mine));
            if (lane == 0) mine->nv += nv;
        }
        team_sync<T>();
        ++it;
        if (leader) {
            double rho;
            const int64_t K2 = ab_bins(team, T, lane, B, true, lead->win.qm, rho);
            if (lane == 0) {
                lead->flag = K2 == 0 ? 1 : 0;
                st->rho = rho;
            }
        }
        team_sync<T>();
        if (lead->flag) break;
        {
            ab_pass<kPassMom, false>(J.vol, w, nullptr, lead->wf, mine->tab, &mine->qu, lane, wt,
                                     T, mine->red);
        }
        team_sync<T>();
        if (leader) {
            if (lane < 6) {
                int64_t mk = 0, ws = 0;
                for (int t = 0; t < T; ++t) {
                    mk += team[t].red[lane];
                    ws += team[t].red[6];
                }
                // 5 (M 2^-pm) / (W 2^-16) = (5 2^(16 - pm)) M / W
                const double hsc = __dmul_rn(5.0, (double)__fdiv_rn(kQW, lead->win.qm));
                st->Hn[lane] =
                    ws > 0 ? __ddiv_rn(__dmul_rn(hsc, (double)mk), (double)ws) : st->H[lane];
            }
            __syncwarp();
            if (lane == 0) {
                // regularise H'
                double *Hn = st->Hn;
                double m = 0.0;
                const int dg[3] = {0, 3, 5};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Hn[dg[a]] = __dadd_rn(Hn[dg[a]], kVoxel);
                    if (Hn[dg[a]] < 1.0) Hn[dg[a]] = 1.0;
                    if (Hn[dg[a]] > m) m = Hn[dg[a]];
                }
                if (m > kHmax) {
                    const double sc = __ddiv_rn(kHmax, m);
#pragma unroll
                    for (int k = 0; k < 6; ++k) Hn[k] = __dmul_rn(Hn[k], sc);
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (Hn[dg[a]] > kHmax) Hn[dg[a]] = kHmax;
                }
                // best so far; stop at a fall of rho
                const double rho = st->rho;
                const double delta = __dsub_rn(st->best, rho);
                if (rho > st->best) {
                    st->best = rho;
                    for (int a = 0; a < 3; ++a) st->xo[a] = st->xn[a];
                    for (int k = 0; k < 6; ++k) st->Ho[k] = Hn[k];
                }
                if (delta > 0.0) {
                    lead->flag = 2;
                } else {
                    lead->flag = 0;
                    for (int a = 0; a < 3; ++a) st->x[a] = st->xn[a];
                    for (int k = 0; k < 6; ++k) st->H[k] = Hn[k];
                }
            }
        }
        team_sync<T>();
        if (lead->flag) {
            stopped = 1;
            break;
        }
    }
    team_sync<T>();
    if (leader) {
        int64_t nv = 0;
        for (int t = 0; t < T; ++t) nv += team[t].nv;
        ks_abmsod_result &o = J.out[si * J.S + ri];
        if (lane < 3) o.x[lane] = st->xo[lane];
        if (lane < 6) o.H[lane] = st->Ho[lane];
        if (lane == 0) {
            o.rho = st->best;
            o.seed = (int32_t)si;
            o.r = r;
            o.iters = it;
            o.stopped = stopped;
            o.voxels = nv;
        }
    }
    team_sync<T>();   // the team's memory is reused by the next item
}

__global__ void __launch_bounds__(kAbWarps * 32, 4) k_abmsod(const __grid_constant__ AbJob J) {
    extern __shared__ __align__(16) uint8_t ab_smem[];
    __shared__ unsigned long long s_ticket;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = J.vol.B;
    // per block: the warps' memories, then per warp B x 32 lane columns
    AbWarpMem *mems = reinterpret_cast<AbWarpMem *>(ab_smem);
    uint32_t *cols = reinterpret_cast<uint32_t *>(ab_smem + kAbWarps * sizeof(AbWarpMem)) +
                     (size_t)wid * B * 32;
    for (int i = lane; i < B * 32; i += 32) cols[i] = 0u;
    if (lane == 0) mems[wid].qu.n = 0;
    __syncwarp();
    const int64_t ns = J.n_seeds;
    // block items: radii index S - S_team .. S - 1, largest first
    const int64_t n_team = ns * J.S_team;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&J.tickets[0], 1ull);
        __syncthreads();
        const int64_t tk = (int64_t)s_ticket;
        __syncthreads();
        if (tk >= n_team) break;
        ab_item<kAbWarps>(J, tk % ns, J.S - 1 - (int)(tk / ns), mems, cols, wid, lane);
    }
    // warp items: radii index 0 .. S - S_team - 1, largest first
    const int S_warp = J.S - J.S_team;
    const int64_t n_warp = ns * S_warp;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(&J.tickets[1], 1ull);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if ((int64_t)tk >= n_warp) break;
        ab_item<1>(J, (int64_t)tk % ns, S_warp - 1 - (int)((int64_t)tk / ns), mems + wid, cols, 0,
                   lane);
    }
}

}  // namespace

size_t abmsod_smem_bytes(int B) {
    return kAbWarps * sizeof(AbWarpMem) + (size_t)kAbWarps * B * 32 * 4;
}

cudaError_t launch_abmsod(const LaunchCtx &lc, const VolDesc &v, const int32_t *seeds,
                          const double *cx, const double *cH, int64_t n_seeds, int r_min,
                          int r_max, int max_iter, int r_team, int r_auto, ks_abmsod_result *out,
                          unsigned long long *tickets) {
    if (cx) {            // candidates: one item each
        r_min = 0;
        r_max = 0;
    }
    const int S = r_max - r_min + 1;
    const int64_t n_items = n_seeds * S;
    if (n_items == 0) return cudaSuccess;
    // byte offsets inside a window's box are 32-bit
    if (v.plane * (2 * kHalo + 2) >= (int64_t)1 << 31) return cudaErrorInvalidValue;
    const size_t smem = abmsod_smem_bytes(v.B);
    cudaError_t e = cudaFuncSetAttribute(k_abmsod, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_abmsod, kAbWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t warps = (int64_t)lc.num_sms * per_sm * kAbWarps;
    int S_team;
    if (cx) {            // all candidates on blocks or all on warps
        S_team = r_team > kRmax ? 0 : (r_team > 0 || n_items < 4 * warps ? 1 : 0);
    } else {
        if (r_team <= 0) r_team = n_items < 4 * warps ? r_auto : kRmax + 1;
        S_team = std::min(S, std::max(0, r_max - r_team + 1));
    }
    const int64_t want = n_seeds * S_team + (n_seeds * (S - S_team) + kAbWarps - 1) / kAbWarps;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)lc.num_sms * per_sm);
    e = cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned long long), lc.stream);
    if (e != cudaSuccess) return e;
    AbJob J;
    J.vol = v;
    J.seeds = seeds;
    J.cx = cx;
    J.cH = cH;
    J.n_seeds = n_seeds;
    J.r_min = r_min;
    J.S = S;
    J.max_iter = max_iter;
    J.S_team = S_team;
    J.out = out;
    J.tickets = tickets;
    J.status = lc.d_status;
    k_abmsod<<<grid, kAbWarps * 32, smem, lc.stream>>>(J);
    return cudaGetLastError();
}

}  // namespace ks
