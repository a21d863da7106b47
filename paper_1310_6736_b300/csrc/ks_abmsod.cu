// Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 7) towards
// the uniform target pmf HQ_b = 1/B.
//
// One warp per (seed, r) item, drawn from a persistent ticket queue with
// the largest starting radius first.  An iteration makes four passes over
// the voxels of the current ellipsoid { s : (s-x)^T H^-1 (s-x) <= 1 }:
//   1. kernel histogram at (x, H) -> w_b = sqrt(HQ_b / HP_b)
//   2. Eq. 6 sums  sum k w o, sum k w            -> x'
//   3. kernel histogram at (x', H) -> w'_b, rho = sum_b sqrt(HQ_b HP'_b)
//   4. Eq. 7 sums  sum w' o o^T, sum w'         -> H' = 5 (M / sum w' + I/12)
// A pass takes the bounding box's x-rows 32 at a time: lane j finds row j's
// span (the root interval of d <= 1 + 1/16 along x), a warp scan packs the
// spans end to end, and the lanes then walk the packed voxels 32 at a time;
// each lane finds its row from a 32-bit mask of the row starts in its step
// (one warp OR-reduction) and a per-warp table of the batch's rows.
// Per-voxel terms are binary32 in one fixed operation order; every sum over
// voxels is an exact int64 sum of the terms rounded to nearest on a
// fixed-point grid (2^-16 for k, 2^-12 for the position terms and w', 2^-8
// for the second moments), so the warp's summation order does not change
// the result.  Histogram sums live in lane-private u32 columns in shared
// memory (no atomics, no bank conflicts).  Everything per bin or per item is
// FP64, one IEEE operation at a time, computed redundantly by all lanes so
// the warp's control flow stays uniform.
#include <algorithm>

#include "ks_internal.cuh"

namespace ks {

namespace {

constexpr int kAbWarps = 8;                 // warps per block, one item each
constexpr float kQK = 65536.0f;             // 2^16: kernel values
constexpr float kQX = 4096.0f;              // 2^12: position terms, weights
constexpr float kQH = 256.0f;               // 2^8: second moments
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

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The bandwidth part of a window: H^-1 rounded to binary32 (adjugate times
// 1/det in FP64) and the box half-widths sqrt(H_aa).  Returns false when H
// is not positive definite (det <= 0).
struct AbShape {
    float h[6];
    double e[3];
};
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
    const double inv = __ddiv_rn(1.0, det);
    sh.h[0] = __double2float_rn(__dmul_rn(c00, inv));
    sh.h[1] = __double2float_rn(__dmul_rn(c01, inv));
    sh.h[2] = __double2float_rn(__dmul_rn(c02, inv));
    sh.h[3] = __double2float_rn(__dmul_rn(c11, inv));
    sh.h[4] = __double2float_rn(__dmul_rn(c12, inv));
    sh.h[5] = __double2float_rn(__dmul_rn(c22, inv));
    sh.e[0] = __dsqrt_rn(a00);
    sh.e[1] = __dsqrt_rn(a11);
    sh.e[2] = __dsqrt_rn(a22);
    return true;
}

// The centre part: floor(x), frac(x) rounded to binary32, and the voxel box
// [lo, hi].  Returns false when the box would leave the halo (not reachable:
// the centre stays in the volume and every diagonal entry of H is at most
// 32^2).
struct AbWin {
    int n[3];
    float f[3];
    int lo[3], hi[3];
};
__device__ __forceinline__ bool ab_place(const double x[3], const AbShape &sh, const int dim[3],
                                         AbWin &w) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(x[a]);
        w.n[a] = (int)fl;
        w.f[a] = __double2float_rn(__dsub_rn(x[a], fl));
        w.lo[a] = (int)ceil(__dsub_rn(x[a], sh.e[a]));
        w.hi[a] = (int)floor(__dadd_rn(x[a], sh.e[a]));
        ok = ok && w.lo[a] >= -kHalo && w.hi[a] < dim[a] + kHalo && w.hi[a] >= w.lo[a];
    }
    return ok;
}

enum AbPass { kPassHist = 0, kPassPos = 1, kPassMom = 2 };

// Per-pass sums.  Hist: s[0] = window voxels of this lane (the sums live in
// shared memory).  Pos: s[0..2] = sum q(k w o_a), s[3] = sum q(k w).  Mom:
// s[0..5] = sum q(w (o_a o_b)), s[6] = sum q(w).
struct AbSums {
    int64_t s[7];
};

// One row of a batch, in the warp's table: where its voxels start in the
// packed order, its first voxel's byte offset from the pass base, the
// binary32 value of its first j = s_x - floor(x_x), and its (o_y, o_z).
struct AbRow {
    int start, off;
    float fj, o1;
    float o2, pad0, pad1, pad2;
};

// One pass of the warp over the window's voxels.
template <int PASS>
__device__ __forceinline__ void ab_pass(const VolDesc &v, const AbShape &sh, const AbWin &w,
                                        uint32_t *col, const float *wf, AbRow *tab, int lane,
                                        AbSums &acc) {
#pragma unroll
    for (int k = 0; k < 7; ++k) acc.s[k] = 0;
    const float h0 = sh.h[0], h1 = sh.h[1], h2 = sh.h[2], h3 = sh.h[3], h4 = sh.h[4],
                h5 = sh.h[5];
    const float f0 = w.f[0], f1 = w.f[1], f2 = w.f[2];
    const int e1 = w.hi[1] - w.lo[1] + 1;
    const int nrows = e1 * (w.hi[2] - w.lo[2] + 1);
    const float jlo = (float)(w.lo[0] - w.n[0]), jhi = (float)(w.hi[0] - w.n[0]);
    const int pitch = (int)v.pitch, plane = (int)v.plane;
    // byte offsets below are relative to voxel (n_x, lo_y, lo_z)
    const uint8_t *base = v.base + (int64_t)w.lo[2] * v.plane + (int64_t)w.lo[1] * v.pitch + w.n[0];
    // lane's row (iy, iz) and the 32-row step
    int iy = lane % e1, iz = lane / e1;
    const int dy = 32 % e1, dz = 32 / e1;
    const unsigned lt = (1u << lane) - 1u;
    for (int rb = 0; rb < nrows; rb += 32) {
        int len = 0, ja = 0, off = 0;
        float o1 = 0.0f, o2 = 0.0f;
        if (rb + lane < nrows) {
            o1 = __fsub_rn((float)(w.lo[1] + iy - w.n[1]), f1);
            o2 = __fsub_rn((float)(w.lo[2] + iz - w.n[2]), f2);
            const float beta = __fadd_rn(__fmul_rn(h1, o1), __fmul_rn(h2, o2));
            const float gamma = __fadd_rn(
                __fmul_rn(__fadd_rn(__fmul_rn(h3, o1), __fmul_rn(__fmul_rn(2.0f, h4), o2)), o1),
                __fmul_rn(__fmul_rn(h5, o2), o2));
            const float disc =
                __fsub_rn(__fmul_rn(beta, beta), __fmul_rn(h0, __fsub_rn(gamma, kSlack)));
            if (disc >= 0.0f) {
                const float sq = __fsqrt_rn(disc);
                const float ulo = __fdiv_rn(__fsub_rn(-beta, sq), h0);
                const float uhi = __fdiv_rn(__fsub_rn(sq, beta), h0);
                const float a = fmaxf(ceilf(__fadd_rn(ulo, f0)), jlo);
                const float b = fminf(floorf(__fadd_rn(uhi, f0)), jhi);
                if (a <= b) {
                    ja = (int)a;
                    len = (int)b - ja + 1;
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
            rw.off = off;
            rw.fj = (float)ja;
            rw.o1 = o1;
            rw.o2 = o2;
        }
        __syncwarp();
        int before = 0;   // nonempty rows that start before this step
        for (int p0 = 0; p0 < total; p0 += 32) {
            const unsigned m = __reduce_or_sync(
                0xffffffffu, (len > 0 && start >= p0 && start < p0 + 32) ? 1u << (start - p0) : 0u);
            const int p = p0 + lane;
            if (p < total) {
                const int k = before + __popc(m & (lt | (1u << lane))) - 1;
                const AbRow &rw = tab[k];
                const int kk = p - rw.start;
                const int b = __ldg(base + rw.off + kk);
                if (b) {
                    const float o0 = __fsub_rn(__fadd_rn(rw.fj, (float)kk), f0);
                    const float r1 = rw.o1, r2 = rw.o2;
                    const float u0 = __fadd_rn(__fadd_rn(__fmul_rn(h0, o0), __fmul_rn(h1, r1)),
                                               __fmul_rn(h2, r2));
                    const float u1 = __fadd_rn(__fadd_rn(__fmul_rn(h1, o0), __fmul_rn(h3, r1)),
                                               __fmul_rn(h4, r2));
                    const float u2 = __fadd_rn(__fadd_rn(__fmul_rn(h2, o0), __fmul_rn(h4, r1)),
                                               __fmul_rn(h5, r2));
                    const float d = __fadd_rn(__fadd_rn(__fmul_rn(o0, u0), __fmul_rn(r1, u1)),
                                              __fmul_rn(r2, u2));
                    if (d >= 0.0f && d <= 1.0f) {
                        if (PASS == kPassHist) {
                            col[(b - 1) * 32] += (uint32_t)ab_rint_small(__fmul_rn(ab_kernel(d), kQK));
                            acc.s[0] += 1;
                        } else if (PASS == kPassPos) {
                            const float tk = __fmul_rn(ab_kernel(d), wf[b - 1]);
                            acc.s[0] += ab_q(__fmul_rn(__fmul_rn(tk, o0), kQX));
                            acc.s[1] += ab_q(__fmul_rn(__fmul_rn(tk, r1), kQX));
                            acc.s[2] += ab_q(__fmul_rn(__fmul_rn(tk, r2), kQX));
                            acc.s[3] += ab_q(__fmul_rn(tk, kQX));
                        } else {
                            const float tw = wf[b - 1];
                            acc.s[0] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, o0)), kQH));
                            acc.s[1] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, r1)), kQH));
                            acc.s[2] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, r2)), kQH));
                            acc.s[3] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(r1, r1)), kQH));
                            acc.s[4] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(r1, r2)), kQH));
                            acc.s[5] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(r2, r2)), kQH));
                            acc.s[6] += ab_q(__fmul_rn(tw, kQX));
                        }
                    }
                }
            }
            before += __popc(m);
        }
        __syncwarp();   // the table is rewritten by the next batch
    }
    if (PASS != kPassHist) {
#pragma unroll
        for (int k = 0; k < 7; ++k) acc.s[k] = warp_sum_i64(acc.s[k]);
    }
}

// Histogram pass + per-bin step (adds this lane's window voxels to nvox):
// P_b from the lane columns (read and cleared), K = sum P_b, weights
// wf_b = (float) sqrt(K / (B P_b)) into shared memory, and, when want_rho,
// rho = (sum_b sqrt(P_b)) / sqrt(B K) with the bins paired (b, b + 32) and
// then summed by a butterfly (the pairwise tree of the definition).
// Returns K.
__device__ __forceinline__ int64_t ab_hist(const VolDesc &v, const AbShape &sh, const AbWin &w,
                                           uint32_t *cols, float *wf, AbRow *tab, int lane,
                                           int B, bool want_rho, double &rho, int64_t &nvox) {
    AbSums cnt;
    ab_pass<kPassHist>(v, sh, w, cols + lane, nullptr, tab, lane, cnt);
    nvox += cnt.s[0];
    __syncwarp();
    int64_t P0 = 0, P1 = 0;
    if (lane < B) {
        uint32_t *c = cols + lane * 32;
        for (int l = 0; l < 32; ++l) {
            const int j = (l + lane) & 31;
            P0 += c[j];
            c[j] = 0u;
        }
    }
    if (lane + 32 < B) {
        uint32_t *c = cols + (lane + 32) * 32;
        for (int l = 0; l < 32; ++l) {
            const int j = (l + lane) & 31;
            P1 += c[j];
            c[j] = 0u;
        }
    }
    const int64_t K = warp_sum_i64(P0 + P1);
    rho = 0.0;
    if (K > 0) {
        const double dK = (double)K, dB = (double)B;
        if (lane < B)
            wf[lane] = P0 > 0 ? __double2float_rn(__dsqrt_rn(__ddiv_rn(dK, __dmul_rn(dB, (double)P0))))
                              : 0.0f;
        if (lane + 32 < B)
            wf[lane + 32] =
                P1 > 0 ? __double2float_rn(__dsqrt_rn(__ddiv_rn(dK, __dmul_rn(dB, (double)P1))))
                       : 0.0f;
        if (want_rho) {
            double t = __dadd_rn(P0 > 0 ? __dsqrt_rn((double)P0) : 0.0,
                                 P1 > 0 ? __dsqrt_rn((double)P1) : 0.0);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, m));
            rho = __ddiv_rn(t, __dsqrt_rn(__dmul_rn(dB, dK)));
        }
    }
    __syncwarp();
    return K;
}

struct AbJob {
    VolDesc vol;
    const int32_t *seeds;
    int64_t n_seeds;
    int r_min, S, max_iter;
    ks_abmsod_result *out;
    unsigned long long *ticket;
    int *status;
};

// Per-warp item state in shared memory (keeps the FP64 state out of the
// registers of the voxel passes).  Every lane writes the same values.
struct AbState {
    double x[3], H[6];     // current centre and bandwidth
    double xn[3], Hn[6];   // this iteration's update
    double xo[3], Ho[6];   // best so far
    double best;
};

constexpr size_t kAbFixedBytes = kAbWarps * (sizeof(AbState) + 32 * sizeof(AbRow));

__global__ void __launch_bounds__(kAbWarps * 32, 4) k_abmsod(const AbJob J) {
    extern __shared__ __align__(16) uint32_t ab_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = J.vol.B;
    // per block: the warps' states, their row tables, then per warp B x 32
    // lane columns and B weights
    AbState *stt = reinterpret_cast<AbState *>(ab_smem) + wid;
    AbRow *tab = reinterpret_cast<AbRow *>(ab_smem + kAbWarps * sizeof(AbState) / 4) + wid * 32;
    uint32_t *cols = ab_smem + kAbFixedBytes / 4 + (size_t)wid * (B * 32 + B);
    float *wf = reinterpret_cast<float *>(cols + B * 32);
    for (int i = lane; i < B * 32; i += 32) cols[i] = 0u;
    __syncwarp();
    const int dim[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    const int64_t n_items = J.n_seeds * J.S;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(J.ticket, 1ull);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if ((int64_t)tk >= n_items) break;
        // largest radius first
        const int ri = J.S - 1 - (int)((int64_t)tk / J.n_seeds);
        const int64_t si = (int64_t)tk % J.n_seeds;
        const int r = J.r_min + ri;
        const double r2 = (double)(r * r);
        if (lane < 3) {
            const double c = (double)J.seeds[3 * si + lane];
            stt->x[lane] = c;
            stt->xo[lane] = c;
        }
        if (lane < 6) {
            const double h = (lane == 0 || lane == 3 || lane == 5) ? r2 : 0.0;
            stt->H[lane] = h;
            stt->Ho[lane] = h;
        }
        if (lane == 0) stt->best = 0.0;
        __syncwarp();
        int it = 0, stopped = 0;
        int64_t nvox = 0;
        while (it < J.max_iter) {
            AbShape sh;
            if (!ab_shape(stt->H, sh)) break;
            AbWin w;
            if (!ab_place(stt->x, sh, dim, w)) {
                if (lane == 0) atomicOr(J.status, kStatusBadInput);
                break;
            }
            double rho;
            const int64_t K = ab_hist(J.vol, sh, w, cols, wf, tab, lane, B, false, rho, nvox);
            if (K == 0) break;
            {
                AbSums sp;
                ab_pass<kPassPos>(J.vol, sh, w, nullptr, wf, tab, lane, sp);
                if (lane < 3) {
                    const int64_t num = lane == 0 ? sp.s[0] : (lane == 1 ? sp.s[1] : sp.s[2]);
                    const int dm = lane == 0 ? dim[0] : (lane == 1 ? dim[1] : dim[2]);
                    const double dl =
                        sp.s[3] > 0 ? __ddiv_rn((double)num, (double)sp.s[3]) : 0.0;
                    double vv = __dadd_rn(stt->x[lane], dl);
                    if (vv < 0.0) vv = 0.0;
                    if (vv > (double)(dm - 1)) vv = (double)(dm - 1);
                    stt->xn[lane] = vv;
                }
            }
            __syncwarp();   // xn written; wf is rewritten by the next histogram
            if (!ab_place(stt->xn, sh, dim, w)) {
                if (lane == 0) atomicOr(J.status, kStatusBadInput);
                break;
            }
            const int64_t K2 = ab_hist(J.vol, sh, w, cols, wf, tab, lane, B, true, rho, nvox);
            ++it;
            if (K2 == 0) break;
            {
                AbSums sm;
                ab_pass<kPassMom>(J.vol, sh, w, nullptr, wf, tab, lane, sm);
                int64_t mk = sm.s[0];
#pragma unroll
                for (int k = 1; k < 6; ++k) mk = lane == k ? sm.s[k] : mk;
                if (lane < 6)
                    stt->Hn[lane] = sm.s[6] > 0 ? __ddiv_rn(__dmul_rn(80.0, (double)mk),
                                                            (double)sm.s[6])
                                                : stt->H[lane];
            }
            __syncwarp();
            // regularise H' (lane 0)
            if (lane == 0) {
                double *Hn = stt->Hn;
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
            }
            __syncwarp();
            const double best = stt->best;
            const double delta = __dsub_rn(best, rho);
            const bool better = rho > best;
            __syncwarp();
            if (better) {
                if (lane < 3) stt->xo[lane] = stt->xn[lane];
                if (lane < 6) stt->Ho[lane] = stt->Hn[lane];
                if (lane == 0) stt->best = rho;
            }
            if (delta > 0.0) {
                stopped = 1;
                __syncwarp();
                break;
            }
            if (lane < 3) stt->x[lane] = stt->xn[lane];
            if (lane < 6) stt->H[lane] = stt->Hn[lane];
            __syncwarp();
        }
        __syncwarp();
        nvox = warp_sum_i64(nvox);
        ks_abmsod_result &o = J.out[si * J.S + ri];
        if (lane < 3) o.x[lane] = stt->xo[lane];
        if (lane < 6) o.H[lane] = stt->Ho[lane];
        if (lane == 0) {
            o.rho = stt->best;
            o.seed = (int32_t)si;
            o.r = r;
            o.iters = it;
            o.stopped = stopped;
            o.voxels = nvox;
        }
        __syncwarp();
    }
}

}  // namespace

size_t abmsod_smem_bytes(int B) { return kAbFixedBytes + (size_t)kAbWarps * (B * 32 + B) * 4; }

cudaError_t launch_abmsod(const LaunchCtx &lc, const VolDesc &v, const int32_t *seeds,
                          int64_t n_seeds, int r_min, int r_max, int max_iter,
                          ks_abmsod_result *out, unsigned long long *ticket) {
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
    const int64_t want = (n_items + kAbWarps - 1) / kAbWarps;
    const int grid = (int)std::min<int64_t>(want, (int64_t)lc.num_sms * per_sm);
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), lc.stream);
    if (e != cudaSuccess) return e;
    AbJob J;
    J.vol = v;
    J.seeds = seeds;
    J.n_seeds = n_seeds;
    J.r_min = r_min;
    J.S = S;
    J.max_iter = max_iter;
    J.out = out;
    J.ticket = ticket;
    J.status = lc.d_status;
    k_abmsod<<<grid, kAbWarps * 32, smem, lc.stream>>>(J);
    return cudaGetLastError();
}

}  // namespace ks
