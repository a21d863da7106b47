// Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 7) towards
// the uniform target pmf HQ_b = 1/B.
//
// One warp per (seed, r) item, drawn from a persistent ticket queue with
// the largest starting radius first.  An iteration makes four passes over
// the voxel box of the current ellipsoid { s : (s-x)^T H^-1 (s-x) <= 1 }:
//   1. kernel histogram at (x, H) -> w_b = sqrt(HQ_b / HP_b)
//   2. Eq. 6 sums  sum k w o, sum k w            -> x'
//   3. kernel histogram at (x', H) -> w'_b, rho = sum_b sqrt(HQ_b HP'_b)
//   4. Eq. 7 sums  sum w' o o^T, sum w'         -> H' = 5 (M / sum w' + I/12)
// The lanes walk the box in linear order, 32 voxels at a time.  Per-voxel
// terms are binary32 in one fixed operation order; every sum over voxels is
// an exact int64 sum of the terms rounded to nearest on a fixed-point grid
// (2^-16 for k, 2^-12 for the position terms and w', 2^-8 for the second
// moments), so the warp's summation order does not change the result.
// Histogram sums live in lane-private u32 columns in shared memory (no
// atomics, no bank conflicts).  Everything per bin or per item is FP64, one
// IEEE operation at a time, computed redundantly by all lanes so the warp's
// control flow stays uniform.
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

// exp(-d/2) for 0 <= d <= 1 by its Taylor series to degree 9 (Horner form;
// truncation error below 3e-10, under half a binary32 ulp).
__device__ __forceinline__ float ab_kernel(float d) {
    const float t = __fmul_rn(-0.5f, d);
    float p = 2.755731922398589e-06f;
    p = __fadd_rn(__fmul_rn(p, t), 2.48015873015873e-05f);
    p = __fadd_rn(__fmul_rn(p, t), 1.984126984126984e-04f);
    p = __fadd_rn(__fmul_rn(p, t), 0.001388888888888889f);
    p = __fadd_rn(__fmul_rn(p, t), 0.008333333333333333f);
    p = __fadd_rn(__fmul_rn(p, t), 0.041666666666666664f);
    p = __fadd_rn(__fmul_rn(p, t), 0.16666666666666666f);
    p = __fadd_rn(__fmul_rn(p, t), 0.5f);
    p = __fadd_rn(__fmul_rn(p, t), 1.0f);
    p = __fadd_rn(__fmul_rn(p, t), 1.0f);
    return p;
}

// Nearest integer (ties to even) of y as int64.  |y| < 2^22: adding
// 1.5 * 2^23 puts y + 1.5 * 2^23 in [2^23, 2^24), where the binary32 ulp
// is 1, so the addition itself rounds y to an integer; its bit pattern is
// then 0x4B400000 + rint(y).  Larger |y| (rare: heavy rare-bin weights)
// use the 64-bit conversion, which rounds the same way.
__device__ __forceinline__ int64_t ab_q(float y) {
    if (fabsf(y) < 4194304.0f)
        return (int64_t)(__float_as_int(__fadd_rn(y, 12582912.0f)) - 0x4B400000);
    return __float2ll_rn(y);
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A window: H^-1 rounded to binary32, the centre as floor + binary32
// fraction, and the voxel box [lo, lo + ext).
struct AbWin {
    float h[6];
    float f[3];
    int n[3];
    int lo[3];
    int ext[3];
};

// H = (00 01 02 11 12 22).  Returns 0, or 1 when H is not positive definite
// (det <= 0), or 2 when the box would leave the halo (not reachable: the
// centre stays in the volume and every diagonal entry of H is at most 32^2).
__device__ __forceinline__ int ab_setup(const double x[3], const double H[6], const int dim[3], AbWin &w) {
    const double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
    const double c00 = __dsub_rn(__dmul_rn(a11, a22), __dmul_rn(a12, a12));
    const double c01 = __dsub_rn(__dmul_rn(a02, a12), __dmul_rn(a01, a22));
    const double c02 = __dsub_rn(__dmul_rn(a01, a12), __dmul_rn(a02, a11));
    const double c11 = __dsub_rn(__dmul_rn(a00, a22), __dmul_rn(a02, a02));
    const double c12 = __dsub_rn(__dmul_rn(a01, a02), __dmul_rn(a00, a12));
    const double c22 = __dsub_rn(__dmul_rn(a00, a11), __dmul_rn(a01, a01));
    const double det =
        __dadd_rn(__dadd_rn(__dmul_rn(a00, c00), __dmul_rn(a01, c01)), __dmul_rn(a02, c02));
    if (!(det > 0.0)) return 1;
    w.h[0] = __double2float_rn(__ddiv_rn(c00, det));
    w.h[1] = __double2float_rn(__ddiv_rn(c01, det));
    w.h[2] = __double2float_rn(__ddiv_rn(c02, det));
    w.h[3] = __double2float_rn(__ddiv_rn(c11, det));
    w.h[4] = __double2float_rn(__ddiv_rn(c12, det));
    w.h[5] = __double2float_rn(__ddiv_rn(c22, det));
    const double dg[3] = {a00, a11, a22};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(x[a]);
        w.n[a] = (int)fl;
        w.f[a] = __double2float_rn(__dsub_rn(x[a], fl));
        const double e = __dsqrt_rn(dg[a]);
        const int lo = (int)ceil(__dsub_rn(x[a], e));
        const int hi = (int)floor(__dadd_rn(x[a], e));
        w.lo[a] = lo;
        w.ext[a] = hi - lo + 1;
        ok = ok && lo >= -kHalo && hi < dim[a] + kHalo && hi >= lo;
    }
    return ok ? 0 : 2;
}

enum AbPass { kPassHist = 0, kPassPos = 1, kPassMom = 2 };

// Per-pass sums.  Hist: nothing here (columns in shared memory).  Pos:
// s[0..2] = sum q(k w o_a), s[3] = sum q(k w).  Mom: s[0..5] = sum
// q(w (o_a o_b)), s[6] = sum q(w).
struct AbSums {
    int64_t s[7];
};

// One pass of the lanes over the window's box.
template <int PASS>
__device__ __forceinline__ void ab_pass(const VolDesc &v, const AbWin &w, uint32_t *col,
                                        const float *wf, int lane, AbSums &acc) {
#pragma unroll
    for (int k = 0; k < 7; ++k) acc.s[k] = 0;
    const int e0 = w.ext[0], e1 = w.ext[1], e2 = w.ext[2];
    const int total = e0 * e1 * e2;
    // lane's first voxel and the 32-voxel step in (x, y, z)
    int ix = lane % e0;
    int q = lane / e0;
    int iy = q % e1, iz = q / e1;
    const int s0 = 32 % e0, t = 32 / e0, s1 = t % e1, s2 = t / e1;
    const float s0f = (float)s0, s1f = (float)s1, s2f = (float)s2;
    const float e0f = (float)e0, e1f = (float)e1;
    // integer-valued binary32 coordinates s_a - floor(x_a)
    float fx = (float)(w.lo[0] - w.n[0] + ix);
    float fy = (float)(w.lo[1] - w.n[1] + iy);
    float fz = (float)(w.lo[2] - w.n[2] + iz);
    const int64_t pitch = v.pitch, plane = v.plane;
    const uint8_t *p = v.base + (int64_t)(w.lo[2] + iz) * plane + (int64_t)(w.lo[1] + iy) * pitch +
                       (w.lo[0] + ix);
    const int64_t dstep = (int64_t)s2 * plane + (int64_t)s1 * pitch + s0;
    const int64_t xwrap = pitch - e0, ywrap = plane - (int64_t)e1 * pitch;
    const float h0 = w.h[0], h1 = w.h[1], h2 = w.h[2], h3 = w.h[3], h4 = w.h[4], h5 = w.h[5];
    const float f0 = w.f[0], f1 = w.f[1], f2 = w.f[2];
#pragma unroll 1
    for (int idx = lane; idx < total; idx += 32) {
        const int b = __ldg(p);
        if (b) {
            const float o0 = __fsub_rn(fx, f0), o1 = __fsub_rn(fy, f1), o2 = __fsub_rn(fz, f2);
            const float u0 =
                __fadd_rn(__fadd_rn(__fmul_rn(h0, o0), __fmul_rn(h1, o1)), __fmul_rn(h2, o2));
            const float u1 =
                __fadd_rn(__fadd_rn(__fmul_rn(h1, o0), __fmul_rn(h3, o1)), __fmul_rn(h4, o2));
            const float u2 =
                __fadd_rn(__fadd_rn(__fmul_rn(h2, o0), __fmul_rn(h4, o1)), __fmul_rn(h5, o2));
            const float d =
                __fadd_rn(__fadd_rn(__fmul_rn(o0, u0), __fmul_rn(o1, u1)), __fmul_rn(o2, u2));
            if (d >= 0.0f && d <= 1.0f) {   // d < 0: rounding of a near-singular H^-1
                if (PASS == kPassHist) {
                    const uint32_t kq = (uint32_t)ab_q(__fmul_rn(ab_kernel(d), kQK));
                    col[(b - 1) * 32] += kq;
                } else if (PASS == kPassPos) {
                    const float tk = __fmul_rn(ab_kernel(d), wf[b - 1]);
                    acc.s[0] += ab_q(__fmul_rn(__fmul_rn(tk, o0), kQX));
                    acc.s[1] += ab_q(__fmul_rn(__fmul_rn(tk, o1), kQX));
                    acc.s[2] += ab_q(__fmul_rn(__fmul_rn(tk, o2), kQX));
                    acc.s[3] += ab_q(__fmul_rn(tk, kQX));
                } else {
                    const float tw = wf[b - 1];
                    acc.s[0] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, o0)), kQH));
                    acc.s[1] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, o1)), kQH));
                    acc.s[2] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o0, o2)), kQH));
                    acc.s[3] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o1, o1)), kQH));
                    acc.s[4] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o1, o2)), kQH));
                    acc.s[5] += ab_q(__fmul_rn(__fmul_rn(tw, __fmul_rn(o2, o2)), kQH));
                    acc.s[6] += ab_q(__fmul_rn(tw, kQX));
                }
            }
        }
        // advance 32 voxels in linear box order
        ix += s0;
        iy += s1;
        iz += s2;
        fx = __fadd_rn(fx, s0f);
        fy = __fadd_rn(fy, s1f);
        fz = __fadd_rn(fz, s2f);
        p += dstep;
        if (ix >= e0) {
            ix -= e0;
            fx = __fsub_rn(fx, e0f);
            ++iy;
            fy = __fadd_rn(fy, 1.0f);
            p += xwrap;
        }
        if (iy >= e1) {
            iy -= e1;
            fy = __fsub_rn(fy, e1f);
            ++iz;
            fz = __fadd_rn(fz, 1.0f);
            p += ywrap;
        }
    }
    if (PASS != kPassHist) {
#pragma unroll
        for (int k = 0; k < 7; ++k) acc.s[k] = warp_sum_i64(acc.s[k]);
    }
}

// Histogram pass + per-bin step: P_b from the lane columns (read and
// cleared), K = sum P_b, weights wf_b = (float) sqrt(HQ / (P_b / K)) into
// shared memory, and the Bhattacharyya terms sqrt(HQ (P_b / K)) for bins
// lane and lane + 32.  Returns K.
__device__ __forceinline__ int64_t ab_hist(const VolDesc &v, const AbWin &w, uint32_t *cols,
                                           float *wf, int lane, int B, double &bt0, double &bt1) {
    AbSums dummy;
    ab_pass<kPassHist>(v, w, cols + lane, nullptr, lane, dummy);
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
    const double hq = __ddiv_rn(1.0, (double)B);
    bt0 = 0.0;
    bt1 = 0.0;
    if (K > 0) {
        const double dK = (double)K;
        if (lane < B) {
            float wv = 0.0f;
            if (P0 > 0) {
                const double hp = __ddiv_rn((double)P0, dK);
                wv = __double2float_rn(__dsqrt_rn(__ddiv_rn(hq, hp)));
                bt0 = __dsqrt_rn(__dmul_rn(hq, hp));
            }
            wf[lane] = wv;
        }
        if (lane + 32 < B) {
            float wv = 0.0f;
            if (P1 > 0) {
                const double hp = __ddiv_rn((double)P1, dK);
                wv = __double2float_rn(__dsqrt_rn(__ddiv_rn(hq, hp)));
                bt1 = __dsqrt_rn(__dmul_rn(hq, hp));
            }
            wf[lane + 32] = wv;
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

__device__ __forceinline__ bool ab_setup_or_flag(const double *x, const double *H,
                                                 const int dim[3], AbWin &w, int lane,
                                                 int *status) {
    const int st = ab_setup(x, H, dim, w);
    if (st == 2 && lane == 0) atomicOr(status, kStatusBadInput);
    return st == 0;
}

__global__ void __launch_bounds__(kAbWarps * 32, 4) k_abmsod(const AbJob J) {
    extern __shared__ __align__(16) uint32_t ab_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = J.vol.B;
    // per warp: its state, B x 32 lane columns, then B weights
    AbState *stt = reinterpret_cast<AbState *>(ab_smem) + wid;
    uint32_t *cols = ab_smem + (kAbWarps * sizeof(AbState)) / 4 + (size_t)wid * (B * 32 + B);
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
        while (it < J.max_iter) {
            AbWin w;
            if (!ab_setup_or_flag(stt->x, stt->H, dim, w, lane, J.status)) break;
            double bt0, bt1;
            const int64_t K = ab_hist(J.vol, w, cols, wf, lane, B, bt0, bt1);
            if (K == 0) break;
            {
                AbSums sp;
                ab_pass<kPassPos>(J.vol, w, nullptr, wf, lane, sp);
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
            if (!ab_setup_or_flag(stt->xn, stt->H, dim, w, lane, J.status)) break;
            const int64_t K2 = ab_hist(J.vol, w, cols, wf, lane, B, bt0, bt1);
            ++it;
            if (K2 == 0) break;
            {
                AbSums sm;
                ab_pass<kPassMom>(J.vol, w, nullptr, wf, lane, sm);
                int64_t mk = sm.s[0];
#pragma unroll
                for (int k = 1; k < 6; ++k) mk = lane == k ? sm.s[k] : mk;
                if (lane < 6)
                    stt->Hn[lane] =
                        sm.s[6] > 0 ? __ddiv_rn(__dmul_rn(5.0, __ddiv_rn((double)mk, 256.0)),
                                                __ddiv_rn((double)sm.s[6], 4096.0))
                                    : stt->H[lane];
            }
            __syncwarp();
            // regularise H' (lane 0), rho at x' in bin order (every lane)
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
            double bh = 0.0;
            for (int b = 0; b < B; ++b) {
                const double tb = __shfl_sync(0xffffffffu, b < 32 ? bt0 : bt1, b & 31);
                bh = __dadd_rn(bh, tb);
            }
            __syncwarp();
            const double best = stt->best;
            const double delta = __dsub_rn(best, bh);
            const bool better = bh > best;
            __syncwarp();
            if (better) {
                if (lane < 3) stt->xo[lane] = stt->xn[lane];
                if (lane < 6) stt->Ho[lane] = stt->Hn[lane];
                if (lane == 0) stt->best = bh;
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
        ks_abmsod_result &o = J.out[si * J.S + ri];
        if (lane < 3) o.x[lane] = stt->xo[lane];
        if (lane < 6) o.H[lane] = stt->Ho[lane];
        if (lane == 0) {
            o.rho = stt->best;
            o.seed = (int32_t)si;
            o.r = r;
            o.iters = it;
            o.stopped = stopped;
        }
        __syncwarp();
    }
}

}  // namespace

size_t abmsod_smem_bytes(int B) {
    return kAbWarps * sizeof(AbState) + (size_t)kAbWarps * (B * 32 + B) * 4;
}

cudaError_t launch_abmsod(const LaunchCtx &lc, const VolDesc &v, const int32_t *seeds,
                          int64_t n_seeds, int r_min, int r_max, int max_iter,
                          ks_abmsod_result *out, unsigned long long *ticket) {
    const int S = r_max - r_min + 1;
    const int64_t n_items = n_seeds * S;
    if (n_items == 0) return cudaSuccess;
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
