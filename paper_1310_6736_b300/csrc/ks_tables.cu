// FP64 lookup tables of the entropy step: T[c] = c ln c and L[n] = ln n,
// each the binary64 value nearest to the exact real number.
//
// The logarithm is evaluated on the device in double-double arithmetic
// (about 104 bits), with the error-free transformations of Dekker (1971)
// and Knuth (TAOCP vol. 2) as arranged by Hida, Li and Bailey's QD library
// (2001), then rounded once to binary64:
//   c = 2^e * m with m in [0.75, 1.5)
//   ln m = 2 atanh(u) = 2 (u + u^3/3 + u^5/5 + ...),  u = (m-1)/(m+1),
//          |u| <= 0.2, 26 terms (u^52 / 53 < 2^-120)
//   ln c = e ln 2 + ln m,  ln 2 as a double-double constant
// The result is the correctly rounded value unless the exact value lies
// within about 2^-98 (relative) of a rounding midpoint.
#include "ks_internal.cuh"

namespace ks {
namespace {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    const dd t = two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo = __dadd_rn(p.lo, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo = __dadd_rn(p.lo, __dmul_rn(a.lo, b));
    return quick_two_sum(p.hi, p.lo);
}
// a / b for doubles a, b, to double-double accuracy (long division: the
// remainder of each quotient digit is exact through one FMA).
__device__ __forceinline__ dd dd_div_dd_d(dd a, double b) {
    const double q1 = __ddiv_rn(a.hi, b);
    const dd p = two_prod(q1, b);
    const double r = __dadd_rn(__dsub_rn(__dsub_rn(a.hi, p.hi), p.lo), a.lo);
    const double q2 = __ddiv_rn(r, b);
    return quick_two_sum(q1, q2);
}

__device__ dd dd_log_int(int64_t c) {
    // c >= 2.  Exponent e and mantissa m = c / 2^e in [0.75, 1.5).
    int e = 63 - __clzll((unsigned long long)c);
    double m = ldexp((double)c, -e);          // [1, 2), exact
    if (m >= 1.5) {
        m = __dmul_rn(m, 0.5);
        e += 1;
    }
    // u = (m - 1) / (m + 1); both operands are exact doubles.
    const dd u = dd_div_dd_d({__dsub_rn(m, 1.0), 0.0}, __dadd_rn(m, 1.0));
    const dd u2 = dd_mul(u, u);
    // Horner for sum_{k=0}^{K} u2^k / (2k+1).
    constexpr int K = 26;
    dd s = dd_div_dd_d({1.0, 0.0}, (double)(2 * K + 1));
    for (int k = K - 1; k >= 0; --k)
        s = dd_add(dd_mul(s, u2), dd_div_dd_d({1.0, 0.0}, (double)(2 * k + 1)));
    dd lnm = dd_mul(u, s);
    lnm.hi = __dmul_rn(lnm.hi, 2.0);
    lnm.lo = __dmul_rn(lnm.lo, 2.0);
    const dd ln2 = {0x1.62e42fefa39efp-1, 0x1.abc9e3b39803fp-56};
    return dd_add(dd_mul_d(ln2, (double)e), lnm);
}

__global__ void k_tables(double *__restrict__ T, double *__restrict__ L, int64_t n) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= n;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c <= 1) {
            T[c] = 0.0;
            L[c] = 0.0;
            continue;
        }
        const dd l = dd_log_int(c);
        L[c] = __dadd_rn(l.hi, l.lo);
        const dd t = dd_mul_d(l, (double)c);
        T[c] = __dadd_rn(t.hi, t.lo);
    }
}

}  // namespace

cudaError_t launch_tables(const LaunchCtx &lc, double *T, double *L, int64_t n) {
    const int threads = 256;
    const int blocks = (int)((n + threads) / threads);
    k_tables<<<blocks, threads, 0, lc.stream>>>(T, L, n);
    return cudaGetLastError();
}

}  // namespace ks
