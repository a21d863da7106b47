/*
 * ks_abmsod_fixed.c -- TEST INFRASTRUCTURE ONLY.
 *
 * NOT the oracle of record for ABMSOD: that is ko_abmsod in ks_oracle.c,
 * the plain binary64 statement of Alg. 2 and Eq. 7.  This file restates
 * the arithmetic the CUDA kernel is specified to use (binary32 window
 * geometry, a degree-9 polynomial for exp(-d/2), fixed-point voxel sums),
 * so that a regression test can check the kernel against its own stated
 * arithmetic bit for bit.  Its distance from the plain statement is bounded
 * by the tolerance test that compares the kernel with ko_abmsod.
 *
 * Built into libks_oracle.so with ks_oracle.c (gcc -O2 -ffp-contract=off;
 * fmaf below is the C library's correctly rounded fused multiply-add).
 *
 * Steps (the same as ko_abmsod): candidate histogram HP at (x, H), weights
 * w_b = sqrt(HQ_b / HP_b), the Eq. 6 step, HP' at (x', H), H' from Eq. 7
 * read as 5 (M / W + I/12) with the diagonal held in [1, 32^2], rho' and
 * the stop at the first fall of rho.
 *
 * Arithmetic.  The window's voxels are found row by row: for the x-row at
 * offsets (o_y, o_z), d as a function of o_x is the quadratic
 * h00 o_x^2 + 2 beta o_x + gamma, and the row's span is where it is at
 * most 1 + 1/16 (binary32 root formula, the division by h00 done as a
 * product with 1/h00); a voxel of the span is in the window when the
 * exact test of the definition holds, (s - x)^T adj(H) (s - x) <= det H in
 * binary64 (ko_ab_inside; the kernel reaches the same set with a binary32
 * test wherever that cannot differ).  Its kernel weight uses d evaluated
 * along the row in binary32 as (h00 o_x + 2 beta) o_x + gamma with fused
 * multiply-adds (beta and gamma once per row).  The rows are those
 * of the box [floor(x_a) - E_a, floor(x_a) + E_a] clipped to the volume,
 * E_a = ceil(sqrt(H_aa)) in binary32.  Offsets are
 * o_a = (s_a - floor(x_a)) - frac(x_a), frac(x_a) rounded to binary32; H^-1
 * is the adjugate times 1/det in FP64, rounded to binary32; k is the
 * degree-9 Taylor polynomial of exp(-d/2) in Horner form with fused
 * multiply-adds.  Every sum over voxels is an exact int64 sum of terms
 * rounded to nearest (ties to even) on a fixed-point grid, so no result
 * depends on the order of summation: 2^-16 for k and for the weights w' of
 * the bandwidth sums; for the position terms k w o and the second moments
 * w' o o^T the finest grids 2^-px, 2^-pm on which no term of the window
 * of weight below 4 reaches 2^22 (px, pm from the box half-width
 * E = max_a E_a, ko_ab_exp: px = 14, pm = 9 for E = 32; px = 18, pm = 16
 * for E = 2).  Per bin: w_b =
 * sqrt(K / (B P_b)) in binary32 (K, B, P_b rounded to binary32) and
 * sqrt(P_b) in FP64; rho = (sum_b sqrt(P_b)) / sqrt(B K), the sum over 64
 * zero-padded slots as a pairwise tree (slot i + m added to slot i, m = 32,
 * 16, ..., 1); H' = (5 2^(16 - pm)) M / W (= 5 (M 2^-pm) / (W 2^-16)) in
 * FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Stored bin value at (x,y,z), or 0 when the voxel lies outside the volume. */
static inline int ko_at(const uint8_t *bins, int nx, int ny, int nz, int x, int y, int z)
{
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0;
    return bins[((int64_t)z * ny + y) * nx + x];
}

#define AB_QK 65536.0f     /* 2^16: kernel values */
#define AB_QW 65536.0f     /* 2^16: the weights of the bandwidth sums */

/* Grid exponents of a window with box half-width E = max_a E_a: the
 * largest p with 4 (E + 1) 2^p <= 2^22 for the position terms and with
 * 4 (E + 1)^2 2^p <= 2^22 for the second moments (|o_a| <= E + 1; the
 * kernel sums terms of weight k w < 4, resp. w < 4, in int32 per batch of
 * rows, the heavier rare-bin terms in int64). */
static int ko_ab_exp(int E, int mult, int deg)
{
    int64_t m = (int64_t)mult * (E + 1);
    if (deg == 2) m *= (E + 1);
    int p = 0;
    while ((m << (p + 1)) <= ((int64_t)1 << 22)) ++p;
    return p;
}
#define AB_HMAX 1024.0     /* 32^2 */
#define AB_VOXEL (5.0 / 12.0)   /* (n+2) x the second moment of a unit voxel */
#define AB_SLACK 1.0625f   /* the row span covers d <= 1 + 1/16 */

/* exp(-d/2) for 0 <= d <= 1: sum_{k=0..9} t^k / k!, t = -d/2, Horner form
 * with fused multiply-adds.  The truncation error is below 3e-10, under
 * half a binary32 ulp. */
float ko_ab_kernel(float d)
{
    const float c[10] = {1.0f, 1.0f, 0.5f, 0.16666666666666666f, 0.041666666666666664f,
                         0.008333333333333333f, 0.001388888888888889f, 1.984126984126984e-04f,
                         2.48015873015873e-05f, 2.755731922398589e-06f};
    const float t = -0.5f * d;
    float p = c[9];
    for (int k = 8; k >= 0; --k) p = fmaf(p, t, c[k]);
    return p;
}

typedef struct {
    double x[3];
    float h[6];                     /* H^-1 rounded to binary32: 00 01 02 11 12 22 */
    int n[3];                       /* floor(x) */
    float f[3];                     /* x - floor(x), rounded to binary32 */
    int lo[3], hi[3];               /* voxel box of the window */
    float qx, qh;                   /* grids of the position and moment terms */
    double hsc;                     /* 5 * 2^16 / qh */
    double adj[6], det;             /* adjugate and determinant of H, FP64 */
} ko_ab_win;

static int ko_ab_setup(ko_ab_win *w, const double x[3], const double H[6], const int dim[3])
{
    const double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22,
                 c02 = a01 * a12 - a02 * a11, c11 = a00 * a22 - a02 * a02,
                 c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.0)) return 0;
    w->adj[0] = c00; w->adj[1] = c01; w->adj[2] = c02;
    w->adj[3] = c11; w->adj[4] = c12; w->adj[5] = c22;
    w->det = det;
    const double inv = 1.0 / det;
    w->h[0] = (float)(c00 * inv); w->h[1] = (float)(c01 * inv); w->h[2] = (float)(c02 * inv);
    w->h[3] = (float)(c11 * inv); w->h[4] = (float)(c12 * inv); w->h[5] = (float)(c22 * inv);
    const double dg[3] = {a00, a11, a22};
    int Emax = 0;
    for (int a = 0; a < 3; ++a) {
        w->x[a] = x[a];
        const double fl = floor(x[a]);
        w->n[a] = (int)fl;
        w->f[a] = (float)(x[a] - fl);   /* exact in FP64 for x >= 0 */
        const int E = (int)ceilf(sqrtf((float)dg[a]));
        if (E > Emax) Emax = E;
        w->lo[a] = w->n[a] - E > 0 ? w->n[a] - E : 0;
        w->hi[a] = w->n[a] + E < dim[a] - 1 ? w->n[a] + E : dim[a] - 1;
    }
    const int px = ko_ab_exp(Emax, 4, 1), pm = ko_ab_exp(Emax, 4, 2);
    w->qx = ldexpf(1.0f, px);
    w->qh = ldexpf(1.0f, pm);
    w->hsc = 5.0 * ldexp(1.0, 16 - pm);
    return 1;
}

/* The x-row at offsets (o1, o2): d = (h00 o_x + b2) o_x + g along it, and
 * the span [*ja, *jb] of j = s_x - floor(x_x), clipped to the box; returns
 * 0 for an empty row. */
static int ko_ab_span(const ko_ab_win *w, float o1, float o2, float *b2, float *g, int *ja,
                      int *jb)
{
    const float *h = w->h;
    const float beta = h[1] * o1 + h[2] * o2;
    const float gamma = (h[3] * o1 + (2.0f * h[4]) * o2) * o1 + (h[5] * o2) * o2;
    *b2 = beta + beta;
    *g = gamma;
    const float disc = beta * beta - h[0] * (gamma - AB_SLACK);
    if (!(disc >= 0.0f)) return 0;
    const float sq = sqrtf(disc);
    const float ih0 = 1.0f / h[0];
    const float ulo = (-beta - sq) * ih0, uhi = (sq - beta) * ih0;
    const float a = fmaxf(ceilf(ulo + w->f[0]), (float)(w->lo[0] - w->n[0]));
    const float b = fminf(floorf(uhi + w->f[0]), (float)(w->hi[0] - w->n[0]));
    if (!(a <= b)) return 0;
    *ja = (int)a;
    *jb = (int)b;
    return 1;
}

static inline int64_t ko_q(float v, float q) { return (int64_t)llrintf(v * q); }

/* Window membership, decided exactly as the definition states it:
 * (s - x)^T adj(H) (s - x) <= det H in binary64, in the operation order of
 * the plain oracle.  The kernel decides in binary32 wherever that cannot
 * differ (|d - 1| above its rounding bound) and takes this test for the
 * rest, so both give this set. */
static int ko_ab_inside(const ko_ab_win *w, int sx, int sy, int sz)
{
    const double o0 = (double)sx - w->x[0], o1 = (double)sy - w->x[1], o2 = (double)sz - w->x[2];
    const double *A = w->adj;
    const double q = A[0] * o0 * o0 + A[3] * o1 * o1 + A[5] * o2 * o2 +
                     2.0 * (A[1] * o0 * o1 + A[2] * o0 * o2 + A[4] * o1 * o2);
    return q <= w->det;
}

enum { AB_HIST = 0, AB_POS = 1, AB_MOM = 2 };

/* One pass over the window.  AB_HIST: P[b] += q(k, 2^16), returns K and
 * adds the window's voxel count to *nvox.  AB_POS: acc[0..2] += q(k w o_a,
 * 2^px), acc[3] += q(k w, 2^px).  AB_MOM: acc[0..5] += q(w (o_a o_b),
 * 2^pm) (00 01 02 11 12 22), acc[6] += q(w, 2^16). */
static int64_t ko_ab_pass(const uint8_t *bins, int nx, int ny, int nz, int B, const ko_ab_win *w,
                          int kind, const float *wf, int64_t *P, int64_t *acc, int64_t *nvox)
{
    int64_t K = 0;
    if (kind == AB_HIST)
        for (int b = 0; b < B; ++b) P[b] = 0;
    else
        for (int k = 0; k < 7; ++k) acc[k] = 0;
    const float *h = w->h;
    for (int sz = w->lo[2]; sz <= w->hi[2]; ++sz)
        for (int sy = w->lo[1]; sy <= w->hi[1]; ++sy) {
            const float o1 = (float)(sy - w->n[1]) - w->f[1];
            const float o2 = (float)(sz - w->n[2]) - w->f[2];
            int ja, jb;
            float b2, g;
            if (!ko_ab_span(w, o1, o2, &b2, &g, &ja, &jb)) continue;
            for (int j = ja; j <= jb; ++j) {
                const int v = ko_at(bins, nx, ny, nz, w->n[0] + j, sy, sz);
                if (!v) continue;
                const float o0 = (float)j - w->f[0];
                const float d = fmaf(fmaf(h[0], o0, b2), o0, g);
                if (!ko_ab_inside(w, w->n[0] + j, sy, sz)) continue;
                if (kind == AB_HIST) {
                    const int64_t k = ko_q(ko_ab_kernel(d), AB_QK);
                    P[v - 1] += k;
                    K += k;
                    ++*nvox;
                } else if (kind == AB_POS) {
                    const float t = ko_ab_kernel(d) * wf[v - 1];
                    acc[0] += ko_q(t * o0, w->qx);
                    acc[1] += ko_q(t * o1, w->qx);
                    acc[2] += ko_q(t * o2, w->qx);
                    acc[3] += ko_q(t, w->qx);
                } else {
                    const float t = wf[v - 1];
                    acc[0] += ko_q(t * (o0 * o0), w->qh);
                    acc[1] += ko_q(t * (o0 * o1), w->qh);
                    acc[2] += ko_q(t * (o0 * o2), w->qh);
                    acc[3] += ko_q(t * (o1 * o1), w->qh);
                    acc[4] += ko_q(t * (o1 * o2), w->qh);
                    acc[5] += ko_q(t * (o2 * o2), w->qh);
                    acc[6] += ko_q(t, AB_QW);
                }
            }
        }
    return K;
}

/* binary32 voxel weights w_b = sqrt(K / (B P_b)) (0 for empty bins) */
static void ko_ab_weights(const int64_t *P, int64_t K, int B, float *wf)
{
    for (int b = 0; b < B; ++b)
        wf[b] = P[b] > 0 ? sqrtf((float)K / ((float)B * (float)P[b])) : 0.0f;
}

/* rho = (sum_b sqrt(P_b)) / sqrt(B K), pairwise over 64 zero-padded slots */
static double ko_ab_rho(const int64_t *P, int64_t K, int B)
{
    double t[64];
    for (int b = 0; b < 64; ++b) t[b] = b < B && P[b] > 0 ? sqrt((double)P[b]) : 0.0;
    for (int m = 32; m >= 1; m >>= 1)
        for (int i = 0; i < m; ++i) t[i] = t[i] + t[i + m];
    return t[0] / sqrt((double)B * (double)K);
}

void ko_abmsod_fixed(const uint8_t *bins, int nx, int ny, int nz, int B,
                     int r_min, int r_max, int max_iter,
                     const int32_t *seeds, int64_t nseeds,
                     const double *cand_x /* NULL, or items x 3 */,
                     const double *cand_H /* items x 6 */, int nthreads,
                     double *x_out /* items x 3 */, double *H_out /* items x 6 */,
                     double *rho_out, int32_t *iters_out, int32_t *stopped_out,
                     int64_t *voxels_out)
{
    const int S = r_max - r_min + 1;
    const int dim[3] = {nx, ny, nz};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t *P = (int64_t *)malloc(sizeof(int64_t) * B);
        float *wf = (float *)malloc(sizeof(float) * B);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t item = 0; item < (cand_x ? nseeds : nseeds * S); ++item) {
            double x[3], H[6];
            if (cand_x) {       /* a given candidate ellipsoid (x, H) */
                for (int a = 0; a < 3; ++a) x[a] = cand_x[3 * item + a];
                for (int c = 0; c < 6; ++c) H[c] = cand_H[6 * item + c];
            } else {            /* seed si with H = r^2 I */
                const int64_t si = item / S;
                const double r2 = (double)(r_min + (int)(item % S)) * (r_min + (int)(item % S));
                x[0] = seeds[3 * si]; x[1] = seeds[3 * si + 1]; x[2] = seeds[3 * si + 2];
                H[0] = r2; H[1] = 0.0; H[2] = 0.0; H[3] = r2; H[4] = 0.0; H[5] = r2;
            }
            double x_opt[3] = {x[0], x[1], x[2]}, H_opt[6];
            for (int k = 0; k < 6; ++k) H_opt[k] = H[k];
            double best = 0.0;
            int it = 0, stopped = 0;
            int64_t nvox = 0, acc[7];
            while (it < max_iter) {
                ko_ab_win w;
                if (!ko_ab_setup(&w, x, H, dim)) break;
                const int64_t K = ko_ab_pass(bins, nx, ny, nz, B, &w, AB_HIST, NULL, P, NULL, &nvox);
                if (K == 0) break;
                ko_ab_weights(P, K, B, wf);
                /* 2. position (Eq. 6) */
                ko_ab_pass(bins, nx, ny, nz, B, &w, AB_POS, wf, NULL, acc, NULL);
                double xn[3];
                for (int a = 0; a < 3; ++a) {
                    const double dl = acc[3] > 0 ? (double)acc[a] / (double)acc[3] : 0.0;
                    double v = x[a] + dl;
                    if (v < 0.0) v = 0.0;
                    if (v > (double)(dim[a] - 1)) v = (double)(dim[a] - 1);
                    xn[a] = v;
                }
                /* 3. histogram and weights at x' */
                ko_ab_win w2;
                if (!ko_ab_setup(&w2, xn, H, dim)) break;
                const int64_t K2 = ko_ab_pass(bins, nx, ny, nz, B, &w2, AB_HIST, NULL, P, NULL, &nvox);
                ++it;
                if (K2 == 0) break;
                ko_ab_weights(P, K2, B, wf);
                /* 4. bandwidth (Eq. 7) */
                ko_ab_pass(bins, nx, ny, nz, B, &w2, AB_MOM, wf, NULL, acc, NULL);
                double Hn[6];
                for (int k = 0; k < 6; ++k)
                    Hn[k] = acc[6] > 0 ? (w2.hsc * (double)acc[k]) / (double)acc[6] : H[k];
                const int dg[3] = {0, 3, 5};
                double m = 0.0;
                for (int a = 0; a < 3; ++a) {
                    Hn[dg[a]] = Hn[dg[a]] + AB_VOXEL;
                    if (Hn[dg[a]] < 1.0) Hn[dg[a]] = 1.0;
                    if (Hn[dg[a]] > m) m = Hn[dg[a]];
                }
                if (m > AB_HMAX) {
                    const double sc = AB_HMAX / m;
                    for (int k = 0; k < 6; ++k) Hn[k] = Hn[k] * sc;
                    for (int a = 0; a < 3; ++a)   /* rounding of m * sc */
                        if (Hn[dg[a]] > AB_HMAX) Hn[dg[a]] = AB_HMAX;
                }
                /* 5. Bhattacharyya coefficient at x' */
                const double bh = ko_ab_rho(P, K2, B);
                const double delta = best - bh;
                if (bh > best) {
                    best = bh;
                    for (int a = 0; a < 3; ++a) x_opt[a] = xn[a];
                    for (int k = 0; k < 6; ++k) H_opt[k] = Hn[k];
                }
                if (delta > 0.0) { stopped = 1; break; }
                for (int a = 0; a < 3; ++a) x[a] = xn[a];
                for (int k = 0; k < 6; ++k) H[k] = Hn[k];
            }
            for (int a = 0; a < 3; ++a) x_out[3 * item + a] = x_opt[a];
            for (int k = 0; k < 6; ++k) H_out[6 * item + k] = H_opt[k];
            rho_out[item] = best;
            iters_out[item] = it;
            stopped_out[item] = stopped;
            voxels_out[item] = nvox;
        }
        free(P);
        free(wf);
    }
}

/* Window membership two ways, for a uniform volume of counted voxels:
 * out[0] = voxels of the box whose quadratic form o^T H^-1 o (binary32, no
 * row form) is in [0, 1], out[1] = those of them that lie in their row's
 * span (equal when the spans lose nothing). */
void ko_ab_window_check(const double x[3], const double H[6], int64_t out[2])
{
    ko_ab_win w;
    const int dim[3] = {1 << 20, 1 << 20, 1 << 20};
    out[0] = out[1] = 0;
    if (!ko_ab_setup(&w, x, H, dim)) return;
    const float *h = w.h;
    for (int sz = w.lo[2]; sz <= w.hi[2]; ++sz)
        for (int sy = w.lo[1]; sy <= w.hi[1]; ++sy) {
            const float o1 = (float)(sy - w.n[1]) - w.f[1];
            const float o2 = (float)(sz - w.n[2]) - w.f[2];
            int ja = 1, jb = 0;
            float b2, g;
            ko_ab_span(&w, o1, o2, &b2, &g, &ja, &jb);
            for (int sx = w.lo[0]; sx <= w.hi[0]; ++sx) {
                const int j = sx - w.n[0];
                const float o0 = (float)j - w.f[0];
                /* d as the quadratic form, independent of the row form */
                const float u0 = h[0] * o0 + h[1] * o1 + h[2] * o2;
                const float u1 = h[1] * o0 + h[3] * o1 + h[4] * o2;
                const float u2 = h[2] * o0 + h[4] * o1 + h[5] * o2;
                const float d = o0 * u0 + o1 * u1 + o2 * u2;
                if (!(d >= 0.0f && d <= 1.0f)) continue;
                out[0] += 1;
                out[1] += (j >= ja && j <= jb);
            }
        }
}
