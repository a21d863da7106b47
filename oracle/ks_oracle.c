/*
 * ks_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of what the Kadir-Brady
 * saliency hot path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library; the product
 * path never calls it and shares no code with it.
 *
 * Built with: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (x86-64 SSE2
 * doubles, so every + - * / and sqrt below is one IEEE binary64 operation
 * rounded to nearest, with no fused multiply-add).
 *
 * Conventions
 *   - Volumes are x-fastest: voxel (x,y,z) is element (z*ny + y)*nx + x.
 *   - Bin volumes hold the STORED value b+1 for bin b in [0,B), and 0 for a
 *     voxel that is not counted (outside the tissue window).  Voxels outside
 *     the volume are never counted either.
 *   - Ball(r) = { o in Z^3 : |o|^2 <= r^2 }.
 *
 * Paper passages followed (arXiv 1310.6736):
 *   Sec. 1 / Sec. 2.1   Kadir-Brady saliency: entropy over multi-scale
 *                       neighbourhoods times the rate of change of the pdf
 *                       with scale, maximised over scale.
 *   Eq. 1-3             entropy of a window; used by the tests as closed forms.
 *   Sec. 2.2, Alg. 1    quadrant (here: octant) hill-climbing.
 *   Sec. 2.3, Eq. 4-6   mean shift towards a uniform target pmf with
 *                       Bhattacharyya weights.
 *   Sec. 2.3, Alg. 2,   adaptive-bandwidth mean shift (ABMSOD) with
 *   Eq. 7               ellipsoidal Gaussian-profile windows.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <quadmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Tables.  T[c] = c*ln(c) and L[n] = ln(n), each correctly rounded to      */
/* binary64.  They are evaluated in binary128 (113-bit) arithmetic with     */
/* libquadmath's logq and rounded once, so the double is the nearest one to */
/* the exact value except for inputs within ~2^-60 ulp of a rounding        */
/* midpoint.  T[0] = T[1] = 0 and L[0] = L[1] = 0.                          */
/* ------------------------------------------------------------------------ */
void ko_tables(int64_t nmax, double *T, double *L)
{
    for (int64_t c = 0; c <= nmax; ++c) {
        if (c <= 1) {
            T[c] = 0.0;
            L[c] = 0.0;
            continue;
        }
        __float128 q = (__float128)c;
        __float128 lq = logq(q);
        T[c] = (double)(q * lq);
        L[c] = (double)lq;
    }
}

/* ------------------------------------------------------------------------ */
/* Binning: the bin index beta(s) of Eq. 4-5, stored as b+1.                 */
/* ------------------------------------------------------------------------ */
/* KO_BIN_STORED: the input is already a bin volume in the stored form (b+1,
 * 0 = not counted); values outside [1, bins] are not counted. */
enum { KO_BIN_CLAMP_SHIFT = 0, KO_BIN_AFFINE_F32 = 1, KO_BIN_WINDOW = 2, KO_BIN_STORED = 3 };

/* Integer inputs (uint8 / int16 widened to int32).
 *   CLAMP_SHIFT: b = (clamp(v, lo, hi) - lo) >> shift
 *   WINDOW:      voxels outside [lo, hi] are not counted (Sec. 3.2's
 *                window-level restriction); inside, b = (v - lo) >> shift. */
void ko_bin_int(const int32_t *v, int64_t n, int kind, int bins, int shift,
                int lo, int hi, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = v[i];
        if (kind == KO_BIN_STORED) {           /* already stored bin values */
            out[i] = (uint8_t)(x >= 1 && x <= bins ? x : 0);
            continue;
        }
        if (kind == KO_BIN_WINDOW && (x < lo || x > hi)) {
            out[i] = 0;
            continue;
        }
        if (x < lo) x = lo;
        if (x > hi) x = hi;
        int32_t b = (x - lo) >> shift;
        if (b > bins - 1) b = bins - 1;
        out[i] = (uint8_t)(b + 1);
    }
}

/* float32 input: b = clamp(floor(bins*(v - vmin) / ((vmax - vmin) + 1e-6)),
 * 0, bins-1), every operation in binary32 rounded to nearest, in this order:
 * a = v - vmin; t = bins*a; d = (vmax - vmin) + 1e-6f; q = t / d.
 * vmin / vmax are the exact minimum and maximum over the whole volume. */
void ko_bin_f32(const float *v, int64_t n, int bins, uint8_t *out,
                float *vmin_out, float *vmax_out)
{
    float vmin = v[0], vmax = v[0];
    for (int64_t i = 1; i < n; ++i) {
        if (v[i] < vmin) vmin = v[i];
        if (v[i] > vmax) vmax = v[i];
    }
    float d = vmax - vmin;
    d = d + 1e-6f;
    float fb = (float)bins;
    for (int64_t i = 0; i < n; ++i) {
        float a = v[i] - vmin;
        float t = fb * a;
        float q = t / d;
        int b = (int)floorf(q);
        if (b < 0) b = 0;
        if (b > bins - 1) b = bins - 1;
        out[i] = (uint8_t)(b + 1);
    }
    if (vmin_out) *vmin_out = vmin;
    if (vmax_out) *vmax_out = vmax;
}

/* ------------------------------------------------------------------------ */
/* Window histograms and the scalar quantities built from them.             */
/* ------------------------------------------------------------------------ */

/* Stored bin value at (x,y,z), or 0 when the voxel lies outside the volume. */
static inline int ko_at(const uint8_t *bins, int nx, int ny, int nz, int x, int y, int z)
{
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0;
    return bins[((int64_t)z * ny + y) * nx + x];
}

/* Brute force: counts c[b] of bin b over Ball(r) centred at (px,py,pz),
 * enumerating the cube [-r, r]^3 and keeping |o|^2 <= r^2. */
void ko_window_counts(const uint8_t *bins, int nx, int ny, int nz, int B,
                      int px, int py, int pz, int r, int64_t *c)
{
    for (int b = 0; b < B; ++b) c[b] = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                if (dx * dx + dy * dy + dz * dz > r * r) continue;
                int s = ko_at(bins, nx, ny, nz, px + dx, py + dy, pz + dz);
                if (s) c[s - 1] += 1;
            }
}

/* Shannon entropy of a window's counts:
 *   H = ln N - (1/N) * sum_b c_b ln c_b
 * which equals -sum_b p_b ln p_b with p_b = c_b / N (Eq. 1).  The sum runs
 * over b = 0..B-1 in order starting from +0.0, then one division and one
 * subtraction.  A window with at most one occupied bin (alpha = 0 in
 * Sec. 2.1, or N <= 1) has H = 0 exactly; the formula would leave rounding
 * noise of order 1e-15 there. */
double ko_entropy(const int64_t *c, int B, const double *T, const double *L)
{
    int64_t N = 0;
    int occupied = 0;
    for (int b = 0; b < B; ++b) { N += c[b]; occupied += c[b] > 0; }
    if (occupied <= 1) return 0.0;
    double s = 0.0;
    for (int b = 0; b < B; ++b) s = s + T[c[b]];
    return L[N] - s / (double)N;
}

/* Kadir-Brady inter-scale weight at radius r from the counts at r (c) and
 * r-1 (cp): W = f(r) * sum_b | c_b/N - cp_b/Np |, evaluated exactly as the
 * integer D = sum_b | c_b*Np - cp_b*N | over the integer N*Np, with the
 * discrete scale normalisation f(r) = r^2 / (2r - 1) (w_norm = 0) or
 * f = 1 (w_norm = 1).  An empty window at either scale gives W = 0. */
double ko_weight(const int64_t *c, const int64_t *cp, int B, int r, int w_norm)
{
    int64_t N = 0, Np = 0;
    for (int b = 0; b < B; ++b) { N += c[b]; Np += cp[b]; }
    if (N == 0 || Np == 0) return 0.0;
    int64_t D = 0;
    for (int b = 0; b < B; ++b) {
        int64_t d = c[b] * Np - cp[b] * N;
        D += d < 0 ? -d : d;
    }
    double f = w_norm == 1 ? 1.0 : (double)(r * r) / (double)(2 * r - 1);
    return f * ((double)D / (double)(N * Np));
}

/* Kadir-Brady saliency at one centre over scales r_min..r_max.
 * H[k], W[k] for r = r_min + k (W[0] = 0: no r_min - 1 histogram).
 * Peaks in scale: interior r (r_min < r < r_max) with H(r-1) < H(r) and
 * H(r) >= H(r+1).  Y(r) = H(r) * W(r).  The best peak is the first peak in
 * ascending r, replaced only by a later peak with strictly larger Y.
 * No peak: Y_best = 0, s_best = 0.
 * brute = 1 enumerates Ball(r) afresh for every r; brute = 0 enumerates
 * Ball(r_max) once, sorted by the shell each offset first enters
 * (the smallest r >= r_min with |o|^2 <= r^2), and adds shell r to the
 * counts of r-1.  Both give the same integer counts. */
typedef struct { int dx, dy, dz, shell; } ko_off;

static int ko_shell_of(int d2, int r_min)
{
    int r = r_min;
    while (r * r < d2) ++r;
    return r;
}

/* Ball(r_max) offsets ordered by shell (stable within a shell: dz, dy, dx).
 * planar = 1 keeps only the offsets with dz = 0: the disk of radius r_max
 * in the centre's z-slice (the 2D windows of Alg. 1 as printed). */
static ko_off *ko_ball_by_shell_p(int r_min, int r_max, int planar, int64_t *count)
{
    int64_t n = 0;
    for (int dz = -r_max; dz <= r_max; ++dz)
        for (int dy = -r_max; dy <= r_max; ++dy)
            for (int dx = -r_max; dx <= r_max; ++dx)
                if (dx * dx + dy * dy + dz * dz <= r_max * r_max && (!planar || dz == 0)) ++n;
    ko_off *o = (ko_off *)malloc(sizeof(ko_off) * (size_t)(n > 0 ? n : 1));
    int64_t k = 0;
    for (int r = r_min; r <= r_max; ++r)
        for (int dz = -r_max; dz <= r_max; ++dz)
            for (int dy = -r_max; dy <= r_max; ++dy)
                for (int dx = -r_max; dx <= r_max; ++dx) {
                    int d2 = dx * dx + dy * dy + dz * dz;
                    if (planar && dz != 0) continue;
                    if (d2 <= r_max * r_max && ko_shell_of(d2, r_min) == r) {
                        o[k].dx = dx; o[k].dy = dy; o[k].dz = dz; o[k].shell = r;
                        ++k;
                    }
                }
    *count = n;
    return o;
}

static ko_off *ko_ball_by_shell(int r_min, int r_max, int64_t *count)
{
    return ko_ball_by_shell_p(r_min, r_max, 0, count);
}

static void ko_kb_core(const uint8_t *bins, int nx, int ny, int nz, int B,
                       int px, int py, int pz, int r_min, int r_max, int w_norm,
                       const double *T, const double *L, int brute,
                       const ko_off *ball, int64_t nball,
                       double *H, double *W, double *Y_best, int *s_best,
                       int64_t *cur, int64_t *prev)
{
    int S = r_max - r_min + 1;
    int64_t k = 0;
    for (int b = 0; b < B; ++b) cur[b] = 0;
    for (int i = 0; i < S; ++i) {
        int r = r_min + i;
        for (int b = 0; b < B; ++b) prev[b] = cur[b];
        if (brute) {
            ko_window_counts(bins, nx, ny, nz, B, px, py, pz, r, cur);
        } else {
            while (k < nball && ball[k].shell == r) {
                int s = ko_at(bins, nx, ny, nz, px + ball[k].dx, py + ball[k].dy, pz + ball[k].dz);
                if (s) cur[s - 1] += 1;
                ++k;
            }
        }
        H[i] = ko_entropy(cur, B, T, L);
        W[i] = i == 0 ? 0.0 : ko_weight(cur, prev, B, r, w_norm);
    }
    double yb = 0.0;
    int sb = 0;
    for (int i = 1; i + 1 < S; ++i) {
        if (H[i - 1] < H[i] && H[i] >= H[i + 1]) {
            double y = H[i] * W[i];
            if (sb == 0 || y > yb) { yb = y; sb = r_min + i; }
        }
    }
    *Y_best = yb;
    *s_best = sb;
}

/* Dense Kadir-Brady sweep over a list of centres (xyz triples), or over
 * every voxel when centres == NULL (then ncentres = nx*ny*nz and centre i
 * is voxel i).  Outputs Y_best (double) and s_best (uint8) per centre, and
 * optionally H / W per centre and scale (ncentres x S, may be NULL). */
void ko_dense(const uint8_t *bins, int nx, int ny, int nz, int B,
              int r_min, int r_max, int w_norm, const double *T, const double *L,
              const int32_t *centres, int64_t ncentres, int brute, int nthreads,
              double *Y, uint8_t *s_out, double *H_out, double *W_out)
{
    int S = r_max - r_min + 1;
    int64_t nball = 0;
    ko_off *ball = ko_ball_by_shell(r_min, r_max, &nball);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * B);
        int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * B);
        double *H = (double *)malloc(sizeof(double) * S);
        double *W = (double *)malloc(sizeof(double) * S);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t i = 0; i < ncentres; ++i) {
            int px, py, pz;
            if (centres) {
                px = centres[3 * i]; py = centres[3 * i + 1]; pz = centres[3 * i + 2];
            } else {
                px = (int)(i % nx); py = (int)((i / nx) % ny); pz = (int)(i / ((int64_t)nx * ny));
            }
            double yb;
            int sb;
            ko_kb_core(bins, nx, ny, nz, B, px, py, pz, r_min, r_max, w_norm, T, L,
                       brute, ball, nball, H, W, &yb, &sb, cur, prev);
            Y[i] = yb;
            s_out[i] = (uint8_t)sb;
            if (H_out) memcpy(H_out + i * S, H, sizeof(double) * S);
            if (W_out) memcpy(W_out + i * S, W, sizeof(double) * S);
        }
        free(cur); free(prev); free(H); free(W);
    }
    free(ball);
}

/* ------------------------------------------------------------------------ */
/* Seed grid (Sec. 2.2: "a uniformly sampled grid of points").               */
/* Positions stride/2 + i*stride < dim per axis; seed index is x-fastest.   */
/* Returns the seed count; writes xyz triples when out != NULL.             */
/* ------------------------------------------------------------------------ */
int64_t ko_seed_grid(int nx, int ny, int nz, int stride, int32_t *out)
{
    int64_t n = 0;
    for (int z = stride / 2; z < nz; z += stride)
        for (int y = stride / 2; y < ny; y += stride)
            for (int x = stride / 2; x < nx; x += stride) {
                if (out) { out[3 * n] = x; out[3 * n + 1] = y; out[3 * n + 2] = z; }
                ++n;
            }
    return n;
}

static inline int ko_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Round half away from zero; exact for every binary64 (C99 round). */
static inline int ko_round(double d) { return (int)round(d); }

/* ------------------------------------------------------------------------ */
/* Octant hill-climbing: the 3D form of Alg. 1 (Sec. 2.2).                   */
/*                                                                          */
/* Octant j (bit0: x<0, bit1: y<0, bit2: z<0) has sign vector sigma_j.  Its */
/* window at scale k is the CLOSED octant of Ball(k) at P: offsets whose    */
/* every nonzero component has the octant's sign (an offset on a coordinate */
/* plane belongs to every octant it touches).  Per iteration:               */
/*   eps_jk  = entropy of window (j, k)                                      */
/*   eps_j   = max_k eps_jk, k_j = argmax (first, i.e. smallest, k on ties)  */
/*   d_j     = k_j * sigma_j  (3D counterpart of the diagonal step sqrt2*k)  */
/*   delta   = sum_j eps_j d_j / sum_j eps_j  (normalised-entropy weights;   */
/*             numerator and denominator summed over j = 0..7 in order, one  */
/*             division per axis; sum_j eps_j = 0 gives delta = 0)           */
/*   P'      = clamp(P + round_half_away(delta), 0, dim-1)                    */
/* The climb stops when P' == P (converged) or after max_iter iterations.    */
/* Afterwards the Kadir-Brady quantities are evaluated on the full ball at  */
/* the final P (Sec. 2.2: the change in pdf about the optimal scale).        */
/* ------------------------------------------------------------------------ */
static int ko_in_octant(int j, int dx, int dy, int dz)
{
    if ((j & 1) ? dx > 0 : dx < 0) return 0;
    if ((j & 2) ? dy > 0 : dy < 0) return 0;
    if ((j & 4) ? dz > 0 : dz < 0) return 0;
    return 1;
}

/* nj = 8: the octants of Ball(k); nj = 4 with a disk `ball`: the four
 * closed quadrants j = 0..3 of Alg. 1 as printed (bit0: x<0, bit1: y<0),
 * whose weighted sum gives a step with no z component. */
static void ko_octant_step(const uint8_t *bins, int nx, int ny, int nz, int B,
                           int r_min, int r_max, const double *T, const double *L,
                           const ko_off *ball, int64_t nball,
                           const int P[3], int step[3], int64_t *cnt /* 8*B */, int nj)
{
    int S = r_max - r_min + 1;
    double eps[8];
    int kopt[8];
    for (int j = 0; j < 8; ++j) {
        for (int b = 0; b < B; ++b) cnt[j * B + b] = 0;
        eps[j] = 0.0;
        kopt[j] = r_min;
    }
    int64_t k = 0;
    for (int i = 0; i < S; ++i) {
        int r = r_min + i;
        while (k < nball && ball[k].shell == r) {
            int dx = ball[k].dx, dy = ball[k].dy, dz = ball[k].dz;
            int s = ko_at(bins, nx, ny, nz, P[0] + dx, P[1] + dy, P[2] + dz);
            if (s)
                for (int j = 0; j < 8; ++j)
                    if (ko_in_octant(j, dx, dy, dz)) cnt[j * B + s - 1] += 1;
            ++k;
        }
        for (int j = 0; j < nj; ++j) {
            double e = ko_entropy(cnt + j * B, B, T, L);
            if (i == 0 || e > eps[j]) { eps[j] = e; kopt[j] = r; }
        }
    }
    double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
    for (int j = 0; j < nj; ++j) {
        /* the quadrant form's sigma_j has no z component */
        int sg[3] = {(j & 1) ? -1 : 1, (j & 2) ? -1 : 1, nj == 8 ? ((j & 4) ? -1 : 1) : 0};
        for (int a = 0; a < 3; ++a) num[a] = num[a] + eps[j] * (double)(kopt[j] * sg[a]);
        den = den + eps[j];
    }
    for (int a = 0; a < 3; ++a) step[a] = den == 0.0 ? 0 : ko_round(num[a] / den);
}

static void ko_climb(const uint8_t *bins, int nx, int ny, int nz, int B,
                     int r_min, int r_max, int max_iter, int w_norm,
                     const double *T, const double *L,
                     const int32_t *seeds, int64_t nseeds, int nthreads, int planar,
                     int32_t *final_xyz, int32_t *iters, int32_t *converged, int32_t *traj,
                     double *Y_best, int32_t *s_best, double *H_best, double *W_best)
{
    int S = r_max - r_min + 1;
    int64_t nball = 0;
    ko_off *ball = ko_ball_by_shell_p(r_min, r_max, planar, &nball);
    int dim[3] = {nx, ny, nz};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 8 * B);
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * B);
        int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * B);
        double *H = (double *)malloc(sizeof(double) * S);
        double *W = (double *)malloc(sizeof(double) * S);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t i = 0; i < nseeds; ++i) {
            int P[3] = {seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2]};
            int it = 0, conv = 0;
            if (traj) for (int a = 0; a < 3; ++a) traj[(i * (max_iter + 1)) * 3 + a] = P[a];
            while (it < max_iter) {
                int step[3], Pn[3];
                ko_octant_step(bins, nx, ny, nz, B, r_min, r_max, T, L, ball, nball, P, step, cnt,
                               planar ? 4 : 8);
                ++it;
                for (int a = 0; a < 3; ++a) Pn[a] = ko_clampi(P[a] + step[a], 0, dim[a] - 1);
                if (Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2]) { conv = 1; break; }
                for (int a = 0; a < 3; ++a) P[a] = Pn[a];
                if (traj) for (int a = 0; a < 3; ++a) traj[(i * (max_iter + 1) + it) * 3 + a] = P[a];
            }
            if (traj)   /* positions after the last move are repeated to the end */
                for (int t = it + (conv ? 0 : 1); t <= max_iter; ++t)
                    for (int a = 0; a < 3; ++a) traj[(i * (max_iter + 1) + t) * 3 + a] = P[a];
            for (int a = 0; a < 3; ++a) final_xyz[3 * i + a] = P[a];
            iters[i] = it;
            converged[i] = conv;
            double yb; int sb;
            ko_kb_core(bins, nx, ny, nz, B, P[0], P[1], P[2], r_min, r_max, w_norm, T, L,
                       0, ball, nball, H, W, &yb, &sb, cur, prev);
            Y_best[i] = yb;
            s_best[i] = sb;
            H_best[i] = sb ? H[sb - r_min] : 0.0;
            W_best[i] = sb ? W[sb - r_min] : 0.0;
        }
        free(cnt); free(cur); free(prev); free(H); free(W);
    }
    free(ball);
}

void ko_octant_climb(const uint8_t *bins, int nx, int ny, int nz, int B,
                     int r_min, int r_max, int max_iter, int w_norm,
                     const double *T, const double *L,
                     const int32_t *seeds, int64_t nseeds, int nthreads,
                     int32_t *final_xyz, int32_t *iters, int32_t *converged,
                     int32_t *traj /* nseeds x (max_iter+1) x 3, or NULL */,
                     double *Y_best, int32_t *s_best, double *H_best, double *W_best)
{
    ko_climb(bins, nx, ny, nz, B, r_min, r_max, max_iter, w_norm, T, L, seeds, nseeds, nthreads,
             0, final_xyz, iters, converged, traj, Y_best, s_best, H_best, W_best);
}

/* ------------------------------------------------------------------------ */
/* Quadrant hill-climbing: Alg. 1 as printed, in 2D (Sec. 2.2), run in the   */
/* z-slice of each seed.  Windows are disks {dx^2 + dy^2 <= k^2, dz = 0};    */
/* quadrant j = 0..3 (bit0: x<0, bit1: y<0) is closed as in the 3D form; the */
/* step is sum_j eps_j k_j sigma_j / sum_j eps_j over the four quadrants     */
/* (d_j = k_j sigma_j = sqrt2 k_j along the quadrant's diagonal direction),   */
/* so P moves within its slice.  The Kadir-Brady evaluation at the final P   */
/* uses the same disks.                                                      */
/* ------------------------------------------------------------------------ */
void ko_quadrant_climb(const uint8_t *bins, int nx, int ny, int nz, int B,
                       int r_min, int r_max, int max_iter, int w_norm,
                       const double *T, const double *L,
                       const int32_t *seeds, int64_t nseeds, int nthreads,
                       int32_t *final_xyz, int32_t *iters, int32_t *converged, int32_t *traj,
                       double *Y_best, int32_t *s_best, double *H_best, double *W_best)
{
    ko_climb(bins, nx, ny, nz, B, r_min, r_max, max_iter, w_norm, T, L, seeds, nseeds, nthreads,
             1, final_xyz, iters, converged, traj, Y_best, s_best, H_best, W_best);
}

/* ------------------------------------------------------------------------ */
/* Mean shift towards a uniform target pmf (Sec. 2.3, Eq. 4-6).              */
/*                                                                          */
/* Item = (seed, r).  The window is Ball(r) at P with a flat profile, so    */
/* p_b = c_b / N (Eq. 4) and -K' is constant in Eq. 6.  With q_b = 1/B the  */
/* voxel weight of Eq. 5 is w(s) = sqrt(q_b / p_b) = sqrt(N / (B c_b)) for  */
/* s in bin b.  Eq. 6 then moves P to the w-weighted centroid:              */
/*   P + delta,  delta = sum_s w(s) o_s / sum_s w(s)                          */
/*              = sum_b w_b m_b / sum_b w_b c_b                               */
/* with m_b = sum of offsets o_s over the voxels of bin b (integers).  The   */
/* two FP64 sums run over b = 0..B-1 in order, skipping empty bins.          */
/*   P' = clamp(P + round_half_away(delta), 0, dim-1); stop when P' == P or   */
/* after max_iter iterations.  At the final P the item reports the           */
/* Bhattacharyya coefficient rho = sum_b sqrt(p_b q_b) = sum_b sqrt(c_b/(N B))*/
/* (bin order) and the window entropy H.                                    */
/* ------------------------------------------------------------------------ */
static void ko_ms_moments(const uint8_t *bins, int nx, int ny, int nz, int B,
                          int r, const int P[3], int64_t *c, int64_t *m /* 3*B */)
{
    for (int b = 0; b < B; ++b) { c[b] = 0; m[3 * b] = m[3 * b + 1] = m[3 * b + 2] = 0; }
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                if (dx * dx + dy * dy + dz * dz > r * r) continue;
                int s = ko_at(bins, nx, ny, nz, P[0] + dx, P[1] + dy, P[2] + dz);
                if (!s) continue;
                c[s - 1] += 1;
                m[3 * (s - 1)] += dx;
                m[3 * (s - 1) + 1] += dy;
                m[3 * (s - 1) + 2] += dz;
            }
}

void ko_meanshift(const uint8_t *bins, int nx, int ny, int nz, int B,
                  int r_min, int r_max, int max_iter, const double *T, const double *L,
                  const int32_t *seeds, int64_t nseeds, int nthreads,
                  int32_t *final_xyz, int32_t *iters, int32_t *converged,
                  double *rho, double *H)
{
    int S = r_max - r_min + 1;
    int dim[3] = {nx, ny, nz};
    int64_t nitems = nseeds * S;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int64_t *c = (int64_t *)malloc(sizeof(int64_t) * B);
        int64_t *m = (int64_t *)malloc(sizeof(int64_t) * 3 * B);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t item = 0; item < nitems; ++item) {
            int64_t sd = item / S;
            int r = r_min + (int)(item % S);
            int P[3] = {seeds[3 * sd], seeds[3 * sd + 1], seeds[3 * sd + 2]};
            int it = 0, conv = 0, fresh = 0;
            while (it < max_iter) {
                ko_ms_moments(bins, nx, ny, nz, B, r, P, c, m);
                fresh = 1;
                ++it;
                int64_t N = 0;
                for (int b = 0; b < B; ++b) N += c[b];
                int step[3] = {0, 0, 0};
                if (N > 0) {
                    double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
                    for (int b = 0; b < B; ++b) {
                        if (c[b] == 0) continue;
                        double w = sqrt((double)N / (double)(B * c[b]));
                        for (int a = 0; a < 3; ++a) num[a] = num[a] + w * (double)m[3 * b + a];
                        den = den + w * (double)c[b];
                    }
                    for (int a = 0; a < 3; ++a) step[a] = ko_round(num[a] / den);
                }
                int Pn[3];
                for (int a = 0; a < 3; ++a) Pn[a] = ko_clampi(P[a] + step[a], 0, dim[a] - 1);
                if (Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2]) { conv = 1; break; }
                for (int a = 0; a < 3; ++a) P[a] = Pn[a];
                fresh = 0;
            }
            if (!fresh) ko_ms_moments(bins, nx, ny, nz, B, r, P, c, m);
            int64_t N = 0;
            for (int b = 0; b < B; ++b) N += c[b];
            double rh = 0.0;
            if (N > 0)
                for (int b = 0; b < B; ++b)
                    if (c[b] > 0) rh = rh + sqrt((double)c[b] / (double)(N * B));
            for (int a = 0; a < 3; ++a) final_xyz[3 * item + a] = P[a];
            iters[item] = it;
            converged[item] = conv;
            rho[item] = rh;
            H[item] = ko_entropy(c, B, T, L);
        }
        free(c); free(m);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-window debug views used by the pins.                                  */
/* ------------------------------------------------------------------------ */

/* Counts of the closed octant j of Ball(r) at P, by brute force. */
void ko_octant_counts(const uint8_t *bins, int nx, int ny, int nz, int B,
                      int px, int py, int pz, int r, int j, int64_t *c)
{
    for (int b = 0; b < B; ++b) c[b] = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                if (dx * dx + dy * dy + dz * dz > r * r) continue;
                if (!ko_in_octant(j, dx, dy, dz)) continue;
                int s = ko_at(bins, nx, ny, nz, px + dx, py + dy, pz + dz);
                if (s) c[s - 1] += 1;
            }
}

/* One octant (planar = 0) or quadrant (planar = 1) step at P (the rounded
 * move, before clamping). */
void ko_octant_one_step(const uint8_t *bins, int nx, int ny, int nz, int B,
                        int r_min, int r_max, const double *T, const double *L,
                        int px, int py, int pz, int planar, int32_t *step_out)
{
    int64_t nball = 0;
    ko_off *ball = ko_ball_by_shell_p(r_min, r_max, planar, &nball);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 8 * B);
    int P[3] = {px, py, pz}, step[3];
    ko_octant_step(bins, nx, ny, nz, B, r_min, r_max, T, L, ball, nball, P, step, cnt,
                   planar ? 4 : 8);
    for (int a = 0; a < 3; ++a) step_out[a] = step[a];
    free(cnt);
    free(ball);
}

/* Mean-shift counts and moments of Ball(r) at P. */
void ko_ms_window(const uint8_t *bins, int nx, int ny, int nz, int B,
                  int px, int py, int pz, int r, int64_t *c, int64_t *m)
{
    int P[3] = {px, py, pz};
    ko_ms_moments(bins, nx, ny, nz, B, r, P, c, m);
}

int ko_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 6 and 7)    */
/* towards the uniform target HQ_b = 1/B, stated plainly in binary64.       */
/*                                                                          */
/* A candidate is a centre x and a symmetric positive definite bandwidth    */
/* matrix H.  Its window is the ellipsoid of counted voxels s with          */
/*   d(s) = (s - x)^T H^-1 (s - x) <= 1,                                     */
/* tested without a division as (s - x)^T adj(H) (s - x) <= det(H) (the     */
/* same set for det > 0; with integer data, as in the first iteration,      */
/* the test is exact, so voxels on the boundary are always inside).  Each   */
/* voxel of the window carries k(s) = exp(-d(s)/2), Alg. 2's c exp(-d/2)    */
/* with the constant c dropped (it cancels in every ratio below).           */
/*                                                                          */
/* One iteration (Alg. 2):                                                   */
/*   1. HP_b = (sum of k over the window's voxels of bin b) / (sum of k),   */
/*      w_b = sqrt(HQ_b / HP_b) for every occupied bin (Eq. 5).             */
/*   2. x' = x + sum_s k w (s - x) / sum_s k w, clamped to the volume       */
/*      (Eq. 6 with the Gaussian profile, whose -K' is proportional to k).  */
/*   3. HP' and w' at (x', H).                                               */
/*   4. H' = (n + 2) (sum_s w' (s - x')(s - x')^T / sum_s w' + I/12), n = 3 */
/*      (Eq. 7; see the readings below); every diagonal entry below 1 is   */
/*      raised to 1, then H' is scaled so that no diagonal entry exceeds    */
/*      32^2.                                                               */
/*   5. rho' = sum_b sqrt(HQ_b HP'_b).  If rho' > best: best = rho',        */
/*      (x_opt, H_opt) = (x', H').  The search stops when rho' < best of    */
/*      the earlier iterations (Alg. 2's THRESHOLD read as 0) or after      */
/*      max_iter iterations; otherwise (x, H) = (x', H').                    */
/* A window without counted voxels ends the search (before the iteration    */
/* is counted when it is the first window of the iteration).  Candidates   */
/* start at every seed with H = r^2 I for r = r_min..r_max, or at given     */
/* candidate ellipsoids (x, H) (Alg. 2's "each candidate ellipsoid W_i      */
/* centred at P_i with bandwidth H_i").                                     */
/*                                                                          */
/* Readings of Eq. 7.  As printed, the second moment of a uniform           */
/* ellipsoid is H/(n+2), so a homogeneous window would shrink by the        */
/* factor n + 2 = 5 every iteration; the factor keeps it at its size.       */
/* I/12 is the second moment of a unit voxel about its centre: without it  */
/* a window whose counted voxels lie on a plane or a line has a singular    */
/* H'.  The bounds on the diagonal keep every window between one voxel and  */
/* 32 voxels along each axis.                                               */
/*                                                                          */
/* Arithmetic: binary64 throughout; exp from libm; adj(H) and det(H) from   */
/* the cofactors; every sum over voxels runs over the bounding box in       */
/* z, y, x order; the box is floor(x_a - sqrt(H_aa)) - 1 ..                 */
/* ceil(x_a + sqrt(H_aa)) + 1 clipped to the volume (the ellipsoid reaches  */
/* sqrt(H_aa) along axis a).                                                */
/*                                                                          */
/* Besides the result, each item reports two margins that say how close    */
/* its discrete decisions came to a tie: edge = the smallest |d - 1| over   */
/* the counted voxels of the boxes of its windows at x' (the centres its    */
/* steps computed), relative to |o|^T |H^-1| |o|, the scale of the rounding */
/* error of an evaluation in a shorter precision -- a voxel this close to   */
/* the boundary may fall on the other side for a centre that differs by    */
/* rounding (ties of an integer x' included) -- and                         */
/* rho_gap = the smallest |rho' - best| over its iterations after the       */
/* first (the stopping test).  An implementation in other arithmetic may    */
/* take another path only where one of them is small.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double x[3];
    double adj[6];       /* adjugate of H: 00 01 02 11 12 22 */
    double det;
    int lo[3], hi[3];    /* bounding box, clipped to the volume */
} ko_abw;

static int ko_abw_setup(ko_abw *w, const double x[3], const double H[6], const int dim[3])
{
    const double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
    w->adj[0] = a11 * a22 - a12 * a12;
    w->adj[1] = a02 * a12 - a01 * a22;
    w->adj[2] = a01 * a12 - a02 * a11;
    w->adj[3] = a00 * a22 - a02 * a02;
    w->adj[4] = a01 * a02 - a00 * a12;
    w->adj[5] = a00 * a11 - a01 * a01;
    w->det = a00 * w->adj[0] + a01 * w->adj[1] + a02 * w->adj[2];
    if (!(w->det > 0.0)) return 0;
    const double dg[3] = {a00, a11, a22};
    for (int a = 0; a < 3; ++a) {
        w->x[a] = x[a];
        const double e = sqrt(dg[a]);
        const int lo = (int)floor(x[a] - e) - 1, hi = (int)ceil(x[a] + e) + 1;
        w->lo[a] = lo > 0 ? lo : 0;
        w->hi[a] = hi < dim[a] - 1 ? hi : dim[a] - 1;
    }
    return 1;
}

/* (s - x)^T adj(H) (s - x) */
static double ko_abw_form(const ko_abw *w, const double o[3])
{
    const double *A = w->adj;
    return A[0] * o[0] * o[0] + A[3] * o[1] * o[1] + A[5] * o[2] * o[2] +
           2.0 * (A[1] * o[0] * o[1] + A[2] * o[0] * o[2] + A[4] * o[1] * o[2]);
}

/* |o|^T |adj(H)| |o|: the scale of the rounding error of any evaluation of
 * the form in a shorter precision */
static double ko_abw_absform(const ko_abw *w, const double o[3])
{
    const double *A = w->adj;
    const double a0 = fabs(o[0]), a1 = fabs(o[1]), a2 = fabs(o[2]);
    const double m = fabs(A[0]) * a0 * a0 + fabs(A[3]) * a1 * a1 + fabs(A[5]) * a2 * a2 +
                     2.0 * (fabs(A[1]) * a0 * a1 + fabs(A[2]) * a0 * a2 + fabs(A[4]) * a1 * a2);
    return m > 0.0 ? m : w->det;
}

enum { ABP_HIST = 0, ABP_POS = 1, ABP_MOM = 2 };

/* One walk over the window.  ABP_HIST: P[b] = sum of k over bin b; returns
 * the sum of k, adds the window's voxel count to *nvox and lowers *edge.
 * ABP_POS: acc[0..2] = sum k w_b (s - x)_a, acc[3] = sum k w_b.
 * ABP_MOM: acc[0..5] = sum w_b (s - x)_a (s - x)_c (00 01 02 11 12 22),
 * acc[6] = sum w_b. */
static double ko_abw_pass(const uint8_t *bins, int nx, int ny, int nz, int B, const ko_abw *w,
                          int kind, const double *wb, double *P, double *acc, int64_t *nvox,
                          double *edge)
{
    double K = 0.0;
    if (kind == ABP_HIST)
        for (int b = 0; b < B; ++b) P[b] = 0.0;
    else
        for (int c = 0; c < 7; ++c) acc[c] = 0.0;
    for (int sz = w->lo[2]; sz <= w->hi[2]; ++sz)
        for (int sy = w->lo[1]; sy <= w->hi[1]; ++sy)
            for (int sx = w->lo[0]; sx <= w->hi[0]; ++sx) {
                const int v = ko_at(bins, nx, ny, nz, sx, sy, sz);
                if (!v) continue;
                const double o[3] = {(double)sx - w->x[0], (double)sy - w->x[1],
                                     (double)sz - w->x[2]};
                const double q = ko_abw_form(w, o);
                if (kind == ABP_HIST && edge) {
                    /* |d - 1| relative to the size of the form's terms */
                    const double gap = fabs(q - w->det) / ko_abw_absform(w, o);
                    if (gap < *edge) *edge = gap;
                }
                if (!(q <= w->det)) continue;
                const double d = q / w->det;
                const int b = v - 1;
                if (kind == ABP_HIST) {
                    const double k = exp(-0.5 * d);
                    P[b] += k;
                    K += k;
                    ++*nvox;
                } else if (kind == ABP_POS) {
                    const double t = exp(-0.5 * d) * wb[b];
                    acc[0] += t * o[0];
                    acc[1] += t * o[1];
                    acc[2] += t * o[2];
                    acc[3] += t;
                } else {
                    const double t = wb[b];
                    acc[0] += t * (o[0] * o[0]);
                    acc[1] += t * (o[0] * o[1]);
                    acc[2] += t * (o[0] * o[2]);
                    acc[3] += t * (o[1] * o[1]);
                    acc[4] += t * (o[1] * o[2]);
                    acc[5] += t * (o[2] * o[2]);
                    acc[6] += t;
                }
            }
    return K;
}

/* w_b = sqrt(HQ_b / HP_b), HQ_b = 1/B, HP_b = P_b / K; 0 for empty bins */
static void ko_abw_weights(const double *P, double K, int B, double *wb)
{
    for (int b = 0; b < B; ++b)
        wb[b] = P[b] > 0.0 ? sqrt((1.0 / B) / (P[b] / K)) : 0.0;
}

/* rho = sum_b sqrt(HQ_b HP_b), bins in order */
static double ko_abw_rho(const double *P, double K, int B)
{
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += sqrt((1.0 / B) * (P[b] / K));
    return s;
}

void ko_abmsod(const uint8_t *bins, int nx, int ny, int nz, int B,
               int r_min, int r_max, int max_iter,
               const int32_t *seeds, int64_t nseeds,
               const double *cand_x /* NULL, or items x 3 */,
               const double *cand_H /* items x 6 */, int nthreads,
               double *x_out /* items x 3 */, double *H_out /* items x 6 */,
               double *rho_out, int32_t *iters_out, int32_t *stopped_out, int64_t *voxels_out,
               double *edge_out, double *rho_gap_out)
{
    const int S = r_max - r_min + 1;
    const int dim[3] = {nx, ny, nz};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *P = (double *)malloc(sizeof(double) * B);
        double *wb = (double *)malloc(sizeof(double) * B);
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
            for (int c = 0; c < 6; ++c) H_opt[c] = H[c];
            double best = 0.0, edge = INFINITY, rho_gap = INFINITY, acc[7];
            int it = 0, stopped = 0;
            int64_t nvox = 0;
            while (it < max_iter) {
                /* 1. candidate histogram and weights at (x, H) */
                ko_abw w;
                if (!ko_abw_setup(&w, x, H, dim)) break;
                const double K = ko_abw_pass(bins, nx, ny, nz, B, &w, ABP_HIST, NULL, P, NULL,
                                             &nvox, NULL);
                if (!(K > 0.0)) break;
                ko_abw_weights(P, K, B, wb);
                /* 2. position (Eq. 6) */
                ko_abw_pass(bins, nx, ny, nz, B, &w, ABP_POS, wb, NULL, acc, NULL, NULL);
                double xn[3];
                for (int a = 0; a < 3; ++a) {
                    double v = x[a] + acc[a] / acc[3];
                    if (v < 0.0) v = 0.0;
                    if (v > (double)(dim[a] - 1)) v = (double)(dim[a] - 1);
                    xn[a] = v;
                }
                /* 3. histogram and weights at (x', H) */
                ko_abw w2;
                if (!ko_abw_setup(&w2, xn, H, dim)) break;
                const double K2 = ko_abw_pass(bins, nx, ny, nz, B, &w2, ABP_HIST, NULL, P, NULL,
                                              &nvox, &edge);
                ++it;
                if (!(K2 > 0.0)) break;
                ko_abw_weights(P, K2, B, wb);
                /* 4. bandwidth (Eq. 7) */
                ko_abw_pass(bins, nx, ny, nz, B, &w2, ABP_MOM, wb, NULL, acc, NULL, NULL);
                double Hn[6];
                for (int c = 0; c < 6; ++c) Hn[c] = 5.0 * (acc[c] / acc[6]);
                const int dg[3] = {0, 3, 5};
                double m = 0.0;
                for (int a = 0; a < 3; ++a) {
                    Hn[dg[a]] += 5.0 / 12.0;
                    if (Hn[dg[a]] < 1.0) Hn[dg[a]] = 1.0;
                    if (Hn[dg[a]] > m) m = Hn[dg[a]];
                }
                if (m > 1024.0)
                    for (int c = 0; c < 6; ++c) Hn[c] *= 1024.0 / m;
                /* 5. Bhattacharyya coefficient at x' and the stopping test */
                const double rho = ko_abw_rho(P, K2, B);
                if (it > 1 && fabs(rho - best) < rho_gap) rho_gap = fabs(rho - best);
                const int fell = rho < best;
                if (rho > best) {
                    best = rho;
                    for (int a = 0; a < 3; ++a) x_opt[a] = xn[a];
                    for (int c = 0; c < 6; ++c) H_opt[c] = Hn[c];
                }
                if (fell) {
                    stopped = 1;
                    break;
                }
                for (int a = 0; a < 3; ++a) x[a] = xn[a];
                for (int c = 0; c < 6; ++c) H[c] = Hn[c];
            }
            for (int a = 0; a < 3; ++a) x_out[3 * item + a] = x_opt[a];
            for (int c = 0; c < 6; ++c) H_out[6 * item + c] = H_opt[c];
            rho_out[item] = best;
            iters_out[item] = it;
            stopped_out[item] = stopped;
            voxels_out[item] = nvox;
            if (edge_out) edge_out[item] = edge;
            if (rho_gap_out) rho_gap_out[item] = rho_gap;
        }
        free(P);
        free(wb);
    }
}
