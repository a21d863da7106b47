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
enum { KO_BIN_CLAMP_SHIFT = 0, KO_BIN_AFFINE_F32 = 1, KO_BIN_WINDOW = 2 };

/* Integer inputs (uint8 / int16 widened to int32).
 *   CLAMP_SHIFT: b = (clamp(v, lo, hi) - lo) >> shift
 *   WINDOW:      voxels outside [lo, hi] are not counted (Sec. 3.2's
 *                window-level restriction); inside, b = (v - lo) >> shift. */
void ko_bin_int(const int32_t *v, int64_t n, int kind, int bins, int shift,
                int lo, int hi, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = v[i];
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
/* Adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3, Alg. 2, Eq. 7) towards  */
/* the uniform target HQ_b = 1/B.                                            */
/*                                                                          */
/* A candidate is a centre x (FP64 vector) with a bandwidth matrix H (FP64, */
/* symmetric positive definite).  Its window is the ellipsoid               */
/* { s : d(s) = (s-x)^T H^-1 (s-x) <= 1 } of counted voxels; each voxel     */
/* carries the kernel k(s) = exp(-d(s)/2) (Alg. 2's c exp(-d/2)).  One      */
/* iteration:                                                                */
/*   1. HP_b = (sum of k over bin b) / (sum of k)  at (x, H)                 */
/*      w_b  = sqrt(HQ_b / HP_b)                                             */
/*   2. x' = x + sum_s k w o / sum_s k w,  o = s - x  (Eq. 6 with the       */
/*      Gaussian profile: -k' is proportional to k); clamp to the volume    */
/*   3. HP' and w' at (x', H)                                                */
/*   4. H' = (n+2) (sum_s w' o' o'^T / sum_s w' + I/12),  o' = s - x',     */
/*      n = 3 (Eq. 7; the factor keeps the window of a homogeneous region   */
/*      at its size: the second moment of a uniform ellipsoid is H/(n+2);   */
/*      I/12 is the second moment of a unit voxel about its centre, which   */
/*      keeps H positive definite when the window's voxels lie on a line or */
/*      a plane); then every diagonal entry below 1 is raised to 1 and H is */
/*      scaled down so that no diagonal entry exceeds 32^2 (the window      */
/*      stays within 32 voxels)                                             */
/*   5. rho = sum_b sqrt(HQ_b HP'_b); the best rho so far keeps its         */
/*      (x', H'); the search stops at the first rho below the best (Alg.    */
/*      2's THRESHOLD read as 0) or after max_iter iterations.              */
/* Candidates start at each seed with H = r^2 I for r = r_min..r_max.       */
/*                                                                          */
/* Arithmetic.  The window's voxels are found row by row: for the x-row at  */
/* offsets (o_y, o_z), d as a function of o_x is the quadratic              */
/* h00 o_x^2 + 2 beta o_x + gamma, and the row's span is where it is at     */
/* most 1 + 1/16 (binary32 root formula, the division by h00 done as a      */
/* product with 1/h00); a voxel of the span is in the window when           */
/* -1/16 <= d <= 1, d evaluated along the row in binary32 as                */
/* (h00 o_x + 2 beta) o_x + gamma with fused multiply-adds (beta and gamma  */
/* once per row; d < 0 arises only from rounding).  The rows are those      */
/* of the box [floor(x_a) - E_a, floor(x_a) + E_a] clipped to the volume,   */
/* E_a = ceil(sqrt(H_aa)) in binary32 (voxels outside the volume are not    */
/* counted).  Offsets are                                                   */
/* o_a = (s_a - floor(x_a)) - frac(x_a), frac(x_a) rounded to binary32; H^-1 */
/* is the adjugate times 1/det in FP64, rounded to binary32; k is the       */
/* degree-9 Taylor polynomial of exp(-d/2) in Horner form with fused        */
/* multiply-adds.  Every sum over voxels is an exact int64 sum of terms     */
/* rounded to nearest (ties to even) on a fixed-point grid (2^-16 for k,    */
/* 2^-12 for the position terms and w', 2^-8 for the second moments), so    */
/* no result depends on the order of summation.  Per bin: w_b =             */
/* sqrt(K / (B P_b)) in binary32 (K, B, P_b rounded to binary32) and        */
/* sqrt(P_b) in FP64; rho =                                                 */
/* (sum_b sqrt(P_b)) / sqrt(B K), the sum over 64 zero-padded slots as a    */
/* pairwise tree (slot i + m added to slot i, m = 32, 16, ..., 1); H' =     */
/* 80 M / W (= 5 (M / 2^8) / (W / 2^12)) in FP64.                           */
/* ------------------------------------------------------------------------ */
#define AB_QK 65536.0f     /* 2^16 */
#define AB_QX 4096.0f      /* 2^12 */
#define AB_QH 256.0f       /* 2^8 */
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
} ko_ab_win;

static int ko_ab_setup(ko_ab_win *w, const double x[3], const double H[6], const int dim[3])
{
    const double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22,
                 c02 = a01 * a12 - a02 * a11, c11 = a00 * a22 - a02 * a02,
                 c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.0)) return 0;
    const double inv = 1.0 / det;
    w->h[0] = (float)(c00 * inv); w->h[1] = (float)(c01 * inv); w->h[2] = (float)(c02 * inv);
    w->h[3] = (float)(c11 * inv); w->h[4] = (float)(c12 * inv); w->h[5] = (float)(c22 * inv);
    const double dg[3] = {a00, a11, a22};
    for (int a = 0; a < 3; ++a) {
        w->x[a] = x[a];
        const double fl = floor(x[a]);
        w->n[a] = (int)fl;
        w->f[a] = (float)(x[a] - fl);   /* exact in FP64 for x >= 0 */
        const int E = (int)ceilf(sqrtf((float)dg[a]));
        w->lo[a] = w->n[a] - E > 0 ? w->n[a] - E : 0;
        w->hi[a] = w->n[a] + E < dim[a] - 1 ? w->n[a] + E : dim[a] - 1;
    }
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

enum { AB_HIST = 0, AB_POS = 1, AB_MOM = 2 };

/* One pass over the window.  AB_HIST: P[b] += q(k, 2^16), returns K and
 * adds the window's voxel count to *nvox.  AB_POS: acc[0..2] += q(k w o_a,
 * 2^12), acc[3] += q(k w, 2^12).  AB_MOM: acc[0..5] += q(w (o_a o_b), 2^8)
 * (00 01 02 11 12 22), acc[6] += q(w, 2^12). */
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
                if (!(d >= -0.0625f && d <= 1.0f)) continue;
                if (kind == AB_HIST) {
                    const int64_t k = ko_q(ko_ab_kernel(d), AB_QK);
                    P[v - 1] += k;
                    K += k;
                    ++*nvox;
                } else if (kind == AB_POS) {
                    const float t = ko_ab_kernel(d) * wf[v - 1];
                    acc[0] += ko_q(t * o0, AB_QX);
                    acc[1] += ko_q(t * o1, AB_QX);
                    acc[2] += ko_q(t * o2, AB_QX);
                    acc[3] += ko_q(t, AB_QX);
                } else {
                    const float t = wf[v - 1];
                    acc[0] += ko_q(t * (o0 * o0), AB_QH);
                    acc[1] += ko_q(t * (o0 * o1), AB_QH);
                    acc[2] += ko_q(t * (o0 * o2), AB_QH);
                    acc[3] += ko_q(t * (o1 * o1), AB_QH);
                    acc[4] += ko_q(t * (o1 * o2), AB_QH);
                    acc[5] += ko_q(t * (o2 * o2), AB_QH);
                    acc[6] += ko_q(t, AB_QX);
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

void ko_abmsod(const uint8_t *bins, int nx, int ny, int nz, int B,
               int r_min, int r_max, int max_iter,
               const int32_t *seeds, int64_t nseeds, int nthreads,
               double *x_out /* items x 3 */, double *H_out /* items x 6 */,
               double *rho_out, int32_t *iters_out, int32_t *stopped_out, int64_t *voxels_out)
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
        for (int64_t item = 0; item < nseeds * S; ++item) {
            const int64_t si = item / S;
            const int r = r_min + (int)(item % S);
            double x[3] = {seeds[3 * si], seeds[3 * si + 1], seeds[3 * si + 2]};
            double H[6] = {(double)r * r, 0.0, 0.0, (double)r * r, 0.0, (double)r * r};
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
                    Hn[k] = acc[6] > 0 ? (80.0 * (double)acc[k]) / (double)acc[6] : H[k];
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
