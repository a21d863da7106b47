// Seed-grid searches: octant hill-climbing (Sec. 2.2, Alg. 1 in 3D) and
// mean shift towards the uniform pmf (Sec. 2.3, Eq. 4-6).
//
// Scheduling.  Work is handed out in tickets: an octant ticket is one seed
// on a block of 256 threads (all its iterations plus the final Kadir-Brady
// evaluation); a mean-shift ticket is one (seed, r) item, on a whole block
// for radii above 20 or more than 32 bins, else on one warp, items taken
// largest radius first.  The same kernel serves a plain launch and the
// persistent batched launch (blocks pull tickets from a device counter until
// the queue is empty), so an item's arithmetic never depends on how it was
// scheduled.
//
// Octant pass.  The block walks the offset tables of Ball(r_max) in row
// order, each entry standing for a set of sign mirrors.  A voxel off the
// coordinate planes lies in exactly one open octant and costs one
// shared-memory atomic.  A plane/axis voxel belongs to every closed octant
// it touches and is added to each; its multiplicity minus one is recorded
// per (shell, bin), so that the full-ball histogram is the sum of the 8
// closed-octant histograms minus that excess.  The Kadir-Brady quantities at
// the final centre therefore come from the last octant pass whenever the
// climb converged (the pass ran at that centre).  A climb whose centre
// repeats stops early (octant_item).
//
// Mean-shift pass.  A thread (block path) or lane (warp path) takes whole
// x-rows of Ball(r) and streams each as aligned 8-byte words.  Per voxel it
// adds the count and the three offset sums, each offset shifted to be
// non-negative, in disjoint bit fields whose bounds are checked below: two
// 32-bit reductions (count and dx sum, then dy and dz sums), or one 64-bit
// reduction where a column's sums need more bits, into columns private to
// a lane or a few threads; the columns are then summed per bin.
//
// Every accumulated quantity is an integer, so neither the order nor the
// grouping of accumulation can change a result; the FP64 steps run
// afterwards in one fixed order (bins ascending, octants 0..7), each step a
// single IEEE operation.
#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kCycleMax = 8;     // longest cycle of centres the octant climb detects
// KINDS bit: a mean-shift launch whose items all take the block path (more
// than 32 bins), compiled without the warp path so that its registers allow
// three blocks per SM.
constexpr int kMsBlockOnly = 1 << 3;

struct SeedShared {
    int step[3];
    int64_t ticket;
    uint32_t N[kMaxScales];
    unsigned long long D[kMaxScales];
    int hist[kCycleMax][3];         // octant climb: centre t at t % kCycleMax
};

__device__ __forceinline__ const uint8_t *voxel_ptr(const VolDesc &v, const int P[3]) {
    return v.base + (int64_t)P[2] * v.plane + (int64_t)P[1] * v.pitch + P[0];
}

// Entropy of counts c[0..B) (bin order), the library's fixed formula.  The
// counts and their table values are gathered eight bins at a time, so the
// table loads of a group are in flight together; the additions still run
// one at a time in bin order.
__device__ double window_entropy(const uint32_t *c, int B, const double *T, const double *L,
                                 uint32_t *N_out) {
    uint32_t N = 0;
    int occ = 0;
    double s = 0.0;
    for (int b0 = 0; b0 < B; b0 += 8) {
        uint32_t x[8];
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = b0 + k < B ? c[b0 + k] : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = __ldg(T + x[k]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            N += x[k];
            occ += x[k] > 0u;
            if (x[k] > 1u) s = __dadd_rn(s, t[k]);
        }
    }
    if (N_out) *N_out = N;
    return entropy_from_sum(s, N, occ, L);
}

// s + p[0] + p[1] + ... + p[n-1], left to right from s = +0.0, with the
// operands read eight at a time (p in shared memory, n a multiple of 8 or
// padded with +0.0 up to one).
__device__ __forceinline__ double chain_sum(const double *p, int n) {
    double s = 0.0;
    for (int b0 = 0; b0 < n; b0 += 8) {
        double t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] = p[b0 + k];
#pragma unroll
        for (int k = 0; k < 8; ++k) s = __dadd_rn(s, t[k]);
    }
    return s;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// ---------------------------------------------------------------- octant
// Closed-octant histograms of every shell at P into cnt[j][si][v] and the
// plane/axis multiplicity excess into extra[si][v] (j = 8); the octant
// histograms are then turned into prefix sums over shells (histograms of
// Ball(r_min + si)), the excess only when kb_from_pass needs it.  Each
// histogram has B + 1 words indexed by the stored value v; word 0 (not
// counted) is a dummy that is never read, so a voxel costs no branch.
// The walk runs over the offset tables of Ball(r_max): an entry with three
// nonzero components stands for its 8 sign mirrors, and mirror m (bit0 -x,
// bit1 -y, bit2 -z) lies in the open octant m, so one entry gives one
// voxel to each octant, all in the entry's shell; an offset on a
// coordinate plane or axis lies in every closed octant it touches.
__device__ void octant_pass(const SeedJob &J, const OffsetTables &ot, uint32_t *cnt,
                            const int P[3]) {
    const int B = J.vol.B, S = J.S, Bs = B + 1;
    const uint32_t SB4 = (uint32_t)(S * Bs * 4);          // bytes per octant
    for (int k = threadIdx.x; k < 9 * S * Bs; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    const uint32_t cnt_s = smem_u32(cnt);
    auto shell = [&](int rho) {   // byte offset of the shell of radius class rho
        return (uint32_t)((rho > J.r_min ? rho - J.r_min : 0) * Bs * 4);
    };
    // three nonzero components (none on the disk dz = 0 of the quadrant climb)
    // Ball(r_max)'s entries sorted by row: the lanes of a warp take
    // neighbouring voxels of a few rows, so each mirror's loads touch few lines
    if (!J.planar) {
        const uint32_t *c8 = ot.c8_rows + __ldg(ot.c8_rows_start + J.r_max);
        const int n8 = __ldg(ot.c8_rows_start + J.r_max + 1) - __ldg(ot.c8_rows_start + J.r_max);
        // two entries per round: their 16 loads are in flight together
        // each round's two entries are loaded one round ahead, so their
        // latency overlaps the previous round's voxel loads
        uint32_t pe0 = threadIdx.x < n8 ? __ldg(c8 + threadIdx.x) : 0u;
        uint32_t pe1 = threadIdx.x + blockDim.x < n8 ? __ldg(c8 + threadIdx.x + blockDim.x) : 0u;
        for (int k = threadIdx.x; k < n8; k += 2 * blockDim.x) {
            const int k2 = k + blockDim.x;
            const uint32_t e0 = pe0;
            const uint32_t e1 = k2 < n8 ? pe1 : 0u;   // 0: the centre, v unused
            const int kn = k + 2 * blockDim.x, kn2 = kn + blockDim.x;
            pe0 = kn < n8 ? __ldg(c8 + kn) : 0u;
            pe1 = kn2 < n8 ? __ldg(c8 + kn2) : 0u;
            uint32_t v[2][8], base[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t e = h ? e1 : e0;
                const int X = (int)(e & 0xffu);
                const int Y = (int)((e >> 8) & 0xffu) * pitch;
                const int Z = (int)((e >> 16) & 0xffu) * plane;
                base[h] = cnt_s + shell((int)(e >> 24));
                const int o[8] = {Z + Y + X, Z + Y - X, Z - Y + X, Z - Y - X,
                                  Y - Z + X, Y - Z - X, -Z - Y + X, -Z - Y - X};
#pragma unroll
                for (int m = 0; m < 8; ++m) v[h][m] = __ldg(c0 + o[m]);
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) red_add_shared(base[0] + (uint32_t)m * SB4 + (v[0][m] << 2), 1u);
            if (k2 < n8) {
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    red_add_shared(base[1] + (uint32_t)m * SB4 + (v[1][m] << 2), 1u);
            }
        }
    }
    // On a coordinate plane or axis: one entry per set of sign mirrors.  Its
    // 8 mirrors name each distinct voxel once per closed octant that voxel
    // touches (2^z times, z = the zero components), so octant m counts
    // mirror m as for c8.  The first mirror of each distinct voxel (the
    // bits of the zero components clear) adds the excess multiplicity
    // 2^z - 1.  Quadrant climb: the entries on the disk dz = 0 only.
    const uint32_t *restm = ot.restm_rows + __ldg(ot.restm_rows_start + J.r_max);
    const int nr = __ldg(ot.restm_rows_start + J.r_max + 1) - __ldg(ot.restm_rows_start + J.r_max);
    uint32_t pf = threadIdx.x < nr ? __ldg(restm + threadIdx.x) : 0u;   // one round ahead
    for (int k = threadIdx.x; k < nr; k += blockDim.x) {
        const uint32_t f = pf;
        pf = k + blockDim.x < nr ? __ldg(restm + k + blockDim.x) : 0u;
        const int X = (int)(f & 0xffu), Yb = (int)((f >> 8) & 0xffu), Zb = (int)((f >> 16) & 0xffu);
        if (J.planar && Zb != 0) continue;
        const uint32_t zm = (X == 0 ? 1u : 0u) | (Yb == 0 ? 2u : 0u) | (Zb == 0 ? 4u : 0u);
        const uint32_t excess = (1u << __popc(zm)) - 1u;
        const int Y = Yb * pitch, Z = Zb * plane;
        const uint32_t base = cnt_s + shell((int)(f >> 24));
        const int o[8] = {Z + Y + X, Z + Y - X, Z - Y + X, Z - Y - X,
                          Y - Z + X, Y - Z - X, -Z - Y + X, -Z - Y - X};
        uint32_t v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = __ldg(c0 + o[m]);
#pragma unroll
        for (int m = 0; m < 8; ++m) red_add_shared(base + (uint32_t)m * SB4 + (v[m] << 2), 1u);
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if ((m & zm) == 0u) red_add_shared(base + 8u * SB4 + (v[m] << 2), excess);
    }
    __syncthreads();
    // prefix over shells per (octant, counted value) column, eight shells at
    // a time: the eight loads are issued before any store of the group.  The
    // dummy value 0 is never read, and the excess column is summed by
    // kb_from_pass, the only reader: 8 B columns, one round for B = 32.
    for (int col = threadIdx.x; col < 8 * B; col += blockDim.x) {
        const int j = col / B, b = 1 + col % B;
        uint32_t *p = cnt + j * S * Bs + b;
        uint32_t run = 0;
        for (int s0 = 0; s0 < S; s0 += 8) {
            uint32_t x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = s0 + k < S ? p[(s0 + k) * Bs] : 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                run += x[k];
                if (s0 + k < S) p[(s0 + k) * Bs] = run;
            }
        }
    }
    __syncthreads();
}

// Alg. 1's update from the octant entropies hb[j*S + si]: eps_j = max over
// scales (the smallest r on ties), d_j = k_j sigma_j, delta = sum_j eps_j
// d_j / sum_j eps_j summed over j = 0..7, rounded half away from zero.
// Called by warp 0 (every operation of the sequential form, spread over the
// lanes: 24 products at once, the four chains side by side, three divisions).
__device__ void octant_step(const SeedJob &J, const double *hb, int step[3]) {
    const int S = J.S;
    const int lane = threadIdx.x & 31;
    // eps_j and k_j: lane 4j + q scans the scales q, q + 4, ... of octant j
    // (the first of equal values kept), then the four lanes of octant j
    // combine, the smaller scale winning ties: the same maximum and the same
    // smallest maximising scale as one scan over all scales
    const int oj = lane >> 2, q = lane & 3;
    double best = -1.0;                       // below every entropy (H >= 0)
    int sb = S;                               // loses every tie
    for (int si = q; si < S; si += 4) {
        const double h = hb[oj * S + si];
        if (h > best) {
            best = h;
            sb = si;
        }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int os = __shfl_xor_sync(0xffffffffu, sb, o);
        if (ob > best || (ob == best && os < sb)) {
            best = ob;
            sb = os;
        }
    }
    // the terms: lane 8a + j holds eps_j k_j sigma_ja (a < 3) or eps_j (a = 3)
    // quadrant climb: the four quadrants j = 0..3 (closed on the plane z = 0,
    // so their histograms are the disk's), sigma without z
    const int nj = J.planar ? 4 : 8;
    const int ta = lane >> 3, tj = lane & 7;
    const double eps = __shfl_sync(0xffffffffu, best, 4 * tj);
    const int kj = J.r_min + __shfl_sync(0xffffffffu, sb, 4 * tj);
    double term = eps;
    if (ta < 3) {
        const int sg = ta == 2 && J.planar ? 0 : (((tj >> ta) & 1) ? -1 : 1);
        term = __dmul_rn(eps, (double)(kj * sg));
    }
    // lane a < 4 adds chain a over j = 0..nj-1 in order: three numerators
    // and the denominator; lanes a < 3 divide
    double sum = 0.0;
    for (int j = 0; j < nj; ++j) {
        const double t = __shfl_sync(0xffffffffu, term, 8 * (lane & 3) + j);
        if (lane < 4) sum = __dadd_rn(sum, t);
    }
    const double den = __shfl_sync(0xffffffffu, sum, 3);
    if (lane < 3) step[lane] = den == 0.0 ? 0 : (int)round(__ddiv_rn(sum, den));
}

// Kadir-Brady on the full ball at the centre of the last octant pass: the
// full histograms (sum of closed octants minus excess, written over the
// excess array), H(r), D(r), peaks, W and Y at peaks.  Histograms have
// B + 1 words, word 0 the not-counted dummy.
__device__ void kb_from_pass(const SeedJob &J, const double *T, const double *L, uint32_t *cnt,
                             uint32_t *full, double *hb, SeedShared &sh, ks_seed_result *o) {
    const int B = J.vol.B, S = J.S, Bs = B + 1;
    // the excess per shell (left unsummed by the pass) -> per Ball(r)
    for (int b = 1 + threadIdx.x; b < Bs; b += blockDim.x) {
        uint32_t run = 0;
        for (int si = 0; si < S; ++si) {
            run += full[si * Bs + b];
            full[si * Bs + b] = run;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < S * Bs; k += blockDim.x) {
        uint32_t s = 0;
        for (int j = 0; j < 8; ++j) s += cnt[j * S * Bs + k];
        full[k] = s - full[k];
    }
    __syncthreads();
    for (int si = threadIdx.x; si < S; si += blockDim.x) {
        uint32_t N;
        hb[si] = window_entropy(full + si * Bs + 1, B, T, L, &N);
        sh.N[si] = N;
    }
    __syncthreads();
    for (int si = 1 + threadIdx.x; si < S; si += blockDim.x) {
        const uint32_t *c = full + si * Bs + 1, *p = full + (si - 1) * Bs + 1;
        const uint32_t N = sh.N[si], Np = sh.N[si - 1];
        uint64_t D = 0;
        for (int b = 0; b < B; ++b) {
            const int64_t d = (int64_t)c[b] * Np - (int64_t)p[b] * N;
            D += (uint64_t)(d < 0 ? -d : d);
        }
        sh.D[si] = D;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double yb = 0.0, hbest = 0.0, wbest = 0.0;
        int sb = 0;
        for (int i = 1; i + 1 < S; ++i) {
            if (hb[i - 1] < hb[i] && hb[i] >= hb[i + 1]) {
                const double W = kb_weight(sh.D[i], sh.N[i], sh.N[i - 1], J.r_min + i, J.w_norm);
                const double y = __dmul_rn(hb[i], W);
                if (sb == 0 || y > yb) {
                    yb = y;
                    sb = J.r_min + i;
                    hbest = hb[i];
                    wbest = W;
                }
            }
        }
        o->s_best = sb;
        o->Y_best = yb;
        o->H_best = hbest;
        o->W_best = wbest;
    }
    __syncthreads();
}

// One seed's climb.  The next centre is a function of the centre alone
// (the pass, the entropies and the step read nothing else), so when the
// centre after iteration t equals the centre after t - p (p >= 2; p = 1 is
// convergence) the search repeats those p centres for good: it never
// converges, and the centre after iteration t' >= t - p is the one after
// t - p + (t' - t + p) mod p.  The search then jumps to iteration max_iter
// and only the final pass at that centre remains: the records (centre,
// iterations, convergence flag, trajectory and the Kadir-Brady values) are
// those of running every iteration.  The last kCycleMax centres are kept
// in shared memory, so cycles up to that length are found.
__device__ void octant_item(const SeedJob &J, int64_t sidx, const OffsetTables &ot,
                            const double *T, const double *L, uint32_t *cnt, double *hb,
                            SeedShared &sh) {
    const int dims[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    const int B = J.vol.B, S = J.S, Bs = B + 1;
    uint32_t *extra = cnt + 8 * S * Bs;
    int P[3] = {J.seeds[3 * sidx], J.seeds[3 * sidx + 1], J.seeds[3 * sidx + 2]};
    const int T1 = J.max_iter + 1;
    int it = 0, conv = 0, fresh = 0;
    int4 *stp = J.state ? J.state + sidx : nullptr;
    if (stp) {
        const int4 st = *stp;
        if (st.w & kItemDone) return;
        if (st.w & kItemStarted) {
            P[0] = st.x;
            P[1] = st.y;
            P[2] = st.z;
            it = st.w & 255;
        }
    }
    if (threadIdx.x == 0 && J.traj && it == 0)
        for (int a = 0; a < 3; ++a) J.traj[(sidx * T1) * 3 + a] = P[a];
    // centres before a resumed search's first iteration are not known
    const int hist_lo = it;
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) sh.hist[it % kCycleMax][a] = P[a];
    const int it_end = J.iter_budget > 0 ? min(J.max_iter, it + J.iter_budget) : J.max_iter;
    while (it < it_end) {
        octant_pass(J, ot, cnt, P);
        fresh = 1;
        for (int w = threadIdx.x; w < 8 * S; w += blockDim.x)
            hb[w] = window_entropy(cnt + w * Bs + 1, B, T, L, nullptr);
        __syncthreads();
        if (threadIdx.x < 32) octant_step(J, hb, sh.step);
        __syncthreads();
        ++it;
        int Pn[3];
        for (int a = 0; a < 3; ++a) Pn[a] = clampi(P[a] + sh.step[a], 0, dims[a] - 1);
        const bool same = Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2];
        int per = 0;                          // the centre after it - per equals Pn
        for (int p = 2; !same && p <= kCycleMax && it - p >= hist_lo; ++p) {
            const int *h = sh.hist[(it - p) % kCycleMax];
            if (h[0] == Pn[0] && h[1] == Pn[1] && h[2] == Pn[2]) {
                per = p;
                break;
            }
        }
        __syncthreads();                      // sh.step and sh.hist read by every thread
        if (same) {
            conv = 1;
            break;
        }
        if (per) {
            // centre after iteration t >= it: the one after it - per + (t - it) % per
            if (threadIdx.x == 0 && J.traj)
                for (int t = it; t <= J.max_iter; ++t)
                    for (int a = 0; a < 3; ++a)
                        J.traj[(sidx * T1 + t) * 3 + a] =
                            sh.hist[(it - per + (t - it) % per) % kCycleMax][a];
            const int *hf = sh.hist[(it - per + (J.max_iter - it) % per) % kCycleMax];
            fresh = hf[0] == P[0] && hf[1] == P[1] && hf[2] == P[2];   // the last pass ran at P
            for (int a = 0; a < 3; ++a) P[a] = hf[a];
            it = J.max_iter;
            break;
        }
        for (int a = 0; a < 3; ++a) P[a] = Pn[a];
        fresh = 0;
        if (threadIdx.x == 0) {
            for (int a = 0; a < 3; ++a) sh.hist[it % kCycleMax][a] = P[a];
            if (J.traj)
                for (int a = 0; a < 3; ++a) J.traj[(sidx * T1 + it) * 3 + a] = P[a];
        }
    }
    if (stp && !conv && it < J.max_iter) {   // the budget ran out: keep the state
        __syncthreads();
        if (threadIdx.x == 0) *stp = make_int4(P[0], P[1], P[2], it | kItemStarted);
        return;
    }
    if (threadIdx.x == 0 && J.traj)
        for (int t = it + (conv ? 0 : 1); t <= J.max_iter; ++t)
            for (int a = 0; a < 3; ++a) J.traj[(sidx * T1 + t) * 3 + a] = P[a];
    if (!fresh) octant_pass(J, ot, cnt, P);     // the last pass was not at P
    ks_seed_result *o = J.oct_out + sidx;
    kb_from_pass(J, T, L, cnt, extra, hb, sh, o);
    if (threadIdx.x == 0) {
        o->x = P[0];
        o->y = P[1];
        o->z = P[2];
        o->seed_x = J.seeds[3 * sidx];
        o->seed_y = J.seeds[3 * sidx + 1];
        o->seed_z = J.seeds[3 * sidx + 2];
        o->iters = it;
        o->converged = conv;
        o->reserved = 0;
        if (stp) {
            *stp = make_int4(P[0], P[1], P[2], it | kItemStarted | kItemDone);
            atomicAdd(J.finished, 1u);
        }
    }
}

// ------------------------------------------------------------ mean shift
// Packed accumulator word: count in bits [0,11), sum(dx+32) in [11,28),
// sum(dy+32) in [28,45), sum(dz+32) in [45,62).  Stored value v >= 1 has
// columns (v - 1) * NC .. v * NC - 1; a not-counted voxel (v = 0) is
// skipped.
//
// Block path (r > kWarpMsRmax or B > kWarpMsBmax): a column is shared by
// 256 / NC threads and a thread walks ceil(rows / 256) rows of at most 2r+1
// voxels, so a column sees at most 8*1*15 = 120 voxels (NC = 32, r <= 7), 4*2*25 = 200 (NC =
// 64, r <= 12) or 2*13*65 = 1690 (NC = 128, r <= 32, at most 3217 rows).
// Warp path (r <= kWarpMsRmax = 20): one warp per item, one column per
// lane, and a lane walks ceil(rows / 32) <= 40 rows (Ball(20) has 1257) of
// at most 41 voxels: at most 1640 voxels.  Either way count < 2^11 and
// each offset sum <= 1690 * 64 < 2^17, so no field carries into the next.
// The warp path uses two 32-bit words per column instead (a 64-bit shared
// reduction costs about 2.5 times a 32-bit one on this part): word A holds
// the count in bits [0,11) and sum(dx+20) in [11,28); word B holds
// sum(dy+20) in [0,16) and sum(dz+20) in [16,32).  A row contributes at
// most (2w+1)(|dy|+20) <= 1056 to a dy sum (the maximum over Ball(20)'s
// rows, at dy = 12), so 40 rows stay below 2^16; the same for dz.
constexpr int kWarpMsRmax = 20;
constexpr int kWarpMsBmax = 32;
constexpr int kRowWords = 6;           // 8-byte words that cover a row of Ball(r <= 20)

// Radii run on the block path: those above kWarpMsRmax, or all of them
// when B > kWarpMsBmax (a warp's columns would take B * 256 bytes, and
// eight such regions would starve the block path of occupancy).
__host__ __device__ inline int ms_block_radii(int r_min, int S, int B) {
    if (B > kWarpMsBmax) return S;
    const int lo = r_min > kWarpMsRmax + 1 ? r_min : kWarpMsRmax + 1;
    const int r_max = r_min + S - 1;
    return r_max >= lo ? r_max - lo + 1 : 0;
}

__device__ __forceinline__ void red_add_shared_u64(uint32_t addr, unsigned long long v) {
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr), "l"(v));
}

// Block path: counts c_b and integer offset sums m_b of Ball(r) at P into
// acc[b][4].  Column words are indexed by the stored value v (0..B): value
// 0 (not counted) has its own columns, never read, so a byte costs no
// branch, and bytes of a row's first and last words outside the row are
// masked to 0.  Each thread takes whole rows (the rows table lists rows of
// like length together, so the lanes of a warp walk similar lengths) and
// streams a row as aligned 8-byte words, the next row's words loaded while
// the current row is counted.
constexpr int kBlkRowWords = 9;   // a row of Ball(r <= 32): <= 65 bins + 7 bytes of alignment
// Block-only launches (more than 32 bins) keep the B words at this fixed
// byte offset from the A words when (B + 1) * 128 words fit below it, so
// the second reduction of a voxel takes the A address plus an immediate.
constexpr uint32_t kMsBOff = 34816;

template <uint32_t OFF>
__device__ __forceinline__ void red_add_shared_at(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF));
}

// The row walk of the block path (W32: two 32-bit words per voxel, else one
// 64-bit word); see ms_pass.
template <bool W32, uint32_t BOFF>
__device__ __forceinline__ void ms_walk_rows(const OffsetTables &ot, int r, const uint8_t *c0,
                                             int plane, int pitch, uint32_t a_addr,
                                             uint32_t b_addr, uint32_t a64, uint32_t stride) {
    const uint32_t *rows = ot.rows + __ldg(ot.rows_start + r);
    const int nrows = __ldg(ot.rows_start + r + 1) - __ldg(ot.rows_start + r);
    // row ri of this thread: its aligned words, the row's offset in the
    // first one, its length and its packed (dy, dz, w)
    auto fetch = [&](int ri, uint32_t &e, int &off, int &n,
                     unsigned long long (&wd)[kBlkRowWords]) {
        e = 0u;
        off = 0;
        n = 0;
        if (ri < nrows) {
            e = __ldg(rows + ri);
            const int dy = (int)(e & 0xffu) - 64, dz = (int)((e >> 8) & 0xffu) - 64;
            const int w = (int)(e >> 16);
            const uintptr_t a = reinterpret_cast<uintptr_t>(c0 + dz * plane + dy * pitch - w);
            off = (int)(a & 7u);
            n = 2 * w + 1;
            const unsigned long long *q =
                reinterpret_cast<const unsigned long long *>(a & ~uintptr_t(7));
            const int nw = (off + n + 7) >> 3;
            // bytes of the first and last words outside the row count as
            // value 0: masked here once, not per word in the walk
            const int hl = off + n - 8 * (nw - 1);        // row bytes in the last word, 1..8
            const unsigned long long last = hl == 8 ? ~0ull : (1ull << (8 * hl)) - 1ull;
#pragma unroll
            for (int k = 0; k < kBlkRowWords; ++k) {
                unsigned long long x = k < nw ? __ldg(q + k) : 0ull;
                if (k == 0) x &= ~0ull << (8 * off);
                wd[k] = x & (k == nw - 1 ? last : ~0ull);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kBlkRowWords; ++k) wd[k] = 0ull;
        }
    };
    uint32_t e;
    int off, n;
    unsigned long long wd[kBlkRowWords];
    fetch(threadIdx.x, e, off, n, wd);
    for (int r0 = 0; r0 < nrows; r0 += blockDim.x) {
        uint32_t en;
        int offn, nn;
        unsigned long long wn[kBlkRowWords];
        fetch(r0 + (int)blockDim.x + (int)threadIdx.x, en, offn, nn, wn);
        const int dy = (int)(e & 0xffu) - 64, dz = (int)((e >> 8) & 0xffu) - 64;
        const int w = (int)(e >> 16);
        // the warp's longest row bounds the words it walks; a shorter row's
        // extra words are zero, so they only add to the value-0 columns
        const int nw_max = __reduce_max_sync(0xffffffffu, (off + n + 7) >> 3);
        // 32-bit words: voxel t (dx = t - w) adds 1 + (t - w + r) << 11 to A
        // and (dy + r) | (dz + r) << 16 to B.  64-bit word: 1 | (t - w + 32)
        // << 11 | (dy + 32) << 28 | (dz + 32) << 45, built from its 32-bit
        // halves (t only changes bits 11..27)
        const uint32_t row_a = W32 ? 1u + ((uint32_t)(r - w) << 11)
                                   : 1u | ((uint32_t)(32 - w) << 11) | ((uint32_t)(dy + 32) << 28);
        const uint32_t row_b = W32 ? (uint32_t)(dy + r) | ((uint32_t)(dz + r) << 16)
                                   : ((uint32_t)(dy + 32) >> 4) | ((uint32_t)(dz + 32) << 13);
#pragma unroll
        for (int k = 0; k < kBlkRowWords; ++k) {
            if (k >= nw_max) break;
            const unsigned long long x = wd[k];           // masked at fetch
            // byte b is voxel t = 8k + b - off (mod 2^32 arithmetic)
            const uint32_t a_k = row_a + ((uint32_t)(8 * k - off) << 11);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t v =
                    __byte_perm(b < 4 ? (uint32_t)x : (uint32_t)(x >> 32), 0u, 0x4440u + (b & 3));
                if constexpr (W32) {
                    const uint32_t av = a_addr + v * stride;
                    red_add_shared(av, a_k + ((uint32_t)b << 11));
                    if constexpr (BOFF != 0u)
                        red_add_shared_at<BOFF>(av, row_b);
                    else
                        red_add_shared(b_addr + v * stride, row_b);
                } else {
                    const unsigned long long inc =
                        ((unsigned long long)row_b << 32) | (a_k + ((uint32_t)b << 11));
                    red_add_shared_u64(a64 + v * 2u * stride, inc);
                }
            }
        }
        e = en;
        off = offn;
        n = nn;
#pragma unroll
        for (int k = 0; k < kBlkRowWords; ++k) wd[k] = wn[k];
    }
}

// FIXB: the launch's layout reserves 2 kMsBOff bytes of columns, and the B
// words go at kMsBOff when they fit (two 32-bit words per voxel only).
template <bool FIXB>
__device__ void ms_pass(const SeedJob &J, const OffsetTables &ot, unsigned long long *cols,
                        int *acc, const int P[3], int r) {
    const int B = J.vol.B;
    const int NC = ms_columns(__ldg(ot.ball_size + r));
    // two 32-bit words per column where the row sums fit (ot.ms32), else
    // one 64-bit word; the column area is (B + 1) * NC * 8 bytes either way
    const bool w32 = __ldg(ot.ms32 + r) != 0;
    const bool fixed = FIXB && w32 && (uint32_t)((B + 1) * NC * 4) <= kMsBOff;
    // 32-bit word index of the B words (64-bit words: the upper half)
    const int boffw = fixed ? (int)(kMsBOff / 4) : (B + 1) * NC;
    uint32_t *colA = reinterpret_cast<uint32_t *>(cols);
    for (int k = threadIdx.x; k < (B + 1) * NC; k += blockDim.x) {
        colA[k] = 0u;
        colA[boffw + k] = 0u;
    }
    __syncthreads();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    const int col = threadIdx.x & (NC - 1);
    // 32-bit words: A of value v at a_addr + 4 NC v, B at b_addr + 4 NC v;
    // 64-bit words: value v at a64 + 8 NC v
    const uint32_t stride = 4u * (uint32_t)NC;
    const uint32_t a_addr = smem_u32(colA + col);
    const uint32_t b_addr = a_addr + 4u * (uint32_t)boffw;
    const uint32_t a64 = smem_u32(cols + col);
    if (fixed)
        ms_walk_rows<true, kMsBOff>(ot, r, c0, plane, pitch, a_addr, b_addr, a64, stride);
    else if (w32)
        ms_walk_rows<true, 0u>(ot, r, c0, plane, pitch, a_addr, b_addr, a64, stride);
    else
        ms_walk_rows<false, 0u>(ot, r, c0, plane, pitch, a_addr, b_addr, a64, stride);
    __syncthreads();
    // column sums: G threads per bin (the largest power of two up to 32 with
    // G B <= blockDim.x).  Thread q of a bin's group reads its NC / G
    // columns q + G ((k + b) mod (NC / G)): rotated by the bin, so the 32
    // lanes of a warp (32 / G bins) read 32 different banks.  The group adds
    // the unpacked fields with xor shuffles.
    int G = 32;
    while (G > 1 && G * B > (int)blockDim.x) G >>= 1;
    const int per = NC / G, q = threadIdx.x & (G - 1);
    const int shift = w32 ? r : 32;   // the offset added to dx, dy, dz
    for (int b0 = 0; b0 < B; b0 += (int)blockDim.x / G) {
        const int b = b0 + (int)threadIdx.x / G;
        int c = 0, sx = 0, sy = 0, sz = 0;
        if (b < B) {
            for (int k = 0; k < per; ++k) {
                const int cc = q + G * ((k + b) & (per - 1));
                if (w32) {
                    const uint32_t xa = colA[(b + 1) * NC + cc], xb = colA[boffw + (b + 1) * NC + cc];
                    c += (int)(xa & 0x7ffu);
                    sx += (int)(xa >> 11);
                    sy += (int)(xb & 0xffffu);
                    sz += (int)(xb >> 16);
                } else {
                    const unsigned long long x = cols[(b + 1) * NC + cc];
                    c += (int)(x & 0x7ffull);
                    sx += (int)((x >> 11) & 0x1ffffull);
                    sy += (int)((x >> 28) & 0x1ffffull);
                    sz += (int)((x >> 45) & 0x1ffffull);
                }
            }
        }
        for (int o = G >> 1; o; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        if (b < B && q == 0) {
            acc[4 * b] = c;
            acc[4 * b + 1] = sx - shift * c;
            acc[4 * b + 2] = sy - shift * c;
            acc[4 * b + 3] = sz - shift * c;
        }
    }
    __syncthreads();
}

// Warp path: the same sums with one column per lane.  cols holds words A
// of value v at colA[v * 32 + lane] and words B at colA[kMswB + v * 32 +
// lane], v = 0..B <= 32: B words at a fixed distance from the A words for
// every bin count, so a voxel's second reduction takes the A address plus
// an immediate.  Value 0 (not counted, and the masked bytes of a row's
// first and last words) is never read, so a byte costs no branch; acc (B *
// 4 ints) is written over the start once the columns have been read.
constexpr int kMswB = 33 * 32;    // word offset of the B words in a warp region
__device__ void ms_pass_warp(const SeedJob &J, const OffsetTables &ot, unsigned long long *cols,
                             int *acc, const int P[3], int r) {
    const int B = J.vol.B, lane = threadIdx.x & 31;
    uint32_t *colA = reinterpret_cast<uint32_t *>(cols);
    for (int k = lane; k < (B + 1) * 32; k += 32) {
        colA[k] = 0u;
        colA[kMswB + k] = 0u;
    }
    __syncwarp();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    const uint32_t a_addr = smem_u32(colA + lane);               // value v: a_addr + 128 v
    const uint32_t *rows = ot.rows + __ldg(ot.rows_start + r);
    const int nrows = __ldg(ot.rows_start + r + 1) - __ldg(ot.rows_start + r);
    // A lane's rows are lane, lane + 32, ...: the words of the next row are
    // loaded before the current row is counted, so one row's loads are
    // always in flight.  A row of Ball(r <= 20) has at most 41 voxels, which
    // with up to 7 bytes of alignment fit in kRowWords aligned words; the
    // words past a row's last one are not loaded.
    auto fetch = [&](int ri, uint32_t &e, int &off, int &n, unsigned long long (&wd)[kRowWords]) {
        e = 0u;
        off = 0;
        n = 0;
        if (ri < nrows) {
            e = __ldg(rows + ri);
            const int dy = (int)(e & 0xffu) - 64, dz = (int)((e >> 8) & 0xffu) - 64;
            const int w = (int)(e >> 16);
            const uintptr_t a = reinterpret_cast<uintptr_t>(c0 + dz * plane + dy * pitch - w);
            off = (int)(a & 7u);
            n = 2 * w + 1;
            const unsigned long long *q =
                reinterpret_cast<const unsigned long long *>(a & ~uintptr_t(7));
            const int nw = (off + n + 7) >> 3;
            // bytes of the first and last words outside the row count as
            // value 0: masked here once, not per word in the walk
            const int hl = off + n - 8 * (nw - 1);        // row bytes in the last word, 1..8
            const unsigned long long last = hl == 8 ? ~0ull : (1ull << (8 * hl)) - 1ull;
#pragma unroll
            for (int k = 0; k < kRowWords; ++k) {
                unsigned long long x = k < nw ? __ldg(q + k) : 0ull;
                if (k == 0) x &= ~0ull << (8 * off);
                wd[k] = x & (k == nw - 1 ? last : ~0ull);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kRowWords; ++k) wd[k] = 0ull;
        }
    };
    uint32_t e;
    int off, n;
    unsigned long long wd[kRowWords];
    fetch(lane, e, off, n, wd);
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        uint32_t en;
        int offn, nn;
        unsigned long long wn[kRowWords];
        fetch(r0 + 32 + lane, en, offn, nn, wn);
        const int dy = (int)(e & 0xffu) - 64, dz = (int)((e >> 8) & 0xffu) - 64;
        const int w = (int)(e >> 16);
        // the warp's longest row bounds the words it walks
        const int nw_max = __reduce_max_sync(0xffffffffu, (off + n + 7) >> 3);
        // voxel t of the row (dx = t - w) adds 1 + (t - w + 20) << 11 to A
        // and the row constant (dy + 20) | (dz + 20) << 16 to B
        const uint32_t row_a = 1u + ((uint32_t)(20 - w) << 11);
        const uint32_t row_b = (uint32_t)(dy + 20) | ((uint32_t)(dz + 20) << 16);
#pragma unroll
        for (int k = 0; k < kRowWords; ++k) {
            if (k >= nw_max) break;
            const unsigned long long x = wd[k];           // masked at fetch
            // byte b is voxel t = 8k + b - off (mod 2^32 arithmetic)
            const uint32_t a_k = row_a + ((uint32_t)(8 * k - off) << 11);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t v =
                    __byte_perm(b < 4 ? (uint32_t)x : (uint32_t)(x >> 32), 0u, 0x4440u + (b & 3));
                const uint32_t av = a_addr + (v << 7);
                red_add_shared(av, a_k + ((uint32_t)b << 11));
                red_add_shared_at<4u * kMswB>(av, row_b);
            }
        }
        e = en;
        off = offn;
        n = nn;
#pragma unroll
        for (int k = 0; k < kRowWords; ++k) wd[k] = wn[k];
    }
    __syncwarp();
    // lane b sums bins b and b + 32 over the 32 columns, starting at its
    // own column so that the lanes' reads fall in different banks
    int s[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int b = lane + 32 * h;
        if (b < B) {
            for (int k = 0; k < 32; ++k) {
                const uint32_t xa = colA[(b + 1) * 32 + ((k + lane) & 31)];
                const uint32_t xb = colA[kMswB + (b + 1) * 32 + ((k + lane) & 31)];
                s[h][0] += (int)(xa & 0x7ffu);
                s[h][1] += (int)(xa >> 11);
                s[h][2] += (int)(xb & 0xffffu);
                s[h][3] += (int)(xb >> 16);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int b = lane + 32 * h;
        if (b < B) {
            acc[4 * b] = s[h][0];
            for (int k = 1; k < 4; ++k) acc[4 * b + k] = s[h][k] - 20 * s[h][0];
        }
    }
    __syncwarp();
}

// Eq. 5-6 with a flat window, run by one whole warp: w_b = sqrt(N / (B c_b));
// delta = sum_b w_b m_b / sum_b w_b c_b, bins ascending, empty bins skipped.
// prod holds 4 * Bp doubles.  Every lane returns the same delta.
__device__ void ms_delta_warp(int B, const int *acc, double *prod, int step[3]) {
    const int lane = threadIdx.x & 31, Bp = (B + 7) & ~7;
    uint32_t n = 0;
    for (int b = lane; b < B; b += 32) n += (uint32_t)acc[4 * b];
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    const uint32_t N = n;
    // The products of the occupied bins, packed in bin order: an empty bin
    // would add +0.0, which leaves every partial sum unchanged (no product
    // and so no partial sum is -0.0), so the chains below run over the
    // occupied bins only and still give the sums over all bins in bin
    // order.  The packed list is padded with +0.0 to a multiple of 8.
    int K = 0;
    for (int b0 = 0; b0 < B; b0 += 32) {
        const int b = b0 + lane;
        const int c = b < B ? acc[4 * b] : 0;
        const unsigned occ = __ballot_sync(0xffffffffu, c > 0);
        if (c > 0) {
            const int k = K + __popc(occ & ((1u << lane) - 1u));
            const double w = __dsqrt_rn(__ddiv_rn((double)N, (double)((int64_t)B * c)));
            for (int a = 0; a < 3; ++a) prod[a * Bp + k] = __dmul_rn(w, (double)acc[4 * b + 1 + a]);
            prod[3 * Bp + k] = __dmul_rn(w, (double)c);
        }
        K += __popc(occ);
    }
    const int Kp = (K + 7) & ~7;
    for (int k = K + lane; k < Kp; k += 32)
        for (int a = 0; a < 4; ++a) prod[a * Bp + k] = 0.0;
    __syncwarp();
    // lane a < 4 sums chain a (three numerators, the denominator)
    const double s = lane < 4 ? chain_sum(prod + lane * Bp, Kp) : 0.0;
    const double den = __shfl_sync(0xffffffffu, s, 3);
    const int d = lane < 3 && N != 0 ? (int)round(__ddiv_rn(s, den)) : 0;
    for (int a = 0; a < 3; ++a) step[a] = __shfl_sync(0xffffffffu, d, a);
    __syncwarp();
}

// The item's result, run by one whole warp: rho = sum_b sqrt(c_b / (N B))
// and H, bins ascending.  Per bin the terms are formed in parallel (+0.0
// for the bins a sum skips: empty bins for rho, c <= 1 for the entropy sum,
// whose table values are +0.0), then lanes 0 and 1 add up one chain each.
__device__ void ms_result_warp(const SeedJob &J, int64_t item, const int *acc, double *prod,
                               const double *T, const double *L, const int P[3], int r, int it,
                               int conv) {
    const int B = J.vol.B, Bp = (B + 7) & ~7, lane = threadIdx.x & 31;
    uint32_t n = 0;
    int occ = 0;
    for (int b = lane; b < B; b += 32) {
        n += (uint32_t)acc[4 * b];
        occ += acc[4 * b] > 0;
    }
    for (int o = 16; o; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        occ += __shfl_xor_sync(0xffffffffu, occ, o);
    }
    const uint32_t N = n;
    for (int b = lane; b < Bp; b += 32) {
        const int c = b < B ? acc[4 * b] : 0;
        prod[b] = c > 0 ? __dsqrt_rn(__ddiv_rn((double)c, (double)((int64_t)N * B))) : 0.0;
        prod[Bp + b] = c > 1 ? __ldg(T + c) : 0.0;
    }
    __syncwarp();
    const double chain = lane < 2 ? chain_sum(prod + lane * Bp, Bp) : 0.0;
    const double s = __shfl_sync(0xffffffffu, chain, 1);
    if (lane == 0) {
        ks_ms_result *o = J.ms_out + item;
        o->x = P[0];
        o->y = P[1];
        o->z = P[2];
        o->r = r;
        o->seed = (int32_t)(item / J.S);
        o->iters = it;
        o->converged = conv;
        o->reserved = 0;
        o->rho = chain;
        o->H = entropy_from_sum(s, N, occ, L);
    }
    __syncwarp();
}

template <bool FIXB>
__device__ void ms_item(const SeedJob &J, int64_t item, const OffsetTables &ot, const double *T,
                        const double *L, unsigned long long *cols, int *acc, double *prod,
                        SeedShared &sh) {
    const int dims[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    const int64_t sidx = item / J.S;
    const int r = J.r_min + (int)(item % J.S);
    int P[3] = {J.seeds[3 * sidx], J.seeds[3 * sidx + 1], J.seeds[3 * sidx + 2]};
    int it = 0, conv = 0, fresh = 0;
    int4 *stp = J.state ? J.state + J.n_seeds + item : nullptr;
    if (stp) {
        const int4 st = *stp;
        if (st.w & kItemDone) return;
        if (st.w & kItemStarted) {
            P[0] = st.x;
            P[1] = st.y;
            P[2] = st.z;
            it = st.w & 255;
        }
    }
    const int it_end = J.iter_budget > 0 ? min(J.max_iter, it + J.iter_budget) : J.max_iter;
    while (it < it_end) {
        ms_pass<FIXB>(J, ot, cols, acc, P, r);
        if (threadIdx.x < 32) {
            int d[3];
            ms_delta_warp(J.vol.B, acc, prod, d);
            if (threadIdx.x == 0)
                for (int a = 0; a < 3; ++a) sh.step[a] = d[a];
        }
        __syncthreads();
        fresh = 1;
        ++it;
        int Pn[3];
        for (int a = 0; a < 3; ++a) Pn[a] = clampi(P[a] + sh.step[a], 0, dims[a] - 1);
        __syncthreads();
        if (Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2]) {
            conv = 1;
            break;
        }
        for (int a = 0; a < 3; ++a) P[a] = Pn[a];
        fresh = 0;
    }
    if (stp && !conv && it < J.max_iter) {   // the budget ran out: keep the state
        __syncthreads();
        if (threadIdx.x == 0) *stp = make_int4(P[0], P[1], P[2], it | kItemStarted);
        return;
    }
    if (!fresh) ms_pass<FIXB>(J, ot, cols, acc, P, r);
    if (threadIdx.x < 32) ms_result_warp(J, item, acc, prod, T, L, P, r, it, conv);
    if (stp && threadIdx.x == 0) {
        *stp = make_int4(P[0], P[1], P[2], it | kItemStarted | kItemDone);
        atomicAdd(J.finished, 1u);
    }
    __syncthreads();
}

// One item on one warp; region is the warp's own 8448 bytes.
__device__ void ms_item_warp(const SeedJob &J, int64_t item, const OffsetTables &ot,
                             const double *T, const double *L, unsigned long long *region) {
    const int dims[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    const int B = J.vol.B;
    int *acc = reinterpret_cast<int *>(region);
    double *prod = reinterpret_cast<double *>(reinterpret_cast<uint8_t *>(region) +
                                              ((B * 16 + 15) & ~15));
    const int64_t sidx = item / J.S;
    const int r = J.r_min + (int)(item % J.S);
    int P[3] = {J.seeds[3 * sidx], J.seeds[3 * sidx + 1], J.seeds[3 * sidx + 2]};
    int it = 0, conv = 0, fresh = 0;
    int4 *stp = J.state ? J.state + J.n_seeds + item : nullptr;
    if (stp) {
        const int4 st = *stp;
        if (st.w & kItemDone) return;
        if (st.w & kItemStarted) {
            P[0] = st.x;
            P[1] = st.y;
            P[2] = st.z;
            it = st.w & 255;
        }
    }
    const int it_end = J.iter_budget > 0 ? min(J.max_iter, it + J.iter_budget) : J.max_iter;
    while (it < it_end) {
        ms_pass_warp(J, ot, region, acc, P, r);
        int d[3];
        ms_delta_warp(B, acc, prod, d);
        fresh = 1;
        ++it;
        int Pn[3];
        for (int a = 0; a < 3; ++a) Pn[a] = clampi(P[a] + d[a], 0, dims[a] - 1);
        if (Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2]) {
            conv = 1;
            break;
        }
        for (int a = 0; a < 3; ++a) P[a] = Pn[a];
        fresh = 0;
    }
    if (stp && !conv && it < J.max_iter) {   // the budget ran out: keep the state
        __syncwarp();
        if ((threadIdx.x & 31) == 0) *stp = make_int4(P[0], P[1], P[2], it | kItemStarted);
        return;
    }
    if (!fresh) ms_pass_warp(J, ot, region, acc, P, r);
    ms_result_warp(J, item, acc, prod, T, L, P, r, it, conv);
    if (stp && (threadIdx.x & 31) == 0) {
        *stp = make_int4(P[0], P[1], P[2], it | kItemStarted | kItemDone);
        atomicAdd(J.finished, 1u);
    }
    __syncwarp();
}

// Shared-memory layout of one block (the octant and mean-shift views
// overlap; a block runs one ticket at a time).  kinds: bit k set when the
// launch carries tickets of kind k.
struct Layout {
    size_t cnt, hb, oct_total;                  // octant: cnt[9][S][B+1] u32, hb[8S] f64
    size_t cols, acc, prod, msb_total;          // mean shift, block path
    size_t msw, msw_stride, msw_total;          // mean shift, warp path: 8 regions
    int kinds;
    __host__ __device__ Layout(int B, int S, int kinds_) : kinds(kinds_) {
        cnt = 0;
        hb = ((size_t)9 * S * (B + 1) * 4 + 15) / 16 * 16;
        oct_total = hb + (size_t)8 * S * 8;
        cols = 0;                                   // (B + 1) * NC words of 8 bytes, NC <= 128
        acc = (size_t)(B + 1) * 128 * 8;
        if ((kinds & kMsBlockOnly) && acc < 2 * (size_t)kMsBOff) acc = 2 * (size_t)kMsBOff;
        prod = acc + (size_t)B * 4 * 4;
        msb_total = prod + (size_t)4 * ((B + 7) & ~7) * 8;   // 4 chains of Bp doubles
        // a warp region holds 2 * 33 * 32 column words, later acc (16 B
        // bytes) and 4 chains of Bp doubles: 16 B + 32 (B + 7) <= 8448
        msw = 0;
        msw_stride = (size_t)kMswB * 8;             // A and B words of 33 values
        msw_total = B <= kWarpMsBmax ? msw + (kSeedThreads / 32) * msw_stride : 0;
    }
    __host__ __device__ size_t total() const {
        size_t t = 0;
        if (kinds & (1 << kOctant)) t = oct_total;
        if (kinds & (1 << kMeanShift)) {
            t = msb_total > t ? msb_total : t;
            t = msw_total > t ? msw_total : t;
        }
        return t;
    }
};

// KINDS: bit k set when the launch carries tickets of kind k; one
// instantiation per combination, so each gets its own register allocation.
template <int KINDS>
__global__ void __launch_bounds__(KINDS == 1 ? kOctThreads : kSeedThreads,
                                  KINDS == 1 ? 6
                                  : KINDS == 2 ? 2
                                  : KINDS == ((1 << kMeanShift) | kMsBlockOnly) ? 3
                                                                                : 1)
    k_seeds(const SeedQueue q, const OffsetTables ot,
                                                        const double *__restrict__ T,
                                                        const double *__restrict__ L,
                                                        int max_B, int max_S, int persistent) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ SeedShared sh;
    const Layout lay(max_B, max_S, KINDS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t round = 0;; ++round) {
        if (threadIdx.x == 0)
            sh.ticket = persistent ? (int64_t)atomicAdd(q.head, 1ull)
                                   : (round == 0 ? (int64_t)blockIdx.x : q.n_tickets);
        __syncthreads();
        const int64_t t = sh.ticket;
        __syncthreads();
        if (t >= q.n_tickets) return;
        int seg = 0;
        while (seg + 1 < q.n_segs && t >= q.seg_start[seg + 1]) ++seg;
        const SeedJob &J = q.jobs[q.seg_job[seg]];
        const int64_t local = t - q.seg_start[seg];
        if (q.seg_kind[seg] == kOctant) {
            if constexpr ((KINDS & (1 << kOctant)) != 0)
                octant_item(J, local, ot, T, L,
                            reinterpret_cast<uint32_t *>(smem + lay.cnt),
                            reinterpret_cast<double *>(smem + lay.hb), sh);
            continue;
        }
        if constexpr ((KINDS & (1 << kMeanShift)) == 0) {
            continue;
        } else {
        if (q.seg_kind[seg] == kMeanShift) {
            // one item of a radius above kWarpMsRmax on the whole block,
            // largest radius first
            const int64_t r_idx = J.S - 1 - local / J.n_seeds;   // a block-path radius
            const int64_t item = (local % J.n_seeds) * J.S + r_idx;
            ms_item<(KINDS & kMsBlockOnly) != 0>(
                J, item, ot, T, L, reinterpret_cast<unsigned long long *>(smem + lay.cols),
                    reinterpret_cast<int *>(smem + lay.acc),
                    reinterpret_cast<double *>(smem + lay.prod), sh);
            continue;
        }
        if constexpr ((KINDS & kMsBlockOnly) != 0) {
            continue;                         // no warp-path items in such a launch
        } else {
        // kMsWarp: items of radii <= kWarpMsRmax, one per warp.  Their
        // segments follow every other segment of the queue, so from the
        // first such ticket on each warp draws its own tickets and the block
        // never synchronises again: an item that takes long holds only its
        // own warp.  (Without a persistent queue a block runs its one ticket
        // on warp 0.)
        unsigned long long *region =
            reinterpret_cast<unsigned long long *>(smem + lay.msw + warp * lay.msw_stride);
        int64_t tw = warp == 0 ? t : -1;
        int sw = seg;
        for (;;) {
            if (tw < 0) {
                if (!persistent) break;
                unsigned long long x = 0;
                if (lane == 0) x = atomicAdd(q.head, 1ull);
                tw = (int64_t)__shfl_sync(0xffffffffu, x, 0);
            }
            if (tw >= q.n_tickets) break;
            while (sw + 1 < q.n_segs && tw >= q.seg_start[sw + 1]) ++sw;
            const SeedJob &Jw = q.jobs[q.seg_job[sw]];
            const int64_t lw = tw - q.seg_start[sw];
            // largest radius first, consecutive seeds side by side (their
            // windows overlap, so concurrent warps share L1 lines)
            const int S_small = Jw.S - ms_block_radii(Jw.r_min, Jw.S, Jw.vol.B);
            const int64_t r_idx = S_small - 1 - lw / Jw.n_seeds;
            ms_item_warp(Jw, (lw % Jw.n_seeds) * Jw.S + r_idx, ot, T, L, region);
            tw = -1;
        }
        return;
        }
        }
    }
}

}  // namespace

int64_t seed_tickets(int kind, int64_t n_seeds, int r_min, int S, int B) {
    if (kind == kOctant) return n_seeds;
    const int S_big = ms_block_radii(r_min, S, B);
    return n_seeds * (kind == kMeanShift ? S_big : S - S_big);
}

// The kinds of the instantiation a launch of these kinds uses with at most
// max_B bins: mean shift alone with more than kWarpMsBmax bins has only
// block-path items.
static int launch_kinds(int kinds, int max_B) {
    return kinds == (1 << kMeanShift) && max_B > kWarpMsBmax ? kinds | kMsBlockOnly : kinds;
}

size_t seed_smem_bytes(int B, int S, int kinds) {
    return Layout(B, S, launch_kinds(kinds, B)).total();
}

using SeedKernel = void (*)(const SeedQueue, const OffsetTables, const double *, const double *,
                            int, int, int);
static int seed_threads(int kinds) { return kinds == (1 << kOctant) ? kOctThreads : kSeedThreads; }

static SeedKernel seed_kernel(int kinds, int max_B) {
    if (launch_kinds(kinds, max_B) & kMsBlockOnly) return k_seeds<(1 << kMeanShift) | kMsBlockOnly>;
    return kinds == (1 << kOctant) ? k_seeds<1 << kOctant>
           : kinds == (1 << kMeanShift) ? k_seeds<1 << kMeanShift>
                                        : k_seeds<(1 << kOctant) | (1 << kMeanShift)>;
}

int seed_blocks_per_sm(int max_B, int max_S, int kinds) {
    // the occupancy query honours the kernel's dynamic shared-memory limit,
    // so raise it to this layout's size first
    const size_t smem = seed_smem_bytes(max_B, max_S, kinds);
    const SeedKernel k = seed_kernel(kinds, max_B);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, seed_threads(kinds), smem);
    return n < 1 ? 1 : n;
}

cudaError_t launch_seeds(const LaunchCtx &lc, const SeedQueue &q, const OffsetTables &ot,
                         const double *T, const double *L, int max_B, int max_S, int kinds,
                         bool persistent, int grid) {
    const size_t smem = seed_smem_bytes(max_B, max_S, kinds);
    const SeedKernel k = seed_kernel(kinds, max_B);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, seed_threads(kinds), smem, lc.stream>>>(q, ot, T, L, max_B, max_S, persistent ? 1 : 0);
    return cudaGetLastError();
}

// Shared-memory histogram-increment rate: each lane adds bytes read from a
// shared byte array into its own conflict-free counter column, the access
// pattern of the dense kernel's inner loop (one byte load and one
// red.shared.add per voxel).
__global__ void __launch_bounds__(256) k_smem_peak(uint32_t *sink, int iters) {
    __shared__ __align__(16) uint8_t bins[4096];
    __shared__ uint32_t cnt[8][33 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) bins[i] = (uint8_t)((i * 7 + (i >> 5)) % 33);
    for (int i = lane; i < 33 * 32; i += 32) cnt[warp][i] = 0;
    __syncthreads();
    const uint32_t col = smem_u32(&cnt[warp][lane]);
    const uint8_t *p = bins + warp * 64 + lane;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t v = p[(it * 16 + u) * 97 & 2047];
            red_add_shared(col + (v << 7), 1u);
        }
    }
    __syncwarp();
    uint32_t acc = 0;
    for (int w = 0; w < 33; ++w) acc += ld_shared_u32(col + (w << 7));
    if (acc == 0xdeadbeefu) sink[blockIdx.x] = acc;   // keeps the work observable
}

// Shared-memory reduction rate alone: the same lane-private columns, but
// every update is a red.shared.add at an address known at compile time
// (the lane's column plus a constant word), so the kernel issues nothing
// else -- no byte loads, no address arithmetic.  The ceiling of any
// histogram kernel that makes one reduction per update.
__global__ void __launch_bounds__(256) k_smem_red_peak(uint32_t *sink, int iters) {
    __shared__ uint32_t cnt[8][33 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = lane; i < 33 * 32; i += 32) cnt[warp][i] = 0;
    __syncwarp();
    const uint32_t col = smem_u32(&cnt[warp][lane]);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) red_add_shared(col + (uint32_t)(((u * 5 + 3) % 33) << 7), 1u);
    }
    __syncwarp();
    uint32_t acc = 0;
    for (int w = 0; w < 33; ++w) acc += ld_shared_u32(col + (w << 7));
    if (acc == 0xdeadbeefu) sink[blockIdx.x] = acc;   // keeps the work observable
}

cudaError_t launch_smem_peak(const LaunchCtx &lc, uint32_t *sink, int blocks, int iters,
                             bool red_only) {
    if (red_only)
        k_smem_red_peak<<<blocks, 256, 0, lc.stream>>>(sink, iters);
    else
        k_smem_peak<<<blocks, 256, 0, lc.stream>>>(sink, iters);
    return cudaGetLastError();
}

// FP64 addition rate: every thread runs 8 independent chains of
// __dadd_rn (the entropy and step sums' operation), so the pipe, not the
// 8-deep dependency, limits the rate once a few warps are resident.
__global__ void __launch_bounds__(256) k_fp64_peak(double *sink, int iters, double inc) {
    double s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = (double)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] = __dadd_rn(s[k], inc);
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = __dadd_rn(acc, s[k]);
    if (acc == -1.0) sink[blockIdx.x] = acc;           // keeps the work observable
}

cudaError_t launch_fp64_peak(const LaunchCtx &lc, double *sink, int blocks, int iters) {
    k_fp64_peak<<<blocks, 256, 0, lc.stream>>>(sink, iters, 1.0e-9);
    return cudaGetLastError();
}

}  // namespace ks
