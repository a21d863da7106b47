// Seed-grid searches: octant hill-climbing (Sec. 2.2, Alg. 1 in 3D) and
// mean shift towards the uniform pmf (Sec. 2.3, Eq. 4-6).
//
// One block of 256 threads owns one item at a time: an octant seed (all
// its iterations plus the final Kadir-Brady evaluation) or one (seed, r)
// mean-shift item.  The same kernel serves a plain launch (block i takes
// item i) and the persistent batched launch (blocks pull items from a
// device counter until the queue is empty), so the arithmetic of an item
// does not depend on how it was scheduled.
//
// Per iteration the block walks the window's offsets (the Ball(32) table,
// sorted by radius class so that Ball(r) is a prefix), threads striding
// over offsets so that a warp reads 32 neighbouring voxels of a row, and
// accumulates integer counts (and, for mean shift, integer offset sums)
// with shared-memory atomics.  Everything accumulated per voxel is an
// integer, so the order of accumulation cannot change any result; the
// FP64 steps run afterwards in one fixed order (bins ascending, octants
// 0..7), each step a single IEEE operation.
#include "ks_internal.cuh"

namespace ks {
namespace {

struct SeedShared {
    int P[3];
    int step[3];
    int64_t item;
    uint32_t N[kMaxScales];
    unsigned long long D[kMaxScales];
};

struct Smem {
    uint32_t *cnt;     // octant: [8][S][B]; final KB: [S][B]; mean shift: [B][4]
    double *hb;        // octant: [8][S] entropies; KB: [S]; mean shift: [4][B]
};

__device__ __forceinline__ const uint8_t *voxel_ptr(const VolDesc &v, const int P[3]) {
    return v.base + (int64_t)P[2] * v.plane + (int64_t)P[1] * v.pitch + P[0];
}

__device__ __forceinline__ void unpack_offset(uint32_t e, int &dx, int &dy, int &dz, int &rho) {
    dx = (int)(e & 0xffu) - 64;
    dy = (int)((e >> 8) & 0xffu) - 64;
    dz = (int)((e >> 16) & 0xffu) - 64;
    rho = (int)(e >> 24);
}

// Entropy of counts c[0..B) (bin order), the library's fixed formula.
__device__ double window_entropy(const uint32_t *c, int B, const double *T, const double *L,
                                 uint32_t *N_out) {
    uint32_t N = 0;
    int occ = 0;
    double s = 0.0;
    for (int b = 0; b < B; ++b) {
        const uint32_t x = c[b];
        N += x;
        occ += x > 0u;
        if (x > 1u) s = __dadd_rn(s, __ldg(T + x));
    }
    if (N_out) *N_out = N;
    return entropy_from_sum(s, N, occ, L);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// ---------------------------------------------------------------- octant
// Counts of the 8 closed octants of every shell at P, then prefix sums over
// shells (so cnt[j][si] is the histogram of octant j of Ball(r_min + si)),
// then the 8*S entropies into hb[j*S + si].
__device__ void octant_histograms(const SeedJob &J, const BallTables &bt, const double *T,
                                  const double *L, const Smem &m, const int P[3]) {
    const int B = J.vol.B, S = J.S;
    for (int k = threadIdx.x; k < 8 * S * B; k += blockDim.x) m.cnt[k] = 0;
    __syncthreads();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int nball = __ldg(bt.ball_size + J.r_max);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    for (int k = threadIdx.x; k < nball; k += blockDim.x) {
        int dx, dy, dz, rho;
        unpack_offset(__ldg(bt.ball + k), dx, dy, dz, rho);
        const uint32_t v = __ldg(c0 + dz * plane + dy * pitch + dx);
        if (v == 0u) continue;
        const int si = rho > J.r_min ? rho - J.r_min : 0;
        // allowed j-bit values per axis: bit 0 -> positive side, bit 1 -> negative
        const int ax = dx > 0 ? 1 : (dx < 0 ? 2 : 3);
        const int ay = dy > 0 ? 1 : (dy < 0 ? 2 : 3);
        const int az = dz > 0 ? 1 : (dz < 0 ? 2 : 3);
        uint32_t *base = m.cnt + si * B + (v - 1);
        for (int jz = 0; jz < 2; ++jz) {
            if (!(az & (1 << jz))) continue;
            for (int jy = 0; jy < 2; ++jy) {
                if (!(ay & (1 << jy))) continue;
                for (int jx = 0; jx < 2; ++jx) {
                    if (!(ax & (1 << jx))) continue;
                    const int j = jx | (jy << 1) | (jz << 2);
                    atomicAdd(base + j * S * B, 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int col = threadIdx.x; col < 8 * B; col += blockDim.x) {
        const int j = col / B, b = col % B;
        uint32_t run = 0;
        for (int si = 0; si < S; ++si) {
            run += m.cnt[(j * S + si) * B + b];
            m.cnt[(j * S + si) * B + b] = run;
        }
    }
    __syncthreads();
    for (int w = threadIdx.x; w < 8 * S; w += blockDim.x)
        m.hb[w] = window_entropy(m.cnt + w * B, B, T, L, nullptr);
    __syncthreads();
}

// Alg. 1's update from the octant entropies: eps_j = max over scales (the
// smallest r on ties), d_j = k_j sigma_j, delta = sum_j eps_j d_j / sum_j
// eps_j summed over j = 0..7, rounded half away from zero.
__device__ void octant_step(const SeedJob &J, const Smem &m, int step[3]) {
    const int S = J.S;
    double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
    for (int j = 0; j < 8; ++j) {
        double best = m.hb[j * S];
        int k = J.r_min;
        for (int si = 1; si < S; ++si)
            if (m.hb[j * S + si] > best) {
                best = m.hb[j * S + si];
                k = J.r_min + si;
            }
        const int sg[3] = {(j & 1) ? -1 : 1, (j & 2) ? -1 : 1, (j & 4) ? -1 : 1};
        for (int a = 0; a < 3; ++a)
            num[a] = __dadd_rn(num[a], __dmul_rn(best, (double)(k * sg[a])));
        den = __dadd_rn(den, best);
    }
    for (int a = 0; a < 3; ++a) step[a] = den == 0.0 ? 0 : (int)round(__ddiv_rn(num[a], den));
}

// Kadir-Brady on the full ball at P (after the climb): H(r), D(r), peaks,
// W and Y at peaks.  Writes s_best, Y_best, H_best, W_best.
__device__ void kb_at(const SeedJob &J, const BallTables &bt, const double *T, const double *L,
                      const Smem &m, SeedShared &sh, const int P[3], int32_t *s_best,
                      double *Y_best, double *H_best, double *W_best) {
    const int B = J.vol.B, S = J.S;
    for (int k = threadIdx.x; k < S * B; k += blockDim.x) m.cnt[k] = 0;
    __syncthreads();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int nball = __ldg(bt.ball_size + J.r_max);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    for (int k = threadIdx.x; k < nball; k += blockDim.x) {
        int dx, dy, dz, rho;
        unpack_offset(__ldg(bt.ball + k), dx, dy, dz, rho);
        const uint32_t v = __ldg(c0 + dz * plane + dy * pitch + dx);
        if (v == 0u) continue;
        const int si = rho > J.r_min ? rho - J.r_min : 0;
        atomicAdd(m.cnt + si * B + (v - 1), 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        uint32_t run = 0;
        for (int si = 0; si < S; ++si) {
            run += m.cnt[si * B + b];
            m.cnt[si * B + b] = run;
        }
    }
    __syncthreads();
    for (int si = threadIdx.x; si < S; si += blockDim.x) {
        uint32_t N;
        m.hb[si] = window_entropy(m.cnt + si * B, B, T, L, &N);
        sh.N[si] = N;
    }
    __syncthreads();
    for (int si = 1 + threadIdx.x; si < S; si += blockDim.x) {
        const uint32_t *c = m.cnt + si * B, *p = m.cnt + (si - 1) * B;
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
        double yb = 0.0, hb = 0.0, wb = 0.0;
        int sb = 0;
        for (int i = 1; i + 1 < S; ++i) {
            if (m.hb[i - 1] < m.hb[i] && m.hb[i] >= m.hb[i + 1]) {
                const double W = kb_weight(sh.D[i], sh.N[i], sh.N[i - 1], J.r_min + i, J.w_norm);
                const double y = __dmul_rn(m.hb[i], W);
                if (sb == 0 || y > yb) {
                    yb = y;
                    sb = J.r_min + i;
                    hb = m.hb[i];
                    wb = W;
                }
            }
        }
        *s_best = sb;
        *Y_best = yb;
        *H_best = hb;
        *W_best = wb;
    }
    __syncthreads();
}

__device__ void octant_item(const SeedJob &J, int64_t sidx, const BallTables &bt,
                            const double *T, const double *L, const Smem &m, SeedShared &sh) {
    const int dims[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    int P[3] = {J.seeds[3 * sidx], J.seeds[3 * sidx + 1], J.seeds[3 * sidx + 2]};
    const int T1 = J.max_iter + 1;
    if (threadIdx.x == 0 && J.traj)
        for (int a = 0; a < 3; ++a) J.traj[(sidx * T1) * 3 + a] = P[a];
    int it = 0, conv = 0;
    while (it < J.max_iter) {
        octant_histograms(J, bt, T, L, m, P);
        if (threadIdx.x == 0) octant_step(J, m, sh.step);
        __syncthreads();
        ++it;
        int Pn[3];
        for (int a = 0; a < 3; ++a) Pn[a] = clampi(P[a] + sh.step[a], 0, dims[a] - 1);
        __syncthreads();
        if (Pn[0] == P[0] && Pn[1] == P[1] && Pn[2] == P[2]) {
            conv = 1;
            break;
        }
        for (int a = 0; a < 3; ++a) P[a] = Pn[a];
        if (threadIdx.x == 0 && J.traj)
            for (int a = 0; a < 3; ++a) J.traj[(sidx * T1 + it) * 3 + a] = P[a];
    }
    if (threadIdx.x == 0 && J.traj)
        for (int t = it + (conv ? 0 : 1); t <= J.max_iter; ++t)
            for (int a = 0; a < 3; ++a) J.traj[(sidx * T1 + t) * 3 + a] = P[a];
    ks_seed_result *o = J.oct_out + sidx;
    int32_t sb;
    double yb, hbv, wbv;
    kb_at(J, bt, T, L, m, sh, P, &sb, &yb, &hbv, &wbv);
    if (threadIdx.x == 0) {
        o->x = P[0];
        o->y = P[1];
        o->z = P[2];
        o->seed_x = J.seeds[3 * sidx];
        o->seed_y = J.seeds[3 * sidx + 1];
        o->seed_z = J.seeds[3 * sidx + 2];
        o->iters = it;
        o->converged = conv;
        o->s_best = sb;
        o->reserved = 0;
        o->Y_best = yb;
        o->H_best = hbv;
        o->W_best = wbv;
    }
}

// ------------------------------------------------------------ mean shift
// Counts c_b and integer offset sums m_b of Ball(r) at P into cnt[b][4].
__device__ void ms_moments(const SeedJob &J, const BallTables &bt, const Smem &m, const int P[3],
                           int r) {
    const int B = J.vol.B;
    int *acc = reinterpret_cast<int *>(m.cnt);
    for (int k = threadIdx.x; k < 4 * B; k += blockDim.x) acc[k] = 0;
    __syncthreads();
    const uint8_t *c0 = voxel_ptr(J.vol, P);
    const int nb = __ldg(bt.ball_size + r);
    const int plane = (int)J.vol.plane, pitch = (int)J.vol.pitch;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        int dx, dy, dz, rho;
        unpack_offset(__ldg(bt.ball + k), dx, dy, dz, rho);
        const uint32_t v = __ldg(c0 + dz * plane + dy * pitch + dx);
        if (v == 0u) continue;
        int *a = acc + 4 * (v - 1);
        atomicAdd(a, 1);
        if (dx) atomicAdd(a + 1, dx);
        if (dy) atomicAdd(a + 2, dy);
        if (dz) atomicAdd(a + 3, dz);
    }
    __syncthreads();
}

// Eq. 5-6 with a flat window: w_b = sqrt(N / (B c_b)); delta = sum_b w_b m_b /
// sum_b w_b c_b, bins ascending, empty bins skipped.
__device__ void ms_step(const SeedJob &J, const Smem &m, SeedShared &sh) {
    const int B = J.vol.B;
    const int *acc = reinterpret_cast<const int *>(m.cnt);
    if (threadIdx.x < 32) {
        uint32_t n = 0;
        for (int b = threadIdx.x; b < B; b += 32) n += (uint32_t)acc[4 * b];
        for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        const uint32_t N = n;
        for (int b = threadIdx.x; b < B; b += 32) {
            const int c = acc[4 * b];
            if (c > 0) {
                const double w = __dsqrt_rn(__ddiv_rn((double)N, (double)((int64_t)B * c)));
                for (int a = 0; a < 3; ++a) m.hb[a * B + b] = __dmul_rn(w, (double)acc[4 * b + 1 + a]);
                m.hb[3 * B + b] = __dmul_rn(w, (double)c);
            }
        }
        __syncwarp();
        if (threadIdx.x == 0) {
            if (N == 0) {
                sh.step[0] = sh.step[1] = sh.step[2] = 0;
            } else {
                double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
                for (int b = 0; b < B; ++b) {
                    if (acc[4 * b] == 0) continue;
                    for (int a = 0; a < 3; ++a) num[a] = __dadd_rn(num[a], m.hb[a * B + b]);
                    den = __dadd_rn(den, m.hb[3 * B + b]);
                }
                for (int a = 0; a < 3; ++a) sh.step[a] = (int)round(__ddiv_rn(num[a], den));
            }
        }
    }
    __syncthreads();
}

__device__ void ms_item(const SeedJob &J, int64_t item, const BallTables &bt, const double *T,
                        const double *L, const Smem &m, SeedShared &sh) {
    const int dims[3] = {J.vol.nx, J.vol.ny, J.vol.nz};
    const int B = J.vol.B;
    const int64_t sidx = item / J.S;
    const int r = J.r_min + (int)(item % J.S);
    int P[3] = {J.seeds[3 * sidx], J.seeds[3 * sidx + 1], J.seeds[3 * sidx + 2]};
    int it = 0, conv = 0, fresh = 0;
    while (it < J.max_iter) {
        ms_moments(J, bt, m, P, r);
        ms_step(J, m, sh);
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
    if (!fresh) ms_moments(J, bt, m, P, r);
    const int *acc = reinterpret_cast<const int *>(m.cnt);
    // rho = sum_b sqrt(c_b / (N B)) and H, bins ascending.
    if (threadIdx.x < 32) {
        uint32_t n = 0;
        for (int b = threadIdx.x; b < B; b += 32) n += (uint32_t)acc[4 * b];
        for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        const uint32_t N = n;
        for (int b = threadIdx.x; b < B; b += 32) {
            const int c = acc[4 * b];
            m.hb[b] = c > 0 ? __dsqrt_rn(__ddiv_rn((double)c, (double)((int64_t)N * B))) : 0.0;
        }
        __syncwarp();
        if (threadIdx.x == 0) {
            double rho = 0.0;
            int occ = 0;
            double s = 0.0;
            for (int b = 0; b < B; ++b) {
                const uint32_t c = (uint32_t)acc[4 * b];
                if (c > 0u) rho = __dadd_rn(rho, m.hb[b]);
                occ += c > 0u;
                if (c > 1u) s = __dadd_rn(s, __ldg(T + c));
            }
            ks_ms_result *o = J.ms_out + item;
            o->x = P[0];
            o->y = P[1];
            o->z = P[2];
            o->r = r;
            o->seed = (int32_t)sidx;
            o->iters = it;
            o->converged = conv;
            o->reserved = 0;
            o->rho = rho;
            o->H = entropy_from_sum(s, N, occ, L);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSeedThreads) k_seeds(const SeedQueue q, const BallTables bt,
                                                        const double *__restrict__ T,
                                                        const double *__restrict__ L,
                                                        int max_B, int max_S, int persistent) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ SeedShared sh;
    Smem m;
    const size_t cnt_bytes = ((size_t)8 * max_S * max_B * 4 + 15) / 16 * 16;
    m.cnt = reinterpret_cast<uint32_t *>(smem);
    m.hb = reinterpret_cast<double *>(smem + cnt_bytes);
    for (int64_t round = 0;; ++round) {
        if (threadIdx.x == 0)
            sh.item = persistent ? (int64_t)atomicAdd(q.head, 1ull)
                                 : (round == 0 ? (int64_t)blockIdx.x : q.n_items);
        __syncthreads();
        const int64_t item = sh.item;
        __syncthreads();
        if (item >= q.n_items) return;
        int seg = 0;
        while (seg + 1 < q.n_segs && item >= q.seg_start[seg + 1]) ++seg;
        const SeedJob &J = q.jobs[q.seg_job[seg]];
        const int64_t local = item - q.seg_start[seg];
        if (q.seg_kind[seg] == kOctant)
            octant_item(J, local, bt, T, L, m, sh);
        else
            ms_item(J, local, bt, T, L, m, sh);
    }
}

}  // namespace

size_t seed_smem_bytes(int B, int S) {
    const size_t cnt = ((size_t)8 * S * B * 4 + 15) / 16 * 16;
    const size_t hb = (size_t)(8 * S > 4 * B ? 8 * S : 4 * B) * 8;
    return cnt + hb;
}

int seed_blocks_per_sm(int max_B, int max_S) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seeds, kSeedThreads,
                                                  seed_smem_bytes(max_B, max_S));
    return n < 1 ? 1 : n;
}

cudaError_t launch_seeds(const LaunchCtx &lc, const SeedQueue &q, const BallTables &bt,
                         const double *T, const double *L, int max_B, int max_S,
                         bool persistent, int grid) {
    const size_t smem = seed_smem_bytes(max_B, max_S);
    cudaError_t e =
        cudaFuncSetAttribute(k_seeds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_seeds<<<grid, kSeedThreads, smem, lc.stream>>>(q, bt, T, L, max_B, max_S,
                                                     persistent ? 1 : 0);
    return cudaGetLastError();
}

// Shared-memory histogram-increment rate: each lane adds bytes read from a
// shared byte array into its own conflict-free counter column, the access
// pattern of the dense kernel's inner loop.
__global__ void __launch_bounds__(512) k_smem_peak(uint32_t *sink, int iters) {
    __shared__ __align__(16) uint8_t bins[4096];
    __shared__ uint32_t cnt[16][17 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) bins[i] = (uint8_t)((i * 7 + (i >> 5)) % 33);
    for (int i = lane; i < 17 * 32; i += 32) cnt[warp][i] = 0;
    __syncthreads();
    const uint32_t col = smem_u32(&cnt[warp][lane]);
    const uint8_t *p = bins + warp * 64 + lane;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t v = p[(it * 16 + u) * 97 & 2047];
            red_add_shared(col + ((v >> 1) << 7), 1u << ((v & 1u) << 4));
        }
    }
    __syncwarp();
    uint32_t acc = 0;
    for (int w = 0; w < 17; ++w) acc += ld_shared_u32(col + (w << 7));
    if (acc == 0xdeadbeefu) sink[blockIdx.x] = acc;   // keeps the work observable
}

cudaError_t launch_smem_peak(const LaunchCtx &lc, uint32_t *sink, int blocks, int iters) {
    k_smem_peak<<<blocks, 512, 0, lc.stream>>>(sink, iters);
    return cudaGetLastError();
}

}  // namespace ks
