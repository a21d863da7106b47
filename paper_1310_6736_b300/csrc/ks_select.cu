// Selection of salient regions among converged seeds (Sec. 2.3, end: maxima
// whose entropy exceeds a threshold are kept and ranked by the change of the
// pdf with scale; Sec. 3.1: the 20 with the highest pdf difference).
//
//   1. keep   candidate i if r_i > 0 (a scale exists) and H_i > h_min;
//   2. merge  candidates with the same (x, y, z, r): one entry, the smallest
//             source index (equal keys have equal H and W: both are functions
//             of the window);
//   3. order  W descending, then H descending, then z, y, x, r ascending;
//   4. take   the first min(top_k, #unique) entries.
//
// Device plan: an open-addressing hash table on the 64-bit key (x, y, z, r)
// holds the smallest source per key (atomicMin); a candidate survives when
// it is kept and its source is that minimum.  Survivors are appended to a
// list; then rounds of block-local bitonic sorts of up to kChunk entries
// each keep the best top_k per chunk until one chunk is left, whose sorted
// prefix is the answer.  Every comparison is a total order on distinct keys,
// so the result does not depend on the order of the appends.
#include <algorithm>
#include <utility>

#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kChunk = 1024;                 // entries per block-local sort
constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long cand_key(const ks_candidate &c) {
    return ((unsigned long long)(uint16_t)c.x) | ((unsigned long long)(uint16_t)c.y << 16) |
           ((unsigned long long)(uint16_t)c.z << 32) | ((unsigned long long)(uint8_t)c.r << 48);
}

__device__ __forceinline__ bool kept(const ks_candidate &c, double h_min) {
    return c.r > 0 && c.H > h_min;
}

// a before b in the selection order
__device__ __forceinline__ bool better(const ks_candidate &a, const ks_candidate &b) {
    if (a.W != b.W) return a.W > b.W;
    if (a.H != b.H) return a.H > b.H;
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    if (a.x != b.x) return a.x < b.x;
    return a.r < b.r;
}

__device__ __forceinline__ uint32_t hash_slot(unsigned long long k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// Insert every kept candidate's key; the slot's value is the smallest source.
__global__ void k_sel_hash(const ks_candidate *in, int64_t n, double h_min,
                           unsigned long long *keys, int *src, uint32_t mask, int *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ks_candidate c = in[i];
        if (!kept(c, h_min)) continue;
        const unsigned long long k = cand_key(c);
        uint32_t s = hash_slot(k, mask);
        // the table has at least twice as many slots as candidates, so a
        // free or matching slot is found within mask + 1 probes
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(keys + s, kEmpty, k);
            if (prev == kEmpty || prev == k) {
                atomicMin(src + s, c.source);
                break;
            }
            s = (s + 1) & mask;
            if (probe == mask) atomicOr(status, kStatusBadInput);
        }
    }
}

// Append the survivors: kept, and the smallest source of their key.
__global__ void k_sel_compact(const ks_candidate *in, int64_t n, double h_min,
                              const unsigned long long *keys, const int *src, uint32_t mask,
                              ks_candidate *out, unsigned long long *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ks_candidate c = in[i];
        if (!kept(c, h_min)) continue;
        const unsigned long long k = cand_key(c);
        uint32_t s = hash_slot(k, mask);
        for (uint32_t probe = 0; probe <= mask && keys[s] != k; ++probe) s = (s + 1) & mask;
        if (keys[s] == k && src[s] == c.source) out[atomicAdd(count, 1ull)] = c;
    }
}

// Block b sorts entries [b * kChunk, min((b + 1) * kChunk, m)) of `in` with a
// bitonic network (missing entries are padding that sorts last) and writes
// its best `keep` entries to out[b * keep ...]; the count written is
// min(keep, entries of the chunk).
__global__ void __launch_bounds__(512) k_sel_topk(const ks_candidate *in, int64_t m, int keep,
                                                  ks_candidate *out) {
    __shared__ ks_candidate buf[kChunk];
    __shared__ unsigned char pad[kChunk];
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int len = (int)(m - base < kChunk ? m - base : kChunk);
    for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
        pad[i] = i >= len;
        if (i < len) buf[i] = in[base + i];
    }
    __syncthreads();
    for (int size = 2; size <= kChunk; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kChunk / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;          // this run ascends in "better"
                const bool hi_first = pad[lo] ? !pad[hi]
                                              : (!pad[hi] && better(buf[hi], buf[lo]));
                if (hi_first == up) {
                    const ks_candidate t = buf[lo];
                    buf[lo] = buf[hi];
                    buf[hi] = t;
                    const unsigned char p = pad[lo];
                    pad[lo] = pad[hi];
                    pad[hi] = p;
                }
            }
            __syncthreads();
        }
    }
    const int n_out = len < keep ? len : keep;
    for (int i = threadIdx.x; i < n_out; i += blockDim.x) out[(int64_t)blockIdx.x * keep + i] = buf[i];
}

// Octant results -> candidates (the Kadir-Brady evaluation at the final
// centre: scale s_best, H_best, W_best).
__global__ void k_oct_cands(const ks_seed_result *in, int64_t n, ks_candidate *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ks_seed_result r = in[i];
        ks_candidate c;
        c.x = r.x;
        c.y = r.y;
        c.z = r.z;
        c.r = r.s_best;
        c.source = (int32_t)i;
        c.reserved = 0;
        c.H = r.H_best;
        c.W = r.W_best;
        out[i] = c;
    }
}

// Distinct final centres of mean-shift results: insert every centre's key
// (x, y, z) into the hash table ...
__global__ void k_ms_centre_keys(const ks_ms_result *in, int64_t n, unsigned long long *keys,
                                 uint32_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)(uint16_t)in[i].x) |
                                     ((unsigned long long)(uint16_t)in[i].y << 16) |
                                     ((unsigned long long)(uint16_t)in[i].z << 32);
        uint32_t s = hash_slot(k, mask);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(keys + s, kEmpty, k);
            if (prev == kEmpty || prev == k) break;
            s = (s + 1) & mask;
        }
    }
}

// ... number the occupied slots and list their centres ...
__global__ void k_ms_centre_list(const unsigned long long *keys, uint32_t slots, int *idx,
                                 int32_t *xyz, unsigned long long *count) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[s];
        if (k == kEmpty) continue;
        const int j = (int)atomicAdd(count, 1ull);
        idx[s] = j;
        xyz[3 * j] = (int32_t)(k & 0xffffu);
        xyz[3 * j + 1] = (int32_t)((k >> 16) & 0xffffu);
        xyz[3 * j + 2] = (int32_t)((k >> 32) & 0xffffu);
    }
}

// ... and give every item the number of its centre.
__global__ void k_ms_centre_of(const ks_ms_result *in, int64_t n, const unsigned long long *keys,
                               const int *idx, uint32_t mask, int *centre) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)(uint16_t)in[i].x) |
                                     ((unsigned long long)(uint16_t)in[i].y << 16) |
                                     ((unsigned long long)(uint16_t)in[i].z << 32);
        uint32_t s = hash_slot(k, mask);
        for (uint32_t probe = 0; probe <= mask && keys[s] != k; ++probe) s = (s + 1) & mask;
        centre[i] = idx[s];
    }
}

// Mean-shift results + H, W of every scale at their distinct final centres
// -> candidates at each item's own scale.
__global__ void k_ms_cands(const ks_ms_result *in, int64_t n, const int *centre, const double *H,
                           const double *W, int r_min, int S, ks_candidate *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const ks_ms_result m = in[i];
        const int64_t si = (int64_t)centre[i] * S + (m.r - r_min);
        ks_candidate c;
        c.x = m.x;
        c.y = m.y;
        c.z = m.z;
        c.r = m.r;
        c.source = (int32_t)i;
        c.reserved = 0;
        c.H = H[si];
        c.W = W[si];
        out[i] = c;
    }
}

}  // namespace

cudaError_t launch_oct_candidates(const LaunchCtx &lc, const ks_seed_result *in, int64_t n,
                                  ks_candidate *out) {
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)lc.num_sms * 8);
    k_oct_cands<<<grid, 256, 0, lc.stream>>>(in, n, out);
    return cudaGetLastError();
}

size_t ms_centres_scratch_bytes(int64_t n) {
    uint32_t slots = 1024;
    while (slots < 2 * (uint64_t)n) slots <<= 1;
    return (size_t)slots * 12 + (size_t)n * 16 + 512;
}

cudaError_t launch_ms_centres(const LaunchCtx &lc, const ks_ms_result *in, int64_t n,
                              void *scratch, unsigned long long *d_count, const int32_t **xyz,
                              const int **centre, int64_t *m) {
    *m = 0;
    if (n == 0) return cudaSuccess;
    uint32_t slots = 1024;
    while (slots < 2 * (uint64_t)n) slots <<= 1;
    uint8_t *p = (uint8_t *)scratch;
    unsigned long long *keys = (unsigned long long *)p;
    int *idx = (int *)(p + (size_t)slots * 8);
    int32_t *list = (int32_t *)(p + (((size_t)slots * 12 + 255) / 256) * 256);
    int *cen = (int *)(list + 3 * n + 64);
    cudaError_t e = cudaMemsetAsync(keys, 0xff, (size_t)slots * 8, lc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, 8, lc.stream);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)lc.num_sms * 8);
    const int sgrid = (int)std::min<int64_t>((slots + 255) / 256, (int64_t)lc.num_sms * 8);
    k_ms_centre_keys<<<grid, 256, 0, lc.stream>>>(in, n, keys, slots - 1);
    k_ms_centre_list<<<sgrid, 256, 0, lc.stream>>>(keys, slots, idx, list, d_count);
    k_ms_centre_of<<<grid, 256, 0, lc.stream>>>(in, n, keys, idx, slots - 1, cen);
    unsigned long long mm = 0;
    e = cudaMemcpyAsync(&mm, d_count, 8, cudaMemcpyDeviceToHost, lc.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lc.stream);
    *xyz = list;
    *centre = cen;
    *m = (int64_t)mm;
    return e;
}

cudaError_t launch_ms_candidates(const LaunchCtx &lc, const ks_ms_result *in, int64_t n,
                                 const int *centre, const double *H, const double *W, int r_min,
                                 int S, ks_candidate *out) {
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)lc.num_sms * 8);
    k_ms_cands<<<grid, 256, 0, lc.stream>>>(in, n, centre, H, W, r_min, S, out);
    return cudaGetLastError();
}

size_t select_scratch_bytes(int64_t n) {
    uint32_t slots = 1024;
    while (slots < 2 * (uint64_t)n) slots <<= 1;
    return (size_t)slots * 12 + 2 * (size_t)n * sizeof(ks_candidate) + 256;
}

cudaError_t launch_select(const LaunchCtx &lc, const ks_candidate *in, int64_t n, double h_min,
                          int top_k, void *scratch, ks_candidate *out,
                          unsigned long long *d_count, int64_t *n_out) {
    *n_out = 0;
    if (n == 0) return cudaSuccess;
    uint32_t slots = 1024;
    while (slots < 2 * (uint64_t)n) slots <<= 1;
    uint8_t *p = (uint8_t *)scratch;
    unsigned long long *keys = (unsigned long long *)p;
    int *src = (int *)(p + (size_t)slots * 8);
    ks_candidate *a = (ks_candidate *)(p + (((size_t)slots * 12 + 255) / 256) * 256);
    ks_candidate *b = a + n;
    cudaError_t e = cudaMemsetAsync(keys, 0xff, (size_t)slots * 8, lc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(src, 0x7f, (size_t)slots * 4, lc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, 8, lc.stream);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)lc.num_sms * 8);
    k_sel_hash<<<grid, 256, 0, lc.stream>>>(in, n, h_min, keys, src, slots - 1, lc.d_status);
    k_sel_compact<<<grid, 256, 0, lc.stream>>>(in, n, h_min, keys, src, slots - 1, a, d_count);
    unsigned long long m = 0;
    e = cudaMemcpyAsync(&m, d_count, 8, cudaMemcpyDeviceToHost, lc.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lc.stream);
    if (e != cudaSuccess) return e;
    // rounds of chunk-wise top_k until one chunk remains
    int64_t len = (int64_t)m;
    ks_candidate *cur = a, *nxt = b;
    do {
        const int64_t chunks = (len + kChunk - 1) / kChunk;
        const int keep = chunks == 1 ? kChunk : top_k;
        k_sel_topk<<<(unsigned)chunks, 512, 0, lc.stream>>>(cur, len, keep, nxt);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        len = chunks == 1 ? std::min<int64_t>(len, kChunk)
                          : (chunks - 1) * (int64_t)top_k + std::min<int64_t>(len - (chunks - 1) * kChunk, top_k);
        std::swap(cur, nxt);
        if (chunks == 1) break;
    } while (true);
    const int64_t k = std::min<int64_t>(len, top_k);
    e = cudaMemcpyAsync(out, cur, (size_t)k * sizeof(ks_candidate), cudaMemcpyDeviceToDevice,
                        lc.stream);
    *n_out = k;
    return e;
}

}  // namespace ks
