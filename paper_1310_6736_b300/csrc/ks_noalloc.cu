// ks_bin_f32_noalloc: the float32 binning pass (the same two kernels as
// ks_create_volume's float32 path) for callers that must not allocate
// device memory.
//
// Who needs it: code that runs under an allocator it does not control or
// inside a region where allocation is off limits -- a framework whose
// caching allocator owns all device memory and forbids side allocations,
// a serving loop that must never take the device-wide synchronisation a
// cudaMalloc/cudaFree can cause, or an application with a hard memory cap
// that has already budgeted every byte.  Such a caller passes its own
// input and output buffers; the only other memory this path touches is a
// fixed scratch array compiled into the library.
//
// The scratch holds one (min, max) partial per block of the reduction pass.
// The pass is grid-stride, so the number of partials does not grow with the
// volume: a call uses 4 blocks per SM, at most kNoAllocPartials.  The array
// is a file-scope __device__ array, so every GPU that loads the library
// holds its 32 KB until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host that name is only a stand-in), so
// every call looks up its device address in the calling thread's current
// context with cudaGetSymbolAddress, which allocates nothing.  A cached
// address would go stale when the module is loaded again (after
// cudaDeviceReset, or in a context the caller created itself).
#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kNoAllocPartials = 4096;     // scratch entries (a 1024-SM part would use them all)
constexpr int kNoAllocMaxDim = 4096;       // the per-axis limit of ks_create_volume

static __device__ __align__(256) float2 g_noalloc_minmax[kNoAllocPartials];

}  // namespace
}  // namespace ks

extern "C" int ks_bin_f32_noalloc(const float *in, int nx, int ny, int nz, int bins,
                                  uint8_t *out, void *cuda_stream) {
    using namespace ks;
    if (!in || !out || nx < 1 || ny < 1 || nz < 1 || bins < 2 || bins > kMaxBins) return KS_EINVAL;
    if (nx > kNoAllocMaxDim || ny > kNoAllocMaxDim || nz > kNoAllocMaxDim) return KS_EINVAL;
    int device = 0, num_sms = 0;
    void *p = nullptr;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_minmax);
    if (e != cudaSuccess) return KS_ECUDA;
    int parts = bin_f32_scratch_blocks(num_sms);
    if (parts > kNoAllocPartials) parts = kNoAllocPartials;
    // Every block of the reduction pass overwrites its own partial, so the
    // scratch needs no clearing between calls.
    LaunchCtx lc{static_cast<cudaStream_t>(cuda_stream), nullptr, num_sms};
    e = launch_bin_f32(lc, in, nx, ny, nz, bins, out, /*pitch=*/nx, /*plane=*/(int64_t)nx * ny,
                       static_cast<float2 *>(p), parts);
    return e == cudaSuccess ? KS_OK : KS_ECUDA;
}
