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
// It is a file-scope __device__ array, so every GPU that loads the library
// holds its 32 KB until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host that name is only a stand-in), so
// the entry point looks up its device address once per device with
// cudaGetSymbolAddress and caches it.
#include <mutex>

#include "ks_internal.cuh"

namespace ks {
namespace {

constexpr int kNoAllocPartials = 4096;                // scratch entries
constexpr int64_t kVoxelsPerPartial = int64_t(1) << 18;
constexpr int64_t kNoAllocMaxVoxels = kNoAllocPartials * kVoxelsPerPartial;   // 2^30
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_minmax[kNoAllocPartials];

std::mutex g_mu;
float2 *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call for that device).
cudaError_t scratch_on_current_device(int *device, float2 **out) {
    cudaError_t e = cudaGetDevice(device);
    if (e != cudaSuccess) return e;
    if (*device < 0 || *device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[*device]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_minmax);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[*device] = static_cast<float2 *>(p);
    }
    *out = g_scratch_ptr[*device];
    return cudaSuccess;
}

}  // namespace
}  // namespace ks

extern "C" int ks_bin_f32_noalloc(const float *in, int nx, int ny, int nz, int bins,
                                  uint8_t *out, void *cuda_stream) {
    using namespace ks;
    if (!in || !out || nx < 1 || ny < 1 || nz < 1 || bins < 2 || bins > kMaxBins) return KS_EINVAL;
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > kNoAllocMaxVoxels) return KS_EINVAL;      // more than the scratch can reduce
    int device = 0;
    float2 *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&device, &scratch);
    int num_sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return KS_ECUDA;
    const int parts = (int)((n + kVoxelsPerPartial - 1) / kVoxelsPerPartial);
    // Every block of the reduction pass overwrites its own partial, so the
    // scratch needs no clearing between calls.
    LaunchCtx lc{static_cast<cudaStream_t>(cuda_stream), nullptr, num_sms};
    e = launch_bin_f32(lc, in, nx, ny, nz, bins, out, /*pitch=*/nx, /*plane=*/(int64_t)nx * ny,
                       scratch, parts);
    return e == cudaSuccess ? KS_OK : KS_ECUDA;
}
