// slrf_gram_noalloc: the Gram product G = X^T Y without a handle and without
// allocating device memory.
//
// Who needs it: callers that are not allowed to allocate device memory of
// their own -- code running inside a framework whose caching allocator or
// fixed-size memory pool owns all device memory (an extra cudaMalloc can fail
// or fragment that pool), and latency-critical loops that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree.  The regular
// slrf_gram takes its split-K scratch from a handle, which allocates.
//
// Scratch: the partial products of the K-split live in one file-scope
// __device__ array of SLRF_NOALLOC_SCRATCH_BYTES (4 MiB).  Every GPU that
// loads this library holds that array until the process exits.  In host code
// the array's name is only a host-side stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress (with that device
// current) on the first call made on that device.  That address belongs to
// the device's primary context (the one the CUDA runtime uses): calls must
// come from that context, and not after cudaDeviceReset in this process.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "slrf.h"

namespace {

constexpr size_t kScratchDoubles = SLRF_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
std::mutex g_setup_mutex;
thread_local std::string g_noalloc_error;

}  // namespace

extern "C" const char *slrf_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" slrf_status slrf_gram_noalloc(int64_t n, int32_t m, const double *X, int64_t ldx, const double *Y,
                                         int64_t ldy, double *G, void *cuda_stream) {
    using namespace slrf;
    g_noalloc_error.clear();
    if (n < 1 || n > (1LL << 31) - 1 || m < 1 || !X || !Y || !G || ldx < m || ldy < m) {
        g_noalloc_error = "invalid argument";
        return SLRF_EINVAL;
    }
    if ((size_t)m * (size_t)m > kScratchDoubles) {
        g_noalloc_error = "m = " + std::to_string(m) + " exceeds the static scratch: m*m must be <= " +
                          std::to_string(kScratchDoubles) + " (m <= 724)";
        return SLRF_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_noalloc_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return SLRF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_noalloc_error = "device index out of range";
        return SLRF_EINVAL;
    }
    double *scratch = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            // The set-up below (symbol lookup, possibly lazy module loading)
            // must not happen while the stream is being captured into a graph.
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            e = cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(cuda_stream), &cap);
            if (e != cudaSuccess) {
                g_noalloc_error = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e);
                return SLRF_ECUDA;
            }
            if (cap != cudaStreamCaptureStatusNone) {
                g_noalloc_error = "the first call on a device must not be made during stream capture";
                return SLRF_EINVAL;
            }
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) {
                g_noalloc_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return SLRF_ECUDA;
            }
            int count = 0;
            e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) {
                g_noalloc_error = std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e);
                return SLRF_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<double *>(ptr);
            g_sm_count[dev] = count;
        }
        scratch = g_scratch_ptr[dev];
        sms = g_sm_count[dev];
    }
    Ctx ctx;
    ctx.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx.sm_count = sms;
    int split = gram_split(ctx, m, n);
    const int max_split = (int)(kScratchDoubles / ((size_t)m * m));
    if (split > max_split) split = max_split;
    // Each K slice writes its whole m x m partial product into the scratch
    // before the fixed-order reduction reads it, so nothing needs clearing.
    dgemm(ctx, 1, 0, m, m, (int)n, X, ldx, Y, ldy, 0.0, G, m, split, scratch, KC_GRAM);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_error = std::string("launch: ") + cudaGetErrorString(e);
        return SLRF_ECUDA;
    }
    return SLRF_OK;
}
