// svt_polar_noalloc: the svt_polar solve for callers that cannot allocate device
// memory and cannot hand the library a workspace of their own.
//
// Who needs this: code that runs where cudaMalloc is off limits at call time
// (a host framework that owns every device allocation through its own pool,
// latency-critical loops that must not hit cudaMalloc's implicit device
// synchronisation or a run-time out-of-memory failure), and plain C callers
// that have no allocator handy at all. They pass only the input A and the
// output Y; all scratch comes from one file-scope device array.
//
// The scratch array is a static __device__ buffer of SVT_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads this library reserves it until the process exits. In
// host code the array's name only denotes a host-side stand-in, so its device
// address is fetched once per device with cudaGetSymbolAddress (with that
// device current) and handed to the kernels through an internal context.
//
// All calls share the one array, and it keeps whatever the last call left in
// it; the solve clears the parts that must start at zero (norm accumulators,
// status word, Gram diagonal) and overwrites every other buffer before reading
// it. Calls whose work overlaps on the GPU (different streams, or another thread)
// race on the array.
//
// Host memory: the first call for each shape and option set builds a launch
// plan, whose one-launch problem table is kept as a small pinned host image
// (cudaMallocHost, a few KB per product of the solve) that every later call
// copies to the array. That allocation can synchronise the device and is not
// allowed under stream capture, so such first calls belong before any capture.
// The internal context keeps at most kMaxPlans plans: a call that finds that many
// cached first waits for the device (their images may still be in copies) and
// drops them all; they are rebuilt, with new pinned images, if used again.
#include <cuda_runtime.h>

#include <mutex>

#include "plan.h"

namespace {

constexpr size_t kScratchBytes = SVT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr size_t kMaxPlans = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
    bool ready = false;
    svt_ctx_t ctx = nullptr;
};

std::mutex g_noalloc_mu;
DeviceScratch g_noalloc_dev[kMaxDevices];

} // namespace

extern "C" svt_status svt_polar_noalloc(int device, const float *A, int64_t m, int64_t n,
                                        int64_t lda, float tau, const svt_options *opt,
                                        float *Y, int64_t ldy, svt_status *d_status,
                                        void *stream)
{
    if (device < 0 || device >= kMaxDevices)
        return SVT_ERR_INVALID;
    svt_status st = svt::validate(A, m, n, lda, tau, Y, ldy);
    if (st != SVT_OK)
        return st;
    size_t need = 0;
    st = svt_workspace_bytes_ex(m, n, opt, &need);
    if (st != SVT_OK)
        return st;
    if (need > kScratchBytes)
        return SVT_ERR_UNSUPPORTED;  // larger than the fixed scratch array

    std::lock_guard<std::mutex> g(g_noalloc_mu);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return SVT_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess)
        return SVT_ERR_CUDA;
    DeviceScratch &d = g_noalloc_dev[device];
    if (!d.ready) {
        // First call on this device: resolve the array's device address with the
        // device current, then wrap it in a context (no device allocation).
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaSetDevice(prev);
            return SVT_ERR_CUDA;
        }
        st = svt_ctx_create(device, ptr, kScratchBytes, &d.ctx);
        if (st != SVT_OK) {
            cudaSetDevice(prev);
            return st;
        }
        d.ready = true;
    }
    {
        // Bound the pinned host images the cached plans hold (see the file comment).
        std::lock_guard<std::mutex> pg(d.ctx->mu);
        if (d.ctx->plans.size() >= kMaxPlans) {
            if (cudaDeviceSynchronize() != cudaSuccess) {
                cudaSetDevice(prev);
                return SVT_ERR_CUDA;
            }
            svt::evict_plans(d.ctx, 0);
        }
    }
    st = svt_polar_ex(d.ctx, A, m, n, lda, tau, opt, Y, ldy, d_status, stream);
    cudaSetDevice(prev);
    return st;
}
