// Allocation-free MIP entry point (vr_render_mip_noalloc).
//
// vr_render's brick path allocates its per-pixel scratch with cudaMalloc the
// first time it meets a larger image.  Some callers cannot allow that:
// real-time loops that must not hit the device-wide synchronisation that
// cudaMalloc may imply, and applications whose device memory is owned by
// another allocator or held to a fixed budget.  This entry point renders the same
// MIP with its scratch -- per-pixel sample ranges, per-pixel running maxima
// and the work counter -- taken from one fixed array compiled into the
// library, and calls no allocating routine.
#include <mutex>

#include "vr_internal.cuh"

namespace {

constexpr long long kPixels = VR_NOALLOC_MAX_PIXELS;
constexpr size_t kRangeBytes = (size_t)kPixels * sizeof(int2);
constexpr size_t kMaxBytes = (size_t)kPixels * sizeof(unsigned int);
constexpr size_t kScratchBytes = kRangeBytes + kMaxBytes + 256;

// One scratch area per device that loads the library, held until the process
// exits.  In host code this name is only a stand-in for the device symbol: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch area on `device`, which must be current.
// Looked up once per device; later calls reuse the cached pointer, so a device
// reset after the first call is not supported (the pointer would be stale).
cudaError_t scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = p;
    }
    *out = g_dev_ptr[device];
    return cudaSuccess;
}

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~CurrentDevice() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" vr_status vr_render_mip_noalloc(vr_ctx* ctx, float* out_rgba, float* out_max,
                                           void* stream) {
    int device = 0;
    long long pixels = 0;
    vr_status st = vr::brick_mip_precheck(ctx, out_rgba, out_max, &device, &pixels);
    if (st != VR_OK) return st;
    if (pixels > kPixels)
        return vr::set_error(ctx, VR_ERR_INVALID_ARG,
                             "vr_render_mip_noalloc: a camera has more than VR_NOALLOC_MAX_PIXELS pixels");
    CurrentDevice guard(device);
    void* base = nullptr;
    cudaError_t e = scratch_address(device, &base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return vr::set_error(ctx, VR_ERR_CUDA, "vr_render_mip_noalloc: cudaGetSymbolAddress failed");
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    int2* krange = reinterpret_cast<int2*>(b);
    unsigned int* enc = reinterpret_cast<unsigned int*>(b + kRangeBytes);
    int* work = reinterpret_cast<int*>(b + kRangeBytes + kMaxBytes);
    // krange and enc are rewritten for every pixel by the set-up kernel of each
    // camera; the work counter is cleared before each brick pass.
    return vr::brick_mip_with_scratch(ctx, out_rgba, out_max, static_cast<cudaStream_t>(stream),
                                      krange, enc, work);
}
