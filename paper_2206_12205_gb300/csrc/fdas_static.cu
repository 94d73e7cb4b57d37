// fdas_plane_static: the f-z plane without a caller-supplied workspace.
//
// Some callers cannot allocate device memory when they need the plane: code that runs while a
// CUDA stream is being captured into a graph, real-time pipelines that reserve all device
// memory at start-up and forbid allocation afterwards (an allocation can block or fail in the
// middle of an observation), and hosts whose own allocator already owns the device's memory.
// For them this entry point keeps its only scratch (the segment spectra) in a file-scope device
// array of fixed size, set up once per device, and allocates nothing itself.
#include <cstdio>
#include <mutex>

#include "fdas_internal.cuh"

struct fdas_plan_s : public fdas::Plan {};

namespace {

constexpr size_t kScratchBytes = FDAS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_plane_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_plane_scratch on device dev, which must be current (looked up once per
// device; in host code the symbol name itself is only a host-side stand-in, never a device
// address).
cudaError_t scratch_on_device(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    cudaError_t e = cudaSuccess;
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_plane_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fdas_status fdas_plane_static(fdas_plan_t plan, const float *d_xhat, void *d_plane, void *stream) {
    if (!plan || !d_xhat || !d_plane) return FDAS_E_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_xhat) & 7) || (reinterpret_cast<uintptr_t>(d_plane) & 15)) return FDAS_E_INVALID;
    fdas::Plan *p = static_cast<fdas::Plan *>(plan);
    if (!p->templates_ready) return FDAS_E_STATE;
    if (p->cfg.precision != FDAS_FP32) {
        p->last_error = "fdas_plane_static: only FDAS_FP32 plans are supported";
        return FDAS_E_UNSUPPORTED;
    }
    const size_t need = sizeof(float2) * (size_t)p->n_seg * (size_t)p->S;
    if (need > kScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "fdas_plane_static: plan needs %zu bytes of segment scratch, the static array holds %zu",
                      need, kScratchBytes);
        p->last_error = msg;
        return FDAS_E_UNSUPPORTED;
    }
    // the plan's templates and twiddles live on the device it was built on: the scratch must be
    // that device's copy of the array
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev != p->device) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "fdas_plane_static: device %d is current, the plan's templates are on device %d",
                      dev, p->device);
        p->last_error = msg;
        return FDAS_E_INVALID;
    }
    void *scratch = nullptr;
    if (e == cudaSuccess) e = scratch_on_device(dev, &scratch);
    if (e == cudaSuccess) {
        p->prof.calls++;
        e = fdas::launch_plane_fp32_scratch(*p, reinterpret_cast<const float2 *>(d_xhat), nullptr,
                                            static_cast<float2 *>(scratch), static_cast<float *>(d_plane),
                                            static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) {
        p->last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
        (void)cudaGetLastError();
        return FDAS_E_CUDA;
    }
    return FDAS_OK;
}
