// build_static.cu -- fif_build_static: the field build without a caller-supplied workspace.
//
// Some callers cannot allocate device memory once they are running: a planner embedded as a
// plug-in in a host application whose own allocator owns the device memory, or a real-time
// loop that forbids cudaMalloc after start-up because it can synchronise the device and take
// unbounded time.  This entry point gives them the build with its scratch (the landmark bins)
// in a fixed array that is part of the library image, so nothing is allocated per call.
//
// The array is FIF_BUILD_STATIC_SCRATCH_BYTES (16 MiB) on every GPU that loads the library,
// held until the process exits.  Host code cannot use the array's name as a device address,
// so the address is looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call that runs on it.
#include <mutex>

#include "fif_internal.h"

namespace {

// scratch for the binning of fif_build_static; every call overwrites it completely
static __device__ __align__(256) unsigned char g_build_scratch[FIF_BUILD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of g_build_scratch on the current device (looked up once per device)
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FIF_ECUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_build_scratch) != cudaSuccess || p == nullptr) return FIF_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FIF_OK;
}

}  // namespace

extern "C" FIF_API int32_t fif_build_static(fif_field* field, const float* d_landmarks, int64_t n,
                                            fif_stream_t stream) {
    // offered for the quadratic-visibility and trace fields only; a GP field is refused
    if (field && field->storage == FIF_STORAGE_GP) return FIF_EINVAL;
    const size_t need = fif_build_workspace_bytes(field, n);
    if (need == 0) return FIF_EINVAL;
    if (need > (size_t)FIF_BUILD_STATIC_SCRATCH_BYTES) return FIF_ERANGE;
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != FIF_OK) return rc;
    // fif_build zeroes the bin counters and statistics itself before using them, and writes
    // the sorted landmarks and bin offsets before reading them, so the contents left by an
    // earlier call do not matter.
    return fif_build(field, d_landmarks, n, scratch, FIF_BUILD_STATIC_SCRATCH_BYTES, stream);
}
