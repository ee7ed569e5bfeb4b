// Allocation-free dual moment reduction.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: code that
// runs inside another framework's device-memory budget (a caching allocator
// that owns the GPU, whose accounting a stray allocation breaks), and
// latency-critical loops that must not take the implicit device-wide
// synchronisation those calls can bring. ad_pic_moments_device serves them:
// the caller passes a device-resident dual particle state and a device output
// buffer, and the per-block partial sums of the reduction live in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits. Nothing is allocated per call.
#include <atomic>

#include "ad_pic.h"
#include "common.cuh"

using namespace adpic;

namespace {

// Blocks of the reduction and the largest padded channel count it accepts.
constexpr int kNoAllocBlocks = 152 * 2;
constexpr int kNoAllocMaxCP = 16;
// [kNoAllocBlocks][15][kNoAllocMaxCP] FP64 partial sums: 583,680 bytes.
static __device__ __align__(256) double g_moment_partials[kNoAllocBlocks * 15 * kNoAllocMaxCP];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_partials_addr[kMaxDevices];

// The array's device address on the current device. In host code the name
// g_moment_partials is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, with that device current. It is looked up again
// on every call made outside stream capture (so a device reset or a new
// primary context, which reload the module, never leave a stale address) and
// cached per device for calls made while `s` is capturing, where the lookup
// is not made. The cache slots are atomic: two host threads may make a first
// call on one device at once.
int partials_address(cudaStream_t s, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AD_PIC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return AD_PIC_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return AD_PIC_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) {
        void* p = g_partials_addr[dev].load();
        if (!p) return AD_PIC_ERR_STATE;      // no call on this device outside capture yet
        *out = p;
        return AD_PIC_OK;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_moment_partials) != cudaSuccess || !p) return AD_PIC_ERR_CUDA;
    g_partials_addr[dev].store(p);
    *out = p;
    return AD_PIC_OK;
}

template <typename T, int C, int CP>
int moments_noalloc(const void* state, int64_t N, double* mom, cudaStream_t s) {
    void* partial = nullptr;
    int st = partials_address(s, &partial);
    if (st) {
        cudaGetLastError();                   // the failed lookup's own error, not an earlier one
        return st;
    }
    MapCoef<T, CP> unused{};
    GeomFuse no_geometry{};          // count == nullptr: no geometry step
    // the MOM variant of the boundary kernel never writes the state and never
    // touches the extrema buffer; every block overwrites all of its partials
    // (a block without particles writes zeros), so nothing needs clearing
    // between calls
    launch_boundary<T, C, CP>(const_cast<T*>(static_cast<const T*>(state)), N, unused, false, true,
                              static_cast<double*>(partial), kNoAllocBlocks, nullptr, no_geometry, s);
    if (cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    launch_moments_reduce(static_cast<const double*>(partial), kNoAllocBlocks, CP, N, mom, s);
    return cudaGetLastError() == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

}  // namespace

extern "C" int ad_pic_moments_device(const void* state_dev, int64_t n_particles, int n_deriv, int precision,
                                     double* mom_dev, void* stream) {
    if (!state_dev || !mom_dev || n_particles < 1) return AD_PIC_ERR_INVALID_ARG;
    if (precision != AD_PIC_FP64 && precision != AD_PIC_FP32_MIXED) return AD_PIC_ERR_INVALID_ARG;
    // only the 7- and 13-derivative channel layouts (CP 8 and 16) are compiled;
    // the partial-sum array holds up to kNoAllocMaxCP = 16 channels per moment
    if (n_deriv != 7 && n_deriv != 13) return AD_PIC_ERR_INVALID_ARG;
    // a CUDA error left pending by an earlier call is handed back untouched:
    // nothing is launched and the error stays pending for its owner
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == AD_PIC_FP64)
        return n_deriv == 7 ? moments_noalloc<double, 8, 8>(state_dev, n_particles, mom_dev, s)
                            : moments_noalloc<double, 14, 16>(state_dev, n_particles, mom_dev, s);
    return n_deriv == 7 ? moments_noalloc<float, 8, 8>(state_dev, n_particles, mom_dev, s)
                        : moments_noalloc<float, 14, 16>(state_dev, n_particles, mom_dev, s);
}
