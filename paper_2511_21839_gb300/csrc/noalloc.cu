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
void* g_partials_addr[kMaxDevices] = {nullptr};

// The array's device address on the current device. In host code the name
// g_moment_partials is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
int partials_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AD_PIC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return AD_PIC_ERR_UNSUPPORTED;
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_moment_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return AD_PIC_ERR_CUDA;
        }
        g_partials_addr[dev] = p;
    }
    *out = g_partials_addr[dev];
    return AD_PIC_OK;
}

template <typename T, int C, int CP>
int moments_noalloc(const void* state, int64_t N, double* mom, cudaStream_t s) {
    void* partial = nullptr;
    int st = partials_address(&partial);
    if (st) return st;
    MapCoef<T, CP> unused{};
    GeomFuse no_geometry{};          // count == nullptr: no geometry step
    // the MOM variant of the boundary kernel never writes the state and never
    // touches the extrema buffer; every block overwrites all of its partials,
    // so nothing needs clearing between calls
    launch_boundary<T, C, CP>(const_cast<T*>(static_cast<const T*>(state)), N, unused, false, true,
                              static_cast<double*>(partial), kNoAllocBlocks, nullptr, no_geometry, s);
    launch_moments_reduce(static_cast<const double*>(partial), kNoAllocBlocks, CP, N, mom, s);
    return cudaGetLastError() == cudaSuccess ? AD_PIC_OK : AD_PIC_ERR_CUDA;
}

}  // namespace

extern "C" int ad_pic_moments_device(const void* state_dev, int64_t n_particles, int n_deriv, int precision,
                                     double* mom_dev, void* stream) {
    if (!state_dev || !mom_dev || n_particles < 1) return AD_PIC_ERR_INVALID_ARG;
    if (precision != AD_PIC_FP64 && precision != AD_PIC_FP32_MIXED) return AD_PIC_ERR_INVALID_ARG;
    // the partial-sum array holds at most kNoAllocMaxCP channels per moment
    if (n_deriv != 7 && n_deriv != 13) return AD_PIC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == AD_PIC_FP64)
        return n_deriv == 7 ? moments_noalloc<double, 8, 8>(state_dev, n_particles, mom_dev, s)
                            : moments_noalloc<double, 14, 16>(state_dev, n_particles, mom_dev, s);
    return n_deriv == 7 ? moments_noalloc<float, 8, 8>(state_dev, n_particles, mom_dev, s)
                        : moments_noalloc<float, 14, 16>(state_dev, n_particles, mom_dev, s);
}
