// Particle kernels: initial distribution, state conversion, the fused
// gather + kick + push (M2 then M1 maps), the period-boundary kernel (dual
// moments in FP64 + half map), and cloud-in-cell deposition of every dual
// channel.
#include "particles_dev.cuh"

namespace adpic {

template <typename T, int C, int CP>
void launch_init(const double* nrm, int64_t N, const double* coef, T* state, cudaStream_t s) {
    if (N <= 0) return;
    init_kernel<T, C, CP><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(nrm, N, coef, state);
}

template <typename T, int CP>
void launch_convert_in(const double* src, T* dst, int64_t N, int C, cudaStream_t s) {
    int64_t tot = 6 * N * CP;
    if (tot > 0) convert_in_kernel<T, CP><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, 6 * N, C);
}
template <typename T, int CP>
void launch_convert_out(const T* src, double* dst, int64_t N, int C, cudaStream_t s) {
    int64_t tot = 6 * N * C;
    if (tot > 0) convert_out_kernel<T, CP><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, dst, 6 * N, C);
}

// resident CTAs of the persistent push, per instantiation (set by setup_push)
template <typename T, int C, int CP, bool TRACK>
static int& push_grid() {
    static int g = 0;
    return g;
}

template <typename T, int C, int CP, bool TRACK>
static void push_attrs() {
    constexpr int TP = push_tile<T, CP>();
    const int smem = (int)push_smem<T, CP>();
    cudaFuncSetAttribute(push_tma_kernel<T, C, CP, TRACK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_tma_kernel<T, C, CP, TRACK>, TP, smem);
    push_grid<T, C, CP, TRACK>() = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

template <typename T, int C, int CP>
void setup_push() {
    push_attrs<T, C, CP, true>();
    push_attrs<T, C, CP, false>();
}

template <typename T, int C, int CP, bool TRACK>
static void launch_push_t(const T* state_in, T* state_out, int64_t N, const T* E, const GeomDev* geom, int nx,
                          int ny, int nz, const MapCoef<T, CP>& A, const KickCoef<T, CP>& K, Ord<T>* mm, int* err,
                          const SortBuf& sb, const GeomFuse& gf, int polls, cudaStream_t s) {
    constexpr int TP = push_tile<T, CP>();
    const int64_t tiles = (N + TP - 1) / TP;
    const int64_t g = push_grid<T, C, CP, TRACK>();
    const unsigned grid = (unsigned)(tiles < g ? tiles : g);
    const size_t smem = push_smem<T, CP>();
    push_tma_kernel<T, C, CP, TRACK><<<grid, TP, smem, s>>>(state_in, state_out, N, E, geom, nx, ny, nz, A, K, mm,
                                                             err, sb, gf, polls >= 0 ? polls : kWaitPolls);
}

template <typename T, int C, int CP>
void launch_push(const T* state_in, T* state_out, int64_t N, const T* E, const GeomDev* geom, int nx, int ny, int nz,
                 const MapCoef<T, CP>& A, const KickCoef<T, CP>& K, bool track, Ord<T>* mm, int* err,
                 const SortBuf& sb, const GeomFuse& gf, int polls, cudaStream_t s) {
    if (N <= 0) return;
    if (track)
        launch_push_t<T, C, CP, true>(state_in, state_out, N, E, geom, nx, ny, nz, A, K, mm, err, sb, gf, polls, s);
    else
        launch_push_t<T, C, CP, false>(state_in, state_out, N, E, geom, nx, ny, nz, A, K, mm, err, sb, gf, polls, s);
}

int scan_blocks(int ncells) { return (ncells + kScanChunk - 1) / kScanChunk; }

void launch_scan(int* hist, int* offs, int* bsum, int ncells, cudaStream_t s) {
    const int nb = scan_blocks(ncells);
    scan_sum_kernel<<<nb, 256, 0, s>>>(hist, ncells, bsum);
    scan_apply_kernel<<<nb, 256, 0, s>>>(hist, ncells, bsum, offs);   // each block prefixes the chunk totals
}
void launch_slots(const int* key, const int* rank, const int* offs, int* dst, int64_t N, cudaStream_t s) {
    if (N > 0) slots_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(key, rank, offs, dst, N);
}
void launch_iota(int* ids, int64_t N, cudaStream_t s) {
    if (N > 0) iota_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ids, N);
}
template <typename T, int CP>
void launch_convert_out_perm(const T* src, const int* ids, double* dst, int64_t N, int C, cudaStream_t s) {
    const int64_t tot = 6 * N * C;
    if (tot > 0) convert_out_perm_kernel<T, CP><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, ids, dst, N, C);
}
int boundary_blocks() { return kBoundaryBlocks; }

int launch_wait_probe(int polls, int* failed, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(polls, failed);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int C, int CP>
void launch_boundary(T* state, int64_t N, const MapCoef<T, CP>& A, bool apply, bool mom, double* partial,
                     int nblocks, Ord<T>* mm, const GeomFuse& gf, cudaStream_t s) {
    if (apply && mom)
        boundary_kernel<T, C, CP, true, true><<<nblocks, 256, 0, s>>>(state, N, A, partial, mm, gf);
    else if (mom)
        boundary_kernel<T, C, CP, true, false><<<nblocks, 256, 0, s>>>(state, N, A, partial, mm, gf);
    else if (apply)
        halfmap_kernel<T, C, CP><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(state, N, A, mm, gf);
}

void launch_moments_reduce(const double* partial, int nblocks, int CP, int64_t N, double* out, cudaStream_t s) {
    moments_reduce_kernel<<<15 * CP, 256, 0, s>>>(partial, nblocks, CP, N, out);
}

template <typename T, int C, int CP>
void launch_deposit(const T* state, int64_t N, const GeomDev* geom, int nx, int ny, int nz, T qm, T* rho, int* err,
                    const SortBuf& sb, int qslot, cudaStream_t s) {
    if (N <= 0) return;
    // warp-sorted, on-chip summed deposition (see deposit_tile_body)
    constexpr int W = dep_tile_warps<CP, T>();
    const size_t sm = (size_t)W * dep_tile_bytes_per_warp<CP, T>();
    const int64_t warps = (N + 31) / 32;
    const unsigned grid = (unsigned)((warps + W - 1) / W);
    if (qslot >= 0)
        deposit_tile_kernel<T, C, CP, W, true><<<grid, W * 32, sm, s>>>(state, N, geom, nx, ny, nz, qm, rho, err, sb,
                                                                        qslot, (T)(1.0 / (double)N));
    else
        deposit_tile_kernel<T, C, CP, W, false><<<grid, W * 32, sm, s>>>(state, N, geom, nx, ny, nz, qm, rho, err, sb,
                                                                         -1, (T)0);
}

template <typename T, int C, int CP>
void setup_deposit() {
    constexpr int W = dep_tile_warps<CP, T>();
    cudaFuncSetAttribute(deposit_tile_kernel<T, C, CP, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((size_t)W * dep_tile_bytes_per_warp<CP, T>()));
    cudaFuncSetAttribute(deposit_tile_kernel<T, C, CP, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((size_t)W * dep_tile_bytes_per_warp<CP, T>()));
}

// ------------------------------------------------------------------ instantiations
#define ADPIC_INST(T, C, CP)                                                                                       \
    template void launch_init<T, C, CP>(const double*, int64_t, const double*, T*, cudaStream_t);                \
    template void launch_push<T, C, CP>(const T*, T*, int64_t, const T*, const GeomDev*, int, int, int,         \
                                        const MapCoef<T, CP>&, const KickCoef<T, CP>&, bool, Ord<T>*, int*,      \
                                        const SortBuf&, const GeomFuse&, int, cudaStream_t);                     \
    template void launch_boundary<T, C, CP>(T*, int64_t, const MapCoef<T, CP>&, bool, bool, double*, int,       \
                                            Ord<T>*, const GeomFuse&, cudaStream_t);                             \
    template void launch_deposit<T, C, CP>(const T*, int64_t, const GeomDev*, int, int, int, T, T*, int*,        \
                                           const SortBuf&, int, cudaStream_t);                                   \
    template void setup_deposit<T, C, CP>();                                                                     \
    template void setup_push<T, C, CP>();
ADPIC_INST(float, 8, 8)
ADPIC_INST(float, 14, 16)
ADPIC_INST(double, 8, 8)
ADPIC_INST(double, 14, 16)
template void launch_convert_in<float, 8>(const double*, float*, int64_t, int, cudaStream_t);
template void launch_convert_in<float, 16>(const double*, float*, int64_t, int, cudaStream_t);
template void launch_convert_in<double, 8>(const double*, double*, int64_t, int, cudaStream_t);
template void launch_convert_in<double, 16>(const double*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out<float, 8>(const float*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out<float, 16>(const float*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out<double, 8>(const double*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out<double, 16>(const double*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out_perm<float, 8>(const float*, const int*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out_perm<float, 16>(const float*, const int*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out_perm<double, 8>(const double*, const int*, double*, int64_t, int, cudaStream_t);
template void launch_convert_out_perm<double, 16>(const double*, const int*, double*, int64_t, int, cudaStream_t);

}  // namespace adpic
