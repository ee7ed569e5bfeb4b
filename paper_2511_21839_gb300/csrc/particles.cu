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

template <typename T, int C, int CP>
void launch_push(const T* state_in, T* state_out, int64_t N, const T* E, const GeomDev* geom, int nx, int ny, int nz,
                 const MapCoef<T, CP>& A, const KickCoef<T, CP>& K, bool track, Ord<T>* mm, int* err,
                 const SortBuf& sb, cudaStream_t s) {
    if (N <= 0) return;
    unsigned blocks = (unsigned)((N + 255) / 256);
    if (track)
        push_kernel<T, C, CP, true><<<blocks, 256, 0, s>>>(state_in, state_out, N, E, geom, nx, ny, nz, A, K, mm, err,
                                                          sb);
    else
        push_kernel<T, C, CP, false><<<blocks, 256, 0, s>>>(state_in, state_out, N, E, geom, nx, ny, nz, A, K, mm,
                                                           err, sb);
}   // cells per block of the scan
int scan_blocks(int ncells) { return (ncells + kScanChunk - 1) / kScanChunk; }

void launch_scan(int* hist, int* offs, int* bsum, int ncells, cudaStream_t s) {
    const int nb = scan_blocks(ncells);
    scan_sum_kernel<<<nb, 256, 0, s>>>(hist, ncells, bsum);
    scan_top_kernel<<<1, 256, 0, s>>>(bsum, nb);
    scan_apply_kernel<<<nb, 256, 0, s>>>(hist, ncells, bsum, offs);
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

template <typename T, int C, int CP>
void launch_boundary(T* state, int64_t N, const MapCoef<T, CP>& A, bool apply, bool mom, double* partial,
                     int nblocks, Ord<T>* mm, cudaStream_t s) {
    if (apply && mom)
        boundary_kernel<T, C, CP, true, true><<<nblocks, 256, 0, s>>>(state, N, A, partial, mm);
    else if (mom)
        boundary_kernel<T, C, CP, true, false><<<nblocks, 256, 0, s>>>(state, N, A, partial, mm);
    else if (apply)
        boundary_kernel<T, C, CP, false, true><<<nblocks, 256, 0, s>>>(state, N, A, partial, mm);
}

void launch_moments_reduce(const double* partial, int nblocks, int CP, int64_t N, double* out, cudaStream_t s) {
    moments_reduce_kernel<<<15 * CP, 256, 0, s>>>(partial, nblocks, CP, N, out);
}

template <typename T, int C, int CP>
void launch_deposit(const T* state, int64_t N, const GeomDev* geom, int nx, int ny, int nz, T qm, T* rho, int* err,
                    const SortBuf& sb, cudaStream_t s) {
    if (N <= 0) return;
    // register-resident runs for the FP32 8-channel dual; the other variants take one particle per
    // thread (their eight node records would not fit in registers)
    constexpr int RUN = (CP == 8 && sizeof(T) == 4) ? 8 : 1;
    const int64_t threads = (N + RUN - 1) / RUN;
    constexpr int BS = RUN > 1 ? 128 : 256;
    deposit_kernel<T, C, CP, RUN><<<(unsigned)((threads + BS - 1) / BS), BS, 0, s>>>(state, N, geom, nx, ny, nz, qm,
                                                                                    rho, err, sb);
}

// ------------------------------------------------------------------ instantiations
#define ADPIC_INST(T, C, CP)                                                                                       \
    template void launch_init<T, C, CP>(const double*, int64_t, const double*, T*, cudaStream_t);                \
    template void launch_push<T, C, CP>(const T*, T*, int64_t, const T*, const GeomDev*, int, int, int,         \
                                        const MapCoef<T, CP>&, const KickCoef<T, CP>&, bool, Ord<T>*, int*,      \
                                        const SortBuf&, cudaStream_t);                                           \
    template void launch_boundary<T, C, CP>(T*, int64_t, const MapCoef<T, CP>&, bool, bool, double*, int,       \
                                            Ord<T>*, cudaStream_t);                                              \
    template void launch_deposit<T, C, CP>(const T*, int64_t, const GeomDev*, int, int, int, T, T*, int*,        \
                                           const SortBuf&, cudaStream_t);
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
