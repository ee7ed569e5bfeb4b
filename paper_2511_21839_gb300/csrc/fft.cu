// Zero-padded (Hockney) FFT convolution of all dual channels with the real,
// even spectrum of the Green's function.
//
// Each 1D transform of length M = 2n is a two-step Cooley-Tukey split
// M = R1 R2: with n = R2 n1 + n2 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_n2 W_R2^(n2 k2) [ W_M^(n2 k1) sum_n1 x[R2 n1 + n2] W_R1^(n1 k1) ].
// Step 1: one thread per (line, n2) does the R1-point DFT over n1 in registers
// and applies W_M^(n2 k1); step 2: one thread per (line, k1) does the
// R2-point DFT over n2 in registers. A line lives in shared memory in the
// padded layout pos(n) = (n / R2) (R2 + 1) + n % R2, so both steps are free of
// bank conflicts and step 1 works in place. In forward transforms of
// zero-padded data the upper half of the inputs (n1 >= R1/2) is known to be
// zero and is never loaded.
//
// Passes (npair = C/2 channel pairs packed as complex, see the x passes):
//   fftx_fwd   rho rows (x < nx)        -> X1 [p][z][y][kx]     (all Mx)
//   ffty<fwd>  X1 columns (y < ny)      -> X2 [p][z][ky][kx]    (all My)
//   fftz       X2 columns (z < nz): forward, times Ghat, inverse, keep z < nz, in place
//   ffty<inv>  X2 columns (all My)      -> X1 (y < ny)
//   fftx_inv   X1 rows (all Mx)         -> phi rows (x < nx), scaled back
// Grids with nz <= 64 take the three-launch slab path instead (fftx_fwd_t,
// fftyz, fftx_inv_t in fft_dev.cuh), with Ghat stored [kx'][kz'][ky'].
#include <algorithm>

#include "fft_dev.cuh"

namespace adpic {

template <typename T, int M>
struct Conv {
    static size_t sm_x(const FFTDims& d) {
        const size_t lines = (size_t)kRowsX * d.npair * Lay<M>::LS;
        return sizeof(V2<T>) * (M + lines) + sizeof(T) * kRowsX * d.nx * d.CP;
    }
    static size_t sm_col() { return sizeof(V2<T>) * (M + (size_t)kTile * Lay<M>::LS); }
    static void attrs() {
        const int mx = 200 * 1024;
        cudaFuncSetAttribute(fftx_fwd_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(ffty_kernel<T, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(ffty_kernel<T, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(fftz_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(fftx_inv_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    }
};

template <typename T, int MX, int MY, int MZ>
void conv_run(T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
              const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    const int rows = d.ny * d.nz;
    const unsigned gx = (unsigned)((rows + kRowsX - 1) / kRowsX);
    fftx_fwd_kernel<T, MX><<<gx, 256, Conv<T, MX>::sm_x(d), s>>>(rho, X1, d, twx, chmax);
    if (spec) cudaStreamWaitEvent(s, spec, 0);
    ffty_kernel<T, MY, false><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, Conv<T, MY>::sm_col(), s>>>(X1, X2, d, twy);
    fftz_kernel<T, MZ><<<dim3(d.Mx / kTile, d.My, d.npair), 256, Conv<T, MZ>::sm_col(), s>>>(X2, Ghat, d, twz);
    ffty_kernel<T, MY, true><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, Conv<T, MY>::sm_col(), s>>>(X2, X1, d, twy);
    fftx_inv_kernel<T, MX><<<gx, 256, Conv<T, MX>::sm_x(d), s>>>(X1, phi, d, twx, chmax);
}
template <typename T, int MX, int MY>
void conv_z(T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
            const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    switch (d.Mz) {
        case 16: conv_run<T, MX, MY, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 32: conv_run<T, MX, MY, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 64: conv_run<T, MX, MY, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 128: conv_run<T, MX, MY, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        default: conv_run<T, MX, MY, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
    }
}

template <typename T, int MX>
void conv_y(T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
            const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    switch (d.My) {
        case 16: conv_z<T, MX, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 32: conv_z<T, MX, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 64: conv_z<T, MX, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 128: conv_z<T, MX, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        default: conv_z<T, MX, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
    }
}

// ---------------------------------------------------------------- slab path

static int lay_ls(int M) {
    switch (M) {
        case 16: return Lay<16>::LS;
        case 32: return Lay<32>::LS;
        case 64: return Lay<64>::LS;
        case 128: return Lay<128>::LS;
        default: return Lay<256>::LS;
    }
}

template <typename T>
static size_t sm_fwd_t(const FFTDims& d, int yt) {
    return sizeof(V2<T>) * ((size_t)d.Mx + (size_t)yt * d.npair * lay_ls(d.Mx)) + sizeof(T) * 16;
}
template <typename T>
static size_t sm_inv_t(const FFTDims& d, int yt) {
    return sm_fwd_t<T>(d, yt) + sizeof(T) * (size_t)yt * ((size_t)d.nx * d.CP + 1);
}
template <typename T>
static size_t sm_yz(const FFTDims& d) {
    return sizeof(V2<T>) * ((size_t)d.My + d.Mz + (size_t)d.nz * lay_ls(d.My) + (size_t)slab_kc<T>() * lay_ls(d.Mz));
}
constexpr size_t kSmemCap = 200 * 1024;

// rows per CTA of the x passes: up to 16 while both x kernels stay within 96 KB
template <typename T>
static int slab_yt(const FFTDims& d) {
    int yt = d.ny < 16 ? d.ny : 16;
    while (yt > 1 && sm_inv_t<T>(d, yt) > 96 * 1024) yt >>= 1;
    return yt;
}

template <typename T>
bool fft_slab_path(const FFTDims& d) {
    return d.nz <= 64 && d.My <= 128 && d.Mz <= 128 && sm_yz<T>(d) <= kSmemCap &&
           sm_inv_t<T>(d, slab_yt<T>(d)) <= kSmemCap;
}

int fft_conv_launches(bool slab) { return slab ? 3 : 5; }

template <typename T>
int fft_slab_yt(const FFTDims& d) { return slab_yt<T>(d); }

template <typename T>
size_t fft_slab_smem(const FFTDims& d, int which) {
    const int yt = slab_yt<T>(d);
    if (which == 0) return sm_fwd_t<T>(d, yt);
    if (which == 1) return sm_yz<T>(d);
    if (which == 2) return sm_inv_t<T>(d, yt);
    return std::max(std::max(sm_fwd_t<T>(d, yt), sm_inv_t<T>(d, yt)), sm_yz<T>(d));
}

template <typename T, int MX, int MY, int MZ>
void conv_slab(T* rho, V2<T>* X1, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx, const V2<T>* twy,
               const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    const int yt = slab_yt<T>(d);
    const dim3 gx((unsigned)(d.ny / yt), (unsigned)d.nz);
    fftx_fwd_t_kernel<T, MX><<<gx, 256, sm_fwd_t<T>(d, yt), s>>>(rho, X1, d, twx, chmax, yt);
    if (spec) cudaStreamWaitEvent(s, spec, 0);
    fftyz_kernel<T, MY, MZ><<<dim3((unsigned)d.Mx, (unsigned)d.npair), 512, sm_yz<T>(d), s>>>(X1, Ghat, d, twy, twz);
    fftx_inv_t_kernel<T, MX><<<gx, 256, sm_inv_t<T>(d, yt), s>>>(X1, phi, d, twx, chmax, yt);
}
template <typename T, int MX, int MY>
void conv_slab_z(T* rho, V2<T>* X1, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx, const V2<T>* twy,
                 const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    switch (d.Mz) {
        case 16: conv_slab<T, MX, MY, 16>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 32: conv_slab<T, MX, MY, 32>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 64: conv_slab<T, MX, MY, 64>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        default: conv_slab<T, MX, MY, 128>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
    }
}
template <typename T, int MX>
void conv_slab_y(T* rho, V2<T>* X1, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx, const V2<T>* twy,
                 const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    switch (d.My) {
        case 16: conv_slab_z<T, MX, 16>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 32: conv_slab_z<T, MX, 32>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 64: conv_slab_z<T, MX, 64>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        default: conv_slab_z<T, MX, 128>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
    }
}

template <typename T>
void launch_fft_conv(T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
                     const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s, cudaEvent_t spec) {
    if (fft_slab_path<T>(d)) {
        switch (d.Mx) {
            case 16: conv_slab_y<T, 16>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
            case 32: conv_slab_y<T, 32>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
            case 64: conv_slab_y<T, 64>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
            case 128: conv_slab_y<T, 128>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
            default: conv_slab_y<T, 256>(rho, X1, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        }
        return;
    }
    switch (d.Mx) {
        case 16: conv_y<T, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 32: conv_y<T, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 64: conv_y<T, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        case 128: conv_y<T, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
        default: conv_y<T, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s, spec); break;
    }
}

template <typename T, int M>
static void slab_x_attrs() {
    cudaFuncSetAttribute(fftx_fwd_t_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(fftx_inv_t_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
}
template <typename T, int MY>
static void slab_yz_attrs() {
    cudaFuncSetAttribute(fftyz_kernel<T, MY, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(fftyz_kernel<T, MY, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(fftyz_kernel<T, MY, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(fftyz_kernel<T, MY, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
}

template <typename T>
void setup_fft() {
    Conv<T, 16>::attrs();
    Conv<T, 32>::attrs();
    Conv<T, 64>::attrs();
    Conv<T, 128>::attrs();
    Conv<T, 256>::attrs();
    slab_x_attrs<T, 16>();
    slab_x_attrs<T, 32>();
    slab_x_attrs<T, 64>();
    slab_x_attrs<T, 128>();
    slab_x_attrs<T, 256>();
    slab_yz_attrs<T, 16>();
    slab_yz_attrs<T, 32>();
    slab_yz_attrs<T, 64>();
    slab_yz_attrs<T, 128>();
}

template void launch_fft_conv<float>(float*, float2*, float2*, const float*, float*, const FFTDims&,
                                     const float2*, const float2*, const float2*, const unsigned int*, cudaStream_t,
                                     cudaEvent_t);
template void launch_fft_conv<double>(double*, double2*, double2*, const double*, double*, const FFTDims&,
                                      const double2*, const double2*, const double2*, const unsigned long long*,
                                      cudaStream_t, cudaEvent_t);
template bool fft_slab_path<float>(const FFTDims&);
template int fft_slab_yt<float>(const FFTDims&);
template size_t fft_slab_smem<float>(const FFTDims&, int);
template bool fft_slab_path<double>(const FFTDims&);
template void setup_fft<float>();
template void setup_fft<double>();

}  // namespace adpic
