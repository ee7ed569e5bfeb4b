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
void conv_run(const T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
              const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s) {
    const int rows = d.ny * d.nz;
    const unsigned gx = (unsigned)((rows + kRowsX - 1) / kRowsX);
    fftx_fwd_kernel<T, MX><<<gx, 256, Conv<T, MX>::sm_x(d), s>>>(rho, X1, d, twx, chmax);
    ffty_kernel<T, MY, false><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, Conv<T, MY>::sm_col(), s>>>(X1, X2, d, twy);
    fftz_kernel<T, MZ><<<dim3(d.Mx / kTile, d.My, d.npair), 256, Conv<T, MZ>::sm_col(), s>>>(X2, Ghat, d, twz);
    ffty_kernel<T, MY, true><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, Conv<T, MY>::sm_col(), s>>>(X2, X1, d, twy);
    fftx_inv_kernel<T, MX><<<gx, 256, Conv<T, MX>::sm_x(d), s>>>(X1, phi, d, twx, chmax);
}
template <typename T, int MX, int MY>
void conv_z(const T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
            const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s) {
    switch (d.Mz) {
        case 16: conv_run<T, MX, MY, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 32: conv_run<T, MX, MY, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 64: conv_run<T, MX, MY, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 128: conv_run<T, MX, MY, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        default: conv_run<T, MX, MY, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
    }
}

template <typename T, int MX>
void conv_y(const T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
            const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s) {
    switch (d.My) {
        case 16: conv_z<T, MX, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 32: conv_z<T, MX, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 64: conv_z<T, MX, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 128: conv_z<T, MX, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        default: conv_z<T, MX, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
    }
}

template <typename T>
void launch_fft_conv(const T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d, const V2<T>* twx,
                     const V2<T>* twy, const V2<T>* twz, const Ord<T>* chmax, cudaStream_t s) {
    switch (d.Mx) {
        case 16: conv_y<T, 16>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 32: conv_y<T, 32>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 64: conv_y<T, 64>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        case 128: conv_y<T, 128>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
        default: conv_y<T, 256>(rho, X1, X2, Ghat, phi, d, twx, twy, twz, chmax, s); break;
    }
}

template <typename T>
void setup_fft() {
    Conv<T, 16>::attrs();
    Conv<T, 32>::attrs();
    Conv<T, 64>::attrs();
    Conv<T, 128>::attrs();
    Conv<T, 256>::attrs();
    float2 f[16];
    double2 dd[16];
    for (int j = 0; j < 16; ++j) {
        const double a = 2.0 * M_PI * (double)j / 16.0;
        dd[j].x = std::cos(a);
        dd[j].y = -std::sin(a);
        f[j].x = (float)dd[j].x;
        f[j].y = (float)dd[j].y;
    }
    cudaMemcpyToSymbol(c_tw16f, f, sizeof(f));
    cudaMemcpyToSymbol(c_tw16d, dd, sizeof(dd));
}

template void launch_fft_conv<float>(const float*, float2*, float2*, const float*, float*, const FFTDims&,
                                     const float2*, const float2*, const float2*, const unsigned int*, cudaStream_t);
template void launch_fft_conv<double>(const double*, double2*, double2*, const double*, double*, const FFTDims&,
                                      const double2*, const double2*, const double2*, const unsigned long long*,
                                      cudaStream_t);
template void setup_fft<float>();
template void setup_fft<double>();

}  // namespace adpic
