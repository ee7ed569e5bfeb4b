// Grid-side kernels: per-kick geometry, the integrated Green's function and
// its real even spectrum, the zero-padded (Hockney) FFT convolution of all
// dual channels, and the central finite-difference field.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace adpic {

__device__ __forceinline__ float ord_dec(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ double ord_dec(unsigned long long u) {
    return __longlong_as_double((long long)((u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u));
}

// ------------------------------------------------------------------ geometry

// Value-part extrema -> nodes x_j = origin + j h with h = (max - min) / (n - 4)
// and origin = min - 1.5 h, so every particle has u = (x - origin)/h in
// [1.5, n - 2.5]: its CIC nodes lie in [1, n-2] and the FD stencil in [0, n-1].
// The geometry is a constant of the kick, not differentiated. Resets the
// extrema and the channel maxima for the next kick.
template <typename T>
__global__ void geom_kernel(Ord<T>* mm, int nx, int ny, int nz, double gamma0, GeomDev* g, Ord<T>* chmax, int CP) {
    const int d = threadIdx.x;
    if (d < 3) {
        const int n = d == 0 ? nx : (d == 1 ? ny : nz);
        double lo = (double)ord_dec(mm[d]), hi = (double)ord_dec(mm[3 + d]);
        if (!(lo <= hi)) { lo = 0.0; hi = 0.0; }
        double w = hi - lo;
        if (!(w > 0.0)) w = 1e-6;
        double h = w / (double)(n - 4);
        double o = lo - 1.5 * h;
        g->o[d] = o;
        g->h[d] = h;
        g->hr[d] = d == 2 ? h * gamma0 : h;
        g->of[d] = (float)o;
        g->ihf[d] = (float)(1.0 / h);
        g->ihd[d] = 1.0 / h;
    }
    __syncthreads();
    if (d < 3) {
        // exact integrals (FP64) for every cell of the FP64 path; in FP32 for
        // the cells whose centre is within 20 h_max, beyond which the
        // expansion is below FP32 rounding
        const int n = d == 0 ? nx : (d == 1 ? ny : nz);
        double hmax = fmax(g->hr[0], fmax(g->hr[1], g->hr[2]));
        int R = (int)ceil(20.0 * hmax / g->hr[d]);
        g->R[d] = (sizeof(T) == 8 || R > n) ? n : R;
    }
    __syncthreads();
    if (d < 3) {
        mm[d] = ~(Ord<T>)0;
        mm[3 + d] = (Ord<T>)0;
    }
    for (int c = d; c < CP; c += blockDim.x) chmax[c] = (Ord<T>)0;
}

template <typename T>
void launch_geom(Ord<T>* mm, int nx, int ny, int nz, double gamma0, GeomDev* geom, Ord<T>* chmax, int CP,
                 cudaStream_t s) {
    geom_kernel<T><<<1, 32, 0, s>>>(mm, nx, ny, nz, gamma0, geom, chmax, CP);
}

// per-channel max |rho| (ordered bits of a non-negative value are its bits)
template <typename T>
__global__ void chmax_kernel(const T* __restrict__ rho, int64_t nodes, int CP, Ord<T>* chmax) {
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // multiple of CP
    T m = (T)0;
    for (int64_t t = t0; t < nodes * CP; t += stride) m = fmax(m, fabs(rho[t]));
    for (int o = CP; o < 32; o <<= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) < CP) {
        if constexpr (sizeof(T) == 4)
            atomicMax(&chmax[threadIdx.x & 31], __float_as_uint(m));
        else
            atomicMax(&chmax[threadIdx.x & 31], (unsigned long long)__double_as_longlong(m));
    }
}

template <typename T>
void launch_chmax(const T* rho, int64_t nodes, int CP, Ord<T>* chmax, cudaStream_t s) {
    chmax_kernel<T><<<152 * 2, 256, 0, s>>>(rho, nodes, CP, chmax);
}

// ------------------------------------------------------------------ Green's function

// An antiderivative of 1/r: d^3 F / dx dy dz = 1/sqrt(x^2 + y^2 + z^2).
__device__ double igf_F(double x, double y, double z) {
    const double r = sqrt(x * x + y * y + z * z);
    return y * z * log(x + r) + x * z * log(y + r) + x * y * log(z + r) - 0.5 * x * x * atan(y * z / (x * r)) -
           0.5 * y * y * atan(x * z / (y * r)) - 0.5 * z * z * atan(x * y / (z * r));
}

// F at the cell corners ((i - 1/2) hx, (j - 1/2) hy, (k - 1/2) hzr), i in [0, Rx+1] etc. (FP64)
// Launched over the full (nx+2)(ny+2)(nz+2) corner lattice; corners outside
// the near box of this kick return at once.
__global__ void green_corner_kernel(const GeomDev* __restrict__ g, int nx, int ny, int nz, double* __restrict__ F) {
    const int cx = nx + 2, cy = ny + 2, cz = nz + 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)cx * cy * cz) return;
    const int i = (int)(t % cx), j = (int)((t / cx) % cy), k = (int)(t / ((int64_t)cx * cy));
    if (i > g->R[0] + 1 || j > g->R[1] + 1 || k > g->R[2] + 1) return;
    F[t] = igf_F((i - 0.5) * g->hr[0], (j - 0.5) * g->hr[1], (k - 0.5) * g->hr[2]);
}

// Cell average of 1/(4 pi eps0 r) over the cell centred at offset (i, j, k):
// the 8-corner difference of F in FP64 inside the near box (exact, every
// cell when `exact`), else 1/r plus its h^2/24 Laplacian-type correction
// (the cell average of a smooth function to O(h^4)), which is below FP32
// rounding beyond 20 h_max.
template <typename T>
__global__ void green_cell_kernel(const GeomDev* __restrict__ g, int nx, int ny, int nz,
                                  const double* __restrict__ F, T* __restrict__ G) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int gx = nx + 1, gy = ny + 1, gz = nz + 1;
    if (t >= (int64_t)gx * gy * gz) return;
    const int i = (int)(t % gx), j = (int)((t / gx) % gy), k = (int)(t / ((int64_t)gx * gy));
    const double hx = g->hr[0], hy = g->hr[1], hz = g->hr[2];
    const double k4 = 1.0 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12);
    if (i <= g->R[0] && j <= g->R[1] && k <= g->R[2]) {
        const int cx = nx + 2, cy = ny + 2;
        auto at = [&](int a, int b, int c) { return F[((int64_t)c * cy + b) * cx + a]; };
        double s = at(i + 1, j + 1, k + 1) - at(i, j + 1, k + 1) - at(i + 1, j, k + 1) - at(i + 1, j + 1, k) +
                   at(i, j, k + 1) + at(i, j + 1, k) + at(i + 1, j, k) - at(i, j, k);
        G[t] = (T)(k4 * s / (hx * hy * hz));
    } else {
        const T x = (T)(i * hx), y = (T)(j * hy), z = (T)(k * hz);
        const T r2 = x * x + y * y + z * z;
        const T ir = rsqrt(r2);
        const T ir2 = ir * ir;
        const T corr = ((T)(hx * hx) * ((T)3 * x * x * ir2 - (T)1) + (T)(hy * hy) * ((T)3 * y * y * ir2 - (T)1) +
                        (T)(hz * hz) * ((T)3 * z * z * ir2 - (T)1)) * ir2 / (T)24;
        G[t] = (T)k4 * ir * ((T)1 + corr);
    }
}

// One DCT-I pass over the leading axis of in [B][A][L] (L = n+1 contiguous)
// into out [Lk][B][A]: out[k][b][a] = sum_l D[k][l] in[b][a][l], D[k][l] =
// w_l cos(pi l k / n), w_0 = w_n = 1, else 2. Three passes give the real
// spectrum of the even extension of G to the 2n-periodic grid.
template <typename T>
__global__ void dct_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ D, int L, int64_t BA) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= BA * L) return;
    const int k = (int)(t / BA);
    const int64_t ba = t % BA;
    const T* src = in + ba * L;
    const T* row = D + (int64_t)k * L;
    T s = (T)0;
    for (int l = 0; l < L; ++l) s = fma(__ldg(row + l), __ldg(src + l), s);
    out[t] = s;
}

template <typename T>
void launch_green(const GeomDev* geom, int nx, int ny, int nz, bool exact, double* corner, T* G, T* Gtmp, T* Ghat,
                  const T* dct_x, const T* dct_y, const T* dct_z, cudaStream_t s) {
    (void)exact;
    const int64_t nc = (int64_t)(nx + 2) * (ny + 2) * (nz + 2);
    green_corner_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(geom, nx, ny, nz, corner);
    const int64_t ng = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    green_cell_kernel<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(geom, nx, ny, nz, corner, G);
    // G [z][y][x] -> pass x -> [x'][z][y] -> pass y -> [y'][x'][z] -> pass z -> [z'][y'][x']
    dct_kernel<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(G, Gtmp, dct_x, nx + 1, (int64_t)(nz + 1) * (ny + 1));
    dct_kernel<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(Gtmp, G, dct_y, ny + 1, (int64_t)(nx + 1) * (nz + 1));
    dct_kernel<T><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(G, Ghat, dct_z, nz + 1, (int64_t)(ny + 1) * (nx + 1));
}

// ------------------------------------------------------------------ FFT convolution

// Radix-2 decimation-in-time FFT of `nlines` lines held in shared memory in
// bit-reversed order (line stride LS), twiddles tw[j] = exp(sign 2 pi i j / M).
template <typename T>
__device__ void smem_fft(V2<T>* buf, int logM, int LS, int nlines, const V2<T>* tw) {
    const int halfM = 1 << (logM - 1);
    const int total = nlines * halfM;
    for (int s = 1; s <= logM; ++s) {
        const int half = 1 << (s - 1);
        const int tsh = logM - s;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int line = t >> (logM - 1);
            const int kk = t & (halfM - 1);
            const int pos = kk & (half - 1);
            const int grp = kk >> (s - 1);
            const int a = line * LS + (grp << s) + pos;
            const int b = a + half;
            const V2<T> w = tw[pos << tsh];
            const V2<T> xb = buf[b], xa = buf[a];
            const T br = xb.x * w.x - xb.y * w.y, bi = xb.x * w.y + xb.y * w.x;
            buf[a].x = xa.x + br; buf[a].y = xa.y + bi;
            buf[b].x = xa.x - br; buf[b].y = xa.y - bi;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int brev(int j, int logM) { return (int)(__brev((unsigned)j) >> (32 - logM)); }

template <typename T>
__device__ __forceinline__ T chan_scale(const Ord<T>* chmax, int c, bool inverse) {
    T m;
    if constexpr (sizeof(T) == 4) m = __uint_as_float(chmax[c]);
    else m = __longlong_as_double((long long)chmax[c]);
    if (!(m > (T)0) || !isfinite(m)) return (T)1;
    int e;
    frexp(m, &e);                         // m = f 2^e, f in [0.5, 1)
    return inverse ? ldexp((T)1, e) : ldexp((T)1, -e);
}

constexpr int kRowsX = 2;   // grid rows per CTA in the x passes
constexpr int kTile = 16;   // lines per CTA in the y and z passes

// x pass, forward: rows (y<ny, z<nz) of every channel pair, zero padded to Mx.
// Channel pair (2p, 2p+1) becomes one complex line (the spectrum of G is
// real and even, so the two real convolutions separate again at the end);
// each channel is scaled by a power of two so both halves of a pair have
// comparable magnitude.
template <typename T>
__global__ void fftx_fwd_kernel(const T* __restrict__ rho, V2<T>* __restrict__ X1, FFTDims d,
                                const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax) {
    extern __shared__ unsigned char smraw[];
    V2<T>* tws = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = tws + d.Mx / 2;
    const int LS = d.Mx + 1;
    const int nl = kRowsX * d.npair;
    for (int j = threadIdx.x; j < d.Mx / 2; j += blockDim.x) tws[j] = tw[j];
    for (int j = threadIdx.x; j < nl * LS; j += blockDim.x) { buf[j].x = (T)0; buf[j].y = (T)0; }
    __syncthreads();
    const int64_t row0 = (int64_t)blockIdx.x * kRowsX;
    const int nrows = d.ny * d.nz;
    for (int t = threadIdx.x; t < kRowsX * d.nx * d.CP; t += blockDim.x) {
        const int r = t / (d.nx * d.CP);
        const int rem = t % (d.nx * d.CP);
        const int x = rem / d.CP, c = rem % d.CP;
        if (row0 + r >= nrows || c >= d.C) continue;
        const T v = rho[((row0 + r) * d.nx + x) * d.CP + c] * chan_scale<T>(chmax, c, false);
        V2<T>& dst = buf[(r * d.npair + (c >> 1)) * LS + brev(x, d.lx)];
        if (c & 1) dst.y = v; else dst.x = v;
    }
    __syncthreads();
    smem_fft<T>(buf, d.lx, LS, nl, tws);
    for (int t = threadIdx.x; t < nl * d.Mx; t += blockDim.x) {
        const int line = t / d.Mx, kx = t % d.Mx;
        const int r = line / d.npair, p = line % d.npair;
        if (row0 + r >= nrows) continue;
        const int64_t z = (row0 + r) / d.ny, y = (row0 + r) % d.ny;
        X1[(((int64_t)p * d.nz + z) * d.ny + y) * d.Mx + kx] = buf[line * LS + kx];
    }
}

// y pass: lines along y for a tile of kTile consecutive kx, for one (z, pair).
// forward: X1 (y < ny) -> X2 (all My); inverse: X2 (all My) -> X1 (y < ny).
template <typename T, bool INV>
__global__ void ffty_kernel(const V2<T>* __restrict__ in, V2<T>* __restrict__ out, FFTDims d,
                            const V2<T>* __restrict__ tw) {
    extern __shared__ unsigned char smraw[];
    V2<T>* tws = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = tws + d.My / 2;
    const int LS = d.My + 1;
    const int kx0 = blockIdx.x * kTile, z = blockIdx.y, p = blockIdx.z;
    const int yin = INV ? d.My : d.ny, yout = INV ? d.ny : d.My;
    for (int j = threadIdx.x; j < d.My / 2; j += blockDim.x) tws[j] = tw[j];
    if (!INV)
        for (int j = threadIdx.x; j < kTile * LS; j += blockDim.x) { buf[j].x = (T)0; buf[j].y = (T)0; }
    __syncthreads();
    const int64_t plane_in = ((int64_t)p * d.nz + z) * yin;
    for (int t = threadIdx.x; t < yin * kTile; t += blockDim.x) {
        const int y = t / kTile, j = t % kTile;
        buf[j * LS + brev(y, d.ly)] = in[(plane_in + y) * d.Mx + kx0 + j];
    }
    __syncthreads();
    smem_fft<T>(buf, d.ly, LS, kTile, tws);
    const int64_t plane_out = ((int64_t)p * d.nz + z) * yout;
    for (int t = threadIdx.x; t < yout * kTile; t += blockDim.x) {
        const int y = t / kTile, j = t % kTile;
        out[(plane_out + y) * d.Mx + kx0 + j] = buf[j * LS + y];
    }
}

// z pass: lines along z (z < nz, zero padded) for a tile of kx at one (ky, pair):
// forward FFT, multiply by the real spectrum of G, bit-reverse, inverse FFT,
// keep z < nz. In place on X2.
template <typename T>
__global__ void fftz_kernel(V2<T>* __restrict__ X2, const T* __restrict__ Ghat, FFTDims d,
                            const V2<T>* __restrict__ twf, const V2<T>* __restrict__ twi) {
    extern __shared__ unsigned char smraw[];
    V2<T>* tf = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* ti = tf + d.Mz / 2;
    V2<T>* buf = ti + d.Mz / 2;
    const int LS = d.Mz + 1;
    const int kx0 = blockIdx.x * kTile, ky = blockIdx.y, p = blockIdx.z;
    for (int j = threadIdx.x; j < d.Mz / 2; j += blockDim.x) { tf[j] = twf[j]; ti[j] = twi[j]; }
    for (int j = threadIdx.x; j < kTile * LS; j += blockDim.x) { buf[j].x = (T)0; buf[j].y = (T)0; }
    __syncthreads();
    const int64_t zstride = (int64_t)d.My * d.Mx;
    V2<T>* base = X2 + (int64_t)p * d.nz * zstride + (int64_t)ky * d.Mx + kx0;
    for (int t = threadIdx.x; t < d.nz * kTile; t += blockDim.x) {
        const int z = t / kTile, j = t % kTile;
        buf[j * LS + brev(z, d.lz)] = base[z * zstride + j];
    }
    __syncthreads();
    smem_fft<T>(buf, d.lz, LS, kTile, tf);
    const int kyr = ky <= d.ny ? ky : d.My - ky;
    for (int t = threadIdx.x; t < kTile * d.Mz; t += blockDim.x) {
        const int j = t / d.Mz, kz = t % d.Mz;
        const int kx = kx0 + j;
        const int kxr = kx <= d.nx ? kx : d.Mx - kx;
        const int kzr = kz <= d.nz ? kz : d.Mz - kz;
        const T gh = Ghat[((int64_t)kzr * (d.ny + 1) + kyr) * (d.nx + 1) + kxr];
        V2<T>& v = buf[j * LS + kz];
        v.x *= gh;
        v.y *= gh;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kTile * d.Mz; t += blockDim.x) {
        const int j = t / d.Mz, z = t % d.Mz;
        const int r = brev(z, d.lz);
        if (z < r) {
            V2<T> tmp = buf[j * LS + z];
            buf[j * LS + z] = buf[j * LS + r];
            buf[j * LS + r] = tmp;
        }
    }
    __syncthreads();
    smem_fft<T>(buf, d.lz, LS, kTile, ti);
    for (int t = threadIdx.x; t < d.nz * kTile; t += blockDim.x) {
        const int z = t / kTile, j = t % kTile;
        base[z * zstride + j] = buf[j * LS + z];
    }
}

// x pass, inverse: rows (y < ny, z < nz) of every pair, keep x < nx, undo the
// channel scaling and the 1/(Mx My Mz) normalisation, write phi [node][CP].
template <typename T>
__global__ void fftx_inv_kernel(const V2<T>* __restrict__ X1, T* __restrict__ phi, FFTDims d,
                                const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax) {
    extern __shared__ unsigned char smraw[];
    V2<T>* tws = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = tws + d.Mx / 2;
    const int LS = d.Mx + 1;
    const int nl = kRowsX * d.npair;
    for (int j = threadIdx.x; j < d.Mx / 2; j += blockDim.x) tws[j] = tw[j];
    const int64_t row0 = (int64_t)blockIdx.x * kRowsX;
    const int nrows = d.ny * d.nz;
    for (int t = threadIdx.x; t < nl * d.Mx; t += blockDim.x) {
        const int line = t / d.Mx, kx = t % d.Mx;
        const int r = line / d.npair, p = line % d.npair;
        V2<T> v;
        v.x = (T)0; v.y = (T)0;
        if (row0 + r < nrows) {
            const int64_t z = (row0 + r) / d.ny, y = (row0 + r) % d.ny;
            v = X1[(((int64_t)p * d.nz + z) * d.ny + y) * d.Mx + kx];
        }
        buf[line * LS + brev(kx, d.lx)] = v;
    }
    __syncthreads();
    smem_fft<T>(buf, d.lx, LS, nl, tws);
    const T norm = (T)(1.0 / ((double)d.Mx * d.My * d.Mz));
    for (int t = threadIdx.x; t < kRowsX * d.nx * d.CP; t += blockDim.x) {
        const int r = t / (d.nx * d.CP);
        const int rem = t % (d.nx * d.CP);
        const int x = rem / d.CP, c = rem % d.CP;
        if (row0 + r >= nrows) continue;
        T v = (T)0;
        if (c < d.C) {
            const V2<T> w = buf[(r * d.npair + (c >> 1)) * LS + x];
            v = ((c & 1) ? w.y : w.x) * norm * chan_scale<T>(chmax, c, true);
        }
        phi[((row0 + r) * d.nx + x) * d.CP + c] = v;
    }
}

template <typename T>
void setup_fft_attrs() {
    const int mx = 200 * 1024;
    cudaFuncSetAttribute(fftx_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(ffty_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(ffty_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(fftz_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(fftx_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <typename T>
void launch_fft_conv(const T* rho, V2<T>* X1, V2<T>* X2, const T* Ghat, T* phi, const FFTDims& d,
                     const V2<T>* twf_x, const V2<T>* twi_x, const V2<T>* twf_y, const V2<T>* twi_y,
                     const V2<T>* twf_z, const V2<T>* twi_z, const Ord<T>* chmax, cudaStream_t s) {
    const int rows = d.ny * d.nz;
    const unsigned gx = (unsigned)((rows + kRowsX - 1) / kRowsX);
    const size_t smx = sizeof(V2<T>) * (d.Mx / 2 + (size_t)kRowsX * d.npair * (d.Mx + 1));
    const size_t smy = sizeof(V2<T>) * (d.My / 2 + (size_t)kTile * (d.My + 1));
    const size_t smz = sizeof(V2<T>) * (d.Mz + (size_t)kTile * (d.Mz + 1));
    fftx_fwd_kernel<T><<<gx, 256, smx, s>>>(rho, X1, d, twf_x, chmax);
    ffty_kernel<T, false><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, smy, s>>>(X1, X2, d, twf_y);
    fftz_kernel<T><<<dim3(d.Mx / kTile, d.My, d.npair), 256, smz, s>>>(X2, Ghat, d, twf_z, twi_z);
    ffty_kernel<T, true><<<dim3(d.Mx / kTile, d.nz, d.npair), 256, smy, s>>>(X2, X1, d, twi_y);
    fftx_inv_kernel<T><<<gx, 256, smx, s>>>(X1, phi, d, twi_x, chmax);
}

// ------------------------------------------------------------------ field

// E = -grad(phi) by central differences on interior nodes, rest-frame
// spacings (hx, hy, gamma0 hz); E layout [node][3][CP].
template <typename T>
__global__ void field_kernel(const T* __restrict__ phi, const GeomDev* __restrict__ g, int nx, int ny, int nz, int CP,
                             T* __restrict__ E) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nodes = (int64_t)nx * ny * nz;
    if (t >= nodes * CP) return;
    const int c = (int)(t % CP);
    const int64_t node = t / CP;
    const int i = (int)(node % nx), j = (int)((node / nx) % ny), k = (int)(node / ((int64_t)nx * ny));
    if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || k < 1 || k > nz - 2) return;
    const T ax = (T)(0.5 / g->hr[0]), ay = (T)(0.5 / g->hr[1]), az = (T)(0.5 / g->hr[2]);
    const int64_t sx = CP, sy = (int64_t)nx * CP, sz = (int64_t)nx * ny * CP;
    const int64_t a = node * CP + c;
    T* e = E + node * 3 * CP + c;
    e[0] = -(phi[a + sx] - phi[a - sx]) * ax;
    e[CP] = -(phi[a + sy] - phi[a - sy]) * ay;
    e[2 * CP] = -(phi[a + sz] - phi[a - sz]) * az;
}

template <typename T>
void launch_field(const T* phi, const GeomDev* geom, int nx, int ny, int nz, int CP, T* E, cudaStream_t s) {
    const int64_t tot = (int64_t)nx * ny * nz * CP;
    field_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(phi, geom, nx, ny, nz, CP, E);
}

#define ADPIC_FIELD_INST(T)                                                                                       \
    template void launch_geom<T>(Ord<T>*, int, int, int, double, GeomDev*, Ord<T>*, int, cudaStream_t);          \
    template void launch_chmax<T>(const T*, int64_t, int, Ord<T>*, cudaStream_t);                                 \
    template void launch_green<T>(const GeomDev*, int, int, int, bool, double*, T*, T*, T*, const T*, const T*,    \
                                  const T*, cudaStream_t);                                                        \
    template void launch_fft_conv<T>(const T*, V2<T>*, V2<T>*, const T*, T*, const FFTDims&, const V2<T>*,        \
                                     const V2<T>*, const V2<T>*, const V2<T>*, const V2<T>*, const V2<T>*,        \
                                     const Ord<T>*, cudaStream_t);                                                \
    template void launch_field<T>(const T*, const GeomDev*, int, int, int, int, T*, cudaStream_t);             \
    template void setup_fft_attrs<T>();
ADPIC_FIELD_INST(float)
ADPIC_FIELD_INST(double)

}  // namespace adpic
