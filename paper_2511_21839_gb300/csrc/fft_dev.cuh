// Device code of fft.cu (helpers, kernel bodies taking an explicit block index,
// and their kernel wrappers), shared by fft.cu and the batched persistent kernel.
#pragma once
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
#include <cmath>

#include "common.cuh"

namespace adpic {

// d * exp(-+ 2 pi i e / 16) for e in [0, 8) (the sign is + for INV). Inside
// unrolled loops e is a compile-time constant, so the switch folds away:
// multiplications by -i cost nothing and the 45-degree ones two adds.
template <typename T, bool INV>
__device__ __forceinline__ V2<T> mul_w16(V2<T> d, int e) {
    constexpr T c1 = (T)0.92387953251128675613;   // cos(pi / 8)
    constexpr T s1 = (T)0.38268343236508977173;   // sin(pi / 8)
    constexpr T h = (T)0.70710678118654752440;    // cos(pi / 4)
    const T sg = INV ? (T)-1 : (T)1;              // exp(-i a) forward, exp(+i a) inverse
    V2<T> r;
    switch (e) {
        case 0: r = d; break;
        case 2: r.x = h * (d.x + sg * d.y); r.y = h * (d.y - sg * d.x); break;
        case 4: r.x = sg * d.y; r.y = -sg * d.x; break;
        case 6: r.x = h * (sg * d.y - d.x); r.y = -h * (d.y + sg * d.x); break;
        default: {
            // exp(-+ i a) with (cos a, sin a) = (c1, s1), (s1, c1), (-s1, c1), (-c1, s1) for e = 1, 3, 5, 7
            const T ca = e == 1 ? c1 : (e == 3 ? s1 : (e == 5 ? -s1 : -c1));
            const T sa = e == 1 ? s1 : (e == 3 ? c1 : (e == 5 ? c1 : s1));
            r.x = fma(d.x, ca, sg * d.y * sa);
            r.y = fma(d.y, ca, -sg * d.x * sa);
        }
    }
    return r;
}

template <typename T>
__device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
    V2<T> r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__host__ __device__ constexpr int brev_c(int k, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((k >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int log2_c(int n) { return n <= 1 ? 0 : 1 + log2_c(n / 2); }

// R-point DFT in registers (R <= 16): radix-2 decimation in frequency, natural
// input order, output X[k] in v[brev(k)]. INV uses the conjugate twiddles.
// HZ: the upper half of the inputs is zero, so the first stage only copies
// and rotates (no additions with zero). HO: only the outputs X[k], k < R/2
// are wanted (v at even positions), so the last stage skips the differences.
template <typename T, int R, bool INV, bool HZ = false, bool HO = false>
__device__ __forceinline__ void dft_reg(V2<T> (&v)[R]) {
#pragma unroll
    for (int len = R; len >= 2; len >>= 1) {
        const int half = len >> 1;
        if (HZ && len == R) {
#pragma unroll
            for (int j = 0; j < half; ++j) v[j + half] = mul_w16<T, INV>(v[j], j * (16 / len));
            continue;
        }
        if (HO && len == 2) {
#pragma unroll
            for (int g = 0; g < R; g += 2) v[g] = v2_add(v[g], v[g + 1]);
            continue;
        }
#pragma unroll
        for (int g = 0; g < R; g += len) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const V2<T> a = v[g + j], b = v[g + j + half];
                v[g + j] = v2_add(a, b);
                v[g + j + half] = mul_w16<T, INV>(v2_sub(a, b), j * (16 / len));
            }
        }
    }
}

template <int M> struct Split;
template <> struct Split<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Split<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Split<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Split<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct Split<256> { static constexpr int R1 = 16, R2 = 16; };

template <int M>
struct Lay {
    static constexpr int R1 = Split<M>::R1, R2 = Split<M>::R2;
    static constexpr int LS = R1 * (R2 + 1) + 1;   // line stride in complex words (odd)
    __device__ static __forceinline__ int pos(int n) { return (n / R2) * (R2 + 1) + n % R2; }
};

// q = n / d and n - q d for 0 <= n < 2^31 and a divisor d >= 1 that is only
// known at run time, by one multiply-high with a precomputed magic number
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (umulhi(m, n) + n) >> l.
struct DivMod {
    int d, l;
    unsigned m;
    __device__ int div(int n) const { return (int)((__umulhi(m, (unsigned)n) + (unsigned)n) >> l); }
};
__device__ __forceinline__ DivMod divmod_of(int d) {
    DivMod r;
    r.d = d;
    r.l = 32 - __clz(d - 1);
    r.m = (unsigned)((((unsigned long long)1 << 32) * (((unsigned long long)1 << r.l) - (unsigned)d)) / (unsigned)d + 1);
    return r;
}
__device__ __forceinline__ int lcount(int n) { return n; }
__device__ __forceinline__ int lcount(const DivMod& n) { return n.d; }
__device__ __forceinline__ int ldiv(int w, int n) { return w / n; }
__device__ __forceinline__ int ldiv(int w, const DivMod& n) { return n.div(w); }

// End of a step-1 item: the R1 outputs (bit-reversed in v) times W_M^(n2 k1),
// stored at b[k1 (R2 + 1)], b = line + n2.
template <typename T, int M, bool INV>
__device__ __forceinline__ void step1_store(const V2<T> (&v)[Lay<M>::R1], V2<T>* b, int n2, const V2<T>* twM) {
    constexpr int R1 = Lay<M>::R1, R2 = Lay<M>::R2;
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        V2<T> y = v[brev_c(k1, log2_c(R1))];
        if (k1 != 0 && n2 != 0) {
            V2<T> t = twM[(n2 * k1) & (M - 1)];
            if (INV) t.y = -t.y;
            y = cmul<T>(y, t);
        }
        b[k1 * (R2 + 1)] = y;
    }
}

// Step 1 for work item w of nlines * R2 (line = w % nlines, n2 = w / nlines):
// R1-point DFT over n1 in place, times W_M^(n2 k1). `half_zero`: inputs with
// n >= M/2 are zero (zero padding) and not read. `nlines` is an int (folded
// when it is a constant of the caller) or a DivMod.
template <typename T, int M, bool INV, typename NL = int>
__device__ __forceinline__ void step1(V2<T>* buf, NL nlines, const V2<T>* twM, bool half_zero) {
    using L = Lay<M>;
    constexpr int R1 = L::R1, R2 = L::R2;
    const int nl = lcount(nlines);
    for (int w = threadIdx.x; w < nl * R2; w += blockDim.x) {
        const int n2 = ldiv(w, nlines), line = w - n2 * nl;
        V2<T>* b = buf + line * L::LS + n2;
        V2<T> v[R1];
        if (half_zero) {
#pragma unroll
            for (int n1 = 0; n1 < R1 / 2; ++n1) v[n1] = b[n1 * (R2 + 1)];
            dft_reg<T, R1, INV, true>(v);
        } else {
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) v[n1] = b[n1 * (R2 + 1)];
            dft_reg<T, R1, INV>(v);
        }
        step1_store<T, M, INV>(v, b, n2, twM);
    }
}

// Step 2 loads for work item w of nlines * R1 (line = w % nlines, k1 = w / nlines)
// the R2 values of row k1 and transforms them; X[k1 + R1 k2] = v[brev(k2)].
// HO: only X[k1 + R1 k2] with k2 < R2/2 are used.
template <typename T, int M, bool INV, bool HO = false>
__device__ __forceinline__ void step2(const V2<T>* buf, int line, int k1, V2<T> (&v)[Lay<M>::R2]) {
    using L = Lay<M>;
    constexpr int R2 = L::R2;
    const V2<T>* b = buf + line * L::LS + k1 * (R2 + 1);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = b[n2];
    dft_reg<T, R2, INV, false, HO>(v);
}

template <typename T>
__device__ __forceinline__ T chan_scale(const Ord<T>* chmax, int c, bool inverse) {
    T m;
    if constexpr (sizeof(T) == 4) m = __uint_as_float(chmax[c]);
    else m = __longlong_as_double((long long)chmax[c]);
    // an identically zero channel (a derivative the beam has not yet picked
    // up) must stay exactly zero: its partner's rounding is not let through
    if (m == (T)0) return inverse ? (T)0 : (T)1;
    if (!isfinite(m)) return (T)1;
    int e;
    frexp(m, &e);                         // m = f 2^e, f in [0.5, 1)
    return inverse ? ldexp((T)1, e) : ldexp((T)1, -e);
}

constexpr int kRowsX = 2;   // grid rows per CTA in the x passes
constexpr int kTile = 16;   // columns per CTA in the y and z passes

// x pass, forward: rows (y < ny, z < nz) of every channel pair. Channel pair
// (2p, 2p+1) becomes one complex line (the spectrum of G is real and even, so
// the two real convolutions separate again at the end); each channel is
// scaled by a power of two so both halves of a pair have comparable magnitude.
// clear: zero each rho value after reading it, so rho is zero for the next
// deposit (read and cleared through one pointer).
template <typename T, int M>
__device__ __forceinline__ void fftx_fwd_kernel_body(T* rho, V2<T>* __restrict__ X1, FFTDims d,
                                                       const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax,
                                                       bool clear,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = twM + M;
    const int nl = kRowsX * d.npair;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    const int64_t row0 = (int64_t)bx_ * kRowsX;
    const int nrows = d.ny * d.nz;
    const int lcp = __ffs(d.CP) - 1;                  // nx = M/2 and CP are powers of two
    constexpr int LNX = log2_c(M) - 1;
    __shared__ T scs[16];                             // channel scales
    if (threadIdx.x < d.CP) scs[threadIdx.x] = chan_scale<T>(chmax, threadIdx.x, false);
    __syncthreads();
    // batches of NB independent loads per thread (one latency per batch)
    constexpr int NB = 8;
    const int total = kRowsX << (LNX + lcp);
    for (int t0 = threadIdx.x; t0 < total; t0 += NB * blockDim.x) {
        T v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, r = t >> (LNX + lcp);
            const int x = (t >> lcp) & ((1 << LNX) - 1), c = t & (d.CP - 1);
            v[b] = (t < total && row0 + r < nrows && c < d.C) ? rho[((row0 + r) * d.nx + x) * d.CP + c] : (T)0;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, r = t >> (LNX + lcp);
            const int x = (t >> lcp) & ((1 << LNX) - 1), c = t & (d.CP - 1);
            if (t >= total || row0 + r >= nrows || c >= d.C) continue;
            V2<T>& dst = buf[(r * d.npair + (c >> 1)) * L::LS + L::pos(x)];
            const T sv = v[b] * scs[c];
            if (c & 1) dst.y = sv; else dst.x = sv;
        }
    }
    __syncthreads();
    if (clear) {
        // the rows just read (contiguous) are cleared after every load of the block
        const int rows = (int)min((int64_t)kRowsX, (int64_t)nrows - row0);
        T* zr = rho + row0 * d.nx * d.CP;
        for (int t = threadIdx.x; t < (rows << (LNX + lcp)); t += blockDim.x) zr[t] = (T)0;
    }
    step1<T, M, false>(buf, nl, twM, true);
    __syncthreads();
    for (int w = threadIdx.x; w < nl * L::R1; w += blockDim.x) {
        const int line = w % nl, k1 = w / nl;
        V2<T> v[L::R2];
        step2<T, M, false>(buf, line, k1, v);
        const int r = line / d.npair, p = line % d.npair;
        if (row0 + r >= nrows) continue;
        const int64_t z = (row0 + r) / d.ny, y = (row0 + r) % d.ny;
        V2<T>* out = X1 + (((int64_t)p * d.nz + z) * d.ny + y) * M;
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) out[k1 + L::R1 * k2] = v[brev_c(k2, log2_c(L::R2))];
    }
}

template <typename T, int M>
static __global__ void __launch_bounds__(256) fftx_fwd_kernel(T* rho, V2<T>* __restrict__ X1, FFTDims d,
                                                       const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax) {
    fftx_fwd_kernel_body<T, M>(rho, X1, d, tw, chmax, true, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// y pass over a tile of kTile consecutive kx for one (z, pair).
// forward: X1 (y < ny) -> X2 (all My); inverse: X2 (all My) -> X1 (y < ny).
template <typename T, int M, bool INV>
__device__ __forceinline__ void ffty_kernel_body(const V2<T>* __restrict__ in, V2<T>* __restrict__ out, FFTDims d,
                                                   const V2<T>* __restrict__ tw,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = twM + M;
    const int kx0 = bx_ * kTile, z = by_, p = bz_;
    const int yin = INV ? M : d.ny, yout = INV ? d.ny : M;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    const int64_t plane_in = ((int64_t)p * d.nz + z) * yin;
    constexpr int NB = 8;                             // independent loads in flight per thread
    for (int t0 = threadIdx.x; t0 < yin * kTile; t0 += NB * blockDim.x) {
        V2<T> v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, y = t / kTile, j = t % kTile;
            if (t < yin * kTile) v[b] = in[(plane_in + y) * d.Mx + kx0 + j];
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, y = t / kTile, j = t % kTile;
            if (t < yin * kTile) buf[j * L::LS + L::pos(y)] = v[b];
        }
    }
    __syncthreads();
    step1<T, M, INV>(buf, kTile, twM, !INV);
    __syncthreads();
    const int64_t plane_out = ((int64_t)p * d.nz + z) * yout;
    for (int w = threadIdx.x; w < kTile * L::R1; w += blockDim.x) {
        const int j = w % kTile, k1 = w / kTile;
        V2<T> v[L::R2];
        step2<T, M, INV, INV>(buf, j, k1, v);       // the inverse keeps y < ny
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) {
            const int y = k1 + L::R1 * k2;
            if (y < yout) out[(plane_out + y) * d.Mx + kx0 + j] = v[brev_c(k2, log2_c(L::R2))];
        }
    }
}

template <typename T, int M, bool INV>
static __global__ void __launch_bounds__(256) ffty_kernel(const V2<T>* __restrict__ in, V2<T>* __restrict__ out, FFTDims d,
                                                   const V2<T>* __restrict__ tw) {
    ffty_kernel_body<T, M, INV>(in, out, d, tw, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// z pass over a tile of kx at one (ky, pair), in place on X2: forward
// transform of the zero-padded column, multiply by Ghat, inverse, keep z < nz.
template <typename T, int M>
__device__ __forceinline__ void fftz_kernel_body(V2<T>* __restrict__ X2, const T* __restrict__ Ghat, FFTDims d,
                                                   const V2<T>* __restrict__ tw,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = twM + M;
    const int kx0 = bx_ * kTile, ky = by_, p = bz_;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    const int64_t zstride = (int64_t)d.My * d.Mx;
    V2<T>* base = X2 + (int64_t)p * d.nz * zstride + (int64_t)ky * d.Mx + kx0;
    constexpr int NB = 8;                             // independent loads in flight per thread
    for (int t0 = threadIdx.x; t0 < d.nz * kTile; t0 += NB * blockDim.x) {
        V2<T> v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, z = t / kTile, j = t % kTile;
            if (t < d.nz * kTile) v[b] = base[z * zstride + j];
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, z = t / kTile, j = t % kTile;
            if (t < d.nz * kTile) buf[j * L::LS + L::pos(z)] = v[b];
        }
    }
    __syncthreads();
    step1<T, M, false>(buf, kTile, twM, true);
    __syncthreads();
    // forward step 2 into registers, times Ghat, back in the input layout
    constexpr int NW = (kTile * L::R1 + 255) / 256;
    V2<T> keep[NW][L::R2];
    const int kyr = ky <= d.ny ? ky : d.My - ky;
#pragma unroll
    for (int s = 0; s < NW; ++s) {
        const int w = threadIdx.x + s * blockDim.x;
        if (w < kTile * L::R1) step2<T, M, false>(buf, w % kTile, w / kTile, keep[s]);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NW; ++s) {
        const int w = threadIdx.x + s * blockDim.x;
        if (w >= kTile * L::R1) continue;
        const int j = w % kTile, k1 = w / kTile;
        const int kx = kx0 + j;
        const int kxr = kx <= d.nx ? kx : d.Mx - kx;
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) {
            const int kz = k1 + L::R1 * k2;
            const int kzr = kz <= d.nz ? kz : M - kz;
            const T gh = Ghat[((int64_t)kzr * (d.ny + 1) + kyr) * (d.nx + 1) + kxr];
            V2<T> v = keep[s][brev_c(k2, log2_c(L::R2))];
            v.x *= gh;
            v.y *= gh;
            buf[j * L::LS + L::pos(kz)] = v;
        }
    }
    __syncthreads();
    step1<T, M, true>(buf, kTile, twM, false);
    __syncthreads();
    for (int w = threadIdx.x; w < kTile * L::R1; w += blockDim.x) {
        const int j = w % kTile, k1 = w / kTile;
        V2<T> v[L::R2];
        step2<T, M, true, true>(buf, j, k1, v);     // keeps z < nz
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) {
            const int z = k1 + L::R1 * k2;
            if (z < d.nz) base[z * zstride + j] = v[brev_c(k2, log2_c(L::R2))];
        }
    }
}

template <typename T, int M>
static __global__ void __launch_bounds__(256) fftz_kernel(V2<T>* __restrict__ X2, const T* __restrict__ Ghat, FFTDims d,
                                                   const V2<T>* __restrict__ tw) {
    fftz_kernel_body<T, M>(X2, Ghat, d, tw, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// x pass, inverse: rows (y < ny, z < nz) of every pair, keep x < nx, undo the
// channel scaling and the 1/(Mx My Mz) normalisation, write phi [node][CP]
// through shared memory so the row is stored contiguously.
template <typename T, int M>
__device__ __forceinline__ void fftx_inv_kernel_body(const V2<T>* __restrict__ X1, T* __restrict__ phi, FFTDims d,
                                                       const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* buf = twM + M;
    const int nl = kRowsX * d.npair;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    const int64_t row0 = (int64_t)bx_ * kRowsX;
    const int nrows = d.ny * d.nz;
    __shared__ T isc[16];                             // channel scales back, times 1/(Mx My Mz)
    if (threadIdx.x < d.CP) isc[threadIdx.x] = (T)d.norm * chan_scale<T>(chmax, threadIdx.x, true);
    constexpr int NB = 8;                             // independent loads in flight per thread
    for (int t0 = threadIdx.x; t0 < nl * M; t0 += NB * blockDim.x) {
        V2<T> v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, line = t / M, kx = t % M;
            const int r = line / d.npair, p = line % d.npair;
            v[b].x = (T)0;
            v[b].y = (T)0;
            if (t < nl * M && row0 + r < nrows) {
                const int64_t z = (row0 + r) / d.ny, y = (row0 + r) % d.ny;
                v[b] = X1[(((int64_t)p * d.nz + z) * d.ny + y) * M + kx];
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int t = t0 + b * blockDim.x, line = t / M, kx = t % M;
            if (t < nl * M) buf[line * L::LS + L::pos(kx)] = v[b];
        }
    }
    __syncthreads();
    step1<T, M, true>(buf, nl, twM, false);
    __syncthreads();
    // outputs x < nx of every line into a row-major staging area [r][x][CP]
    T* stage = reinterpret_cast<T*>(buf + nl * L::LS);
    for (int w = threadIdx.x; w < nl * L::R1; w += blockDim.x) {
        const int line = w % nl, k1 = w / nl;
        V2<T> v[L::R2];
        step2<T, M, true, true>(buf, line, k1, v);   // keeps x < nx
        const int r = line / d.npair, p = line % d.npair;
        const T sa = isc[2 * p], sb = isc[2 * p + 1];
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) {
            const int x = k1 + L::R1 * k2;
            if (x < d.nx) {
                const V2<T> q = v[brev_c(k2, log2_c(L::R2))];
                stage[(r * d.nx + x) * d.CP + 2 * p] = q.x * sa;
                stage[(r * d.nx + x) * d.CP + 2 * p + 1] = q.y * sb;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kRowsX * d.nx * d.CP; t += blockDim.x) {
        const int r = t / (d.nx * d.CP);
        const int c = t % d.CP;
        if (row0 + r >= nrows) continue;
        phi[row0 * d.nx * d.CP + t] = c < d.C ? stage[t] : (T)0;
    }
}

template <typename T, int M>
static __global__ void __launch_bounds__(256) fftx_inv_kernel(const V2<T>* __restrict__ X1, T* __restrict__ phi, FFTDims d,
                                                       const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax) {
    fftx_inv_kernel_body<T, M>(X1, phi, d, tw, chmax, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// ------------------------------------------------------------------ slab path
// For grids whose (z, 2ny) slab of one channel pair fits in shared memory
// (n <= 64): the x passes exchange data with X1 in the layout
// [pair][kx][z][y] (y fastest), and one CTA per (kx, pair) runs the y and z
// transforms, the multiplication by Ghat and both inverses on its slab
// without leaving shared memory. Ghat is then stored [kx'][kz'][ky'] so a
// CTA reads one contiguous plane. Three launches instead of five, and the
// (2ny)(2nx) nz intermediate never exists.

// x pass, forward: rows (z, y0 .. y0 + yt - 1) of every pair -> X1 [p][kx][z][y]
template <typename T, int M>
__device__ __forceinline__ void fftx_fwd_t_kernel_body(T* rho, V2<T>* __restrict__ X1, FFTDims d,
                                                         const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax,
                                                         int yt, bool clear, const int bx_, const int by_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    T* sc = reinterpret_cast<T*>(twM + M);            // channel scales [16]
    V2<T>* buf = reinterpret_cast<V2<T>*>(sc + 16);   // [npair * yt][LS], line = p * yt + r
    const int nl = yt * d.npair;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    if (threadIdx.x < d.CP) sc[threadIdx.x] = chan_scale<T>(chmax, threadIdx.x, false);
    __syncthreads();
    const int y0 = bx_ * yt, z = by_;
    // channel pairs (2p, 2p+1) of a node are one V2 load; nx = M/2, CP and yt
    // are powers of two, so the indices are shifts and masks
    constexpr int LNX = log2_c(M) - 1;
    const int lpn = __ffs(d.CP) - 2;                  // log2(CP / 2)
    const int lyt = __ffs(yt) - 1;
    V2<T>* src = reinterpret_cast<V2<T>*>(rho + ((int64_t)z * d.ny + y0) * d.nx * d.CP);
    // batches of 16 independent loads per thread (one latency per batch)
    constexpr int NBL = 16;
    const int total = yt << (LNX + lpn);
    for (int t0 = threadIdx.x; t0 < total; t0 += NBL * blockDim.x) {
        V2<T> v[NBL];
#pragma unroll
        for (int b = 0; b < NBL; ++b) {
            const int t = t0 + b * blockDim.x;
            if (t < total && (t & ((1 << lpn) - 1)) < d.npair) v[b] = src[t];
        }
#pragma unroll
        for (int b = 0; b < NBL; ++b) {
            const int t = t0 + b * blockDim.x;
            const int p = t & ((1 << lpn) - 1), x = (t >> lpn) & ((1 << LNX) - 1), r = t >> (lpn + LNX);
            if (t < total && p < d.npair) {
                v[b].x *= sc[2 * p];
                v[b].y *= sc[2 * p + 1];
                buf[(p * yt + r) * L::LS + L::pos(x)] = v[b];
            }
        }
    }
    __syncthreads();
    if (clear) {
        // the rows just read (contiguous: yt rows of nx CP values) are cleared
        // with 16-byte stores, after every load of the block
        float4* zr = reinterpret_cast<float4*>(src);
        const int n16 = (yt << (LNX + lpn)) * (int)sizeof(V2<T>) / 16;
        for (int t = threadIdx.x; t < n16; t += blockDim.x) zr[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    step1<T, M, false>(buf, divmod_of(nl), twM, true);
    __syncthreads();
    const int64_t kstride = (int64_t)d.nz * d.ny;
    V2<T>* dst0 = X1 + (int64_t)z * d.ny + y0;
    // work items with r fastest (consecutive y in the stores), then k1, then p
    for (int w = threadIdx.x; w < nl * L::R1; w += blockDim.x) {
        const int r = w & (yt - 1), k1 = (w >> lyt) & (L::R1 - 1), p = w >> (lyt + log2_c(L::R1));
        const int line = p * yt + r;
        V2<T> v[L::R2];
        step2<T, M, false>(buf, line, k1, v);
        V2<T>* o = dst0 + (int64_t)p * M * kstride + r;
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) o[(int64_t)(k1 + L::R1 * k2) * kstride] = v[brev_c(k2, log2_c(L::R2))];
    }
}

template <typename T, int M>
static __global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) fftx_fwd_t_kernel(T* rho, V2<T>* __restrict__ X1,
                                                                  FFTDims d, const V2<T>* __restrict__ tw,
                                                                  const Ord<T>* __restrict__ chmax, int yt) {
    fftx_fwd_t_kernel_body<T, M>(rho, X1, d, tw, chmax, yt, true, (int)blockIdx.x, (int)blockIdx.y);
}

// Pieces of the two-step transform used by the slab kernel (M = R1 R2, see
// the file comment). With k = k1 + R1 k2 and n = R2 n1 + n2 the inverse
// splits the same way,
//   y[R2 n1 + n2] = sum_k1 W_R1^(-n1 k1) W_M^(-n2 k1) [ sum_k2 Y[k1 + R1 k2] W_R2^(-n2 k2) ],
// so the thread that ends the forward transform for one k1 (holding every
// k2) can begin the inverse in registers. Spectra stay in the "k1-major"
// layout of the forward step 2: position k1 (R2 + 1) + m of a line holds the
// bin k1 + R1 brev(m).

// forward step 2 in place: line data at k1 (R2+1) + n2 -> bins k1 + R1 brev(m) at k1 (R2+1) + m
template <typename T, int M>
__device__ __forceinline__ void step2_fwd_inplace(V2<T>* line, int k1) {
    using L = Lay<M>;
    V2<T>* b = line + k1 * (L::R2 + 1);
    V2<T> v[L::R2];
#pragma unroll
    for (int n2 = 0; n2 < L::R2; ++n2) v[n2] = b[n2];
    dft_reg<T, L::R2, false>(v);
#pragma unroll
    for (int m = 0; m < L::R2; ++m) b[m] = v[m];
}

// first half of the inverse for one k1: spectrum bins u[k2] = Y[k1 + R1 k2]
// -> Z[n2] W_M^(-n2 k1) stored at k1 (R2+1) + n2
template <typename T, int M>
__device__ __forceinline__ void inv_half1_store(V2<T>* line, int k1, V2<T> (&u)[Lay<M>::R2], const V2<T>* twM) {
    using L = Lay<M>;
    dft_reg<T, L::R2, true>(u);
    V2<T>* b = line + k1 * (L::R2 + 1);
#pragma unroll
    for (int n2 = 0; n2 < L::R2; ++n2) {
        V2<T> z = u[brev_c(n2, log2_c(L::R2))];
        if (n2 != 0 && k1 != 0) {
            V2<T> t = twM[(n2 * k1) & (M - 1)];
            t.y = -t.y;
            z = cmul<T>(z, t);
        }
        b[n2] = z;
    }
}

// second half of the inverse for one n2: R1-point inverse DFT over k1 of
// line[k1 (R2+1) + n2]; out[n1] = y[R2 n1 + n2] for n1 < R1/2 (the kept half)
template <typename T, int M>
__device__ __forceinline__ void inv_half2(const V2<T>* line, int n2, V2<T> (&out)[Lay<M>::R1]) {
    using L = Lay<M>;
    V2<T> v[L::R1];
#pragma unroll
    for (int k1 = 0; k1 < L::R1; ++k1) v[k1] = line[k1 * (L::R2 + 1) + n2];
    dft_reg<T, L::R1, true, false, true>(v);     // callers keep n1 < R1/2
#pragma unroll
    for (int n1 = 0; n1 < L::R1 / 2; ++n1) out[n1] = v[brev_c(n1, log2_c(L::R1))];
}

template <int M>
__device__ __forceinline__ int kmajor_pos(int k) {
    using L = Lay<M>;
    return (k % L::R1) * (L::R2 + 1) + brev_c(k / L::R1, log2_c(L::R2));
}

template <typename T>
__host__ __device__ constexpr int slab_kc() { return sizeof(T) == 4 ? 32 : 16; }   // z columns per chunk

// y and z transforms of the slab of one (kx, pair), in place on X1: forward
// y (inputs y < ny); for slab_kc columns ky at a time: forward z (inputs
// z < nz), times Ghat, inverse z (outputs z < nz); inverse y (outputs
// y < ny). The slab lives in A as nz lines of 2ny; a chunk of columns is
// copied to B as z lines and back.
template <typename T, int MY, int MZ>
__device__ __forceinline__ void fftyz_kernel_body(V2<T>* __restrict__ X1, const T* __restrict__ Ghat, FFTDims d,
                                                    const V2<T>* __restrict__ twy, const V2<T>* __restrict__ twz,
                                                    const int bx_, const int by_) {
    using LY = Lay<MY>;
    using LZ = Lay<MZ>;
    // columns per chunk, at most the MY columns there are (an 8-node y grid has 16)
    constexpr int KC = slab_kc<T>() < MY ? slab_kc<T>() : MY;
    extern __shared__ unsigned char smraw[];
    V2<T>* tY = reinterpret_cast<V2<T>*>(smraw);
    V2<T>* tZ = tY + MY;
    V2<T>* A = tZ + MZ;                        // [nz][LY::LS]
    V2<T>* B = A + d.nz * LY::LS;              // [KC][LZ::LS]
    const int kx = bx_, p = by_;
    constexpr int nz = MZ / 2, ny = MY / 2;         // zero-padded lengths M = 2n
    for (int j = threadIdx.x; j < MY; j += blockDim.x) tY[j] = twy[j];
    for (int j = threadIdx.x; j < MZ; j += blockDim.x) tZ[j] = twz[j];
    V2<T>* slab = X1 + ((int64_t)p * d.Mx + kx) * nz * ny;
    __syncthreads();
    // forward y: step 1 straight from the slab (inputs y >= ny are zero; item
    // (z, n2) reads y = R2 n1 + n2, consecutive threads take consecutive n2 so
    // the loads are coalesced) into A, then step 2 in place -> k1-major spectra
    for (int w = threadIdx.x; w < nz * LY::R2; w += blockDim.x) {
        const int n2 = w % LY::R2, z = w / LY::R2;
        V2<T> v[LY::R1];
#pragma unroll
        for (int n1 = 0; n1 < LY::R1 / 2; ++n1) v[n1] = slab[z * ny + LY::R2 * n1 + n2];
        dft_reg<T, LY::R1, false, true>(v);
        step1_store<T, MY, false>(v, A + z * LY::LS + n2, n2, tY);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < nz * LY::R1; w += blockDim.x)
        step2_fwd_inplace<T, MY>(A + (w % nz) * LY::LS, w / nz);
    __syncthreads();
    const int kxr = kx <= d.nx ? kx : d.Mx - kx;
    const T* Gp = Ghat + (int64_t)kxr * (d.nz + 1) * (d.ny + 1);     // plane [kz'][ky']
    for (int c0 = 0; c0 < MY; c0 += KC) {
        // forward z step 1 for KC columns, read straight from the y spectra in A
        // (column c0 + j of row z is A[z][kmajor(c0 + j)]; rows z >= nz are zero)
        for (int w = threadIdx.x; w < KC * LZ::R2; w += blockDim.x) {
            const int j = w % KC, n2 = w / KC;
            const V2<T>* a = A + kmajor_pos<MY>(c0 + j);
            V2<T> v[LZ::R1];
#pragma unroll
            for (int n1 = 0; n1 < LZ::R1 / 2; ++n1) v[n1] = a[(LZ::R2 * n1 + n2) * LY::LS];
            dft_reg<T, LZ::R1, false, true>(v);
            step1_store<T, MZ, false>(v, B + j * LZ::LS + n2, n2, tZ);
        }
        __syncthreads();
        // per (column, k1): forward R2-point DFT, times Ghat, first half of the inverse
        for (int w = threadIdx.x; w < KC * LZ::R1; w += blockDim.x) {
            const int j = w % KC, k1 = w / KC;
            const int ky = c0 + j;
            const int kyr = ky <= ny ? ky : MY - ky;
            V2<T>* line = B + j * LZ::LS;
            V2<T> v[LZ::R2];
#pragma unroll
            for (int n2 = 0; n2 < LZ::R2; ++n2) v[n2] = line[k1 * (LZ::R2 + 1) + n2];
            dft_reg<T, LZ::R2, false>(v);
            V2<T> u[LZ::R2];
#pragma unroll
            for (int k2 = 0; k2 < LZ::R2; ++k2) {
                const int kz = k1 + LZ::R1 * k2;
                const int kzr = kz <= nz ? kz : MZ - kz;
                const T gh = Gp[kzr * (ny + 1) + kyr];
                u[k2] = v[brev_c(k2, log2_c(LZ::R2))];
                u[k2].x *= gh;
                u[k2].y *= gh;
            }
            inv_half1_store<T, MZ>(line, k1, u, tZ);
        }
        __syncthreads();
        // per (column, n2): second half of the inverse, outputs z < nz back into A
        for (int w = threadIdx.x; w < KC * LZ::R2; w += blockDim.x) {
            const int j = w % KC, n2 = w / KC;
            V2<T> o[LZ::R1];
            inv_half2<T, MZ>(B + j * LZ::LS, n2, o);
            const int pa = kmajor_pos<MY>(c0 + j);
#pragma unroll
            for (int n1 = 0; n1 < LZ::R1 / 2; ++n1) A[(LZ::R2 * n1 + n2) * LY::LS + pa] = o[n1];
        }
        __syncthreads();
    }
    // inverse y from the k1-major spectra: first half in place per (z, k1) ...
    for (int w = threadIdx.x; w < nz * LY::R1; w += blockDim.x) {
        const int z = w % nz, k1 = w / nz;
        V2<T>* line = A + z * LY::LS;
        V2<T> u[LY::R2];
#pragma unroll
        for (int k2 = 0; k2 < LY::R2; ++k2) u[k2] = line[k1 * (LY::R2 + 1) + brev_c(k2, log2_c(LY::R2))];
        inv_half1_store<T, MY>(line, k1, u, tY);
    }
    __syncthreads();
    // ... then per (z, n2), outputs y < ny to the slab (n2 fastest: consecutive y)
    for (int w = threadIdx.x; w < nz * LY::R2; w += blockDim.x) {
        const int n2 = w % LY::R2, z = w / LY::R2;
        V2<T> o[LY::R1];
        inv_half2<T, MY>(A + z * LY::LS, n2, o);
#pragma unroll
        for (int n1 = 0; n1 < LY::R1 / 2; ++n1) slab[z * ny + LY::R2 * n1 + n2] = o[n1];
    }
}

template <typename T, int MY, int MZ>
static __global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) fftyz_kernel(V2<T>* __restrict__ X1, const T* __restrict__ Ghat, FFTDims d,
                                                             const V2<T>* __restrict__ twy, const V2<T>* __restrict__ twz) {
    fftyz_kernel_body<T, MY, MZ>(X1, Ghat, d, twy, twz, (int)blockIdx.x, (int)blockIdx.y);
}

// x pass, inverse: X1 [p][kx][z][y] for rows (z, y0 .. y0 + yt - 1) -> phi rows
// (x < nx), channel scaling and 1/(Mx My Mz) undone, staged so each row is
// stored contiguously (stage rows padded by one word against bank conflicts)
template <typename T, int M>
__device__ __forceinline__ void fftx_inv_t_kernel_body(const V2<T>* __restrict__ X1, T* __restrict__ phi, FFTDims d,
                                                         const V2<T>* __restrict__ tw, const Ord<T>* __restrict__ chmax,
                                                         int yt, const int bx_, const int by_) {
    using L = Lay<M>;
    extern __shared__ unsigned char smraw[];
    V2<T>* twM = reinterpret_cast<V2<T>*>(smraw);
    T* sc = reinterpret_cast<T*>(twM + M);
    V2<T>* buf = reinterpret_cast<V2<T>*>(sc + 16);
    const int nl = yt * d.npair;
    T* stage = reinterpret_cast<T*>(buf + nl * L::LS);   // [yt][nx * CP + 1]
    const int SR = d.nx * d.CP + 1;
    for (int j = threadIdx.x; j < M; j += blockDim.x) twM[j] = tw[j];
    if (threadIdx.x < d.CP) sc[threadIdx.x] = (T)d.norm * chan_scale<T>(chmax, threadIdx.x, true);
    const int y0 = bx_ * yt, z = by_;
    const int64_t kstride = (int64_t)d.nz * d.ny;
    const V2<T>* src0 = X1 + (int64_t)z * d.ny + y0;
    const int lyt = __ffs(yt) - 1;                    // yt, nx, CP are powers of two
    // batches of 16 independent loads per thread (one latency per batch)
    constexpr int NBL = 16;
    for (int t0 = threadIdx.x; t0 < nl * M; t0 += NBL * blockDim.x) {
        V2<T> v[NBL];
#pragma unroll
        for (int b = 0; b < NBL; ++b) {
            const int t = t0 + b * blockDim.x;
            const int r = t & (yt - 1), rest = t >> lyt;
            const int kx = rest & (M - 1), p = rest >> log2_c(M);
            if (t < nl * M) v[b] = src0[((int64_t)p * M + kx) * kstride + r];
        }
#pragma unroll
        for (int b = 0; b < NBL; ++b) {
            const int t = t0 + b * blockDim.x;
            const int r = t & (yt - 1), rest = t >> lyt;
            const int kx = rest & (M - 1), p = rest >> log2_c(M);
            if (t < nl * M) buf[(p * yt + r) * L::LS + L::pos(kx)] = v[b];
        }
    }
    __syncthreads();
    step1<T, M, true>(buf, divmod_of(nl), twM, false);
    __syncthreads();
    for (int w = threadIdx.x; w < nl * L::R1; w += blockDim.x) {
        const int r = w & (yt - 1), k1 = (w >> lyt) & (L::R1 - 1), p = w >> (lyt + log2_c(L::R1));
        const int line = p * yt + r;
        V2<T> v[L::R2];
        step2<T, M, true, true>(buf, line, k1, v);   // keeps x < nx
        const T sa = sc[2 * p], sb = sc[2 * p + 1];
#pragma unroll
        for (int k2 = 0; k2 < L::R2; ++k2) {
            const int x = k1 + L::R1 * k2;
            if (x < d.nx) {
                const V2<T> q = v[brev_c(k2, log2_c(L::R2))];
                stage[r * SR + x * d.CP + 2 * p] = q.x * sa;
                stage[r * SR + x * d.CP + 2 * p + 1] = q.y * sb;
            }
        }
    }
    __syncthreads();
    T* dst = phi + ((int64_t)z * d.ny + y0) * d.nx * d.CP;
    const int lrow = log2_c(M) - 1 + __ffs(d.CP) - 1;      // log2(nx CP)
    for (int t = threadIdx.x; t < (yt << lrow); t += blockDim.x) {
        const int r = t >> lrow, rem = t & ((1 << lrow) - 1);
        const int c = rem & (d.CP - 1);
        dst[t] = c < d.C ? stage[r * SR + rem] : (T)0;
    }
}

template <typename T, int M>
static __global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) fftx_inv_t_kernel(const V2<T>* __restrict__ X1, T* __restrict__ phi,
                                                                  FFTDims d, const V2<T>* __restrict__ tw,
                                                                  const Ord<T>* __restrict__ chmax, int yt) {
    fftx_inv_t_kernel_body<T, M>(X1, phi, d, tw, chmax, yt, (int)blockIdx.x, (int)blockIdx.y);
}

}  // namespace adpic
