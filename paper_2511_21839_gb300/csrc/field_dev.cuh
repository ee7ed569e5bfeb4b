// Device code of field.cu (helpers, kernel bodies taking an explicit block index,
// and their kernel wrappers), shared by field.cu and the batched persistent kernel.
#pragma once
// Grid-side kernels: per-kick geometry, the integrated Green's function and
// its real even spectrum, the zero-padded (Hockney) FFT convolution of all
// dual channels, and the central finite-difference field.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <type_traits>

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
__device__ __forceinline__ void geom_kernel_body(Ord<T>* mm, int nx, int ny, int nz, double gamma0, GeomDev* g, Ord<T>* chmax, int CP,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int d = threadIdx.x;
    if (d < 3) {
        const int n = d == 0 ? nx : (d == 1 ? ny : nz);
        double lo = (double)ord_dec(__ldcg(&mm[d])), hi = (double)ord_dec(__ldcg(&mm[3 + d]));
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
        const double hr = d == 2 ? h * gamma0 : h;
        g->fdd[d] = 0.5 / hr;
        g->fdf[d] = (float)(0.5 / hr);
    }
    __syncthreads();
    if (d < 3) {
        // exact integrals (FP64) for every cell of the FP64 path; in FP32 for
        // the cells whose centre is within 10 h_max, beyond which the
        // fourth-order expansion is below FP32 rounding
        const int n = d == 0 ? nx : (d == 1 ? ny : nz);
        double hmax = fmax(g->hr[0], fmax(g->hr[1], g->hr[2]));
        int R = (int)ceil(10.0 * hmax / g->hr[d]);
        g->R[d] = (sizeof(T) == 8 || R > n) ? n : R;
    }
    __syncthreads();
    if (d < 3) {
        mm[d] = ~(Ord<T>)0;
        mm[3 + d] = (Ord<T>)0;
    }
    for (int c = d; c < CP; c += blockDim.x) chmax[c] = (Ord<T>)0;
}

// The geometry step run by the last block of the kernel that produced the
// extrema (every block calls this after its extrema atomics; all threads of
// the block take part): a counter of finished blocks picks the last one,
// which derives the geometry and resets the counter. Fences order each
// block's atomics before its count and the last block's reads after it.
// (a call, not inlined: the host kernel's register allocation stays its own)
template <typename T>
__device__ __noinline__ void geom_step(const GeomFuse gf, Ord<T>* mm) {
    geom_kernel_body<T>(mm, gf.nx, gf.ny, gf.nz, gf.gamma0, gf.g, reinterpret_cast<Ord<T>*>(gf.chmax), gf.CP, 0, 0, 0, 1);
}
template <typename T>
__device__ __forceinline__ void geom_last_block(const GeomFuse& gf, Ord<T>* mm) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(gf.count, 1u) == gridDim.x * gridDim.y * gridDim.z - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    geom_step<T>(gf, mm);
    if (threadIdx.x == 0) *gf.count = 0u;
}

// per-channel max |rho| (ordered bits of a non-negative value are its bits).
// Each thread keeps four independent running maxima over a grid-stride loop
// (element t belongs to channel t % CP; the stride is a multiple of CP).
template <typename T>
__device__ __forceinline__ void chmax_kernel_body(const T* __restrict__ rho, int64_t nodes, int CP, Ord<T>* chmax,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int64_t t0 = bx_ * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)nbx_ * blockDim.x;   // multiple of CP
    const int64_t total = nodes * CP;
    T m0 = (T)0, m1 = (T)0, m2 = (T)0, m3 = (T)0;
    int64_t t = t0;
    for (; t + 3 * stride < total; t += 4 * stride) {
        m0 = fmax(m0, fabs(rho[t]));
        m1 = fmax(m1, fabs(rho[t + stride]));
        m2 = fmax(m2, fabs(rho[t + 2 * stride]));
        m3 = fmax(m3, fabs(rho[t + 3 * stride]));
    }
    for (; t < total; t += stride) m0 = fmax(m0, fabs(rho[t]));
    T m = fmax(fmax(m0, m1), fmax(m2, m3));
    for (int o = CP; o < 32; o <<= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // across the block's warps, then one atomic per channel
    __shared__ T wm[32][16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane < CP) wm[w][lane] = m;
    __syncthreads();
    if ((int)threadIdx.x < CP) {
        T b = wm[0][threadIdx.x];
        for (int j = 1; j < nw; ++j) b = fmax(b, wm[j][threadIdx.x]);
        if constexpr (sizeof(T) == 4)
            atomicMax(&chmax[threadIdx.x], __float_as_uint(b));
        else
            atomicMax(&chmax[threadIdx.x], (unsigned long long)__double_as_longlong(b));
    }
}

template <typename T>
static __global__ void chmax_kernel(const T* __restrict__ rho, int64_t nodes, int CP, Ord<T>* chmax) {
    chmax_kernel_body<T>(rho, nodes, CP, chmax, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// The same maxima with 16-byte loads: vector j of rho holds the EPV channels
// starting at (j % VPN) EPV of node j / VPN. The grid stride and the block
// size are multiples of VPN, so a thread's channel group is that of its lane
// and stays fixed; lanes whose indices differ by a multiple of VPN share it.
template <typename T, int CP>
static __global__ void __launch_bounds__(256) chmax_vec_kernel(const T* __restrict__ rho, int64_t nodes, Ord<T>* chmax) {
    constexpr int EPV = 16 / (int)sizeof(T), VPN = CP / EPV;
    static_assert(CP % EPV == 0 && (VPN & (VPN - 1)) == 0 && VPN <= 32, "channel groups");
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const V* r = reinterpret_cast<const V*>(rho);
    const int64_t nv = nodes * VPN;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    T m[EPV];
#pragma unroll
    for (int e = 0; e < EPV; ++e) m[e] = (T)0;
    auto upd = [&](const V& a) {
        T v[EPV];
        memcpy(v, &a, sizeof(V));
#pragma unroll
        for (int e = 0; e < EPV; ++e) m[e] = fmax(m[e], fabs(v[e]));
    };
    for (; t + 3 * stride < nv; t += 4 * stride) {
        V a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = r[t + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) upd(a[u]);
    }
    for (; t < nv; t += stride) upd(r[t]);
#pragma unroll
    for (int o = VPN; o < 32; o <<= 1)
#pragma unroll
        for (int e = 0; e < EPV; ++e) m[e] = fmax(m[e], __shfl_xor_sync(0xffffffffu, m[e], o));
    __shared__ T wm[8][CP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane < VPN)
#pragma unroll
        for (int e = 0; e < EPV; ++e) wm[w][lane * EPV + e] = m[e];
    __syncthreads();
    if ((int)threadIdx.x < CP) {
        T b = wm[0][threadIdx.x];
        for (int j = 1; j < nw; ++j) b = fmax(b, wm[j][threadIdx.x]);
        if constexpr (sizeof(T) == 4)
            atomicMax(&chmax[threadIdx.x], __float_as_uint(b));
        else
            atomicMax(&chmax[threadIdx.x], (unsigned long long)__double_as_longlong(b));
    }
}

// The central differences with one thread per (node, 32-byte piece of its
// channels): six 32-byte loads of phi and three 32-byte stores of E, the
// same arithmetic per value as field_kernel_body.
template <typename T, int CP>
static __global__ void __launch_bounds__(256) field_vec_kernel(const T* __restrict__ phi, const GeomDev* __restrict__ g,
                                                              int nx, int ny, int nz, T* __restrict__ E) {
    constexpr int EPC = 32 / (int)sizeof(T), CPN = CP / EPC, LCPN = CPN == 1 ? 0 : (CPN == 2 ? 1 : 2);
    static_assert(CP % EPC == 0 && CPN <= 4, "32-byte pieces");
    const unsigned t = (unsigned)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ((unsigned)nx * ny * nz << LCPN)) return;
    const int lx = __ffs(nx) - 1, ly = __ffs(ny) - 1;
    const unsigned piece = t & (CPN - 1), node = t >> LCPN;
    const int i = node & (nx - 1), j = (node >> lx) & (ny - 1), k = node >> (lx + ly);
    if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || k < 1 || k > nz - 2) return;
    const T a[3] = {sizeof(T) == 4 ? (T)g->fdf[0] : (T)g->fdd[0], sizeof(T) == 4 ? (T)g->fdf[1] : (T)g->fdd[1],
                    sizeof(T) == 4 ? (T)g->fdf[2] : (T)g->fdd[2]};
    const int64_t s[3] = {CP, (int64_t)nx * CP, (int64_t)nx * ny * CP};
    const T* p = phi + (int64_t)node * CP + piece * EPC;
    T* e = E + (int64_t)node * 3 * CP + piece * EPC;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        T hi[EPC], lo[EPC], r[EPC];
        ldg_v<T, EPC>(p + s[d], hi);
        ldg_v<T, EPC>(p - s[d], lo);
#pragma unroll
        for (int c = 0; c < EPC; ++c) r[c] = -(hi[c] - lo[c]) * a[d];
        stg_v<T, EPC>(e + d * CP, r);
    }
}

// ------------------------------------------------------------------ Green's function

// An antiderivative of 1/r: d^3 F / dx dy dz = 1/sqrt(x^2 + y^2 + z^2).
__device__ __forceinline__ double igf_F(double x, double y, double z) {
    const double r = sqrt(x * x + y * y + z * z);
    return y * z * log(x + r) + x * z * log(y + r) + x * y * log(z + r) - 0.5 * x * x * atan(y * z / (x * r)) -
           0.5 * y * y * atan(x * z / (y * r)) - 0.5 * z * z * atan(x * y / (z * r));
}

// F at the cell corners ((i - 1/2) hx, (j - 1/2) hy, (k - 1/2) hzr) of the near
// box i in [0, Rx+1], j in [0, Ry+1], k in [0, Rz+1] (FP64), stored in the
// (nx+2)(ny+2)(nz+2) corner lattice. The box is mapped onto the first threads
// so its FP64 work spreads over consecutive small blocks; callers launch at
// least (nx+2)(ny+2)(nz+2) threads (R <= n), the rest return at once.
__device__ __forceinline__ void green_corner_kernel_body(const GeomDev* __restrict__ g, int nx, int ny, int nz, double* __restrict__ F,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const int cx = nx + 2, cy = ny + 2;
    const int t = bx_ * blockDim.x + threadIdx.x;
    const int ex = g->R[0] + 2, ey = g->R[1] + 2, ez = g->R[2] + 2;
    if (t >= ex * ey * ez) return;
    const int i = t % ex, j = (t / ex) % ey, k = t / (ex * ey);
    F[((int64_t)k * cy + j) * cx + i] = igf_F((i - 0.5) * g->hr[0], (j - 0.5) * g->hr[1], (k - 0.5) * g->hr[2]);
}

static __global__ void green_corner_kernel(const GeomDev* __restrict__ g, int nx, int ny, int nz, double* __restrict__ F) {
    green_corner_kernel_body(g, nx, ny, nz, F, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

// The same integrals from a fixed grid of blocks that strides over the near
// box (its size is known on the device only), instead of one thread per
// corner of the whole lattice of which all but the box return at once:
// block b of nb.
__device__ __forceinline__ void green_corner_strided_body(const GeomDev* __restrict__ g, int nx, int ny,
                                                          double* __restrict__ F, int b, int nb) {
    const int ex = g->R[0] + 2, ey = g->R[1] + 2, ez = g->R[2] + 2;
    const int cx = nx + 2, cy = ny + 2;
    for (int t = b * blockDim.x + threadIdx.x; t < ex * ey * ez; t += nb * blockDim.x) {
        const int i = t % ex, j = (t / ex) % ey, k = t / (ex * ey);
        F[((int64_t)k * cy + j) * cx + i] = igf_F((i - 0.5) * g->hr[0], (j - 0.5) * g->hr[1], (k - 0.5) * g->hr[2]);
    }
}
static __global__ void __launch_bounds__(64) green_corner_strided_kernel(const GeomDev* __restrict__ g, int nx, int ny,
                                                                       int nz, double* __restrict__ F) {
    (void)nz;
    green_corner_strided_body(g, nx, ny, F, (int)blockIdx.x, (int)gridDim.x);
}

// dF/dz of the antiderivative above, in closed form (differentiating F's six
// terms and collecting): y log(x + r) + x log(y + r) - z atan(x y / (z r))
// + z^2 (x + y)(x y + z^2) / ((x^2 + z^2)(y^2 + z^2)).
__device__ __forceinline__ double igf_Fz(double x, double y, double z) {
    const double r = sqrt(x * x + y * y + z * z);
    const double z2 = z * z;
    return y * log(x + r) + x * log(y + r) - z * atan(x * y / (z * r)) +
           z2 * (x + y) * (x * y + z2) / ((x * x + z2) * (y * y + z2));
}

// The kinetic energy as a dual input moves the rest-frame spacing hzr =
// gamma0 hz and with it every corner z = (k - 1/2) hzr: FE holds
// dF/dhzr = (k - 1/2) dF/dz at the corners of the same near box as F.
static __global__ void __launch_bounds__(64) green_corner_dz_kernel(const GeomDev* __restrict__ g, int nx, int ny,
                                                                  int nz, double* __restrict__ FE) {
    const int ex = g->R[0] + 2, ey = g->R[1] + 2, ez = g->R[2] + 2;
    const int cx = nx + 2, cy = ny + 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ex * ey * ez; t += gridDim.x * blockDim.x) {
        const int i = t % ex, j = (t / ex) % ey, k = t / (ex * ey);
        FE[((int64_t)k * cy + j) * cx + i] =
            (k - 0.5) * igf_Fz((i - 0.5) * g->hr[0], (j - 0.5) * g->hr[1], (k - 0.5) * g->hr[2]);
    }
}

// Cell average of 1/(4 pi eps0 r) over the cell centred at offset (i, j, k):
// the 8-corner difference of F in FP64 inside the near box (every cell on
// the FP64 path), else the Taylor expansion of the box average of a smooth
// function, f + (1/24) sum_d h_d^2 f_dd + (1/1920) sum_d h_d^4 f_dddd
// + (1/576) sum_{d<e} h_d^2 h_e^2 f_ddee, with the derivatives of 1/r
// f_dd = (3 d^2 - r^2)/r^5, f_dddd = 3 (35 d^4 - 30 d^2 r^2 + 3 r^4)/r^9,
// f_ddee = 3 (35 d^2 e^2 - 5 r^2 (d^2 + e^2) + r^4)/r^9; its O(h^6) remainder
// is below FP32 rounding beyond 10 h_max.
// G is stored [k][j][i] (order 0, i fastest) or [i][k][j] (order 1, j fastest).
template <typename T>
__device__ __forceinline__ T green_cell_value(const GeomDev* __restrict__ g, int nx, int ny,
                                              const double* __restrict__ F, int i, int j, int k) {
    const double hx = g->hr[0], hy = g->hr[1], hz = g->hr[2];
    const double k4 = 1.0 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12);
    if (i <= g->R[0] && j <= g->R[1] && k <= g->R[2]) {
        const int cx = nx + 2, cy = ny + 2;
        auto at = [&](int a, int b, int c) { return F[((int64_t)c * cy + b) * cx + a]; };
        double s = at(i + 1, j + 1, k + 1) - at(i, j + 1, k + 1) - at(i + 1, j, k + 1) - at(i + 1, j + 1, k) +
                   at(i, j, k + 1) + at(i, j + 1, k) + at(i + 1, j, k) - at(i, j, k);
        return (T)(k4 * s / (hx * hy * hz));
    }
    // in units of r: direction cosines c_d = d / r and ratios t_d = h_d / r
    const T x = (T)i * (T)hx, y = (T)j * (T)hy, z = (T)k * (T)hz;
    const T ir = rsqrt(x * x + y * y + z * z);
    const T c2[3] = {x * x * ir * ir, y * y * ir * ir, z * z * ir * ir};
    const T t2[3] = {(T)hx * (T)hx * ir * ir, (T)hy * (T)hy * ir * ir, (T)hz * (T)hz * ir * ir};
    T s2 = (T)0, s4 = (T)0, s22 = (T)0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s2 += t2[d] * ((T)3 * c2[d] - (T)1);
        s4 += t2[d] * t2[d] * (T)3 * ((T)35 * c2[d] * c2[d] - (T)30 * c2[d] + (T)3);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int e = (d + 1) % 3;
        s22 += t2[d] * t2[e] * (T)3 * ((T)35 * c2[d] * c2[e] - (T)5 * (c2[d] + c2[e]) + (T)1);
    }
    return (T)k4 * ir * ((T)1 + s2 / (T)24 + s4 / (T)1920 + s22 / (T)576);
}

// a first-order dual of one variable (value, derivative), for the far-field
// expansion of the cell average differentiated in hzr (Eqs. 1-4)
template <typename T>
struct D1 {
    T v, d;
};
template <typename T> __device__ __forceinline__ D1<T> operator+(D1<T> a, D1<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __device__ __forceinline__ D1<T> operator-(D1<T> a, D1<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __device__ __forceinline__ D1<T> operator*(D1<T> a, D1<T> b) {
    return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <typename T> __device__ __forceinline__ D1<T> operator*(T c, D1<T> a) { return {c * a.v, c * a.d}; }
template <typename T> __device__ __forceinline__ D1<T> d1_rsqrt(D1<T> a) {
    const T r = rsqrt(a.v);
    return {r, (T)-0.5 * r * r * r * a.d};
}

// dG/dhzr of the cell average at offset (i, j, k), the offset k hzr moving
// with hzr: inside the near box from the corner values, G = c S / (hx hy hzr)
// with S the 8-corner difference of F, so dG/dhzr = c (S' - S / hzr) /
// (hx hy hzr) with S' the same difference of FE; outside it the expansion of
// green_cell_value carried through in dual arithmetic.
template <typename T>
__device__ __forceinline__ T green_cell_dvalue(const GeomDev* __restrict__ g, int nx, int ny,
                                               const double* __restrict__ F, const double* __restrict__ FE, int i,
                                               int j, int k) {
    const double hx = g->hr[0], hy = g->hr[1], hz = g->hr[2];
    const double k4 = 1.0 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12);
    if (i <= g->R[0] && j <= g->R[1] && k <= g->R[2]) {
        const int cx = nx + 2, cy = ny + 2;
        auto diff = [&](const double* A) {
            auto at = [&](int a, int b, int c) { return A[((int64_t)c * cy + b) * cx + a]; };
            return at(i + 1, j + 1, k + 1) - at(i, j + 1, k + 1) - at(i + 1, j, k + 1) - at(i + 1, j + 1, k) +
                   at(i, j, k + 1) + at(i, j + 1, k) + at(i + 1, j, k) - at(i, j, k);
        };
        const double S = diff(F), Sd = diff(FE);
        return (T)(k4 * (Sd - S / hz) / (hx * hy * hz));
    }
    const D1<T> H = {(T)hz, (T)1};
    const T x = (T)i * (T)hx, y = (T)j * (T)hy;
    const D1<T> z = (T)k * H;
    const D1<T> r2 = D1<T>{x * x + y * y, (T)0} + z * z;
    const D1<T> ir = d1_rsqrt(r2);
    const D1<T> ir2 = ir * ir;
    const D1<T> c2[3] = {(x * x) * ir2, (y * y) * ir2, z * z * ir2};
    const D1<T> t2[3] = {((T)hx * (T)hx) * ir2, ((T)hy * (T)hy) * ir2, H * H * ir2};
    const D1<T> one = {(T)1, (T)0};
    D1<T> s2 = {(T)0, (T)0}, s4 = {(T)0, (T)0}, s22 = {(T)0, (T)0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s2 = s2 + t2[d] * ((T)3 * c2[d] - one);
        s4 = s4 + (T)3 * (t2[d] * t2[d] * ((T)35 * (c2[d] * c2[d]) - (T)30 * c2[d] + (T)3 * one));
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int e = (d + 1) % 3;
        s22 = s22 + (T)3 * (t2[d] * t2[e] * ((T)35 * (c2[d] * c2[e]) - (T)5 * (c2[d] + c2[e]) + one));
    }
    const D1<T> bracket = one + ((T)1 / (T)24) * s2 + ((T)1 / (T)1920) * s4 + ((T)1 / (T)576) * s22;
    return ((T)k4 * (ir * bracket)).d;
}

// (i, j, k) of element l of DCT line ba in G's layout: order 0 G[z][y][x]
// (lines along x), order 1 G[x][z][y] (lines along y)
__device__ __forceinline__ void green_cell_index(int ba, int l, int nx, int ny, int nz, int order, int& i, int& j,
                                                 int& k) {
    if (order == 0) {
        i = l; j = ba % (ny + 1); k = ba / (ny + 1);
    } else {
        j = l; k = ba % (nz + 1); i = ba / (nz + 1);
    }
}

template <typename T>
__device__ __forceinline__ void green_cell_kernel_body(const GeomDev* __restrict__ g, int nx, int ny, int nz,
                                  const double* __restrict__ F, T* __restrict__ G,
    const int bx_, const int by_, const int bz_, const int nbx_, int order = 0) {
    const int t = bx_ * blockDim.x + threadIdx.x;     // < 129^3
    const int gx = nx + 1, gy = ny + 1, gz = nz + 1;
    if (t >= gx * gy * gz) return;
    const int L = order == 0 ? gx : gy;
    int i, j, k;
    green_cell_index(t / L, t % L, nx, ny, nz, order, i, j, k);
    G[t] = green_cell_value<T>(g, nx, ny, F, i, j, k);
}

template <typename T>
static __global__ void green_cell_kernel(const GeomDev* __restrict__ g, int nx, int ny, int nz,
                                  const double* __restrict__ F, T* __restrict__ G, int order) {
    green_cell_kernel_body<T>(g, nx, ny, nz, F, G, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x,
                              order);
}

// One DCT-I pass over the contiguous axis of in [BA][L] (L = n+1) into
// out [L][BA]: out[k][ba] = sum_l D[k][l] in[ba][l], D[k][l] = w_l cos(pi l k / n),
// w_0 = w_n = 1, else 2. Three passes (rotating the axes) give the real
// spectrum of the even extension of G to the 2n-periodic grid. A block of
// nw warps stages kDctLines = 32 input lines and the matrix D in shared
// memory; lane l of warp w accumulates out[k][line l] for k = w, w + nw, ...
// in registers (the D reads are warp-wide broadcasts, the line stride L is
// odd so the line reads are conflict-free, and the stores of one k are 32
// consecutive words).
constexpr int kDctLines = 32;
constexpr int kDctAcc = 8;

// ACC accumulators per lane: one sweep over l covers every output when
// ACC * (warps per block) >= L.
// CELL: the lines are not read from `in` but computed here as the cell
// averages of the Green's function (green_cell_value; lines of G's layout for
// `order`), so the cell pass and the first DCT pass are one launch.
// CELL == 2: the lines are the energy derivative dG/dE = dG/dhzr * hz / (m c^2)
// (escale = 1 / (m c^2) in 1/eV) from F and FE (green_cell_dvalue).
template <typename T, int ACC = kDctAcc, int CELL = 0>
__device__ __forceinline__ void dct_kernel_body(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ D, int L, int64_t BA,
    const int bx_, const int by_, const int bz_, const int nbx_, const GeomDev* __restrict__ g = nullptr,
    int nx = 0, int ny = 0, int nz = 0, const double* __restrict__ F = nullptr, int order = 0,
    const double* __restrict__ FE = nullptr, double escale = 0.0) {
    extern __shared__ unsigned char smraw[];
    T* Ds = reinterpret_cast<T*>(smraw);            // [L][L]
    T* xs = Ds + L * L;                             // [kDctLines][L] (room for [kDctLines][L + 1])
    const int64_t ba0 = (int64_t)bx_ * kDctLines;
    const int nl = (int)min((int64_t)kDctLines, BA - ba0);
    // global -> shared in batches of 8 independent loads per thread (one latency per batch)
    auto stage = [&](const T* __restrict__ src, T* dst, int count, int total) {
        for (int t0 = threadIdx.x; t0 < total; t0 += 8 * blockDim.x) {
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int t = t0 + q * blockDim.x;
                v[q] = t < count ? src[t] : (T)0;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int t = t0 + q * blockDim.x;
                if (t < total) dst[t] = v[q];
            }
        }
    };
    stage(D, Ds, L * L, L * L);
    if constexpr (CELL != 0) {
        const T es = CELL == 2 ? (T)(g->h[2] * escale) : (T)0;
        for (int t = threadIdx.x; t < kDctLines * L; t += blockDim.x) {
            const int line = t / L, lp = t - line * L;
            T v = (T)0;
            if (line < nl) {
                int i, j, k;
                green_cell_index((int)(ba0 + line), lp, nx, ny, nz, order, i, j, k);
                if constexpr (CELL == 2) v = green_cell_dvalue<T>(g, nx, ny, F, FE, i, j, k) * es;
                else v = green_cell_value<T>(g, nx, ny, F, i, j, k);
            }
            xs[t] = v;
        }
    } else {
        stage(in + ba0 * L, xs, nl * L, kDctLines * L);
    }
    __syncthreads();
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T* x = xs + l * L;
    for (int k0 = w; k0 < L; k0 += nw * ACC) {
        T acc[ACC];
        const T* row[ACC];
#pragma unroll
        for (int q = 0; q < ACC; ++q) {
            acc[q] = (T)0;
            row[q] = Ds + min(k0 + q * nw, L - 1) * L;
        }
        for (int c = 0; c < L; ++c) {
            const T xv = x[c];
#pragma unroll
            for (int q = 0; q < ACC; ++q) acc[q] = fma(row[q][c], xv, acc[q]);
        }
        if (l < nl) {
#pragma unroll
            for (int q = 0; q < ACC; ++q) {
                const int k = k0 + q * nw;
                if (k < L) out[(int64_t)k * BA + ba0 + l] = acc[q];
            }
        }
    }
}

template <typename T, int ACC = kDctAcc>
static __global__ void dct_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ D, int L, int64_t BA) {
    dct_kernel_body<T, ACC>(in, out, D, L, BA, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}
// Green's cell averages and the first DCT pass in one launch
template <typename T, int ACC>
static __global__ void cell_dct_kernel(T* __restrict__ out, const T* __restrict__ D, int L, int64_t BA,
                                       const GeomDev* __restrict__ g, int nx, int ny, int nz,
                                       const double* __restrict__ F, int order) {
    dct_kernel_body<T, ACC, 1>(nullptr, out, D, L, BA, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                               (int)gridDim.x, g, nx, ny, nz, F, order);
}
// dG/dE's cell values and the first DCT pass in one launch
template <typename T, int ACC>
static __global__ void cell_dct_energy_kernel(T* __restrict__ out, const T* __restrict__ D, int L, int64_t BA,
                                              const GeomDev* __restrict__ g, int nx, int ny, int nz,
                                              const double* __restrict__ F, const double* __restrict__ FE,
                                              double escale, int order) {
    dct_kernel_body<T, ACC, 2>(nullptr, out, D, L, BA, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                               (int)gridDim.x, g, nx, ny, nz, F, order, FE, escale);
}

// ------------------------------------------------------------------ field

// E = -grad(phi) by central differences on interior nodes, rest-frame
// spacings (hx, hy, gamma0 hz); E layout [node][3][CP]. One thread per
// (node, channel); nx, ny, CP are powers of two, so the node coordinates come
// from shifts and masks (32-bit: nodes * CP < 2^31).
template <typename T>
__device__ __forceinline__ void field_kernel_body(const T* __restrict__ phi, const GeomDev* __restrict__ g, int nx, int ny, int nz, int CP,
                             T* __restrict__ E,
    const int bx_, const int by_, const int bz_, const int nbx_) {
    const unsigned t = (unsigned)bx_ * blockDim.x + threadIdx.x;
    const unsigned total = (unsigned)nx * ny * nz * CP;
    if (t >= total) return;
    const int lcp = __ffs(CP) - 1, lx = __ffs(nx) - 1, ly = __ffs(ny) - 1;
    const unsigned c = t & (CP - 1), node = t >> lcp;
    const int i = node & (nx - 1), j = (node >> lx) & (ny - 1), k = node >> (lx + ly);
    if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || k < 1 || k > nz - 2) return;
    const T ax = sizeof(T) == 4 ? (T)g->fdf[0] : (T)g->fdd[0];
    const T ay = sizeof(T) == 4 ? (T)g->fdf[1] : (T)g->fdd[1];
    const T az = sizeof(T) == 4 ? (T)g->fdf[2] : (T)g->fdd[2];
    const unsigned sx = CP, sy = (unsigned)nx * CP, sz = (unsigned)nx * ny * CP;
    T* e = E + (size_t)node * 3 * CP + c;
    e[0] = -(phi[t + sx] - phi[t - sx]) * ax;
    e[CP] = -(phi[t + sy] - phi[t - sy]) * ay;
    e[2 * CP] = -(phi[t + sz] - phi[t - sz]) * az;
}

// The same field for R consecutive 256-element blocks (rb = R bx + r): the
// loads of all R are issued before any store, for callers whose block
// dispatch is costly.
template <typename T, int R>
__device__ __forceinline__ void field_multi_body(const T* __restrict__ phi, const GeomDev* __restrict__ g, int nx,
                                                 int ny, int nz, int CP, T* __restrict__ E, const int bx_) {
    const unsigned total = (unsigned)nx * ny * nz * CP;
    const int lcp = __ffs(CP) - 1, lx = __ffs(nx) - 1, ly = __ffs(ny) - 1;
    const T ax = sizeof(T) == 4 ? (T)g->fdf[0] : (T)g->fdd[0];
    const T ay = sizeof(T) == 4 ? (T)g->fdf[1] : (T)g->fdd[1];
    const T az = sizeof(T) == 4 ? (T)g->fdf[2] : (T)g->fdd[2];
    const unsigned sx = CP, sy = (unsigned)nx * CP, sz = (unsigned)nx * ny * CP;
    T dx[R], dy[R], dz[R];
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const unsigned t = ((unsigned)bx_ * R + r) * blockDim.x + threadIdx.x;
        const unsigned node = t >> lcp;
        const int i = node & (nx - 1), j = (node >> lx) & (ny - 1), k = node >> (lx + ly);
        ok[r] = t < total && i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
        dx[r] = ok[r] ? phi[t + sx] - phi[t - sx] : (T)0;
        dy[r] = ok[r] ? phi[t + sy] - phi[t - sy] : (T)0;
        dz[r] = ok[r] ? phi[t + sz] - phi[t - sz] : (T)0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const unsigned t = ((unsigned)bx_ * R + r) * blockDim.x + threadIdx.x;
        T* e = E + (size_t)(t >> lcp) * 3 * CP + (t & (CP - 1));
        e[0] = -dx[r] * ax;
        e[CP] = -dy[r] * ay;
        e[2 * CP] = -dz[r] * az;
    }
}

template <typename T>
static __global__ void field_kernel(const T* __restrict__ phi, const GeomDev* __restrict__ g, int nx, int ny, int nz, int CP,
                             T* __restrict__ E) {
    field_kernel_body<T>(phi, g, nx, ny, nz, CP, E, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x);
}

}  // namespace adpic
