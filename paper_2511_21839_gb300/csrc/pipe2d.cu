// 2D dual-number PIC in a rectangular, perfectly conducting pipe (Sec. 4:
// the paper's own field solver). A coasting beam: coordinates (x, px, y,
// py) as dual numbers; bilinear deposit of the normalised density; the
// Poisson equation with phi = 0 on the walls solved by the sine series of
// Sec. 4 (rho^lm from the nodes, phi^lm = rho^lm / gamma_lm^2, sine sums
// back); central-difference fields; the kick of H2 = K phi / 2 with the
// perveance K = q I / (2 pi eps0 p0 v0^2 gamma0^2) (I optionally an AD
// variable); the quadrupole maps of Eq. "quadtr" in x and y.
//
// The sine transforms are dense: at the grid sizes of a 2D pipe (up to
// 512 x 512 cells) a matrix of sin(pi l i / n) per dimension is small,
// exact to rounding, and every channel of the dual density shares it. The
// particle state is [6][N][CP] with the z rows zero so the moment reduction
// and the opening half map of the 3D runtime serve unchanged.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>
#include <type_traits>

#include "ad_pic.h"
#include "common.cuh"
#include "hostdual.h"

using namespace adpic;
using namespace adpic_host;

namespace {

constexpr double kC = 299792458.0;
constexpr double kQE = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ kernels

// cell index and offset along one dimension (pipe coordinate u = (x + half
// width) / h); a particle within one cell of a wall is flagged and clamped
template <typename T>
__device__ __forceinline__ int cell2d(T x, T off, T ih, int n, T& f, int& bad) {
    T u = (x + off) * ih;
    T fl = floor(u);
    int i = (int)fl;
    if (!(fl >= (T)1 && fl <= (T)(n - 2))) {
        bad |= isfinite(x) ? kErrOutOfGrid : kErrNonfinite;
        i = i < 1 ? 1 : (i > n - 2 ? n - 2 : i);
        if (!isfinite(x)) i = 1;
        fl = (T)i;
        u = fmin(fmax(u, fl), fl + (T)1);
        if (!isfinite(x)) u = fl;
    }
    f = u - fl;
    return i;
}

// bilinear deposit of the normalised density (q = 1 / (N hx hy)); node
// records [ny+1][nx+1][CP]; channel k of W = wx wy carries dW = dwx wy + wx dwy
// with dwx = +-x_k / hx (Eq. 2 on the weight product)
template <typename T, int C, int CP>
__global__ void __launch_bounds__(256) deposit2d_kernel(const T* __restrict__ st, int64_t N, int nx, int ny, T offx,
                                                        T offy, T ihx, T ihy, T q, T* __restrict__ rho,
                                                        int* __restrict__ err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    T x[CP], y[CP];
    ldv<T, CP>(st + (0 * N + i) * CP, x);
    ldv<T, CP>(st + (2 * N + i) * CP, y);
    int bad = 0;
    T fx, fy;
    const int ix = cell2d<T>(x[0], offx, ihx, nx, fx, bad);
    const int iy = cell2d<T>(y[0], offy, ihy, ny, fy, bad);
    if (bad) atomicOr(err, bad);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const T wx = a ? fx : (T)1 - fx, sx = a ? (T)1 : (T)-1;
            const T wy = b ? fy : (T)1 - fy, sy = b ? (T)1 : (T)-1;
            T* r = rho + ((int64_t)(iy + b) * (nx + 1) + (ix + a)) * CP;
            if constexpr (sizeof(T) == 4) {
                // FP32: the node record in 16-byte vector reductions (records are
                // 16-byte aligned, CP a multiple of 4), a quarter of the atomics
                T rec[CP];
                rec[0] = q * (wx * wy);
#pragma unroll
                for (int k = 1; k < CP; ++k) rec[k] = k < C ? q * (sx * x[k] * ihx * wy + sy * y[k] * ihy * wx) : (T)0;
                float4* r4 = reinterpret_cast<float4*>(r);
#pragma unroll
                for (int v = 0; v < CP / 4; ++v)
                    atomicAdd(r4 + v, make_float4(rec[4 * v], rec[4 * v + 1], rec[4 * v + 2], rec[4 * v + 3]));
            } else {
                atomicAdd(r, q * (wx * wy));
#pragma unroll
                for (int k = 1; k < C; ++k) atomicAdd(r + k, q * (sx * x[k] * ihx * wy + sy * y[k] * ihy * wx));
            }
        }
}

// Sine sums as small matrix products, one block per (line, 64 outputs): the
// line's CP-channel records are staged in shared memory with 16-byte loads;
// each thread accumulates all CP channels of one output in the order of the
// sum index (one load of S per term, the records read as broadcast vectors).
constexpr int kSineThreads = 64;
template <typename T>
using SineVec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;

// out[j][l][c] = sum_i S[l][i] in[j][i][c] along the rows (x), S = sin(pi l i / nx)
template <typename T, int CP>
__global__ void __launch_bounds__(kSineThreads) sine_rows_kernel(const T* __restrict__ in, const T* __restrict__ S,
                                                                 int nx, int ny, T* __restrict__ out) {
    using V = SineVec<T>;
    constexpr int EPV = 16 / (int)sizeof(T), VPR = CP / EPV;
    extern __shared__ __align__(16) unsigned char sine_sm[];
    V* rowv = reinterpret_cast<V*>(sine_sm);          // [nx + 1][VPR]
    const int j = blockIdx.y, l = blockIdx.x * blockDim.x + threadIdx.x;
    const int nv = (nx + 1) * VPR;
    const V* src = reinterpret_cast<const V*>(in + (int64_t)j * (nx + 1) * CP);
    for (int t0 = threadIdx.x; t0 < nv; t0 += 8 * blockDim.x) {
        V v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (t0 + b * (int)blockDim.x < nv) v[b] = src[t0 + b * blockDim.x];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (t0 + b * (int)blockDim.x < nv) rowv[t0 + b * blockDim.x] = v[b];
    }
    __syncthreads();
    if (l > nx) return;
    T acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = (T)0;
    const T* sl = S + (int64_t)l * (nx + 1);
    for (int i = 1; i < nx; ++i) {
        const T w = sl[i];
#pragma unroll
        for (int q = 0; q < VPR; ++q) {
            const V a = rowv[i * VPR + q];
            T e[EPV];
            memcpy(e, &a, sizeof(V));
#pragma unroll
            for (int k = 0; k < EPV; ++k) acc[q * EPV + k] = fma(w, e[k], acc[q * EPV + k]);
        }
    }
    V* dst = reinterpret_cast<V*>(out + ((int64_t)j * (nx + 1) + l) * CP);
#pragma unroll
    for (int q = 0; q < VPR; ++q) {
        V a;
        memcpy(&a, acc + q * EPV, sizeof(V));
        dst[q] = a;
    }
}

// out[m][l][c] = scale[m][l] sum_j S[m][j] in[j][l][c] along the columns (y)
template <typename T, int CP>
__global__ void __launch_bounds__(kSineThreads) sine_cols_kernel(const T* __restrict__ in, const T* __restrict__ S,
                                                                 const T* __restrict__ scale, int nx, int ny,
                                                                 T* __restrict__ out) {
    using V = SineVec<T>;
    constexpr int EPV = 16 / (int)sizeof(T), VPR = CP / EPV;
    extern __shared__ __align__(16) unsigned char sine_sm[];
    V* colv = reinterpret_cast<V*>(sine_sm);          // [ny + 1][VPR]
    const int l = blockIdx.y, m = blockIdx.x * blockDim.x + threadIdx.x;
    const int nv = (ny + 1) * VPR;
    const V* src = reinterpret_cast<const V*>(in);
    for (int t0 = threadIdx.x; t0 < nv; t0 += 8 * blockDim.x) {
        V v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int t = t0 + b * blockDim.x;
            if (t < nv) v[b] = src[((int64_t)(t / VPR) * (nx + 1) + l) * VPR + t % VPR];
        }
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (t0 + b * (int)blockDim.x < nv) colv[t0 + b * blockDim.x] = v[b];
    }
    __syncthreads();
    if (m > ny) return;
    T acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = (T)0;
    const T* sm = S + (int64_t)m * (ny + 1);
    for (int jj = 1; jj < ny; ++jj) {
        const T w = sm[jj];
#pragma unroll
        for (int q = 0; q < VPR; ++q) {
            const V a = colv[jj * VPR + q];
            T e[EPV];
            memcpy(e, &a, sizeof(V));
#pragma unroll
            for (int k = 0; k < EPV; ++k) acc[q * EPV + k] = fma(w, e[k], acc[q * EPV + k]);
        }
    }
    const T f = scale ? scale[(int64_t)m * (nx + 1) + l] : (T)1;
    V* dst = reinterpret_cast<V*>(out + ((int64_t)m * (nx + 1) + l) * CP);
#pragma unroll
    for (int q = 0; q < VPR; ++q) {
        T e[EPV];
#pragma unroll
        for (int k = 0; k < EPV; ++k) e[k] = scale ? acc[q * EPV + k] * f : acc[q * EPV + k];
        V a;
        memcpy(&a, e, sizeof(V));
        dst[q] = a;
    }
}

// FP64: one thread per (output, channel) (the FP64 units bound these sums,
// and this form keeps more of them busy than the staged one)
// out[j][l][c] = sum_i S[l][i] in[j][i][c] along the rows (x), S = sin(pi l i / nx)
template <typename T, int CP>
__global__ void sine_rows_point_kernel(const T* __restrict__ in, const T* __restrict__ S, int nx, int ny, T* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(ny + 1) * (nx + 1) * CP;
    if (t >= tot) return;
    const int c = (int)(t % CP);
    const int l = (int)((t / CP) % (nx + 1));
    const int j = (int)(t / ((int64_t)CP * (nx + 1)));
    T s = (T)0;
    const T* row = in + (int64_t)j * (nx + 1) * CP + c;
    const T* sl = S + (int64_t)l * (nx + 1);
    for (int i = 1; i < nx; ++i) s = fma(sl[i], row[(int64_t)i * CP], s);
    out[t] = s;
}

// out[m][l][c] = scale[m][l] sum_j S[m][j] in[j][l][c] along the columns (y)
template <typename T, int CP>
__global__ void sine_cols_point_kernel(const T* __restrict__ in, const T* __restrict__ S, const T* __restrict__ scale, int nx,
                                 int ny, T* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(ny + 1) * (nx + 1) * CP;
    if (t >= tot) return;
    const int c = (int)(t % CP);
    const int l = (int)((t / CP) % (nx + 1));
    const int m = (int)(t / ((int64_t)CP * (nx + 1)));
    T s = (T)0;
    const T* col = in + (int64_t)l * CP + c;
    const T* sm = S + (int64_t)m * (ny + 1);
    for (int j = 1; j < ny; ++j) s = fma(sm[j], col[(int64_t)j * (nx + 1) * CP], s);
    out[t] = scale ? s * scale[(int64_t)m * (nx + 1) + l] : s;
}

// E = -grad phi at interior nodes (central differences), zero on the walls;
// records [ny+1][nx+1][2][CP]
template <typename T, int CP>
__global__ void field2d_kernel(const T* __restrict__ phi, int nx, int ny, T fx, T fy, T* __restrict__ E) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(ny + 1) * (nx + 1) * CP;
    if (t >= tot) return;
    const int c = (int)(t % CP);
    const int64_t node = t / CP;
    const int i = (int)(node % (nx + 1)), j = (int)(node / (nx + 1));
    T ex = (T)0, ey = (T)0;
    if (i >= 1 && i <= nx - 1 && j >= 1 && j <= ny - 1) {
        ex = -(phi[t + CP] - phi[t - CP]) * fx;
        ey = -(phi[t + (int64_t)(nx + 1) * CP] - phi[t - (int64_t)(nx + 1) * CP]) * fy;
    }
    E[node * 2 * CP + c] = ex;
    E[node * 2 * CP + CP + c] = ey;
}

// gather of the dual field, the kick p += a E (dual product with the dual
// kick factor 2 pi K tau), then the dual map A of the x and y planes; in place
template <typename T, int C, int CP>
__global__ void __launch_bounds__(128) push2d_kernel(T* __restrict__ st, int64_t N, const T* __restrict__ E, int nx,
                                                     int ny, T offx, T offy, T ihx, T ihy, const MapCoef<T, CP> A,
                                                     const KickCoef<T, CP> K, int* __restrict__ err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    T u[4][CP];
#pragma unroll
    for (int c = 0; c < 4; ++c) ldv<T, CP>(st + ((int64_t)c * N + i) * CP, u[c]);
    int bad = 0;
    T fx, fy;
    const int ix = cell2d<T>(u[0][0], offx, ihx, nx, fx, bad);
    const int iy = cell2d<T>(u[2][0], offy, ihy, ny, fy, bad);
    if (bad) atomicOr(err, bad);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        T Ev[CP];
        T gx = (T)0, gy = (T)0;
#pragma unroll
        for (int k = 0; k < CP; ++k) Ev[k] = (T)0;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const T wx = a ? fx : (T)1 - fx, sx = a ? (T)1 : (T)-1;
                const T wy = b ? fy : (T)1 - fy, sy = b ? (T)1 : (T)-1;
                T en[CP];
                ldv<T, CP>(E + (((int64_t)(iy + b) * (nx + 1) + (ix + a)) * 2 + d) * CP, en);
                const T W = wx * wy;
#pragma unroll
                for (int k = 0; k < CP; ++k) Ev[k] = fma(W, en[k], Ev[k]);
                gx = fma(sx * wy, en[0], gx);
                gy = fma(wx * sy, en[0], gy);
            }
        gx *= ihx;
        gy *= ihy;
        T* p = u[2 * d + 1];
        const T a0 = K.a[d][0], E0 = Ev[0];
#pragma unroll
        for (int k = 1; k < CP; ++k) {
            const T Ek = fma(u[0][k], gx, fma(u[2][k], gy, Ev[k]));
            p[k] = fma(a0, Ek, fma(K.a[d][k], E0, p[k]));
        }
        p[0] = fma(a0, E0, p[0]);
    }
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
        T* x = u[2 * pl];
        T* p = u[2 * pl + 1];
        const T a0 = A.m[pl][0][0], b0 = A.m[pl][1][0], c0 = A.m[pl][2][0], d0 = A.m[pl][3][0];
        const T x0 = x[0], p0 = p[0];
#pragma unroll
        for (int k = 1; k < CP; ++k) {
            const T xk = x[k], pk = p[k];
            x[k] = fma(a0, xk, fma(b0, pk, fma(A.m[pl][0][k], x0, A.m[pl][1][k] * p0)));
            p[k] = fma(c0, xk, fma(d0, pk, fma(A.m[pl][2][k], x0, A.m[pl][3][k] * p0)));
        }
        x[0] = fma(a0, x0, b0 * p0);
        p[0] = fma(c0, x0, d0 * p0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) stv<T, CP>(st + ((int64_t)c * N + i) * CP, u[c]);
}

template <typename T, int CP>
__global__ void convert_in2d_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t rows4, int C) {
    // host [4][N][C] doubles into the first four coordinate rows [4][N][CP]
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows4 * CP) return;
    const int64_t r = t / CP;
    const int k = (int)(t % CP);
    dst[t] = k < C ? (T)src[r * C + k] : (T)0;
}

template <typename T, int CP>
__global__ void convert_out2d_kernel(const T* __restrict__ src, double* __restrict__ dst, int64_t rows4, int C) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows4 * C) return;
    dst[t] = (double)src[(t / C) * CP + (t % C)];
}

unsigned nblk(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ====================================================================== handle

struct ad_pic2d {
    int prec = 0, P = 7, C = 8, CP = 8;
    int nx = 0, ny = 0;
    double a = 0, b = 0;
    int64_t N = 0;
    double gamma0 = 0, beta0 = 0, p0 = 0, brho = 0, K_per_A = 0, current = 0;
    int current_slot = -1;
    bool beam_set = false, lattice_set = false, particles_set = false;
    ad_pic_lattice lat{};
    int kpp = 0;
    int64_t kick = 0;
    bool first_record = true;
    cudaStream_t stream = nullptr;
    void* state = nullptr;           // [6][N][CP], z rows zero
    void *rho = nullptr, *phi = nullptr, *T1 = nullptr, *T2 = nullptr, *E = nullptr;
    void *Sx = nullptr, *Sy = nullptr, *scale = nullptr;
    void* mm = nullptr;              // extrema scratch of the shared half-map kernel
    int* err = nullptr;
    double* partial = nullptr;
    double* records = nullptr;
    int records_cap = 0;
    double* staging = nullptr;
    std::vector<void*> allocs;
    std::vector<unsigned char> half, comp, kcoef;
    std::vector<double> hist;        // records [3][5][C] (z plane zero)
};

namespace {

int alloc2d(ad_pic2d* h, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return AD_PIC_ERR_OOM;
    }
    h->allocs.push_back(*p);
    return AD_PIC_OK;
}

template <typename T, int C, int CP>
struct Impl2 {
    using M = MapCoef<T, CP>;
    using K = KickCoef<T, CP>;

    static M to_map(const HMap& a) {
        M r;
        for (int p = 0; p < 3; ++p)
            for (int e = 0; e < 4; ++e)
                for (int k = 0; k < CP; ++k) r.m[p][e][k] = (T)a.m[p][e].v[k];
        return r;
    }

    // per-kick half maps (x, y planes; z identity), their compositions and the dual kick factor
    static void build_coef(ad_pic2d* h) {
        const ad_pic_lattice& L = h->lat;
        const int len_param[5] = {0, 1, 3, 4, 6};
        int kpp = 0;
        for (int e = 0; e < 5; ++e) kpp += L.kicks[e];
        h->kpp = kpp;
        std::vector<HMap> halfm(kpp);
        std::vector<K> kc(kpp);
        const HD I = hvar(h->current, h->current_slot);
        const HD twopiK = hmul(hc(2.0 * kPi * h->K_per_A), I);          // K is linear in the current
        int s = 0;
        for (int e = 0; e < 5; ++e) {
            const HD Le = hvar(L.L[e], L.deriv_slot[len_param[e]]);
            const HD tau = hdiv(Le, hc((double)L.kicks[e]));
            const HD t = hmul(tau, hc(0.5));
            HD kx = hc(0.0), ky = hc(0.0);
            if (e == 1 || e == 3) {
                const HD g = hvar(L.g[e == 1 ? 0 : 1], L.deriv_slot[e == 1 ? 2 : 5]);
                kx = hdiv(g, hc(h->brho));
                ky = hneg(kx);
            }
            HMap m;
            plane_map(kx, t, m.m[0]);
            plane_map(ky, t, m.m[1]);
            m.m[2][0] = hc(1.0); m.m[2][1] = hc(0.0); m.m[2][2] = hc(0.0); m.m[2][3] = hc(1.0);
            const HD ak = hmul(twopiK, tau);
            K kk;
            for (int k = 0; k < CP; ++k) { kk.a[0][k] = (T)ak.v[k]; kk.a[1][k] = (T)ak.v[k]; kk.a[2][k] = (T)0; }
            for (int j = 0; j < L.kicks[e]; ++j, ++s) { halfm[s] = m; kc[s] = kk; }
        }
        h->half.resize(sizeof(M) * kpp);
        h->comp.resize(sizeof(M) * kpp);
        h->kcoef.resize(sizeof(K) * kpp);
        for (int i = 0; i < kpp; ++i) {
            M a = to_map(halfm[i]);
            M c = to_map(compose(halfm[(i + 1) % kpp], halfm[i]));
            std::memcpy(h->half.data() + sizeof(M) * i, &a, sizeof(M));
            std::memcpy(h->comp.data() + sizeof(M) * i, &c, sizeof(M));
            std::memcpy(h->kcoef.data() + sizeof(K) * i, &kc[i], sizeof(K));
        }
    }
    static const M& half(ad_pic2d* h, int64_t g) { return ((const M*)h->half.data())[g % h->kpp]; }
    static const M& comp(ad_pic2d* h, int64_t g) { return ((const M*)h->comp.data())[g % h->kpp]; }
    static const K& kick(ad_pic2d* h, int64_t g) { return ((const K*)h->kcoef.data())[g % h->kpp]; }

    static int allocate(ad_pic2d* h) {
        const int64_t nodes = (int64_t)(h->nx + 1) * (h->ny + 1);
        int r = 0;
        r |= alloc2d(h, &h->state, sizeof(T) * 6 * h->N * CP);
        r |= alloc2d(h, &h->rho, sizeof(T) * nodes * CP);
        r |= alloc2d(h, &h->phi, sizeof(T) * nodes * CP);
        r |= alloc2d(h, &h->T1, sizeof(T) * nodes * CP);
        r |= alloc2d(h, &h->T2, sizeof(T) * nodes * CP);
        r |= alloc2d(h, &h->E, sizeof(T) * nodes * 2 * CP);
        r |= alloc2d(h, &h->Sx, sizeof(T) * (h->nx + 1) * (h->nx + 1));
        r |= alloc2d(h, &h->Sy, sizeof(T) * (h->ny + 1) * (h->ny + 1));
        r |= alloc2d(h, &h->scale, sizeof(T) * nodes);
        r |= alloc2d(h, &h->mm, sizeof(Ord<T>) * 6);
        r |= alloc2d(h, (void**)&h->err, sizeof(int));
        r |= alloc2d(h, (void**)&h->partial, sizeof(double) * boundary_blocks() * 15 * CP);
        if (r) return AD_PIC_ERR_OOM;
        // sine matrices (rows 0 and n exactly zero: phi = 0 on the walls) and
        // the spectral factors 4 / (nx ny gamma_lm^2), gamma_lm^2 = (l pi/a)^2 + (m pi/b)^2
        auto sines = [](int n) {
            std::vector<T> S((size_t)(n + 1) * (n + 1), (T)0);
            for (int l = 1; l < n; ++l)
                for (int i = 1; i < n; ++i) {
                    const long long q = ((long long)l * i) % (2LL * n);      // exact argument reduction
                    S[(size_t)l * (n + 1) + i] = (T)std::sin(kPi * (double)q / (double)n);
                }
            return S;
        };
        std::vector<T> Sx = sines(h->nx), Sy = sines(h->ny), sc((size_t)nodes, (T)0);
        for (int m = 1; m < h->ny; ++m)
            for (int l = 1; l < h->nx; ++l) {
                const double al = kPi * l / h->a, be = kPi * m / h->b;
                sc[(size_t)m * (h->nx + 1) + l] = (T)(4.0 / ((double)h->nx * h->ny) / (al * al + be * be));
            }
        // the staged line of the sine sums: up to 513 records of CP values
        if constexpr (sizeof(T) == 4) {
            cudaFuncSetAttribute(sine_rows_kernel<T, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            cudaFuncSetAttribute(sine_cols_kernel<T, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        }
        if (cudaMemcpy(h->Sx, Sx.data(), sizeof(T) * Sx.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->Sy, Sy.data(), sizeof(T) * Sy.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->scale, sc.data(), sizeof(T) * sc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(h->state, 0, sizeof(T) * 6 * h->N * CP) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        return AD_PIC_OK;
    }

    static void field(ad_pic2d* h) {
        cudaStream_t s = h->stream;
        const int64_t nodes = (int64_t)(h->nx + 1) * (h->ny + 1);
        const unsigned g = nblk(nodes * CP);
        const T hx = (T)(h->a / h->nx), hy = (T)(h->b / h->ny);
        cudaMemsetAsync(h->rho, 0, sizeof(T) * nodes * CP, s);
        deposit2d_kernel<T, C, CP><<<nblk(h->N), 256, 0, s>>>(
            (const T*)h->state, h->N, h->nx, h->ny, (T)(0.5 * h->a), (T)(0.5 * h->b), (T)1 / hx, (T)1 / hy,
            (T)(1.0 / ((double)h->N * (h->a / h->nx) * (h->b / h->ny))), (T*)h->rho, h->err);
        // rho^lm (rows, then columns with the spectral factor), then phi by the sine sums back
        if constexpr (sizeof(T) == 4) {
            const dim3 gr((unsigned)((h->nx + kSineThreads) / kSineThreads), (unsigned)(h->ny + 1));
            const dim3 gc((unsigned)((h->ny + kSineThreads) / kSineThreads), (unsigned)(h->nx + 1));
            const size_t smr = sizeof(T) * (size_t)(h->nx + 1) * CP, smc = sizeof(T) * (size_t)(h->ny + 1) * CP;
            sine_rows_kernel<T, CP><<<gr, kSineThreads, smr, s>>>((const T*)h->rho, (const T*)h->Sx, h->nx, h->ny,
                                                                  (T*)h->T1);
            sine_cols_kernel<T, CP><<<gc, kSineThreads, smc, s>>>((const T*)h->T1, (const T*)h->Sy,
                                                                  (const T*)h->scale, h->nx, h->ny, (T*)h->T2);
            sine_cols_kernel<T, CP><<<gc, kSineThreads, smc, s>>>((const T*)h->T2, (const T*)h->Sy, nullptr, h->nx,
                                                                  h->ny, (T*)h->T1);
            sine_rows_kernel<T, CP><<<gr, kSineThreads, smr, s>>>((const T*)h->T1, (const T*)h->Sx, h->nx, h->ny,
                                                                  (T*)h->phi);
        } else {
            sine_rows_point_kernel<T, CP><<<g, 256, 0, s>>>((const T*)h->rho, (const T*)h->Sx, h->nx, h->ny,
                                                            (T*)h->T1);
            sine_cols_point_kernel<T, CP><<<g, 256, 0, s>>>((const T*)h->T1, (const T*)h->Sy, (const T*)h->scale,
                                                            h->nx, h->ny, (T*)h->T2);
            sine_cols_point_kernel<T, CP><<<g, 256, 0, s>>>((const T*)h->T2, (const T*)h->Sy, nullptr, h->nx, h->ny,
                                                            (T*)h->T1);
            sine_rows_point_kernel<T, CP><<<g, 256, 0, s>>>((const T*)h->T1, (const T*)h->Sx, h->nx, h->ny,
                                                            (T*)h->phi);
        }
        field2d_kernel<T, CP><<<g, 256, 0, s>>>((const T*)h->phi, h->nx, h->ny, (T)0.5 / hx, (T)0.5 / hy, (T*)h->E);
    }

    static void push(ad_pic2d* h, const M& A, const K& Kc) {
        push2d_kernel<T, C, CP><<<nblk(h->N, 128), 128, 0, h->stream>>>(
            (T*)h->state, h->N, (const T*)h->E, h->nx, h->ny, (T)(0.5 * h->a), (T)(0.5 * h->b),
            (T)(h->nx / h->a), (T)(h->ny / h->b), A, Kc, h->err);
    }

    static void reduce(ad_pic2d* h, int r) {
        launch_moments_reduce(h->partial, boundary_blocks(), CP, h->N, h->records + (int64_t)r * 15 * CP, h->stream);
    }

    static M identity() {
        HMap I;
        for (int p = 0; p < 3; ++p) { I.m[p][0] = hc(1); I.m[p][1] = hc(0); I.m[p][2] = hc(0); I.m[p][3] = hc(1); }
        return to_map(I);
    }

    static int run(ad_pic2d* h, int n) {
        build_coef(h);
        cudaStream_t s = h->stream;
        const int nb = boundary_blocks();
        GeomFuse nofuse{};
        const int need = (h->first_record ? 1 : 0) + 1 + n / h->kpp + 1;
        if (need > h->records_cap) {
            if (h->records) cudaFree(h->records);
            for (auto& p : h->allocs) if (p == h->records) p = nullptr;
            h->records = nullptr;
            if (alloc2d(h, (void**)&h->records, sizeof(double) * 15 * CP * need)) return AD_PIC_ERR_OOM;
            h->records_cap = need;
        }
        cudaMemsetAsync(h->err, 0, sizeof(int), s);
        int nrec = 0;
        const int64_t g0 = h->kick;
        if (n == 0) {
            launch_boundary<T, C, CP>((T*)h->state, h->N, identity(), false, true, h->partial, nb, (Ord<T>*)h->mm,
                                      nofuse, s);
            reduce(h, nrec++);
        } else {
            launch_boundary<T, C, CP>((T*)h->state, h->N, half(h, g0), true, h->first_record, h->partial, nb,
                                      (Ord<T>*)h->mm, nofuse, s);
            if (h->first_record) reduce(h, nrec++);
            for (int i = 0; i < n; ++i) {
                const int64_t g = g0 + i;
                field(h);
                const bool last = i == n - 1, pend = ((g + 1) % h->kpp) == 0;
                if (last || pend) {
                    push(h, half(h, g), kick(h, g));
                    launch_boundary<T, C, CP>((T*)h->state, h->N, half(h, g + 1), !last, true, h->partial, nb,
                                              (Ord<T>*)h->mm, nofuse, s);
                    reduce(h, nrec++);
                } else {
                    push(h, comp(h, g), kick(h, g));
                }
            }
        }
        if (cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        std::vector<double> rec((size_t)nrec * 15 * CP);
        int errw = 0;
        if (cudaMemcpyAsync(rec.data(), h->records, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&errw, h->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        for (int r = 0; r < nrec; ++r)
            for (int q = 0; q < 15; ++q)
                for (int k = 0; k < C; ++k) h->hist.push_back(rec[((size_t)r * 15 + q) * CP + k]);
        h->kick += n;
        h->first_record = false;
        if (errw & kErrNonfinite) return AD_PIC_ERR_NONFINITE;
        if (errw & kErrOutOfGrid) return AD_PIC_ERR_OUT_OF_GRID;
        return AD_PIC_OK;
    }

    static int staging(ad_pic2d* h) {
        if (!h->staging && alloc2d(h, (void**)&h->staging, sizeof(double) * 4 * h->N * C)) return AD_PIC_ERR_OOM;
        return AD_PIC_OK;
    }

    static int set_particles(ad_pic2d* h, const double* src) {
        if (staging(h)) return AD_PIC_ERR_OOM;
        cudaStream_t s = h->stream;
        if (cudaMemcpyAsync(h->staging, src, sizeof(double) * 4 * h->N * C, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        convert_in2d_kernel<T, CP><<<nblk(4 * h->N * CP), 256, 0, s>>>(h->staging, (T*)h->state, 4 * h->N, C);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
        h->particles_set = true;
        h->kick = 0;
        h->first_record = true;
        h->hist.clear();
        return AD_PIC_OK;
    }

    static int get_particles(ad_pic2d* h, double* dst) {
        if (staging(h)) return AD_PIC_ERR_OOM;
        cudaStream_t s = h->stream;
        convert_out2d_kernel<T, CP><<<nblk(4 * h->N * C), 256, 0, s>>>((const T*)h->state, h->staging, 4 * h->N, C);
        if (cudaMemcpyAsync(dst, h->staging, sizeof(double) * 4 * h->N * C, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return AD_PIC_ERR_CUDA;
        return AD_PIC_OK;
    }

    // per plane u = sqrt(eps beta) n1, p = sqrt(eps/beta) (n2 - alpha n1), sample mean removed (host FP64)
    static int beam_init(ad_pic2d* h, const ad_pic_beam* b, const double* normals) {
        std::vector<double> st((size_t)4 * h->N * C, 0.0);
        const double bg = h->beta0 * h->gamma0;
        for (int pl = 0; pl < 2; ++pl) {
            const double eps = b->eps_n[pl] / bg, beta = b->beta[pl], alpha = b->alpha[pl];
            double m1 = 0.0, m2 = 0.0;
            for (int64_t i = 0; i < h->N; ++i) { m1 += normals[(2 * pl) * h->N + i]; m2 += normals[(2 * pl + 1) * h->N + i]; }
            m1 /= (double)h->N;
            m2 /= (double)h->N;
            for (int64_t i = 0; i < h->N; ++i) {
                const double n1 = normals[(2 * pl) * h->N + i] - m1, n2 = normals[(2 * pl + 1) * h->N + i] - m2;
                st[((size_t)(2 * pl) * h->N + i) * C] = std::sqrt(eps * beta) * n1;
                st[((size_t)(2 * pl + 1) * h->N + i) * C] = std::sqrt(eps / beta) * (n2 - alpha * n1);
            }
        }
        return set_particles(h, st.data());
    }
};

#define DISPATCH2(h, expr)                                                                                  \
    do {                                                                                                    \
        if ((h)->prec == AD_PIC_FP64 && (h)->P == 7) { using I = Impl2<double, 8, 8>; return expr; }        \
        if ((h)->prec == AD_PIC_FP64 && (h)->P == 13) { using I = Impl2<double, 14, 16>; return expr; }     \
        if ((h)->prec == AD_PIC_FP32_MIXED && (h)->P == 7) { using I = Impl2<float, 8, 8>; return expr; }   \
        if ((h)->prec == AD_PIC_FP32_MIXED && (h)->P == 13) { using I = Impl2<float, 14, 16>; return expr; } \
        return AD_PIC_ERR_INVALID_ARG;                                                                      \
    } while (0)

}  // namespace

extern "C" {

int ad_pic2d_create(int nx, int ny, double a, double b, int64_t n_particles, int n_deriv, int precision,
                    ad_pic2d** out) {
    if (!out) return AD_PIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < 8 || nx > 512 || ny < 8 || ny > 512 || !(a > 0) || !(b > 0) || n_particles < 1 ||
        n_particles > ((int64_t)1 << 31) - 1 || (n_deriv != 7 && n_deriv != 13) ||
        (precision != AD_PIC_FP64 && precision != AD_PIC_FP32_MIXED))
        return AD_PIC_ERR_INVALID_ARG;
    ad_pic2d* h = new (std::nothrow) ad_pic2d();
    if (!h) return AD_PIC_ERR_OOM;
    h->prec = precision;
    h->P = n_deriv;
    h->C = n_deriv + 1;
    h->CP = n_deriv == 7 ? 8 : 16;
    h->nx = nx; h->ny = ny; h->a = a; h->b = b;
    h->N = n_particles;
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return AD_PIC_ERR_CUDA;
    }
    auto alloc = [&]() -> int { DISPATCH2(h, I::allocate(h)); };
    const int st = alloc();
    if (st) { ad_pic2d_destroy(h); return st; }
    *out = h;
    return AD_PIC_OK;
}

int ad_pic2d_set_beam(ad_pic2d* h, const ad_pic_beam* b, double current_A, int current_deriv_slot,
                      const double* normals) {
    if (!h || !b || !(b->kinetic_eV > 0) || !(b->mass_eV > 0) || b->charge_e == 0 || !(current_A >= 0) ||
        current_deriv_slot < -1 || current_deriv_slot >= h->P)
        return AD_PIC_ERR_INVALID_ARG;
    if (b->energy_deriv_slot != -1) return AD_PIC_ERR_UNSUPPORTED;   // the pipe's energy derivative is not built
    for (int d = 0; d < 2; ++d)
        if (!(b->eps_n[d] > 0) || !(b->beta[d] > 0) || !std::isfinite(b->alpha[d])) return AD_PIC_ERR_INVALID_ARG;
    const double q = b->charge_e * kQE;
    const double mass_kg = b->mass_eV * kQE / (kC * kC);
    h->gamma0 = 1.0 + b->kinetic_eV / b->mass_eV;
    h->beta0 = std::sqrt(1.0 - 1.0 / (h->gamma0 * h->gamma0));
    h->p0 = h->gamma0 * h->beta0 * mass_kg * kC;
    h->brho = h->p0 / q;
    const double v0 = h->beta0 * kC;
    h->K_per_A = q / (2.0 * kPi * kEps0 * h->p0 * v0 * v0 * h->gamma0 * h->gamma0);
    h->current = current_A;
    h->current_slot = current_deriv_slot;
    h->beam_set = true;
    if (!normals) return AD_PIC_OK;
    DISPATCH2(h, I::beam_init(h, b, normals));
}

int ad_pic2d_set_particles(ad_pic2d* h, const double* state) {
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    DISPATCH2(h, I::set_particles(h, state));
}

int ad_pic2d_get_particles(const ad_pic2d* hc_, double* state) {
    ad_pic2d* h = const_cast<ad_pic2d*>(hc_);
    if (!h || !state) return AD_PIC_ERR_INVALID_ARG;
    if (!h->particles_set) return AD_PIC_ERR_STATE;
    DISPATCH2(h, I::get_particles(h, state));
}

int ad_pic2d_set_lattice(ad_pic2d* h, const ad_pic_lattice* L) {
    if (!h || !L) return AD_PIC_ERR_INVALID_ARG;
    for (int e = 0; e < 5; ++e)
        if (!(L->L[e] > 0) || L->kicks[e] < 1 || L->kicks[e] > 100000) return AD_PIC_ERR_INVALID_ARG;
    if (!(L->g[0] != 0) || !(L->g[1] != 0) || !std::isfinite(L->g[0]) || !std::isfinite(L->g[1]))
        return AD_PIC_ERR_INVALID_ARG;
    for (int j = 0; j < 7; ++j)
        if (L->deriv_slot[j] < -1 || L->deriv_slot[j] >= h->P) return AD_PIC_ERR_INVALID_ARG;
    h->lat = *L;
    h->lattice_set = true;
    return AD_PIC_OK;
}

int ad_pic2d_run(ad_pic2d* h, int n_steps) {
    if (!h || n_steps < 0) return AD_PIC_ERR_INVALID_ARG;
    if (!h->beam_set || !h->lattice_set || !h->particles_set) return AD_PIC_ERR_STATE;
    if (cudaPeekAtLastError() != cudaSuccess) return AD_PIC_ERR_CUDA;
    DISPATCH2(h, I::run(h, n_steps));
}

int ad_pic2d_moments(const ad_pic2d* h, double* values, double* derivs) {
    if (!h || !values) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    if (h->hist.size() < rs) return AD_PIC_ERR_STATE;
    const double* rec = h->hist.data() + h->hist.size() - rs;
    for (int pl = 0; pl < 2; ++pl) {
        // centred second moments and the dual emittance (Sec. 4)
        HD m[5];
        for (int q = 0; q < 5; ++q) {
            m[q] = hc(0.0);
            for (int k = 0; k < h->C; ++k) m[q].v[k] = rec[(pl * 5 + q) * h->C + k];
        }
        const HD a = hadd(m[2], hneg(hmul(m[0], m[0])));
        const HD b = hadd(m[3], hneg(hmul(m[0], m[1])));
        const HD c = hadd(m[4], hneg(hmul(m[1], m[1])));
        const HD e = hsqrt(hadd(hmul(a, c), hneg(hmul(b, b))));
        values[pl] = e.v[0];
        if (derivs)
            for (int k = 0; k < h->P; ++k) derivs[pl * h->P + k] = e.v[1 + k];
    }
    return AD_PIC_OK;
}

int ad_pic2d_moments_full(const ad_pic2d* h, double* mom) {
    if (!h || !mom) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    if (h->hist.size() < rs) return AD_PIC_ERR_STATE;
    std::memcpy(mom, h->hist.data() + h->hist.size() - rs, sizeof(double) * 10 * h->C);
    return AD_PIC_OK;
}

int ad_pic2d_history(const ad_pic2d* h, double* hist, int max_records, int* n_records) {
    if (!h || !n_records || max_records < 0) return AD_PIC_ERR_INVALID_ARG;
    const size_t rs = (size_t)15 * h->C;
    const int n = (int)(h->hist.size() / rs);
    *n_records = n;
    if (hist)
        for (int r = 0; r < n && r < max_records; ++r)
            std::memcpy(hist + (size_t)r * 10 * h->C, h->hist.data() + (size_t)r * rs, sizeof(double) * 10 * h->C);
    return AD_PIC_OK;
}

void ad_pic2d_destroy(ad_pic2d* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    if (h->stream) cudaStreamDestroy(h->stream);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
